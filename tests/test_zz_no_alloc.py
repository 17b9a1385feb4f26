"""The workspace-free error norm (lc_error_norm_noalloc), for callers that cannot
allocate device memory: it must give lc_error_norm's result, call after call, through
the C ABI.  Kept in a file of its own that runs last."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


def _sums_with_workspace(lc, out, ref, dt, stream):
    import torch
    lib = lc.load()
    ws = ctypes.c_size_t(0)
    lc.check(lib.lc_error_norm_workspace_size(out.numel(), ctypes.byref(ws)))
    work = torch.empty(ws.value // 8 + 2, dtype=torch.float64, device="cuda")
    sums = torch.empty(2, dtype=torch.float64, device="cuda")
    lc.check(lib.lc_error_norm(out.data_ptr(), dt, ref.data_ptr(), out.numel(), sums.data_ptr(), work.data_ptr(),
                               ws.value, stream))
    return sums


def test_noalloc_matches_workspace_version_twice(lc):
    import torch
    lib = lc.load()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(7)
    for n, dtype, dt in ((3_000_001, np.float32, lc.DTYPE_F32), (65536 * 3 + 17, np.float64, lc.DTYPE_F64)):
        sums_nd = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        # two calls in a row on different data: the shared array must not leak state
        for call in range(2):
            ref = rng.standard_normal(n) * 10.0 ** rng.uniform(-2, 2, n)
            out = (ref * (1 + rng.normal(0, 1e-5, n))).astype(dtype)
            ref_d = torch.from_numpy(ref).cuda()
            out_d = torch.from_numpy(out).cuda()
            want = _sums_with_workspace(lc, out_d, ref_d, dt, stream)
            st = lib.lc_error_norm_noalloc(out_d.data_ptr(), dt, ref_d.data_ptr(), n, sums_nd.data_ptr(), stream)
            assert st == 0, lc.STATUS[st]
            torch.cuda.synchronize()
            got, exp = sums_nd.cpu().numpy(), want.cpu().numpy()
            assert np.allclose(got, exp, rtol=1e-12, atol=0), (call, got, exp)
            rel_got, rel_exp = np.sqrt(got[0] / got[1]), np.sqrt(exp[0] / exp[1])
            assert abs(rel_got - rel_exp) <= 1e-12 * rel_exp


def test_noalloc_rejects_oversize_and_bad_arguments(lc):
    import torch
    lib = lc.load()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert lib.lc_error_norm_noalloc(p, lc.DTYPE_F64, p, (1 << 28) + 1, p, None) == 6  # beyond the array's capacity
    assert lib.lc_error_norm_noalloc(p, lc.DTYPE_F64, p, 0, p, None) == 1
    assert lib.lc_error_norm_noalloc(p, 7, p, 4, p, None) == 1
    assert lib.lc_error_norm_noalloc(None, lc.DTYPE_F64, p, 4, p, None) == 1
