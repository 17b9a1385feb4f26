"""GPU FP64 error norm (lc_error_norm) against the oracle's relative Frobenius error."""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 255, 1000003, 1 << 22])
def test_error_norm_matches_oracle(lc, dtype, n):
    import torch
    rng = np.random.default_rng(n)
    ref = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
    out = (ref * (1 + rng.normal(0, 1e-6, n))).astype(dtype)
    got = lc.error_norm(torch.from_numpy(out).cuda(), torch.from_numpy(ref).cuda())
    want = oracle.rel_fro_error(out, ref)
    assert abs(got - want) <= 1e-10 * want + 1e-300


def test_error_norm_exact_zero_and_known_value(lc):
    import torch
    ref = torch.tensor([3.0, 4.0], dtype=torch.float64, device="cuda")
    assert lc.error_norm(ref.clone(), ref) == 0.0
    out = torch.tensor([3.3, 4.4], dtype=torch.float64, device="cuda")
    assert abs(lc.error_norm(out, ref) - 0.1) < 1e-15
