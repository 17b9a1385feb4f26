"""GPU parity of the host-array entry point (lc_contract_host): chunked, overlapped copies
in and out around the contraction must give exactly what one lc_contract of the whole
batch gives (every element's arithmetic is the same), and agree with the CPU FP64 oracle.
Chunks: up to 8 of whole 128-element tiles, at least 2^16 elements each; the sizes below
cover one chunk, several chunks with a ragged last one, and both layouts."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


CASES = [
    (1000, 35, 3, "elem", "bf16x3"),           # one chunk
    ((1 << 18) + 77, 35, 3, "elem", "bf16x3"),  # four chunks, the last ragged
    ((1 << 18) + 77, 35, 3, "node", "bf16x3"),
    ((1 << 19) + 128, 20, 2, "elem", "fp32"),   # eight chunks, SIMT engine
    ((1 << 17) + 5, 84, 4, "node", "bf16"),
    ((1 << 18) + 3, 20, 1, "elem", "fp64"),   # FP64 storage (8-byte elements), four chunks
    ((1 << 18) + 3, 20, 1, "node", "fp64"),
]


@pytest.mark.parametrize("E,N,F,layout,prec", CASES)
def test_host_entry_matches_device_entry(lc, E, N, F, layout, prec):
    import torch
    dtype = np.float64 if prec == "fp64" else np.float32
    D, u = synth.operands(E, N, F, dtype, seed=E % 1000 + N)
    uu = np.ascontiguousarray(synth.to_node_major(u) if layout == "node" else u)
    kernel = lc.Kernel() if F > 1 else lc.Kernel("{ [e,i,j]: 0<=e<E and 0<=i,j<N }", "out[e,i] = sum(j, D[i,j]*u[e,j])")
    v = lc.variant_default(kernel, E, N, F, layout, prec)
    shape = (F, N, E) if layout == "node" else (F, E, N)
    Dd, ud = torch.from_numpy(D).cuda(), torch.from_numpy(uu).cuda()
    want = lc.contract(kernel, v, Dd, ud, torch.empty(shape, dtype=Dd.dtype, device="cuda"))
    torch.cuda.synchronize()
    want = want.cpu().numpy()

    Dh, uh = torch.from_numpy(D).pin_memory(), torch.from_numpy(uu).pin_memory()
    oh = torch.full(shape, float("nan"), dtype=Dd.dtype).pin_memory()
    D2, u2, o2 = torch.empty_like(Dd), torch.empty_like(ud), torch.empty(shape, dtype=Dd.dtype, device="cuda")
    stream = torch.cuda.Stream()
    lc.contract_host(kernel, v, Dh, uh, oh, D2, u2, o2, stream=stream)
    stream.synchronize()
    assert lc.device_error() == 0
    got = oh.numpy()
    assert np.array_equal(got, want), float(np.nanmax(np.abs(got - want)))
    # and against the FP64 oracle on sampled elements
    rows = np.unique(np.concatenate([np.arange(64), np.random.default_rng(0).integers(0, E, 500), [E - 1]]))
    ref = oracle.contract_rows(D, u, rows)
    sub = got[:, :, rows].transpose(0, 2, 1) if layout == "node" else got[:, rows, :]
    tol = {"bf16": 1e-2, "bf16x3": 1e-6, "fp32": 1e-6, "fp64": 1e-13}[prec]
    assert oracle.rel_fro_error(sub, ref) <= tol


def test_host_entry_runs_after_queued_work(lc):
    """The copies wait for work already queued on the caller's stream: a device-side write
    of the input buffer queued before the call must not race with the call's own copy."""
    import torch
    E, N, F = (1 << 17) + 256, 35, 3
    D, u = synth.operands(E, N, F, np.float32, seed=3)
    kernel = lc.Kernel()
    v = lc.variant_default(kernel, E, N, F, "elem", "bf16x3")
    Dh, uh = torch.from_numpy(D).pin_memory(), torch.from_numpy(u).pin_memory()
    oh = torch.empty((F, E, N)).pin_memory()
    D2, u2, o2 = torch.empty(D.shape, device="cuda"), torch.empty(u.shape, device="cuda"), \
        torch.empty((F, E, N), device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(3):
            u2.fill_(7.0)  # queued writes of the same device buffers
            o2.fill_(7.0)
    lc.contract_host(kernel, v, Dh, uh, oh, D2, u2, o2, stream=stream)
    stream.synchronize()
    rows = np.arange(0, E, 997)
    ref = oracle.contract_rows(D, u, rows)
    assert oracle.rel_fro_error(oh.numpy()[:, rows, :], ref) <= 1e-6
