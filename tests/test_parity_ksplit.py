"""GPU parity of the K-split SIMT engine (FP32: 8 x 8 register blocks, the j reduction in
chunks whose D^T rows are fetched one chunk ahead) against the CPU FP64 oracle.

Bars: integer-valued inputs bit-exact (every partial sum is exact in FP32); random inputs
within the FP32 FMA-chain bound of the exact result; sentinel elements around every
output untouched; the full-size precision-sweep and N = 165 problems on sampled rows.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import CanaryOut, fma_bound, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


def ks_variant(lc, layout, bm, bk, stages, max_ctas=0):
    return lc.Variant(engine="ksplit", layout=layout, precision="fp32", tile_e=bm, elems_per_thread=8,
                      split_i=8, unroll=bk, prefetch_smem=1, stages=stages, max_ctas=max_ctas)


def run(lc, kernel, v, D, u, layout):
    import torch
    F, N, _ = D.shape
    E = u.shape[1] if layout == "node" else u.shape[0]
    co = CanaryOut((F, N, E) if layout == "node" else (F, E, N), np.float32)
    lc.contract(kernel, v, to_dev(D), to_dev(u), co.out)
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    assert co.intact(), "write outside the output"
    return co.out.cpu().numpy().astype(np.float64)


# (E, N, F): ragged tails, N not a multiple of 4 or of the chunk, several column blocks,
# the largest N and F, a single element
SHAPES = [(1000, 35, 3), (333, 84, 4), (517, 20, 1), (64, 4, 2), (1, 5, 1), (300, 16, 3), (129, 120, 2),
          (257, 165, 3), (130, 256, 8), (4099, 10, 3), (200, 128, 1)]


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_integer_inputs_bit_exact(lc, layout):
    kernel = lc.Kernel()
    for si, (E, N, F) in enumerate(SHAPES):
        D, u = synth.integer_operands(E, N, F, seed=E + N)
        uu = synth.to_node_major(u) if layout == "node" else u
        want = oracle.contract(D, uu, layout)
        ran = 0
        for bm, bk, st, mc in ((128, 16, 2, 0), (64, 8, 1, 0), (128, 8, 1, 3), (64, 16, 2, 2)):
            v = ks_variant(lc, layout, bm, bk, st, mc)
            if lc.variant_validate(kernel, E, N, F, v) != 0:
                continue
            got = run(lc, kernel, v, D, uu, layout)
            assert np.array_equal(got, want), (E, N, F, layout, bm, bk, st, mc)
            ran += 1
        assert ran >= 2, (E, N, F)


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_random_inputs_within_bound(lc, layout):
    kernel = lc.Kernel()
    for si, (E, N, F) in enumerate(SHAPES):
        D, u = synth.operands(E, N, F, np.float32, seed=300 + si, scale_exp=3.0 if si % 2 else None)
        uu = synth.to_node_major(u) if layout == "node" else u
        v = ks_variant(lc, layout, 64, 16, 2)
        got = run(lc, kernel, v, D, uu, layout)
        ref = oracle.contract(D, uu, layout)
        assert np.all(np.abs(got - ref) <= fma_bound(D, uu, layout, 2.0 ** -24)), (E, N, F)


def test_unaligned_node_major_rows(lc):
    """Node-major with E % 4 != 0: u rows copied element by element, outputs stored one by one."""
    kernel = lc.Kernel()
    E, N, F = 1023, 56, 2
    D, u = synth.integer_operands(E, N, F, seed=7)
    uu = synth.to_node_major(u)
    for bm in (64, 128):
        got = run(lc, kernel, ks_variant(lc, "node", bm, 8, 2), D, uu, "node")
        assert np.array_equal(got, oracle.contract(D, uu, "node"))


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("shape", ["precision", "n165"])
def test_full_size_sampled(lc, layout, shape):
    """The precision-sweep problem (E = 2^20, N = 84, F = 4, u scaled by 10^k) and the
    uneven-batching workload's largest group (E = 564445, N = 165, F = 3) at full size,
    sampled rows against the oracle within the FMA bound."""
    import torch
    if shape == "precision":
        D, u = synth.precision_sweep()
    else:
        D, u = synth.operands(564445, 165, 3, np.float32, seed=4)
    F, N, _ = D.shape
    E = u.shape[0]
    kernel = lc.Kernel()
    uu = synth.to_node_major(u) if layout == "node" else u
    v = ks_variant(lc, layout, 128, 16, 2)
    out = lc.contract(kernel, v, to_dev(D), to_dev(uu))
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    rows = np.unique(np.concatenate([np.arange(300), np.random.default_rng(5).integers(0, E, 3000),
                                     np.arange(E - 300, E)]))
    idx = torch.from_numpy(rows).cuda()
    got = out.index_select(2 if layout == "node" else 1, idx).cpu().numpy().astype(np.float64)
    if layout == "node":
        got = got.transpose(0, 2, 1)
    ref = oracle.contract_rows(D, u, rows)
    assert np.all(np.abs(got - ref) <= fma_bound(D, u[rows], "elem", 2.0 ** -24))
