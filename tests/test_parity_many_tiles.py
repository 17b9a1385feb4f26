"""GPU parity with every CTA walking many element tiles (the descriptor's `max_ctas`
bounds the persistent grid), so that each pipeline resource wraps several times:

  * tensor cores (tcgen05): both TMEM accumulators, mbarrier phase flips, the u stage
    ring (stages 1/2/3), A buffers handed over K-block by K-block (K-blocks 16/32/64),
    element-major staging slots reused behind the bulk-store read waits (out_buffers
    1/2/4, store_rows 32/64/128), column blocks of operators, both layouts;
  * SIMT: the bulk-copy prefetch ring (stages 1/2), register blocks, unroll factors.

Inputs are integer-valued (exact in bf16 and in FP32 sums), so every variant must match
the oracle bit for bit (Section 2.3: the transformations of Section 2.4 preserve the
result).  Element counts leave a ragged last tile (the guard of Eq. 1).
"""

import itertools

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import CanaryOut, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


def run(lc, kernel, v, D, u, layout):
    import torch
    F, N, _ = D.shape
    E = u.shape[1] if layout == "node" else u.shape[0]
    co = CanaryOut((F, N, E) if layout == "node" else (F, E, N), D.dtype)
    lc.contract(kernel, v, to_dev(D), to_dev(u), co.out)
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    assert co.intact(), "write outside the output"
    return co.out.cpu().numpy().astype(np.float64)


def tiles_per_cta(lc, kernel, E, N, F, v):
    p = lc.variant_plan(kernel, E, N, F, v)
    return p["tiles"] * p["column_blocks"] / p["grid"]


TC_SHAPES = [(3000 + 77, 35, 3), (2000 + 5, 84, 4), (1500 + 33, 20, 2), (2000 + 1, 56, 1)]


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_tc_descriptor_grid_many_tiles(lc, layout, prec):
    kernel = lc.Kernel()
    ran = 0
    for E, N, F in TC_SHAPES:
        D, u = synth.integer_operands(E, N, F, seed=E + N + F)
        uu = synth.to_node_major(u) if layout == "node" else u
        ref = oracle.contract(D, uu, layout)
        combos = itertools.product((1, 2, 3), (16, 32, 64), ((32, 1), (64, 2), (128, 4), (0, 0)), (0, 1))
        for k, (stages, kbw, (rows, ob), split) in enumerate(combos):
            tpr = 1 + k % 4  # epilogue threads per tile row: 1..4
            if layout == "node" and (rows, ob) != (0, 0):
                continue  # staging slots and store rows are element-major fields
            for nb_ctas in (1, 3):
                v = lc.Variant(engine="tcgen05", layout=layout, precision=prec, tile_e=128, elems_per_thread=kbw,
                               split_i=split, unroll=tpr, prefetch_smem=1, stages=stages, out_buffers=ob,
                               store_rows=rows)
                if lc.variant_validate(kernel, E, N, F, v) != 0:
                    continue
                nblocks = lc.variant_plan(kernel, E, N, F, v)["column_blocks"]
                v.max_ctas = nb_ctas * nblocks
                assert lc.variant_validate(kernel, E, N, F, v) == 0
                assert tiles_per_cta(lc, kernel, E, N, F, v) >= 4
                got = run(lc, kernel, v, D, uu, layout)
                assert np.array_equal(got, ref), (E, N, F, stages, kbw, rows, ob, split, tpr, v.max_ctas)
                ran += 1
    assert ran >= 40, ran


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_tc_large_n_many_tiles(lc, layout, prec):
    """Many K-blocks per tile and many tiles per CTA at once (N = 120 and 165)."""
    kernel = lc.Kernel()
    for E, N, F, kbw in ((1300 + 9, 120, 2, 16), (1100 + 3, 165, 1, 16), (1100 + 3, 165, 2, 32)):
        D, u = synth.integer_operands(E, N, F, seed=N * F)
        uu = synth.to_node_major(u) if layout == "node" else u
        v = lc.Variant(engine="tcgen05", layout=layout, precision=prec, tile_e=128, elems_per_thread=kbw, split_i=0,
                       unroll=2, prefetch_smem=1, stages=1)
        if lc.variant_validate(kernel, E, N, F, v) != 0:
            continue
        v.max_ctas = lc.variant_plan(kernel, E, N, F, v)["column_blocks"] * 2
        assert tiles_per_cta(lc, kernel, E, N, F, v) >= 4
        got = run(lc, kernel, v, D, uu, layout)
        assert np.array_equal(got, oracle.contract(D, uu, layout)), (E, N, F, kbw)


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_simt_descriptor_grid_many_tiles(lc, layout, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    V = 2 if prec == "fp64" else 4
    kernel = lc.Kernel()
    ran = 0
    for E, N, F in ((2000 + 13, 35, 3), (900 + 7, 84, 2), (1500 + 3, 9, 4)):
        D, u = synth.integer_operands(E, N, F, dt, seed=E)
        uu = synth.to_node_major(u) if layout == "node" else u
        ref = oracle.contract(D, uu, layout)
        for re_, rc, unr, (pf, st), te_mul in itertools.product((V, 2 * V), (V, 2 * V), (1, 2, 4, 8),
                                                                ((0, 1), (1, 1), (1, 2)), (4, 16)):
            v = lc.Variant(engine="simt", layout=layout, precision=prec, tile_e=re_ * te_mul, elems_per_thread=re_,
                           split_i=rc, unroll=unr, prefetch_smem=pf, stages=st, ctas_per_sm=1)
            if lc.variant_validate(kernel, E, N, F, v) != 0:
                continue
            v.max_ctas = lc.variant_plan(kernel, E, N, F, v)["column_blocks"] * 2
            if tiles_per_cta(lc, kernel, E, N, F, v) < 4:
                continue
            got = run(lc, kernel, v, D, uu, layout)
            assert np.array_equal(got, ref), (E, N, F, re_, rc, unr, pf, st, te_mul)
            ran += 1
    assert ran >= 20, ran




EARLY_SHAPES = [(3000 + 77, 35, 3), (1500 + 33, 20, 2), (1200 + 7, 17, 3), (900 + 1, 48, 1), (2000 + 5, 84, 4)]


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_tc_early_release_many_tiles(lc, layout, prec):
    """prefetch_smem = 2: each converting thread takes its chunks of the u tile into registers
    and hands the stage back before converting (one K-block, at most three chunks a thread;
    otherwise the plain path runs), bit-exact on integer inputs with every CTA walking several
    tiles; chunks past the last node are the zeros written at set-up."""
    kernel = lc.Kernel()
    ran = 0
    for E, N, F in EARLY_SHAPES:
        D, u = synth.integer_operands(E, N, F, seed=E + 2 * N + F)
        uu = synth.to_node_major(u) if layout == "node" else u
        ref = oracle.contract(D, uu, layout)
        combos = itertools.product((1, 2), (1, 64), ((128, 2), (32, 1), (0, 0)), (0, 1))
        for k, (stages, kbw, (rows, ob), split) in enumerate(combos):
            tpr = 1 + k % 4
            if layout == "node" and (rows, ob) != (0, 0):
                continue
            v = lc.Variant(engine="tcgen05", layout=layout, precision=prec, tile_e=128, elems_per_thread=kbw,
                           split_i=split, unroll=tpr, prefetch_smem=2, stages=stages, out_buffers=ob,
                           store_rows=rows)
            if lc.variant_validate(kernel, E, N, F, v) != 0:
                continue
            v.max_ctas = 2 * lc.variant_plan(kernel, E, N, F, v)["column_blocks"]
            assert tiles_per_cta(lc, kernel, E, N, F, v) >= 4
            got = run(lc, kernel, v, D, uu, layout)
            assert np.array_equal(got, ref), (E, N, F, stages, kbw, rows, ob, split, tpr)
            ran += 1
    assert ran >= 30, ran

