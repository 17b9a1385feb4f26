"""GPU parity of the SIMT and small-N warp kernels against the CPU FP64 oracle.

Every descriptor must reproduce the oracle (the unordered semantics of
Section 2.3: transformations preserve the result). Bars:
  * integer-valued inputs: bit-exact (all sums exact in FP32/FP64);
  * random inputs: each output within the N-term FMA error bound
    (N + 2) * u * sum_j |D_ij| |u_j| (u = 2^-24 for FP32, 2^-53 for FP64), and the
    relative Frobenius error at most 1e-6 (FP32) or 1e-13 (FP64);
  * sentinel elements around every output stay untouched (tail guards of Eq. 1).
"""

import itertools

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


def run(lc, kernel, v, D, u, layout):
    import torch
    F, N, _ = D.shape
    E = u.shape[1] if layout == "node" else u.shape[0]
    shape = (F, N, E) if layout == "node" else (F, E, N)
    co = CanaryOut(shape, D.dtype)
    lc.contract(kernel, v, to_dev(D), to_dev(u), co.out)
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    assert co.intact(), "write outside the output"
    return co.out.cpu().numpy()


def check(got, D, u, layout, fp64):
    ref = oracle.contract(D, u, layout)
    unit = 2.0 ** -53 if fp64 else 2.0 ** -24
    bound = fma_bound(D, u, layout, unit)
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= bound), f"max excess {np.max(err / bound)}"
    tol = 1e-13 if fp64 else 1e-6
    assert oracle.rel_fro_error(got, ref) <= tol


SHAPES = [(1000, 35, 3), (517, 20, 1), (333, 7, 2), (64, 84, 4), (1, 5, 1), (129, 165, 3), (4097, 12, 2),
          (300, 250, 2), (777, 84, 4)]


def simt_variants(fp64):
    V = 2 if fp64 else 4
    for re_, rc, unr, (pf, st), ctas in itertools.product((V, 2 * V), (V, 2 * V), (1, 4),
                                                         ((0, 1), (1, 1), (1, 2)), (0, 2)):
        yield dict(engine="simt", elems_per_thread=re_, split_i=rc, unroll=unr, prefetch_smem=pf, stages=st,
                   tile_e=re_ * 16, ctas_per_sm=ctas)
    # other tile shapes: narrow tiles (wide warps along columns) and wide tiles
    for te, re_ in ((4 * V, V), (8 * V, 2 * V), (64 * V, V)):
        for pf, st in ((0, 1), (1, 2)):
            yield dict(engine="simt", elems_per_thread=re_, split_i=2 * V, unroll=2, prefetch_smem=pf, stages=st,
                       tile_e=te, ctas_per_sm=1)


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_simt_descriptor_grid_random(lc, layout, prec):
    fp64 = prec == "fp64"
    dt = np.float64 if fp64 else np.float32
    kernel = lc.Kernel()
    for si, (E, N, F) in enumerate(SHAPES):
        D, u = synth.operands(E, N, F, dt, seed=100 + si)
        uu = synth.to_node_major(u) if layout == "node" else u
        for vd in simt_variants(fp64):
            v = lc.Variant(layout=layout, precision=prec, **vd)
            if lc.variant_validate(kernel, E, N, F, v) != 0:
                continue
            got = run(lc, kernel, v, D, uu, layout)
            check(got, D, uu, layout, fp64)


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_simt_unroll_all_factors(lc, layout):
    kernel = lc.Kernel()
    D, u = synth.operands(777, 35, 3, np.float32, seed=7)
    uu = synth.to_node_major(u) if layout == "node" else u
    for unr in (1, 2, 4, 8):
        v = lc.Variant(layout=layout, unroll=unr, tile_e=64)
        check(run(lc, kernel, v, D, uu, layout), D, uu, layout, False)


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_integer_inputs_bit_exact(lc, layout, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    kernel = lc.Kernel()
    for E, N, F in [(1000, 35, 3), (300, 165, 2), (77, 9, 4)]:
        D, u = synth.integer_operands(E, N, F, dt, seed=E)
        uu = synth.to_node_major(u) if layout == "node" else u
        ref = oracle.contract(D, uu, layout)
        for vd in list(simt_variants(prec == "fp64"))[:8]:
            v = lc.Variant(layout=layout, precision=prec, **vd)
            if lc.variant_validate(kernel, E, N, F, v) != 0:
                continue
            got = run(lc, kernel, v, D, uu, layout)
            assert np.array_equal(got.astype(np.float64), ref)


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_warp_engine_small_n(lc, layout):
    kernel = lc.Kernel()
    for E, N, F in [(1000, 4, 3), (513, 10, 3), (333, 20, 1), (100, 32, 4), (5, 3, 2)]:
        D, u = synth.operands(E, N, F, np.float32, seed=N)
        uu = synth.to_node_major(u) if layout == "node" else u
        per = 32 // N
        for warps in (1, 4, 8):
            v = lc.Variant(engine="warp", layout=layout, tile_e=per * warps, elems_per_thread=1, split_i=1,
                           unroll=1, prefetch_smem=0)
            assert lc.variant_validate(kernel, E, N, F, v) == 0
            check(run(lc, kernel, v, D, uu, layout), D, uu, layout, False)
        Di, ui = synth.integer_operands(E, N, F, seed=3)
        uui = synth.to_node_major(ui) if layout == "node" else ui
        got = run(lc, kernel, v, Di, uui, layout)
        assert np.array_equal(got.astype(np.float64), oracle.contract(Di, uui, layout))


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_warp_engine_fp64_single_operator(lc, layout):
    """FP64 warp engine above 16 nodes (one operator's row in registers): N = 20 (the FP64
    workload's size, one element per warp, 12 lanes idle) and N = 32."""
    kernel = lc.Kernel("{ [e,i,j]: 0<=e<E and 0<=i,j<N }", "out[e,i] = sum(j, D[i,j]*u[e,j])")
    for E, N in [(4096, 20), (777, 20), (130, 32)]:
        D, u = synth.operands(E, N, 1, np.float64, seed=N + E)
        uu = synth.to_node_major(u) if layout == "node" else u
        for warps in (1, 8):
            v = lc.Variant(engine="warp", layout=layout, precision="fp64", tile_e=(32 // N) * warps,
                           elems_per_thread=1, split_i=1, unroll=1, prefetch_smem=0)
            assert lc.variant_validate(kernel, E, N, 1, v) == 0
            check(run(lc, kernel, v, D, uu, layout), D, uu, layout, True)
    # two operators above 16 nodes do not fit the registers: rejected before launch
    v = lc.Variant(engine="warp", layout=layout, precision="fp64", tile_e=8, elems_per_thread=1, split_i=1,
                   unroll=1, prefetch_smem=0)
    assert lc.variant_validate(lc.Kernel(), 100, 20, 2, v) != 0


def test_tail_free_under_assumption(lc):
    kernel = lc.Kernel(assumptions="E mod 128 = 0")
    D, u = synth.operands(1024, 35, 3, np.float32, seed=9)
    v = lc.Variant(tile_e=64, tail_free=1)
    check(run(lc, kernel, v, D, u, "elem"), D, u, "elem", False)
    # the same descriptor without the assumption is rejected before launch
    assert lc.variant_validate(lc.Kernel(), 1024, 35, 3, v) == 3
    # a problem size that breaks the assumption is rejected
    assert lc.variant_validate(kernel, 1000, 35, 3, v) == 4


def test_empty_and_single_element(lc):
    import torch
    kernel = lc.Kernel()
    D, u = synth.operands(1, 35, 3, np.float32, seed=1)
    v = lc.Variant()
    check(run(lc, kernel, v, D, u, "elem"), D, u, "elem", False)
    out = torch.empty((3, 0, 35), device="cuda")
    lc.contract(kernel, v, to_dev(D), torch.empty((0, 35), device="cuda"), out)


def test_fp64_single_operator_config(lc):
    """E=4096, N=20, F=1, FP64 in the single-operator form of the instruction."""
    kernel = lc.Kernel("{ [e,i,j]: 0<=e<E and 0<=i,j<N }", "out[e,i] = sum(j, D[i,j]*u[e,j])")
    D, u = synth.fp64_single()
    for layout in ("elem", "node"):
        uu = synth.to_node_major(u) if layout == "node" else u
        v = lc.variant_default(kernel, 4096, 20, 1, layout, "fp64")
        check(run(lc, kernel, v, D, uu, layout), D, uu, layout, True)


def test_full_size_fp32_three_sampled(lc):
    """E=2^21, N=35, F=3 at full size: sampled elements against the oracle, both layouts."""
    import torch
    D, u = synth.fp32_three()
    kernel = lc.Kernel()
    rows = np.unique(np.concatenate([np.arange(64), np.random.default_rng(0).integers(0, 1 << 21, 4000),
                                     np.arange((1 << 21) - 64, 1 << 21)]))
    ref = oracle.contract_rows(D, u, rows)
    bound = fma_bound(D, u[rows], "elem", 2.0 ** -24)
    for layout in ("elem", "node"):
        uu = synth.to_node_major(u) if layout == "node" else u
        v = lc.variant_default(kernel, 1 << 21, 35, 3, layout, "fp32")
        out = lc.contract(kernel, v, to_dev(D), to_dev(uu))
        torch.cuda.synchronize()
        idx = torch.from_numpy(rows).cuda()
        got = out.index_select(2 if layout == "node" else 1, idx).cpu().numpy()
        if layout == "node":
            got = got.transpose(0, 2, 1)
        assert np.all(np.abs(got - ref) <= bound)
        del out


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_column_blocks_and_row_splits(lc, layout):
    """Operators spread over CTA column blocks (F=8) and, at N=256, one operator's rows
    split over several blocks because its D^T does not fit shared memory."""
    kernel = lc.Kernel()
    for E, N, F in [(1000, 120, 8), (513, 256, 3)]:
        D, u = synth.operands(E, N, F, np.float32, seed=N)
        uu = synth.to_node_major(u) if layout == "node" else u
        # the SIMT engine (the default for this N is the K-split one): the largest tile that fits
        re_, tile = (8, 128) if layout == "elem" else (4, 64)
        while True:
            v = lc.Variant(layout=layout, elems_per_thread=re_, split_i=8, tile_e=tile, unroll=1, prefetch_smem=1,
                           stages=1, ctas_per_sm=2)
            if lc.variant_validate(kernel, E, N, F, v) == 0:
                break
            assert tile > re_
            tile //= 2
        check(run(lc, kernel, v, D, uu, layout), D, uu, layout, False)
        Di, ui = synth.integer_operands(E, N, F, seed=1)
        uui = synth.to_node_major(ui) if layout == "node" else ui
        got = run(lc, kernel, v, Di, uui, layout)
        assert np.array_equal(got.astype(np.float64), oracle.contract(Di, uui, layout))
