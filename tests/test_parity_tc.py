"""GPU parity of the tcgen05 tensor-core paths (BF16, three-term split BF16X3) against
the CPU FP64 oracle.

Bars:
  * integer-valued inputs (exact in bf16, all partial sums exact in FP32): bit-exact;
  * random inputs: each output within an FP32-accumulation bound of the oracle's exact
    result for the same reduced-precision operands (contract_bf16 / contract_bf16x3),
    and the relative Frobenius error against the exact FP64 result at most 1e-2 (BF16)
    or 1e-6 (BF16X3);
  * sentinel elements around every output stay untouched.
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


def accum_bound(D, u, layout, prec):
    """|err| <= 2 * (products + 2) * 2^-24 * sum |terms| (FP32 accumulation of the kept products)."""
    N = D.shape[-1]
    npairs = 6 if prec == "bf16x3" else 1
    mag = oracle.contract(np.abs(D.astype(np.float64)), np.abs(u.astype(np.float64)), layout)
    return 2.0 * (npairs * N + 2) * 2.0 ** -24 * mag * 1.01 + 1e-30


SHAPES = [(1000, 35, 3), (333, 84, 4), (517, 20, 1), (64, 4, 2), (1, 5, 1), (300, 16, 3), (129, 120, 2),
          (4099, 10, 3)]


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_integer_inputs_bit_exact(lc, layout, prec):
    kernel = lc.Kernel()
    for E, N, F in SHAPES:
        D, u = synth.integer_operands(E, N, F, seed=E + N)
        uu = synth.to_node_major(u) if layout == "node" else u
        # K-block widths: 1 = widest that divides K padded to 16; 32 and 64 leave all-zero K steps
        for stages, tpr, kbw in ((1, 1, 1), (2, 2, 64), (3, 3, 1), (2, 3, 32), (1, 4, 64)):
            v = lc.Variant(engine="tcgen05", layout=layout, precision=prec, tile_e=128, elems_per_thread=kbw,
                           split_i=0, unroll=tpr, prefetch_smem=1, stages=stages)
            if lc.variant_validate(kernel, E, N, F, v) != 0:
                continue
            got = run(lc, kernel, v, D, uu, layout)
            assert np.array_equal(got, oracle.contract(D, uu, layout)), (E, N, F, stages, kbw)


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_random_inputs_within_bounds(lc, layout, prec):
    kernel = lc.Kernel()
    for si, (E, N, F) in enumerate(SHAPES):
        D, u = synth.operands(E, N, F, np.float32, seed=200 + si, scale_exp=3.0 if si % 2 else None)
        uu = synth.to_node_major(u) if layout == "node" else u
        try:
            v = lc.variant_default(kernel, E, N, F, layout, prec)
        except lc.LcError:
            # the shared-memory plan of the three-term path does not fit for large N
            assert prec == "bf16x3" and N > 96
            continue
        got = run(lc, kernel, v, D, uu, layout)
        if lc.variant_dict(v)["engine"] != "tcgen05":
            # no tensor-core default for this N: an FP32 kernel, within the FP32 FMA bound
            assert prec == "bf16x3" and N > 96
            assert np.all(np.abs(got - oracle.contract(D, uu, layout)) <= fma_bound(D, uu, layout, 2.0 ** -24))
            continue
        target = oracle.contract_bf16x3(D, uu, layout) if prec == "bf16x3" else oracle.contract_bf16(D, uu, layout)
        # the operand terms as the kernel sees them
        if prec == "bf16x3":
            Ds, us = oracle.bf16_split3(D), oracle.bf16_split3(uu)
            Dm = np.abs(Ds[0]) + np.abs(Ds[1]) + np.abs(Ds[2])
            um = np.abs(us[0]) + np.abs(us[1]) + np.abs(us[2])
        else:
            Dm, um = np.abs(oracle.bf16_round(D)), np.abs(oracle.bf16_round(uu))
        bound = accum_bound(Dm, um, layout, prec)
        assert np.all(np.abs(got - target) <= bound), (E, N, F, float(np.max(np.abs(got - target) / bound)))
        err = oracle.rel_fro_error(got, oracle.contract(D, uu, layout))
        assert err <= (1e-6 if prec == "bf16x3" else 1e-2), (E, N, F, err)
        if prec == "bf16" and E * N > 1000:
            assert err > 1e-4  # operand rounding to bf16 really happens


@pytest.mark.parametrize("layout,split", [("elem", 1), ("node", 1), ("node", 2), ("elem", 3)])
def test_column_blocks_split_operators(lc, layout, split):
    """Operators split over CTA column blocks (split_i = operators per block, last block partial)."""
    kernel = lc.Kernel()
    N = 84 if split < 3 else 20
    D, u = synth.operands(700, N, 4, np.float32, seed=5)
    uu = synth.to_node_major(u) if layout == "node" else u
    v = lc.Variant(engine="tcgen05", layout=layout, precision="bf16x3", tile_e=128, elems_per_thread=1,
                   split_i=split, unroll=2, prefetch_smem=1, stages=1)
    assert lc.variant_validate(kernel, 700, N, 4, v) == 0
    got = run(lc, kernel, v, D, uu, layout)
    assert oracle.rel_fro_error(got, oracle.contract(D, uu, layout)) <= 1e-6


def test_full_size_precision_sweep_sampled(lc):
    """E=2^20, N=84, F=4 (u scaled by 10^k): sampled rows against the oracle, both tensor paths."""
    import torch
    D, u = synth.precision_sweep()
    kernel = lc.Kernel()
    rows = np.unique(np.concatenate([np.arange(130), np.random.default_rng(1).integers(0, 1 << 20, 3000),
                                     np.arange((1 << 20) - 130, 1 << 20)]))
    ref = oracle.contract_rows(D, u, rows)
    idx = torch.from_numpy(rows).cuda()
    Dd, ud = to_dev(D), to_dev(u)
    for prec, tol in (("bf16", 1e-2), ("bf16x3", 1e-6)):
        v = lc.variant_default(kernel, 1 << 20, 84, 4, "elem", prec)
        out = lc.contract(kernel, v, Dd, ud)
        torch.cuda.synchronize()
        got = out.index_select(1, idx).cpu().numpy()
        assert oracle.rel_fro_error(got, ref) <= tol
        del out
    assert lc.device_error() == 0


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_store_groups_and_slots(lc, prec):
    """Element-major epilogue: bulk stores of 32, 64 or 128 tile rows from 1, 2 or 4 staging
    slots; ragged last tiles, and the plain-copy path (E*N not a multiple of 4)."""
    kernel = lc.Kernel()
    for E, N, F in ((1000, 35, 3), (1001, 35, 3), (333, 84, 4), (515, 20, 2)):
        D, u = synth.integer_operands(E, N, F, seed=E + 7 * N)
        ref = oracle.contract(D, u, "elem")
        ran = 0
        for rows in (32, 64, 128):
            for ob in (1, 2, 4):
                v = lc.Variant(engine="tcgen05", layout="elem", precision=prec, tile_e=128, elems_per_thread=1,
                               split_i=0, unroll=2, prefetch_smem=1, stages=1, out_buffers=ob, store_rows=rows)
                if lc.variant_validate(kernel, E, N, F, v) != 0:
                    continue
                got = run(lc, kernel, v, D, u, "elem")
                assert np.array_equal(got, ref), (E, N, F, rows, ob)
                ran += 1
        assert ran >= 3, (E, N, F, ran)


@pytest.mark.parametrize("E,N,F,layout,prec,kbw", [
    (1000, 165, 1, "node", "bf16", 16),   # 11 K-blocks handed over one by one
    (1000, 165, 2, "node", "bf16", 32),   # two column blocks, a ragged last K-block
    (777, 120, 2, "elem", "bf16", 16),    # 8 K-blocks, element-major staging
    (333, 100, 1, "node", "bf16x3", 16),  # stacked terms, 7 K-blocks
    (500, 64, 4, "elem", "bf16x3", 16),   # unstacked (MMA N = 256), products outermost over 4 K-blocks
    (500, 64, 4, "node", "bf16x3", 64),
])
def test_large_n_k_blocks_bit_exact(lc, E, N, F, layout, prec, kbw):
    """Integer-valued inputs at large N: every K-block handover, both MMA orders, exact."""
    kernel = lc.Kernel()
    D, u = synth.integer_operands(E, N, F, seed=N + F)
    uu = synth.to_node_major(u) if layout == "node" else u
    v = lc.Variant(engine="tcgen05", layout=layout, precision=prec, tile_e=128, elems_per_thread=kbw, split_i=0,
                   unroll=2, prefetch_smem=1, stages=1)
    assert lc.variant_validate(kernel, E, N, F, v) == 0
    got = run(lc, kernel, v, D, uu, layout)
    assert np.array_equal(got, oracle.contract(D, uu, layout)), (E, N, F, layout, prec, kbw)


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_full_size_fp32_three_tensor_sampled(lc, layout):
    """E=2^21, N=35, F=3 on the tensor cores (BF16X3, the default descriptor and the bench's
    launch configuration), sampled rows against the oracle: per-output FP32-accumulation
    bound against the exact split products, and the relative error within 1e-6."""
    import torch
    E, N, F = 1 << 21, 35, 3
    D, u = synth.fp32_three()
    kernel = lc.Kernel()
    uu = synth.to_node_major(u) if layout == "node" else u
    v = lc.variant_default(kernel, E, N, F, layout, "bf16x3")
    assert lc.variant_dict(v)["engine"] == "tcgen05"
    rows = np.unique(np.concatenate([np.arange(300), np.random.default_rng(3).integers(0, E, 4000),
                                     np.arange(E - 300, E)]))
    out = lc.contract(kernel, v, to_dev(D), to_dev(uu))
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    idx = torch.from_numpy(rows).cuda()
    got = out.index_select(2 if layout == "node" else 1, idx).cpu().numpy().astype(np.float64)
    if layout == "node":
        got = got.transpose(0, 2, 1)
    us = u[rows]
    target = oracle.contract_bf16x3(D, us)
    Ds, uss = oracle.bf16_split3(D), oracle.bf16_split3(us)
    bound = accum_bound(np.abs(Ds[0]) + np.abs(Ds[1]) + np.abs(Ds[2]), np.abs(uss[0]) + np.abs(uss[1]) + np.abs(uss[2]),
                        "elem", "bf16x3")
    assert np.all(np.abs(got - target) <= bound)
    assert oracle.rel_fro_error(got, oracle.contract_rows(D, u, rows)) <= 1e-6


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("E,N,F", [(1000, 35, 3), (517, 100, 2), (300, 120, 3), (129, 128, 1), (777, 56, 4)])
def test_bf16x3_a_in_tensor_memory(lc, layout, E, N, F):
    """Three-term split with the A terms in tensor memory (a_operand = 2; the planner's plan
    for N above about 100): integer inputs bit-exact, random inputs within the FP32
    accumulation bound of the split products and 1e-6 of the exact result."""
    kernel = lc.Kernel()
    for kbw, tpr in ((1, 4), (64, 2), (32, 3)):
        v = lc.Variant(engine="tcgen05", layout=layout, precision="bf16x3", tile_e=128, elems_per_thread=kbw,
                       split_i=0, unroll=tpr, prefetch_smem=1, stages=1, a_operand=2)
        if lc.variant_validate(kernel, E, N, F, v) != 0:
            continue
        assert lc.variant_plan(kernel, E, N, F, v)["a_in_tmem"] == 1
        D, u = synth.integer_operands(E, N, F, seed=E + N + kbw)
        uu = synth.to_node_major(u) if layout == "node" else u
        got = run(lc, kernel, v, D, uu, layout)
        assert np.array_equal(got, oracle.contract(D, uu, layout)), (E, N, F, kbw, tpr)
        D, u = synth.operands(E, N, F, np.float32, seed=E + 3 * N)
        uu = synth.to_node_major(u) if layout == "node" else u
        got = run(lc, kernel, v, D, uu, layout)
        Ds, us = oracle.bf16_split3(D), oracle.bf16_split3(uu)
        bound = accum_bound(np.abs(Ds[0]) + np.abs(Ds[1]) + np.abs(Ds[2]), np.abs(us[0]) + np.abs(us[1]) + np.abs(us[2]),
                            layout, "bf16x3")
        assert np.all(np.abs(got - oracle.contract_bf16x3(D, uu, layout)) <= bound), (E, N, F, kbw)
        assert oracle.rel_fro_error(got, oracle.contract(D, uu, layout)) <= 1e-6
    if N >= 120:
        # the default from N of about 100 (no shared-memory plan): A in tensor memory, one
        # operator per column block, 32-row stores; checked the same way
        v = lc.variant_default(kernel, E, N, F, layout, "bf16x3")
        assert lc.variant_dict(v)["engine"] == "tcgen05" and lc.variant_plan(kernel, E, N, F, v)["a_in_tmem"] == 1
        D, u = synth.integer_operands(E, N, F, seed=E + N + 7)
        uu = synth.to_node_major(u) if layout == "node" else u
        assert np.array_equal(run(lc, kernel, v, D, uu, layout), oracle.contract(D, uu, layout)), (E, N, F)
        D, u = synth.operands(E, N, F, np.float32, seed=E + 5 * N, scale_exp=3.0)
        uu = synth.to_node_major(u) if layout == "node" else u
        got = run(lc, kernel, v, D, uu, layout)
        Ds, us = oracle.bf16_split3(D), oracle.bf16_split3(uu)
        bound = accum_bound(np.abs(Ds[0]) + np.abs(Ds[1]) + np.abs(Ds[2]), np.abs(us[0]) + np.abs(us[1]) + np.abs(us[2]),
                            layout, "bf16x3")
        assert np.all(np.abs(got - oracle.contract_bf16x3(D, uu, layout)) <= bound), (E, N, F)
        assert oracle.rel_fro_error(got, oracle.contract(D, uu, layout)) <= 1e-6



@pytest.mark.parametrize("layout", ["elem", "node"])
def test_three_term_early_release_random(lc, layout):
    """BF16X3 with early release of the stage (prefetch_smem = 2): random inputs within the
    per-output bound of the six-product target and 1e-6 of the exact result."""
    kernel = lc.Kernel()
    for si, (E, N, F) in enumerate(((1000, 35, 3), (517, 20, 1), (300, 17, 2), (4099, 10, 3))):
        D, u = synth.operands(E, N, F, np.float32, seed=800 + si, scale_exp=3.0 if si % 2 else None)
        uu = synth.to_node_major(u) if layout == "node" else u
        v = lc.Variant(engine="tcgen05", layout=layout, precision="bf16x3", tile_e=128, elems_per_thread=64,
                       split_i=0, unroll=4, prefetch_smem=2, stages=1)
        assert lc.variant_validate(kernel, E, N, F, v) == 0
        got = run(lc, kernel, v, D, uu, layout)
        Ds, us = oracle.bf16_split3(D), oracle.bf16_split3(uu)
        bound = accum_bound(np.abs(Ds[0]) + np.abs(Ds[1]) + np.abs(Ds[2]),
                            np.abs(us[0]) + np.abs(us[1]) + np.abs(us[2]), layout, "bf16x3")
        target = oracle.contract_bf16x3(D, uu, layout)
        assert np.all(np.abs(got - target) <= bound), (E, N, F)
        assert oracle.rel_fro_error(got, oracle.contract(D, uu, layout)) <= 1e-6, (E, N, F)

