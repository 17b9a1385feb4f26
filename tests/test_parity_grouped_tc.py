"""GPU parity of the grouped launch on the tensor cores (BF16 and BF16X3 variants): one
tcgen05 launch over every group with a tensor-core plan, each CTA running one (group,
column block) unit of its group's plan, then the FP32 SIMT grouped launch for the groups
without one (N = 165), against the CPU FP64 oracle group by group.

Bars (as for the single-problem tensor-core path):
  * integer-valued inputs: bit-exact in every group;
  * random inputs: every output of a tensor-core group within the FP32-accumulation bound
    of the oracle's exact result for the split operands, every output of a SIMT group
    within the FP32 FMA bound of the exact result.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import fma_bound, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


SIZES = [(4, 3000), (10, 777), (20, 1), (35, 4096), (56, 513), (84, 2000), (120, 300), (165, 257)]


def tc_variant(lc, layout, prec, kbw=64, tpr=4, stages=1, pf=1):
    return lc.Variant(engine="tcgen05", layout=layout, precision=prec, tile_e=128, elems_per_thread=kbw,
                      split_i=0, unroll=tpr, prefetch_smem=pf, stages=stages,
                      store_rows=0 if layout == "node" else 128)


def accum_bound(D, u, layout, prec):
    """|err| <= 2 * (products + 2) * 2^-24 * sum |terms| (FP32 accumulation of the kept products)."""
    N = D.shape[-1]
    npairs = 6 if prec == "bf16x3" else 1
    mag = oracle.contract(np.abs(D.astype(np.float64)), np.abs(u.astype(np.float64)), layout)
    return 2.0 * (npairs * N + 2) * 2.0 ** -24 * mag * 1.01 + 1e-30


def on_tensor_cores(lc, plan, k):
    v = plan.group_variant(k)
    return v.engine == lc.ENGINE["tcgen05"]


def make_groups(sizes, data, layout):
    import torch
    groups, host = [], []
    for (N, E), (D, u) in zip(sizes, data):
        uu = synth.to_node_major(u) if layout == "node" else u
        out = torch.full((3, N, E) if layout == "node" else (3, E, N), float("nan"), device="cuda")
        groups.append((to_dev(D), to_dev(uu), out))
        host.append((D, uu))
    return groups, host


def run_plan(lc, plan, groups, stream):
    import torch
    for _, _, out in groups:
        out.fill_(float("nan"))
    torch.cuda.synchronize()  # the fills run on torch's stream, the plan on `stream`
    plan.run(stream)
    stream.synchronize()
    assert lc.device_error() == 0


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_grouped_tc_integer_exact(lc, layout, prec):
    import torch
    kernel = lc.Kernel()
    data = [synth.integer_operands(E, N, 3, seed=k) for k, (N, E) in enumerate(SIZES)]
    groups, host = make_groups(SIZES, data, layout)
    stream = torch.cuda.Stream()
    # (the last two release the u stage early: prefetch_smem = 2)
    for kbw, tpr, stages, graph, pf in ((64, 4, 1, True, 1), (1, 2, 2, False, 1), (1, 3, 1, True, 1),
                                        (64, 3, 1, True, 2), (1, 2, 2, False, 2)):
        v = tc_variant(lc, layout, prec, kbw, tpr, stages, pf)
        plan = lc.GroupedPlan(kernel, v, groups, use_graph=graph, stream=stream)
        on_tc = [on_tensor_cores(lc, plan, k) for k in range(len(SIZES))]
        assert all(on_tc[:6]), (prec, kbw, on_tc)  # every group up to N = 84 runs on the tensor cores
        if prec == "bf16x3":
            assert not on_tc[7]  # N = 165: no three-term tensor-core plan, FP32 SIMT
        for rep in range(2):  # the result must not depend on the previous run
            run_plan(lc, plan, groups, stream)
            for (D, uu), (_, _, out) in zip(host, groups):
                assert np.array_equal(out.cpu().numpy().astype(np.float64), oracle.contract(D, uu, layout)), \
                    (D.shape, layout, prec, kbw)
        del plan


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_grouped_tc_random_within_bounds(lc, layout, prec):
    import torch
    kernel = lc.Kernel()
    data = synth.grouped_operands(SIZES, F=3, seed=7)
    groups, host = make_groups(SIZES, data, layout)
    stream = torch.cuda.Stream()
    for pf in (1, 2):
        _check_random(lc, kernel, tc_variant(lc, layout, prec, pf=pf), groups, host, stream, layout, prec)


def _check_random(lc, kernel, v, groups, host, stream, layout, prec):
    plan = lc.GroupedPlan(kernel, v, groups, use_graph=True, stream=stream)
    run_plan(lc, plan, groups, stream)
    for k, ((N, E), (D, uu), (_, _, out)) in enumerate(zip(SIZES, host, groups)):
        got = out.cpu().numpy().astype(np.float64)
        if on_tensor_cores(lc, plan, k):
            if prec == "bf16x3":
                target = oracle.contract_bf16x3(D, uu, layout)
                Ds, us = oracle.bf16_split3(D), oracle.bf16_split3(uu)
                Dm = np.abs(Ds[0]) + np.abs(Ds[1]) + np.abs(Ds[2])
                um = np.abs(us[0]) + np.abs(us[1]) + np.abs(us[2])
            else:
                target = oracle.contract_bf16(D, uu, layout)
                Dm, um = np.abs(oracle.bf16_round(D)), np.abs(oracle.bf16_round(uu))
            bound = accum_bound(Dm, um, layout, prec)
        else:
            assert N > 84
            target = oracle.contract(D, uu, layout)
            bound = fma_bound(D, uu, layout, 2.0 ** -24)
        assert np.all(np.abs(got - target) <= bound), (N, E, layout, prec)


def _sample_rows(E, rng, k=400):
    if E <= 2 * 130 + k:
        return np.arange(E)
    return np.unique(np.concatenate([np.arange(130), rng.integers(0, E, k), np.arange(E - 130, E)]))


def _check_sampled(lc, kernel, v, sizes, data, layout):
    import torch
    groups, _ = make_groups(sizes, data, layout)
    stream = torch.cuda.Stream()
    plan = lc.GroupedPlan(kernel, v, groups, use_graph=True, stream=stream)
    rng = np.random.default_rng(11)
    run_plan(lc, plan, groups, stream)
    for k, ((N, E), (D, u), (_, _, out)) in enumerate(zip(sizes, data, groups)):
        rows = _sample_rows(E, rng)
        idx = torch.from_numpy(rows).cuda()
        got = out.index_select(2 if layout == "node" else 1, idx).cpu().numpy().astype(np.float64)
        if layout == "node":
            got = got.transpose(0, 2, 1)
        us = u[rows]
        if on_tensor_cores(lc, plan, k):
            target = oracle.contract_bf16x3(D, us)
            Ds, uss = oracle.bf16_split3(D), oracle.bf16_split3(us)
            bound = accum_bound(np.abs(Ds[0]) + np.abs(Ds[1]) + np.abs(Ds[2]),
                                np.abs(uss[0]) + np.abs(uss[1]) + np.abs(uss[2]), "elem", "bf16x3")
        else:
            target = oracle.contract_rows(D, u, rows)
            bound = fma_bound(D, us, "elem", 2.0 ** -24)
        assert np.all(np.abs(got - target) <= bound), (N, E)
    info = plan.info()
    del plan, groups
    torch.cuda.empty_cache()
    return info


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_grouped_tc_strided_large_groups(lc, layout):
    """Two groups of about 2^18 elements beside tiny ones: the large units get many CTAs
    that stride over their tiles, the tiny ones one CTA each."""
    kernel = lc.Kernel()
    sizes = [(4, 700), (84, 1 << 18), (10, 33), (35, (1 << 18) + 77), (165, 129)]
    data = synth.grouped_operands(sizes, F=3, seed=2)
    info = _check_sampled(lc, kernel, tc_variant(lc, layout, "bf16x3"), sizes, data, layout)
    assert info["segments"] >= 100  # one segment per tensor-core CTA: the SMs are shared out


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_grouped_tc_full_size_sampled(lc, layout):
    """The uneven-batching workload at full size (8 groups, N in {4, ..., 165}, 3,554,987
    elements, F = 3) in the bench's launch configuration: BF16X3 grouped tensor-core launch
    for N <= 84, a tensor-core launch with the A terms in tensor memory for N = 120, a K-split
    launch for N = 165, one graph; sampled rows of every group."""
    kernel = lc.Kernel()
    sizes = synth.grouped_sizes(0)
    data = synth.grouped_operands(sizes, F=3, seed=0)
    _check_sampled(lc, kernel, tc_variant(lc, layout, "bf16x3"), sizes, data, layout)
