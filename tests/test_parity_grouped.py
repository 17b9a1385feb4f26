"""GPU parity of the grouped persistent kernel (several problems of different N in one
launch, replayed from a CUDA graph) against the CPU FP64 oracle, group by group."""

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


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("graph", [True, False])
def test_grouped_matches_oracle(lc, layout, graph):
    import torch
    kernel = lc.Kernel()
    data = synth.grouped_operands(SIZES, F=3, seed=1)
    groups, host = [], []
    for (N, E), (D, u) in zip(SIZES, data):
        uu = synth.to_node_major(u) if layout == "node" else u
        out = torch.full((3, N, E) if layout == "node" else (3, E, N), float("nan"), device="cuda")
        groups.append((to_dev(D), to_dev(uu), out))
        host.append((D, uu))
    stream = torch.cuda.Stream()
    for re_, rc, unr, pf, st in [(8, 4, 4, 1, 2), (4, 8, 1, 0, 1), (8, 8, 1, 1, 1), (4, 8, 1, 1, 2)]:
        v = lc.Variant(layout=layout, elems_per_thread=re_, split_i=rc, unroll=unr, prefetch_smem=pf, stages=st,
                       ctas_per_sm=2)
        plan = lc.GroupedPlan(kernel, v, groups, use_graph=graph, stream=stream)
        for rep in range(2):  # replay twice: the result must not depend on the previous run
            for _, _, out in groups:
                out.fill_(float("nan"))
            torch.cuda.synchronize()  # the fills run on torch's stream, the plan on `stream`
            plan.run(stream)
            stream.synchronize()
            assert lc.device_error() == 0
            for (D, uu), (_, _, out) in zip(host, groups):
                got = out.cpu().numpy().astype(np.float64)
                ref = oracle.contract(D, uu, layout)
                assert np.all(np.abs(got - ref) <= fma_bound(D, uu, layout, 2.0 ** -24)), (D.shape, layout)
        info = plan.info()
        assert info["segments"] >= len([n for n, _ in SIZES if n < 96]) - 1
        # N >= 96: one K-split launch each (D^T streamed in chunks), the rest in the persistent launch
        for k, (N, E) in enumerate(SIZES):
            assert lc.variant_dict(plan.group_variant(k))["engine"] == ("ksplit" if N >= 96 else "simt"), (N, E)
        del plan


def test_grouped_integer_exact(lc):
    import torch
    kernel = lc.Kernel()
    groups, host = [], []
    for k, (N, E) in enumerate(SIZES):
        D, u = synth.integer_operands(E, N, 3, seed=k)
        groups.append((to_dev(D), to_dev(u), torch.empty((3, E, N), device="cuda")))
        host.append((D, u))
    v = lc.Variant(elems_per_thread=8, split_i=4, unroll=4, prefetch_smem=1, stages=2, ctas_per_sm=1)
    plan = lc.GroupedPlan(kernel, v, groups, use_graph=False)
    plan.run()
    torch.cuda.synchronize()
    for (D, u), (_, _, out) in zip(host, groups):
        assert np.array_equal(out.cpu().numpy().astype(np.float64), oracle.contract(D, u))


def _sample_rows(E, rng, k=400):
    if E <= 2 * 130 + k:
        return np.arange(E)
    return np.unique(np.concatenate([np.arange(130), rng.integers(0, E, k), np.arange(E - 130, E)]))


def _check_groups_sampled(lc, kernel, v, sizes, data, layout, graph, reps=2):
    """Run the grouped plan on (D, u) per group; compare sampled element rows of every group
    with the oracle within the FP32 FMA bound, twice in a row (replay)."""
    import torch
    groups = []
    for (N, E), (D, u) in zip(sizes, data):
        uu = synth.to_node_major(u) if layout == "node" else u
        out = torch.empty((3, N, E) if layout == "node" else (3, E, N), device="cuda")
        groups.append((to_dev(D), to_dev(uu), out))
    stream = torch.cuda.Stream()
    plan = lc.GroupedPlan(kernel, v, groups, use_graph=graph, stream=stream)
    rng = np.random.default_rng(5)
    for rep in range(reps):
        for _, _, out in groups:
            out.fill_(float("nan"))
        torch.cuda.synchronize()  # the fills run on torch's stream, the plan on `stream`
        plan.run(stream)
        stream.synchronize()
        assert lc.device_error() == 0
        for (N, E), (D, u), (_, _, out) in zip(sizes, data, groups):
            rows = _sample_rows(E, rng)
            idx = torch.from_numpy(rows).cuda()
            got = out.index_select(2 if layout == "node" else 1, idx).cpu().numpy().astype(np.float64)
            if layout == "node":
                got = got.transpose(0, 2, 1)
            ref = oracle.contract_rows(D, u, rows)
            bound = fma_bound(D, u[rows], "elem", 2.0 ** -24)
            assert np.all(np.abs(got - ref) <= bound), (N, E, rep)
    info = plan.info()
    del plan, groups
    torch.cuda.empty_cache()
    return info


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_grouped_strided_ctas_large_groups(lc, layout):
    """Two groups of about 2^18 elements beside tiny ones: the planner hands each large
    (group, column block) unit to several CTAs that stride over its tiles."""
    kernel = lc.Kernel()
    sizes = [(4, 700), (84, 1 << 18), (10, 33), (35, (1 << 18) + 77), (165, 129)]
    data = synth.grouped_operands(sizes, F=3, seed=2)
    v = lc.Variant(layout=layout, elems_per_thread=8, split_i=8, unroll=1, prefetch_smem=1, stages=1, ctas_per_sm=2)
    info = _check_groups_sampled(lc, kernel, v, sizes, data, layout, graph=True)
    assert info["segments"] > info["grid"] // 2  # many CTAs hold a strided share of a unit


@pytest.mark.parametrize("layout", ["elem", "node"])
def test_grouped_full_size_sampled(lc, layout):
    """The uneven-batching workload at full size: 8 groups, N in {4, ..., 165}, E_g from
    the seeded log-uniform draw (3,554,987 elements in all), F = 3, one graph launch;
    sampled rows of every group against the oracle."""
    kernel = lc.Kernel()
    sizes = synth.grouped_sizes(0)
    assert [n for n, _ in sizes] == [4, 10, 20, 35, 56, 84, 120, 165]
    assert sum(e for _, e in sizes) == 3554987
    data = synth.grouped_operands(sizes, F=3, seed=0)
    v = lc.Variant(layout=layout, elems_per_thread=8, split_i=8, unroll=1, prefetch_smem=1, stages=1, ctas_per_sm=2)
    _check_groups_sampled(lc, kernel, v, sizes, data, layout, graph=True, reps=1)
