"""GPU parity of the volume derivative with per-element geometric factors,
out[d,e,i] = sum_f r[e,d,f] * sum_j D[f,i,j] u[e,j] (the dG FEM volume workload of Table 1
with the chain rule in the kernel), against the CPU FP64 oracle (oracle.contract_geo).

Bars: integer-valued inputs (exact in bf16, every sum exact in FP32) bit-exact, both
layouts, F = 2 and 3, ragged element counts, every CTA walking many tiles; random inputs
within a per-output bound and within 1e-6 (BF16X3) or 1e-2 (BF16) relative Frobenius error;
sentinels around the output untouched; sampled rows at full size (E = 2^21, N = 35, F = 3).
"""

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


def factors(E, F, layout, seed, integer=False):
    rng = np.random.default_rng(seed)
    r = rng.integers(-3, 4, size=(E, F, F)).astype(np.float32) if integer else \
        rng.uniform(-2, 2, size=(E, F, F)).astype(np.float32)
    return np.ascontiguousarray(r.transpose(1, 2, 0)) if layout == "node" else r


def run(lc, kernel, v, D, u, r, layout):
    import torch
    F, N, _ = D.shape
    E = u.shape[1] if layout == "node" else u.shape[0]
    co = CanaryOut((F, N, E) if layout == "node" else (F, E, N), np.float32)
    lc.contract_geo(kernel, v, to_dev(D), to_dev(u), to_dev(r), co.out)
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    assert co.intact(), "write outside the output"
    return co.out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_integer_inputs_bit_exact(lc, layout, prec):
    kernel = lc.Kernel(lc.GEO_DOMAIN, lc.GEO_INSTRUCTION)
    ran = 0
    for E, N, F in ((3000 + 77, 35, 3), (2000 + 5, 20, 2), (1500 + 1, 48, 3), (1200 + 3, 64, 2), (700, 4, 3),
                    (1, 10, 2)):
        D, u = synth.integer_operands(E, N, F, seed=E + N)
        uu = synth.to_node_major(u) if layout == "node" else u
        r = factors(E, F, layout, seed=N, integer=True)
        ref = oracle.contract_geo(D, uu, r, layout)
        for stages, tpr, kbw, aop in ((2, 3, 64, 0), (1, 4, 1, 1), (3, 2, 64, 2), (2, 1, 16, 0)):
            v = lc.Variant(engine="tcgen05", layout=layout, precision=prec, tile_e=128, elems_per_thread=kbw,
                           split_i=0, unroll=tpr, prefetch_smem=1, stages=stages, a_operand=aop)
            if lc.variant_validate(kernel, E, N, F, v) != 0:
                continue
            p = lc.variant_plan(kernel, E, N, F, v)
            v.max_ctas = 2 if p["tiles"] >= 8 else 0  # two CTAs walk every tile
            got = run(lc, kernel, v, D, uu, r, layout)
            assert np.array_equal(got, ref), (E, N, F, stages, tpr, kbw, aop)
            ran += 1
    assert ran >= 10, ran


@pytest.mark.parametrize("layout", ["elem", "node"])
@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_random_inputs_within_bounds(lc, layout, prec):
    kernel = lc.Kernel(lc.GEO_DOMAIN, lc.GEO_INSTRUCTION)
    for si, (E, N, F) in enumerate(((5000 + 3, 35, 3), (1000, 48, 3), (777, 64, 2))):
        D, u = synth.operands(E, N, F, np.float32, seed=300 + si, scale_exp=2.0 if si else None)
        uu = synth.to_node_major(u) if layout == "node" else u
        r = factors(E, F, layout, seed=si)
        v = lc.variant_default(kernel, E, N, F, layout, prec)
        got = run(lc, kernel, v, D, uu, r, layout)
        ref = oracle.contract_geo(D, uu, r, layout)
        # per output: each partial within the FP32-accumulation bound of its kept products,
        # weighted by |r|, plus F FP32 roundings of the weighted sum
        rabs = np.abs(r.astype(np.float64))
        part_mag = oracle.contract(np.abs(D.astype(np.float64)), np.abs(uu.astype(np.float64)), layout)
        npairs = 6 if prec == "bf16x3" else 1
        part_bound = 2.0 * (npairs * N + 2) * 2.0 ** -24 * part_mag * 1.01
        if prec == "bf16":
            part_bound = part_bound + 2 * 2.0 ** -8 * part_mag  # operands rounded to bf16
        sum_mag = oracle.contract_geo(np.abs(D.astype(np.float64)), np.abs(uu.astype(np.float64)), rabs, layout)
        if layout == "node":
            wb = np.einsum("dfe,fie->die", rabs, part_bound)
        else:
            wb = np.einsum("edf,fei->dei", rabs, part_bound)
        bound = wb + (F + 2) * 2.0 ** -24 * sum_mag + 1e-30
        assert np.all(np.abs(got - ref) <= bound), (E, N, F, float(np.max(np.abs(got - ref) / bound)))
        err = oracle.rel_fro_error(got, ref)
        assert err <= (1e-6 if prec == "bf16x3" else 1e-2), (E, N, F, err)


def test_full_size_sampled(lc):
    """E = 2^21, N = 35, F = 3 (the bench's launch configuration), sampled rows."""
    import torch
    E, N, F = 1 << 21, 35, 3
    D, u = synth.fp32_three()
    r = factors(E, F, "elem", seed=9)
    kernel = lc.Kernel(lc.GEO_DOMAIN, lc.GEO_INSTRUCTION)
    v = lc.variant_default(kernel, E, N, F, "elem", "bf16x3")
    out = lc.contract_geo(kernel, v, to_dev(D), to_dev(u), to_dev(r))
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    rows = np.unique(np.concatenate([np.arange(200), np.random.default_rng(4).integers(0, E, 3000),
                                     np.arange(E - 200, E)]))
    got = out.index_select(1, torch.from_numpy(rows).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.contract_geo_rows(D, u, r, rows)
    assert oracle.rel_fro_error(got, ref) <= 1e-6

