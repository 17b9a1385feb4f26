"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
symbol include/lc.h declares, parses the loop-domain / instruction / assumption
texts of Section 2.1, prints kernels, and validates descriptors before any launch.
"""

import ctypes
import os
import re

import pytest

from paper_1405_7470_gb300 import lc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1405_7470_gb300 import build
    build()
    return lc.load()


def header_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(lc_\w+)\s*\(", text, flags=re.M))
    return names


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert "lc_contract" in names and "lc_kernel_create" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    # and the binding knows every one of them
    assert names <= set(lc.SIGNATURES), names - set(lc.SIGNATURES)


def _create(lib, dom, insn, asm=None):
    h = ctypes.c_void_p()
    st = lib.lc_kernel_create(dom.encode(), insn.encode(), asm.encode() if asm else None, ctypes.byref(h))
    if st == 0:
        lib.lc_kernel_destroy(h)
    return st


@pytest.mark.parametrize("dom,insn,asm", [
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }", "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])", None),
    ("[F,E,N] -> {[f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i<N and 0<=j<N}", "out[f,e,i]=sum(j,u[e,j]*D[f,i,j])", None),
    ("{ [e,i,j,f]: e>=0 and E>e and 0<=i,j<=N-1 and 0<=f<F }", "res[f,e,i] = sum(j, A[f,i,j]*x[e,j])",
     "E mod 128 = 0 and N >= 4"),
    ("{ [e,i,j]: 0<=e<E and 0<=i,j<N }", "out[e,i] = sum(j, D[i,j]*u[e,j])", "N > 0"),
    ("{ [k,a,b]: 0<=k<nel and 0<=a,b<nn }", "y[k,a] = sum(b, u[k,b]*M[a,b])", None),
])
def test_parse_accepts(lib, dom, insn, asm):
    assert _create(lib, dom, insn, asm) == 0


@pytest.mark.parametrize("dom,insn,asm", [
    ("{ [f,e,i,j]: 1<=f<F and 0<=e<E and 0<=i,j<N }", "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])", None),  # lower bound 1
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i<N and 0<=j<M }", "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])", None),  # non-square
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }", "out[f,e,i] = sum(j, D[f,j,i]*u[e,j])", None),  # transposed D
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }", "out[f,e,i] = sum(i, D[f,i,j]*u[e,j])", None),
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }", "out[f,e,i] = D[f,i,j]*u[e,j]", None),  # no reduction
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }", "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])", "Q mod 4 = 0"),
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }", "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])", "E mod 0 = 0"),
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E }", "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])", None),  # unbounded inames
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N", "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])", None),  # no brace
    ("{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }", "out[f,e,i] = sum(j, D[f,i,j]*D[e,j])", None),  # same array
])
def test_parse_rejects(lib, dom, insn, asm):
    assert _create(lib, dom, insn, asm) == 2


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.lc_kernel_create(None, b"x", None, ctypes.byref(h)) == 1
    assert lib.lc_status_string(8) == b"LC_ERR_TIMEOUT"
    assert lib.lc_status_string(99) == b"LC_ERR_UNKNOWN"


def test_print_sections(lib):
    k = lc.Kernel(assumptions="E mod 64 = 0")
    text = k.print()
    for sec in ("ARGUMENTS:", "DOMAINS:", "ASSUMPTIONS: E mod 64 = 0", "INSTRUCTIONS:",
                "out[f, e, i] <- sum(j, D[f, i, j]*u[e, j])"):
        assert sec in text
    v = lc.Variant(tile_e=64, tail_free=1, layout="node")
    t2 = k.print(v)
    assert "split_iname(e, 64)" in t2 and "no guard: assumption E mod 64 = 0" in t2
    assert "u: GlobalArg, type: float32, shape: (E, N), dim_tags: (stride:1, stride:E)" in t2
    # a too-small buffer reports the needed size and truncates safely
    need = ctypes.c_size_t(0)
    buf = ctypes.create_string_buffer(10)
    assert lib.lc_kernel_print(k.handle, None, buf, 10, ctypes.byref(need)) == 6
    assert need.value == len(text) + 1 and len(buf.value) == 9


def test_variant_validation_rules(lib):
    k = lc.Kernel()
    ok = lc.Variant()
    assert lc.variant_validate(k, 1 << 21, 35, 3, ok) == 0
    bad = [
        dict(elems_per_thread=3), dict(split_i=16), dict(unroll=3), dict(prefetch_smem=2), dict(tile_e=66),
        dict(tail_free=1), dict(stages=0), dict(stages=3), dict(stages=2, prefetch_smem=0), dict(engine="tcgen05", precision="fp32"), dict(precision="bf16"),
        dict(ctas_per_sm=-1), dict(tile_e=4096 * 8, elems_per_thread=8),
    ]
    for b in bad:
        assert lc.variant_validate(k, 1 << 21, 35, 3, lc.Variant(**b)) == 3, b
    assert lc.variant_validate(k, 1 << 21, 300, 3, ok) == 1      # N out of range
    assert lc.variant_validate(k, -1, 35, 3, ok) == 1
    # shared-memory plan too large for one CTA
    assert lc.variant_validate(k, 1 << 21, 256, 8, lc.Variant(tile_e=1024, elems_per_thread=8)) == 3
    # warp engine only for N <= 32 and one warp-multiple tile
    w = lc.Variant(engine="warp", tile_e=8 * 4, elems_per_thread=1, split_i=1, unroll=1, prefetch_smem=0)
    assert lc.variant_validate(k, 1000, 4, 3, w) == 0
    assert lc.variant_validate(k, 1000, 40, 3, w) == 3
    # single-operator kernels take F = 1 only
    k1 = lc.Kernel("{ [e,i,j]: 0<=e<E and 0<=i,j<N }", "out[e,i] = sum(j, D[i,j]*u[e,j])")
    assert lc.variant_validate(k1, 100, 20, 1, ok) == 0
    assert lc.variant_validate(k1, 100, 20, 2, ok) == 1


def test_assumptions_checked_against_sizes(lib):
    k = lc.Kernel(assumptions="E mod 128 = 0 and N >= 8 and F <= 4")
    v = lc.Variant()
    assert lc.variant_validate(k, 1024, 35, 3, v) == 0
    assert lc.variant_validate(k, 1000, 35, 3, v) == 4
    assert lc.variant_validate(k, 1024, 4, 3, v) == 4
    assert lc.variant_validate(k, 1024, 35, 5, v) == 4


def test_contract_rejects_before_launch(lib):
    k = lc.Kernel()
    v = lc.Variant()
    assert lc.lc_contract(k, v, 0, 0, 0, 10, 35, 3, 0) == 1           # null pointers
    assert lc.lc_contract(k, v, 0x1000, 0x2008, 0x30000, 10, 35, 3, 0) == 5  # misaligned u
    bad = lc.Variant(unroll=5)
    assert lc.lc_contract(k, bad, 0x1000, 0x2000, 0x30000, 10, 35, 3, 0) in (3, 9)


def test_default_variant_fits(lib):
    k = lc.Kernel()
    for E, N, F in [(1 << 21, 35, 3), (1 << 20, 84, 4), (4096, 165, 4), (100, 4, 1), (1 << 23, 256, 8)]:
        for layout in ("elem", "node"):
            v = lc.variant_default(k, E, N, F, layout, "fp32")
            assert lc.variant_validate(k, E, N, F, v) == 0


def test_default_engine_per_size(lib):
    """The defaults the autotuner's measurements chose: FP32 on the warp engine up to N = 12,
    SIMT tiles below N = 96 (element-major 4 x 8 blocks, unrolled; node-major not unrolled
    from N = 25), K-split from N = 96; BF16X3 on the tensor cores with the A terms in shared
    memory, then (about N = 100 to 128) in tensor memory, then the K-split FP32 kernel."""
    k = lc.Kernel()
    eng = lambda E, N, F, layout, prec: lc.variant_dict(lc.variant_default(k, E, N, F, layout, prec))
    for layout in ("elem", "node"):
        assert eng(360273, 4, 3, layout, "fp32")["engine"] == "warp"
        d = eng(1 << 20, 56, 3, layout, "fp32")
        assert d["engine"] == "simt" and d["elems_per_thread"] == 4 and d["split_i"] == 8
        assert d["unroll"] == (4 if layout == "elem" else 1) and d["stages"] == 2
        assert eng(1 << 20, 120, 3, layout, "fp32")["engine"] == "ksplit"
        v = lc.variant_default(k, 1 << 21, 35, 3, layout, "bf16x3")
        assert lc.variant_dict(v)["engine"] == "tcgen05" and lc.variant_plan(k, 1 << 21, 35, 3, v)["a_in_tmem"] == 0
        v = lc.variant_default(k, 310977, 120, 3, layout, "bf16x3")
        assert lc.variant_dict(v)["engine"] == "tcgen05" and lc.variant_plan(k, 310977, 120, 3, v)["a_in_tmem"] == 1
        assert eng(564445, 165, 3, layout, "bf16x3")["engine"] == "ksplit"


def test_variant_plan_reports_the_resolved_launch(lib):
    """lc_variant_plan: the tensor plan of the default BF16X3 descriptor, a SIMT plan, and
    the argument checks (host only; without a GPU a 148-SM part is assumed)."""
    k = lc.Kernel()
    v = lc.Variant(engine="tcgen05", layout="elem", precision="bf16x3", tile_e=128, elems_per_thread=64,
                   split_i=0, unroll=4, prefetch_smem=1, stages=1, store_rows=128, mma_order=1)
    p = lc.variant_plan(k, 1 << 21, 35, 3, v)
    assert p["tiles"] == (1 << 21) // 128 and p["column_blocks"] == 1 and p["ops_per_block"] == 3
    assert p["k_mma"] == 48 and p["k_block"] == 64
    # the three operators packed without padding: 105 columns, MMA N 112, the D terms stacked
    # (MMA N 224): 5 MMAs per K step
    assert p["cols_per_op"] == 35 and p["mma_n"] == 112 and p["stacked"] == 1 and p["mma_per_tile"] == 15
    assert p["threads"] == 128 * (4 + 2) + 96 and p["store_rows"] == 128
    assert 0 < p["smem_bytes"] <= 232448 and p["a_in_tmem"] == 0 and p["tmem_cols"] == 512
    # BF16 with the A terms in tensor memory: two accumulators of 128 columns and two A
    # buffers of 24 columns; no A in shared memory
    w = lc.Variant(engine="tcgen05", layout="elem", precision="bf16", tile_e=128, elems_per_thread=64, split_i=0,
                   unroll=4, prefetch_smem=1, stages=2, store_rows=128, a_operand=2)
    q = lc.variant_plan(k, 1 << 21, 35, 3, w)
    assert q["a_in_tmem"] == 1 and q["stacked"] == 0 and q["mma_per_tile"] == 3 and q["a_buffers"] == 2
    assert q["cols_per_op"] == 40 and q["mma_n"] == 128 and q["tmem_cols"] == 512
    w.a_operand = 1
    assert lc.variant_plan(k, 1 << 21, 35, 3, w)["a_in_tmem"] == 0
    v.a_operand = 2  # the three-term path keeps A in shared memory
    assert lib.lc_variant_validate(k.handle, 1 << 21, 35, 3, ctypes.byref(v)) == 3
    v.mma_order, v.a_operand, v.stages = 1, 0, 1
    s = lc.variant_plan(k, 1 << 21, 35, 3, lc.variant_default(k, 1 << 21, 35, 3, "elem", "fp32"))
    assert s["mma_per_tile"] == 0 and s["grid"] > 0 and s["tiles"] > 0
    bad = lc.lc_plan()
    bad.struct_size = 3
    assert lib.lc_variant_plan(k.handle, 1 << 21, 35, 3, ctypes.byref(v), ctypes.byref(bad)) == 1
    v.unroll = 9
    with pytest.raises(lc.LcError):
        lc.variant_plan(k, 1 << 21, 35, 3, v)


def test_early_release_and_store_warp_plan(lib):
    """prefetch_smem = 2 (early release of the u stage) is a valid tensor-core descriptor for
    both reduced-precision paths; every tensor-core CTA carries the producer, MMA and store
    warps beside its epilogue and conversion warps."""
    k = lc.Kernel()
    for prec in ("bf16", "bf16x3"):
        v = lc.Variant(engine="tcgen05", layout="elem", precision=prec, tile_e=128, elems_per_thread=64,
                       split_i=0, unroll=4, prefetch_smem=2, stages=1, store_rows=128)
        assert lib.lc_variant_validate(k.handle, 1 << 21, 35, 3, ctypes.byref(v)) == 0
        assert lc.variant_plan(k, 1 << 21, 35, 3, v)["threads"] == 128 * (4 + 2) + 96
    s = lc.variant_default(k, 4096, 35, 3, "elem", "fp32")
    s.prefetch_smem = 2
    assert lib.lc_variant_validate(k.handle, 4096, 35, 3, ctypes.byref(s)) != 0


def test_max_ctas_bounds_the_grid(lib):
    """The descriptor's grid bound: honoured by the plan in whole column-block sets; a bound
    below one set of column blocks, or a negative one, is rejected before any launch."""
    kernel = lc.Kernel()
    for prec, N, F in (("bf16x3", 84, 4), ("fp32", 35, 3), ("bf16", 165, 3)):
        v = lc.variant_default(kernel, 1 << 16, N, F, "elem", prec)
        p = lc.variant_plan(kernel, 1 << 16, N, F, v)
        nb = p["column_blocks"]
        v.max_ctas = 2 * nb + 1
        # the K-split engine runs every column block of a tile in one CTA: any grid size
        whole = 1 if lc.variant_dict(v)["engine"] == "ksplit" else nb
        assert lc.variant_plan(kernel, 1 << 16, N, F, v)["grid"] == (2 * nb + 1) // whole * whole
        v.max_ctas = 10 ** 6
        assert lc.variant_plan(kernel, 1 << 16, N, F, v)["grid"] == p["grid"]
        if whole > 1:
            v.max_ctas = nb - 1
            assert lc.variant_validate(kernel, 1 << 16, N, F, v) == 3  # LC_ERR_INVALID_VARIANT
        v.max_ctas = -1
        assert lc.variant_validate(kernel, 1 << 16, N, F, v) == 3


def test_variant_features_and_pick_arguments(lib):
    """The cost model's features come from the library (host only): LC_FEATURES finite values
    with consistent one-hot groups; lc_pick_variant rejects bad arguments before any work."""
    import numpy as np
    kernel = lc.Kernel()
    for path, layout in (("bf16x3", "elem"), ("fp32", "node"), ("bf16", "node")):
        for v in lc.enumerate_variants(kernel, 100000, 35, 3, layout, path):
            x = lc.variant_features(kernel, 100000, 35, 3, layout, path, v)
            assert x.shape == (lc.FEATURES,) and np.all(np.isfinite(x))
            # engine one-hot over simt / tcgen05 / warp; the K-split engine is all zeros there
            # (and tells itself apart by its register-block and chunk fields)
            ks = v.engine == lc.ENGINE["ksplit"]
            assert x[4:7].sum() == 1 and x[7:9].sum() == 1 and x[12:15].sum() == (0 if ks else 1)
    need = ctypes.c_size_t(0)
    assert lib.lc_pick_workspace_size(ctypes.byref(need)) == 0 and need.value >= 256 * 33 * 4
    v = lc.lc_variant()
    assert lib.lc_pick_variant(kernel.handle, 1000, 35, 3, 0, 3, None, None, 0, ctypes.byref(v), None, None) == 1
    assert lib.lc_pick_variant(kernel.handle, 1000, 35, 3, 0, 3, 16, 16, 8, ctypes.byref(v), None, None) == 6
    # the ensemble form: at least one model, the same workspace rule
    assert lib.lc_pick_variant_ensemble(kernel.handle, 1000, 35, 3, 0, 3, 16, 0, 16, need.value, ctypes.byref(v),
                                        None, None) == 1
    assert lib.lc_pick_variant_ensemble(kernel.handle, 1000, 35, 3, 0, 3, 16, 3, 16, 8, ctypes.byref(v), None,
                                        None) == 6
    assert lib.lc_pick_variant_ensemble(kernel.handle, 1000, 35, 3, 0, 3, 18, 3, 16, need.value, ctypes.byref(v),
                                        None, None) == 5


def test_enumeration_leaves_out_one_warp_plans(lib):
    """Large N with one operator (E=43715, N=145): a SIMT descriptor whose tile does not fit
    shared memory resolves to many column blocks of one warp each; such plans stay valid but
    are not candidates (one of them ran 12x slower than the best in the autotuner)."""
    kernel = lc.Kernel("{ [e,i,j]: 0<=e<E and 0<=i,j<N }", "out[e,i] = sum(j, D[i,j]*u[e,j])")
    E, N, F = 43715, 145, 1
    cands = lc.enumerate_variants(kernel, E, N, F, "elem", "bf16")
    assert cands
    for v in cands:
        assert lc.variant_plan(kernel, E, N, F, v)["threads"] >= 64
    v = lc.Variant(engine="simt", tile_e=128, elems_per_thread=8, split_i=4, unroll=1, prefetch_smem=1, stages=2,
                   ctas_per_sm=2)
    assert lc.variant_validate(kernel, E, N, F, v) == 0
    assert lc.variant_plan(kernel, E, N, F, v)["threads"] < 64
    assert lc.variant_dict(v) not in [lc.variant_dict(c) for c in cands]


GEO_DOM = "{ [d,f,e,i,j]: 0<=d<F and 0<=f<F and 0<=e<E and 0<=i,j<N }"


@pytest.mark.parametrize("insn,ok", [
    ("out[d,e,i] = sum((f,j), G[e,d,f]*D[f,i,j]*u[e,j])", True),
    ("y[d,e,i] = sum((j,f), u[e,j]*Dr[f,i,j]*rx[e,d,f])", True),
    ("out[d,e,i] = sum((f,j), G[e,f,d]*D[f,i,j]*u[e,j])", False),   # transposed factors
    ("out[d,e,i] = sum((f,j), G[e,d,f]*D[f,j,i]*u[e,j])", False),   # transposed operator
    ("out[d,e,i] = sum((f,j), G[e,d,f]*D[f,i,j]*G[e,j])", False),   # repeated array
    ("out[d,e,i] = sum(j, D[d,i,j]*u[e,j])", False),                # not this domain's inames
])
def test_parse_geometric_factor_form(lib, insn, ok):
    assert (_create(lib, GEO_DOM, insn) == 0) == ok
    # d and f must share one bound
    assert _create(lib, "{ [d,f,e,i,j]: 0<=d<P and 0<=f<F and 0<=e<E and 0<=i,j<N }",
                   "out[d,e,i] = sum((f,j), G[e,d,f]*D[f,i,j]*u[e,j])") == 2


def test_geometric_factor_kernel_rules(lib):
    """The two instruction forms have their own entry points; the fused epilogue needs every
    operator in one column block of the tensor-core engine, F = 2 or 3."""
    kg = lc.Kernel(lc.GEO_DOMAIN, lc.GEO_INSTRUCTION)
    kc = lc.Kernel()
    v = lc.variant_default(kg, 1 << 20, 35, 3, "elem", "bf16x3")
    assert lc.variant_dict(v)["engine"] == "tcgen05" and lc.variant_plan(kg, 1 << 20, 35, 3, v)["column_blocks"] == 1
    assert lc.load().lc_contract(kg.handle, ctypes.byref(v), 16, 16, 16, 0, 35, 3, None) == 2
    assert lib.lc_contract_geo(kc.handle, ctypes.byref(v), 16, 16, 16, 16, 0, 35, 3, None) == 2
    for bad in (dict(split_i=1), dict(engine="simt", precision="fp32", tile_e=64, elems_per_thread=4, split_i=8)):
        d = lc.variant_dict(v)
        d.update(bad)
        assert lc.variant_validate(kg, 1 << 20, 35, 3, lc.Variant(**d)) == 3, bad
    assert lc.variant_validate(kg, 1 << 20, 35, 4, v) == 3  # F = 4: no kernel instance
    text = kg.print(v)
    assert "out[d, e, i] <- sum((f, j), G[e, d, f]*D[f, i, j]*u[e, j])" in text
    assert "G: GlobalArg" in text


def test_grouped_tensor_plan_arguments(lib):
    """Grouped plans on the tensor cores: at most 16 groups, BF16 / BF16X3 only, null or
    misaligned buffers refused before any device query."""
    kernel = lc.Kernel()
    G = lc.lc_group
    arr = (G * 17)()
    for g in arr:
        g.E, g.N, g.F, g.D_dev, g.u_dev, g.out_dev = 100, 35, 3, 256, 512, 1024
    need = ctypes.c_size_t(0)
    v = lc.Variant(engine="tcgen05", precision="bf16x3", tile_e=128, elems_per_thread=64, unroll=4, stages=1,
                   store_rows=128)
    assert lib.lc_grouped_workspace_size(kernel.handle, ctypes.byref(v), arr, 17, ctypes.byref(need)) == 1
    vf = lc.Variant(engine="tcgen05", precision="fp32", tile_e=128, elems_per_thread=64, unroll=4, stages=1)
    assert lib.lc_grouped_workspace_size(kernel.handle, ctypes.byref(vf), arr, 2, ctypes.byref(need)) == 3
    arr[0].D_dev = 0
    assert lib.lc_grouped_workspace_size(kernel.handle, ctypes.byref(v), arr, 2, ctypes.byref(need)) == 1
    arr[0].D_dev = 258
    assert lib.lc_grouped_workspace_size(kernel.handle, ctypes.byref(v), arr, 2, ctypes.byref(need)) == 5
