"""The general front end for elementwise instructions (a loop domain of one or two inames
plus one assignment, Section 2.1), generated into CUDA with split_iname's bulk, edge and
corner code (Section 2.4).

CPU: parsing and its errors, the argument signature, descriptor validation (assumption-
gated guard-free code), the generated source's structure.  GPU: every instruction, domain
size and descriptor reproduces the oracle's IEEE single-precision evaluation bit for bit
(tiles cut by one bound, by both, and whole), with sentinels around the output.
"""

import itertools

import numpy as np
import pytest

from oracle import elementwise as ew_oracle
from paper_1405_7470_gb300 import lc

SAXPY = ("{ [i]: 0<=i<n }", "z[i] = a*x[i] + y[i]")
CASES = [
    ("{ [i]: 0<=i<n }", "z[i] = a*x[i] + y[i]"),
    ("{ [i]: 0<=i<n }", "w[i] = -(x[i] - y[i]) / (1.5 + x[i]*x[i]) + 2e-3*s"),
    ("{ [i,j]: 0<=i<n and 0<=j<m }", "b[i,j] = c[j] - 2.5*d[i] / (a[i,j] + 3)"),
    ("{ [r,c]: 0<=r<R and 0<=c<C }", "o[r,c] = alpha*A[r,c] + beta*B[r,c]*B[r,c] - v[c]"),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1405_7470_gb300 import build
    build()
    return lc.load()


def test_parse_and_signature(lib):
    k = lc.Kernel(*CASES[1])
    assert lc.kernel_args(k) == dict(arrays=["w", "x", "y"], params=["s"], dims=["n"])
    k2 = lc.Kernel(*CASES[2])
    assert lc.kernel_args(k2) == dict(arrays=["b", "c", "d", "a"], params=[], dims=["n", "m"])
    text = k2.print(lc.variant_default(k2, 100, 100, 1, "elem", "fp32"))
    assert "KERNEL: elementwise" in text and "split_iname(j, 256)" in text and "corner" in text


@pytest.mark.parametrize("dom,insn", [
    ("{ [i]: 0<=i<n }", "z[j] = x[j]"),                     # index not an iname of the domain
    ("{ [i]: 0<=i<n }", "z[i] = x[i] + z[i]"),              # reads the output
    ("{ [i,j]: 0<=i<n and 0<=j<m }", "b[i,j] = c[j,i]"),    # indices out of domain order
    ("{ [i,j]: 0<=i<n and 0<=j<m }", "b[j,i] = c[j]"),      # output not in domain order
    ("{ [i]: 0<=i<n }", "z[i] = x[i] + x"),                 # one name, array and scalar... as two
    ("{ [i]: 0<=i<n }", "z[i] = x[i] +"),                   # incomplete
    ("{ [i]: 0<=i<n }", "z[i] = i * 2"),                    # an iname as a value
    ("{ [i,j,k]: 0<=i<n and 0<=j<m and 0<=k<p }", "o[i,j,k] = x[i,j,k]"),  # three inames
])
def test_parse_rejects(lib, dom, insn):
    import ctypes
    h = ctypes.c_void_p()
    st = lib.lc_kernel_create(dom.encode(), insn.encode(), None, ctypes.byref(h))
    if st == 0:
        lib.lc_kernel_destroy(h)
    assert st == 2, (dom, insn)


def test_descriptor_rules(lib):
    k = lc.Kernel(*SAXPY, assumptions="n mod 4096 = 0")
    v = lc.variant_default(k, 1 << 20, 1, 1, "elem", "fp32")
    assert lc.variant_validate(k, 1 << 20, 1, 1, v) == 0
    v.tail_free = 1            # guard-free code: the assumption makes the tile (4096) divide n
    assert lc.variant_validate(k, 1 << 20, 1, 1, v) == 0
    assert lc.variant_validate(k, (1 << 20) + 4, 1, 1, v) == 4   # the assumption fails
    v.unroll = 2               # tile 2048 divides n too
    assert lc.variant_validate(k, 1 << 20, 1, 1, v) == 0
    k2 = lc.Kernel(*SAXPY)
    assert lc.variant_validate(k2, 1 << 20, 1, 1, v) == 3       # no assumption: guards needed
    for bad in (dict(unroll=3), dict(elems_per_thread=2), dict(stages=2), dict(precision="bf16"),
                dict(tile_e=100), dict(engine="tcgen05")):
        d = lc.variant_dict(lc.variant_default(k2, 100, 1, 1, "elem", "fp32"))
        d.update(bad)
        assert lc.variant_validate(k2, 100, 1, 1, lc.Variant(**d)) == 3, bad
    p = lc.variant_plan(k2, 10 ** 6, 1, 1, lc.variant_default(k2, 10 ** 6, 1, 1, "elem", "fp32"))
    assert p["tiles"] == -(-10 ** 6 // 4096) and p["threads"] == 256
    # the other entry points refuse an elementwise kernel
    assert lc.lc_contract(k2, v, 16, 16, 16, 0, 35, 3, 0) == 2


def test_generated_source_structure(lib):
    k = lc.Kernel(*CASES[2])
    v = lc.variant_default(k, 100, 100, 1, "elem", "fp32")
    src = lc.elementwise_source(k, v, (100, 100))
    for part in ("bulk: no guard", "edge cut by n0", "edge cut by n1", "corner: both guards", "__fdiv_rn",
                 "__ldcs(reinterpret_cast<const float4 *>"):
        assert part in src, part
    k1 = lc.Kernel(*SAXPY, assumptions="n mod 4096 = 0")
    v1 = lc.variant_default(k1, 4096, 1, 1, "elem", "fp32")
    v1.tail_free = 1
    assert "i < n0 && i < base + T" not in lc.elementwise_source(k1, v1, (8192,))
    assert "i < n0 && i < base + T" in lc.elementwise_source(k1, lc.variant_default(k1, 4096, 1, 1, "elem", "fp32"),
                                                             (8192,))


# ------------------------------------------------------------------------------- GPU

@pytest.mark.gpu
@pytest.mark.parametrize("case", range(len(CASES)))
def test_elementwise_bit_exact(case):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lc.load()
    dom, insn = CASES[case]
    kernel = lc.Kernel(dom, insn)
    args = lc.kernel_args(kernel)
    inames = [t.strip() for t in dom[dom.index("[") + 1:dom.index("]")].split(",")]
    # which inames each array is indexed by (from the instruction text)
    idx = {}
    for name in args["arrays"]:
        pos = insn.index(name + "[")
        idx[name] = [t.strip() for t in insn[pos + len(name) + 1:insn.index("]", pos)].split(",")]
    sizes_list = ([(1,), (4095,), (4096,), (4097,), (100003,), (1 << 20,)] if len(inames) == 1 else
                  [(1, 1), (3, 257), (16, 256), (17, 255), (64, 1024), (129, 300), (1000, 1000)])
    rng = np.random.default_rng(case)
    for sizes in sizes_list:
        ext = dict(zip(args["dims"], sizes))
        host = {}
        for name in args["arrays"][1:]:
            shape = tuple(sizes[inames.index(n)] for n in idx[name])
            host[name] = (rng.standard_normal(shape) * 3).astype(np.float32)
        params = {p: float(rng.uniform(-2, 2)) for p in args["params"]}
        want = ew_oracle.evaluate(insn, inames, sizes, host, params)
        for unroll, vec, ctas in itertools.product((1, 4, 8), (4, 1), (1, 0)):
            v = lc.variant_default(kernel, sizes[0], sizes[-1], 1, "elem", "fp32")
            v.unroll, v.elems_per_thread = unroll, vec
            v.max_ctas = ctas  # 1: one CTA walks every tile
            n = int(np.prod(sizes))
            buf = torch.full((n + 128,), 777.0, device="cuda")
            out = buf[64:64 + n].view(*sizes)
            devs = [out] + [torch.from_numpy(host[nm]).cuda() for nm in args["arrays"][1:]]
            lc.elementwise(kernel, v, devs, [params[p] for p in args["params"]], extents=sizes)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.array_equal(got, want, equal_nan=True), (insn, sizes, unroll, vec, ctas)
            b = buf.cpu().numpy()
            assert np.all(b[:64] == 777.0) and np.all(b[64 + n:] == 777.0)
