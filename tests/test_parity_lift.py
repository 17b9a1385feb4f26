"""The surface lift of the dG operator (the dG FEM surface workload of Table 1):
out[e,i] (+)= sum_{f,p} L[i,f,p] s[e,f] (u[e,fmask[f,p]] - u_flat[vmapP[e,f,p]]).

CPU: the instruction form is parsed (names free) and malformed ones are refused; argument
checks before any launch.  GPU: integer-valued inputs bit-exact against the oracle (both
overwrite and accumulate), random inputs within the FP32 bound, every CTA walking many
tiles, an out-of-range index reported through the device error word (its flux is NaN, no
access outside u), and the full-size synthetic mesh sampled.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth
from paper_1405_7470_gb300 import lc


@pytest.fixture(scope="module")
def lib():
    from paper_1405_7470_gb300 import build
    build()
    return lc.load()


@pytest.mark.parametrize("insn,ok", [
    (lc.LIFT_INSTRUCTION, True),
    ("y[e,i] = sum((f,p), LIFT[i,f,p]*Fs[e,f]*(q[e,Fm[f,p]] - q[vP[e,f,p]]))", True),
    ("out[e,i] = sum((f,p), L[i,f,p]*s[e,f]*(u[e,fmask[f,p]] + u[vmapP[e,f,p]]))", False),  # not a jump
    ("out[e,i] = sum((f,p), L[i,f,p]*s[e,p]*(u[e,fmask[f,p]] - u[vmapP[e,f,p]]))", False),  # scale per node
    ("out[e,i] = sum((f,p), L[i,f,p]*s[e,f]*(u[e,fmask[f,p]] - w[vmapP[e,f,p]]))", False),  # two fields
])
def test_parse(lib, insn, ok):
    h = ctypes.c_void_p()
    st = lib.lc_kernel_create(lc.LIFT_DOMAIN.encode(), insn.encode(), None, ctypes.byref(h))
    if st == 0:
        lib.lc_kernel_destroy(h)
    assert (st == 0) == ok, (insn, st)


def test_rejects_before_launch(lib):
    k = lc.Kernel(lc.LIFT_DOMAIN, lc.LIFT_INSTRUCTION)
    v = lc.variant_default(k, 100, 35, 1, "elem", "fp32")
    f = lib.lc_lift
    assert f(k.handle, ctypes.byref(v), 16, 16, 16, 16, 16, 16, 10, 200, 4, 15, 0, None) == 1   # N > 128
    assert f(k.handle, ctypes.byref(v), 16, 16, 16, 16, 16, 18, 10, 35, 4, 15, 0, None) == 5   # misaligned
    assert f(k.handle, ctypes.byref(v), 16, 16, 16, 16, 16, 16, 10, 35, 4, 15, 2, None) == 1   # accumulate 2
    kc = lc.Kernel()
    assert f(kc.handle, ctypes.byref(v), 16, 16, 16, 16, 16, 16, 10, 35, 4, 15, 0, None) == 2  # other kind
    bad = lc.variant_default(kc, 100, 35, 3, "elem", "bf16x3")
    assert f(k.handle, ctypes.byref(bad), 16, 16, 16, 16, 16, 16, 10, 35, 4, 15, 0, None) == 3
    # no launch plan without the face counts
    with pytest.raises(lc.LcError):
        lc.variant_plan(k, 100, 35, 1, v)
    for st, te in ((0, 64), (3, 64), (1, 32), (1, 256)):  # one or two staging buffers, 64 or 128 elements
        w = lc.variant_default(k, 100, 35, 1, "elem", "fp32")
        w.stages, w.tile_e = st, te
        assert lc.variant_validate(k, 100, 35, 1, w) == 3
        assert f(k.handle, ctypes.byref(w), 16, 16, 16, 16, 16, 16, 10, 35, 4, 15, 0, None) == 3


def _dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _needs_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lc.load()
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("accumulate", [False, True])
@pytest.mark.parametrize("prefetch", [1, 0])
def test_integer_inputs_bit_exact(accumulate, prefetch):
    """Both trace paths: the staged u window (prefetch 1; width 200 puts two faces' neighbours
    outside the 64-element halo, read from global memory) and global loads only (prefetch 0)."""
    torch = _needs_gpu()
    k = lc.Kernel(lc.LIFT_DOMAIN, lc.LIFT_INSTRUCTION)
    for E, order, width in ((5000 + 13, 4, 64), (777, 2, 8), (64, 3, 4), (1, 1, 1), (3000, 5, 32),
                            (5000, 4, 200)):
        L, fmask, vmapP, s, u = synth.surface_mesh(E, order=order, width=width, seed=E)
        rng = np.random.default_rng(order)
        L = rng.integers(-3, 4, L.shape).astype(np.float32)
        s = rng.integers(1, 4, s.shape).astype(np.float32)
        u = rng.integers(-8, 9, u.shape).astype(np.float32)
        out0 = rng.integers(-5, 6, u.shape).astype(np.float32)
        want = oracle.lift(L, fmask, vmapP, s, u, out=out0 if accumulate else None)
        for ctas, stages, te in ((0, 1, 64), (2, 1, 64), (0, 2, 64), (3, 2, 64), (0, 1, 128), (2, 2, 128)):
            v = lc.variant_default(k, E, u.shape[1], 1, "elem", "fp32")
            v.max_ctas = ctas
            v.prefetch_smem = prefetch
            v.stages = stages
            v.tile_e = te
            Ld, fd, vd, sd, ud, od = _dev(L, fmask, vmapP, s, u, out0 if accumulate else np.zeros_like(u))
            lc.lift(k, v, Ld, fd, vd, sd, ud, od, accumulate=accumulate)
            torch.cuda.synchronize()
            assert lc.device_error() == 0
            assert np.array_equal(od.cpu().numpy().astype(np.float64), want), (E, order, ctas, stages, te)


@pytest.mark.gpu
def test_random_inputs_within_bound():
    torch = _needs_gpu()
    k = lc.Kernel(lc.LIFT_DOMAIN, lc.LIFT_INSTRUCTION)
    L, fmask, vmapP, s, u = synth.surface_mesh(20000 + 7, order=4, width=64, seed=1)
    v = lc.variant_default(k, u.shape[0], u.shape[1], 1, "elem", "fp32")
    Ld, fd, vd, sd, ud = _dev(L, fmask, vmapP, s, u)
    out = lc.lift(k, v, Ld, fd, vd, sd, ud)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.lift(L, fmask, vmapP, s, u)
    Nfp = fmask.size // 4
    # per output: the jump and the scale round once each, then an M-term FP32 FMA chain
    mag = (np.repeat(np.abs(s.astype(np.float64)), Nfp, axis=1) *
           (np.abs(u[:, fmask].astype(np.float64)) + np.abs(u.ravel()[vmapP].astype(np.float64)))) @ np.abs(L.T)
    bound = (fmask.size + 4) * 2.0 ** -24 * mag + 1e-30
    assert np.all(np.abs(got - want) <= bound)
    assert oracle.rel_fro_error(got, want) <= 1e-6


@pytest.mark.gpu
def test_out_of_range_index_is_reported():
    torch = _needs_gpu()
    k = lc.Kernel(lc.LIFT_DOMAIN, lc.LIFT_INSTRUCTION)
    L, fmask, vmapP, s, u = synth.surface_mesh(500, order=2, width=8, seed=2)
    bad = vmapP.copy()
    bad[7, 3] = u.size + 1000  # past the end of u
    v = lc.variant_default(k, u.shape[0], u.shape[1], 1, "elem", "fp32")
    Ld, fd, vd, sd, ud = _dev(L, fmask, bad, s, u)
    out = lc.lift(k, v, Ld, fd, vd, sd, ud)
    torch.cuda.synchronize()
    assert lc.device_error() == 11  # LC_ERR_INDEX (and cleared)
    got = out.cpu().numpy()
    assert np.all(np.isnan(got[7])) and np.all(np.isfinite(np.delete(got, 7, axis=0)))
    assert lc.device_error() == 0


@pytest.mark.gpu
def test_full_size_sampled():
    """E = 2^21 tetrahedra of degree 4 (N = 35, 4 faces x 15 nodes), the bench's workload."""
    torch = _needs_gpu()
    E = 1 << 21
    L, fmask, vmapP, s, u = synth.surface_mesh(E, order=4, width=64, seed=0)
    k = lc.Kernel(lc.LIFT_DOMAIN, lc.LIFT_INSTRUCTION)
    v = lc.variant_default(k, E, 35, 1, "elem", "fp32")
    Ld, fd, vd, sd, ud = _dev(L, fmask, vmapP, s, u)
    out = lc.lift(k, v, Ld, fd, vd, sd, ud)
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    rows = np.unique(np.concatenate([np.arange(200), np.random.default_rng(3).integers(0, E, 5000),
                                     np.arange(E - 200, E)]))
    got = out.index_select(0, torch.from_numpy(rows).cuda()).cpu().numpy()
    want = oracle.lift(L, fmask, vmapP, s, u)[rows]
    assert oracle.rel_fro_error(got, want) <= 1e-6


@pytest.mark.gpu
def test_window_from_unaligned_u():
    """u starting 4 bytes past a 16-byte boundary: no bulk copies, every operand read from
    global memory (the staged path needs 16-byte aligned u, vmapP and s)."""
    torch = _needs_gpu()
    k = lc.Kernel(lc.LIFT_DOMAIN, lc.LIFT_INSTRUCTION)
    L, fmask, vmapP, s, u = synth.surface_mesh(3001, order=4, width=64, seed=5)
    rng = np.random.default_rng(9)
    u = rng.integers(-8, 9, u.shape).astype(np.float32)
    Ld, fd, vd, sd, _ = _dev(L, fmask, vmapP, s, u)
    flat = torch.empty(u.size + 4, dtype=torch.float32, device="cuda")
    ud = flat[1:1 + u.size].view(u.shape)
    ud.copy_(torch.from_numpy(u))
    v = lc.variant_default(k, u.shape[0], u.shape[1], 1, "elem", "fp32")
    assert v.prefetch_smem == 1
    out = lc.lift(k, v, Ld, fd, vd, sd, ud)
    torch.cuda.synchronize()
    assert lc.device_error() == 0
    want = oracle.lift(L, fmask, vmapP, s, u)
    got = out.cpu().numpy().astype(np.float64)
    Nfp = fmask.size // 4
    mag = (np.repeat(np.abs(s.astype(np.float64)), Nfp, axis=1) *
           (np.abs(u[:, fmask].astype(np.float64)) + np.abs(u.ravel()[vmapP].astype(np.float64)))) @ np.abs(L.T)
    assert np.all(np.abs(got - want) <= (fmask.size + 4) * 2.0 ** -24 * mag + 1e-30)
