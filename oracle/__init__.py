"""CPU FP64 oracle for the batched element-local contraction (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package. The library never imports it, and it imports nothing
from the library: the two share no code.

What it computes (all in float64, no reordering of any sum):

* ``contract``            out[f,e,i] = sum_j D[f,i,j] u[e,j], the untransformed
                          loop nest of the dG FEM volume workload (Table 1), in the
                          loop-domain-plus-instruction form of Section 2.1.
* ``contract_rows``       the same for a chosen subset of elements (sampled checks
                          at full size).
* ``bf16_round``          binary32 -> bfloat16, round-to-nearest-even.
* ``bf16_split3``         x = hi + mid + lo, three bfloat16 terms.
* ``contract_bf16`` /     the exact result of the reduced-precision tensor-core
  ``contract_bf16x3``     paths: bf16-rounded operands (or the kept split products)
                          multiplied exactly, summed in float64.
* ``mlp_forward`` / ``mlp_loss_grad`` / ``adam_step``  the cost model's network.
* ``contract_geo``        out[d,e,i] = sum_f r[e,d,f] sum_j D[f,i,j] u[e,j]: the volume
                          derivative with per-element geometric factors.
* ``lift``                the surface part of the dG operator: jumps of the traces at
                          the face nodes, scaled per face, lifted by the lift matrix.
* ``rel_fro_error``       ||out - ref||_F / ||ref||_F in float64.
* ``elementwise.evaluate`` one elementwise assignment over a rectangular loop domain,
                          every operation one IEEE float32 operation (module
                          ``oracle.elementwise``).

Parity pins: every function here is pinned by tests in ``tests/test_oracle_pins.py``
against brute force, closed forms, a library routine, or finite differences.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# The layout of the cost model's parameter vector (see oracle.c).
MLP_HIDDEN = 64

# The six kept products of the three-term split: (D term, u term), hi=0, mid=1, lo=2.
BF16X3_PAIRS = ((0, 0), (0, 1), (1, 0), (0, 2), (2, 0), (1, 1))


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, IEEE arithmetic, OpenMP over elements)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.oracle_contract.argtypes = [P, P, P, i64, i32, i32, i32, i32]
            lib.oracle_contract.restype = None
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_contract_geo.argtypes = [P, P, P, P, i64, i32, i32, i32, i32, i32]
            lib.oracle_contract_geo.restype = None
            lib.oracle_lift.argtypes = [P, P, P, P, P, P, i64, i32, i32, i32, i32, i32]
            lib.oracle_lift.restype = None
            lib.oracle_bf16_round.argtypes = [P, P, i64]
            lib.oracle_bf16_split3.argtypes = [P, P, P, P, i64]
            lib.oracle_mlp_param_count.argtypes = [i32, i32]
            lib.oracle_mlp_param_count.restype = i64
            lib.oracle_mlp_forward.argtypes = [P, P, P, i64, i32, i32]
            lib.oracle_mlp_loss_grad.argtypes = [P, P, P, i64, i32, i32, P]
            lib.oracle_mlp_loss_grad.restype = f64
            lib.oracle_adam_step.argtypes = [P, P, P, P, i64, i32, f64, f64, f64, f64]
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def contract(D, u, layout: str = "elem", threads: int = 0) -> np.ndarray:
    """out[f,e,i] = sum_j D[f,i,j] u[e,j] in float64.

    D: (F, N, N). u: (E, N) if layout == "elem", (N, E) if layout == "node".
    Returns (F, E, N) for "elem" and (F, N, E) for "node". Inputs are upcast to
    float64 exactly (every binary32 value is a binary64 value).
    """
    lib = _load()
    D = _f64(D)
    u = _f64(u)
    if D.ndim == 2:
        D = D[None]
    F, N, N2 = D.shape
    assert N == N2
    node = layout == "node"
    if node:
        assert u.shape[0] == N
        E = u.shape[1]
        out = np.empty((F, N, E), dtype=np.float64)
    else:
        assert u.shape[1] == N
        E = u.shape[0]
        out = np.empty((F, E, N), dtype=np.float64)
    if E > 0 and N > 0 and F > 0:
        lib.oracle_contract(_ptr(D), _ptr(u), _ptr(out), E, N, F, int(node), int(threads))
    return out


def contract_rows(D, u, rows, layout: str = "elem", threads: int = 0) -> np.ndarray:
    """Oracle outputs for the elements ``rows`` only, as (F, len(rows), N)."""
    rows = np.asarray(rows, dtype=np.int64)
    u = np.asarray(u)
    sub = u[rows] if layout == "elem" else u[:, rows].T
    return contract(D, sub, "elem", threads)


def contract_geo(D, u, r, layout: str = "elem", threads: int = 0) -> np.ndarray:
    """out[d,e,i] = sum_f r[e,d,f] * sum_j D[f,i,j] u[e,j] in float64 (volume derivative
    with per-element geometric factors).

    D: (F, N, N). u: (E, N) or (N, E) per layout. r: (E, Dd, F) element-major or
    (Dd, F, E) node-major. Returns (Dd, E, N) or (Dd, N, E).
    """
    lib = _load()
    D, u, r = _f64(D), _f64(u), _f64(r)
    F, N, N2 = D.shape
    assert N == N2
    node = layout == "node"
    if node:
        Dd, F2, E = r.shape
        assert u.shape == (N, E)
        out = np.empty((Dd, N, E), dtype=np.float64)
    else:
        E, Dd, F2 = r.shape
        assert u.shape == (E, N)
        out = np.empty((Dd, E, N), dtype=np.float64)
    assert F2 == F
    if E > 0 and N > 0 and F > 0 and Dd > 0:
        lib.oracle_contract_geo(_ptr(D), _ptr(u), _ptr(r), _ptr(out), E, N, F, Dd, int(node), int(threads))
    return out


def contract_geo_rows(D, u, r, rows, layout: str = "elem", threads: int = 0) -> np.ndarray:
    """contract_geo for the elements ``rows`` only, as (Dd, len(rows), N)."""
    rows = np.asarray(rows, dtype=np.int64)
    u, r = np.asarray(u), np.asarray(r)
    if layout == "node":
        return contract_geo(D, u[:, rows].T, np.ascontiguousarray(r[:, :, rows].transpose(2, 0, 1)), "elem", threads)
    return contract_geo(D, u[rows], r[rows], "elem", threads)


def lift(L, fmask, vmapP, s, u, out=None, threads: int = 0) -> np.ndarray:
    """Surface part of the dG operator in float64:
    out[e,i] (+)= sum_m L[i,m] * s[e, m // Nfp] * (u[e, fmask[m]] - u.flat[vmapP[e,m]]).

    L: (N, M); fmask: (M,) ints; vmapP: (E, M) ints into u.ravel(); s: (E, Nf); u: (E, N).
    With ``out`` given (E, N) the result is added to a float64 copy of it, else it is returned.
    """
    lib = _load()
    L, s_, u = _f64(L), _f64(s), _f64(u)
    fmask = np.ascontiguousarray(fmask, dtype=np.int32)
    vmapP = np.ascontiguousarray(vmapP, dtype=np.int32)
    E, N = u.shape
    Nf = s_.shape[1]
    M = L.shape[1]
    assert L.shape[0] == N and M % Nf == 0 and fmask.shape == (M,) and vmapP.shape == (E, M)
    res = np.zeros((E, N)) if out is None else _f64(out).copy()
    if E > 0:
        lib.oracle_lift(_ptr(L), _ptr(fmask), _ptr(vmapP), _ptr(s_), _ptr(u), _ptr(res), E, N, Nf, M // Nf,
                        0 if out is None else 1, int(threads))
    return res


def bf16_round(x) -> np.ndarray:
    """binary32 -> nearest-even bfloat16, returned as float32 values."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    y = np.empty_like(x)
    if x.size:
        lib.oracle_bf16_round(_ptr(x), _ptr(y), x.size)
    return y


def bf16_split3(x):
    """(hi, mid, lo) bfloat16 terms (as float32 values) with x = hi + mid + lo."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    hi, mid, lo = np.empty_like(x), np.empty_like(x), np.empty_like(x)
    if x.size:
        lib.oracle_bf16_split3(_ptr(x), _ptr(hi), _ptr(mid), _ptr(lo), x.size)
    return hi, mid, lo


def contract_bf16(D, u, layout: str = "elem", threads: int = 0) -> np.ndarray:
    """Exact contraction of the bf16-rounded operands (the plain BF16 path's target)."""
    return contract(bf16_round(D), bf16_round(u), layout, threads)


def contract_bf16x3(D, u, layout: str = "elem", threads: int = 0,
                    pairs=BF16X3_PAIRS) -> np.ndarray:
    """Exact sum of the kept split products: sum over (a, b) in pairs of D_a . u_b.

    With the default pairs (hh, hm, mh, hl, lh, mm) this is the target of the
    split-BF16 tensor-core path; the dropped products (ml, lm, ll) are below
    2^-24 relative.
    """
    Ds = bf16_split3(D)
    us = bf16_split3(u)
    out = None
    for a, b in pairs:
        r = contract(Ds[a], us[b], layout, threads)
        out = r if out is None else out + r
    return out


def rel_fro_error(out, ref) -> float:
    """||out - ref||_F / ||ref||_F in float64."""
    o = np.asarray(out, dtype=np.float64).ravel()
    r = np.asarray(ref, dtype=np.float64).ravel()
    den = float(np.sqrt(np.dot(r, r)))
    d = o - r
    num = float(np.sqrt(np.dot(d, d)))
    return num / den if den > 0 else num


# ---------------------------------------------------------------- MLP cost model

def mlp_param_count(din: int, H: int = MLP_HIDDEN) -> int:
    return int(_load().oracle_mlp_param_count(din, H))


def mlp_forward(p, x, H: int = MLP_HIDDEN) -> np.ndarray:
    lib = _load()
    p = _f64(p)
    x = _f64(x)
    B, din = x.shape
    assert p.size == mlp_param_count(din, H)
    y = np.empty(B, dtype=np.float64)
    lib.oracle_mlp_forward(_ptr(p), _ptr(x), _ptr(y), B, din, H)
    return y


def mlp_loss_grad(p, x, t, H: int = MLP_HIDDEN):
    """(loss, grad) for L = mean_s (y_s - t_s)^2."""
    lib = _load()
    p = _f64(p)
    x = _f64(x)
    t = _f64(t)
    B, din = x.shape
    g = np.empty_like(p)
    loss = lib.oracle_mlp_loss_grad(_ptr(p), _ptr(x), _ptr(t), B, din, H, _ptr(g))
    return float(loss), g


def adam_step(p, g, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays p, m, v (step t >= 1)."""
    lib = _load()
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib.oracle_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.size, int(t), lr, beta1, beta2, eps)
