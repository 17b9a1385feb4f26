"""Seeded synthetic inputs for the batched element-local contraction.

    out[f, e, i] = sum_j D_f[i, j] * u[e, j]

This module only draws numbers. It holds none of the contraction's arithmetic and
is the one piece of code shared by the CPU oracle's tests and the CUDA path's tests
and benchmark. Every array is drawn in float64 with numpy's PCG64 generator
(``np.random.default_rng(seed)``) and then rounded (round-to-nearest-even) to the
storage dtype, so both sides receive bit-identical inputs.

Draw order for one problem: D_0 .. D_{F-1} (each N x N, row-major ``D[f][i][j]``),
then any extra operator material, then u (E x N, element-major), then any
per-element scale exponents. Node-major inputs are the element-major values
transposed (``u_nm[j][e] = u[e][j]``), so one seed yields the same problem in
both layouts.

Workloads (the dG FEM volume contraction of Table 1, sized as stated beside each):

* ``fp64_single``   E=4096, N=20, F=1, D ~ U[-1,1), u ~ N(0,1), float64.
* ``fp32_three``    E=2^21, N=35, F=3, D ~ U[-1,1), u ~ N(0,1), float32.
* ``precision``     E=2^20, N=84, F=4, D_0..2 ~ U[-1,1), D_3 = A A^T/84 + I with
                    A ~ U[-1,1) (84 x 84), u ~ N(0,1) * 10^k, k ~ U[-3,3) per element.
* ``grouped``       8 groups, N in {4,10,20,35,56,84,120,165},
                    E_g = floor(2^U(14,21)) drawn in N order, F=3, float32.
* ``picker``        600 shapes: N ~ U{4..165}, E = floor(2^U(12,23)), F ~ U{1..4},
                    path in {fp32, bf16, bf16x3}, layout in {elem, node}.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "operands",
    "integer_operands",
    "fp64_single",
    "fp32_three",
    "precision_sweep",
    "grouped_sizes",
    "grouped_operands",
    "picker_shapes",
    "to_node_major",
    "GROUP_NS",
]

GROUP_NS = (4, 10, 20, 35, 56, 84, 120, 165)


def _round(x: np.ndarray, dtype) -> np.ndarray:
    # numpy's float64 -> float32 cast rounds to nearest even.
    return np.ascontiguousarray(x.astype(dtype))


def operands(E: int, N: int, F: int, dtype=np.float32, seed: int = 0,
             spd_last: bool = False, scale_exp: float | None = None):
    """Draw (D, u) for one contraction problem, element-major.

    D: (F, N, N) with entries U[-1, 1). If ``spd_last``, the last operator is
    replaced by A A^T / N + I with A ~ U[-1, 1) (N x N), drawn after D_0..D_{F-2}.
    u: (E, N) standard normal; if ``scale_exp`` is given, each element's row is
    multiplied by 10^k with k ~ U[-scale_exp, scale_exp) (drawn after u).
    """
    rng = np.random.default_rng(seed)
    nplain = F - 1 if spd_last else F
    D = np.empty((F, N, N), dtype=np.float64)
    for f in range(nplain):
        D[f] = rng.uniform(-1.0, 1.0, size=(N, N))
    if spd_last:
        A = rng.uniform(-1.0, 1.0, size=(N, N))
        D[F - 1] = A @ A.T / N + np.eye(N)
    u = rng.standard_normal(size=(E, N))
    if scale_exp is not None:
        k = rng.uniform(-scale_exp, scale_exp, size=E)
        u *= (10.0 ** k)[:, None]
    return _round(D, dtype), _round(u, dtype)


def integer_operands(E: int, N: int, F: int, dtype=np.float32, seed: int = 0, lim: int = 8):
    """Integer-valued (D, u) with entries in [-lim, lim].

    With lim = 8 and N <= 165 every product is at most 64 in magnitude and every
    partial sum stays below 2^24, so the contraction is exact in float32, float64
    and in bf16 x bf16 -> float32 tensor-core arithmetic, in any summation order.
    """
    rng = np.random.default_rng(seed)
    D = rng.integers(-lim, lim + 1, size=(F, N, N)).astype(np.float64)
    u = rng.integers(-lim, lim + 1, size=(E, N)).astype(np.float64)
    return _round(D, dtype), _round(u, dtype)


def fp64_single(seed: int = 0, E: int = 4096, N: int = 20):
    """FP64 single-operator problem: E=4096, N=20, F=1."""
    return operands(E, N, 1, np.float64, seed)


def fp32_three(seed: int = 0, E: int = 1 << 21, N: int = 35):
    """FP32 three-operator problem: E=2^21, N=35, F=3."""
    return operands(E, N, 3, np.float32, seed)


def precision_sweep(seed: int = 0, E: int = 1 << 20, N: int = 84):
    """Precision-sweep problem: E=2^20, N=84, F=4 (last operator SPD), u scaled by 10^k."""
    return operands(E, N, 4, np.float32, seed, spd_last=True, scale_exp=3.0)


def grouped_sizes(seed: int = 0, lo: float = 14.0, hi: float = 21.0):
    """[(N_g, E_g)] for the 8 uneven groups, E_g = floor(2^U(lo, hi)) drawn in N order."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=len(GROUP_NS))
    E = np.floor(2.0 ** x).astype(np.int64)
    return [(int(n), int(e)) for n, e in zip(GROUP_NS, E)]


def grouped_operands(sizes, F: int = 3, seed: int = 0, dtype=np.float32):
    """Per-group (D_g, u_g) for ``sizes`` = [(N_g, E_g)]; group g uses seed (seed, g)."""
    out = []
    for g, (n, e) in enumerate(sizes):
        D, u = operands(e, n, F, dtype, seed=[seed, g + 1])
        out.append((D, u))
    return out


PATHS = ("fp32", "bf16", "bf16x3")
LAYOUTS = ("elem", "node")


def picker_shapes(seed: int = 0, count: int = 600, e_lo: float = 12.0, e_hi: float = 23.0):
    """Random shapes for the learned variant picker.

    Returns a list of dicts {E, N, F, path, layout} with N ~ U{4..165},
    E = floor(2^U(e_lo, e_hi)), F ~ U{1..4}; for the full experiment the first 500
    train the model and the last 100 are held out.
    """
    rng = np.random.default_rng(seed)
    N = rng.integers(4, 166, size=count)
    E = np.floor(2.0 ** rng.uniform(e_lo, e_hi, size=count)).astype(np.int64)
    F = rng.integers(1, 5, size=count)
    p = rng.integers(0, len(PATHS), size=count)
    lay = rng.integers(0, len(LAYOUTS), size=count)
    return [dict(E=int(E[k]), N=int(N[k]), F=int(F[k]), path=PATHS[p[k]], layout=LAYOUTS[lay[k]])
            for k in range(count)]


def to_node_major(u: np.ndarray) -> np.ndarray:
    """u[e][j] -> u_nm[j][e] (same values, contiguous)."""
    return np.ascontiguousarray(u.T)
