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
    "tet_nodes",
    "surface_mesh",
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


def tet_nodes(order: int):
    """Nodes (a, b, c), a + b + c <= order, of a degree-`order` tetrahedron in lexicographic order,
    and its four faces' node lists (c = 0, b = 0, a = 0, a + b + c = order), each ascending."""
    nodes = [(a, b, c) for a in range(order + 1) for b in range(order + 1 - a) for c in range(order + 1 - a - b)]
    faces = [[k for k, (a, b, c) in enumerate(nodes) if cond(a, b, c)]
             for cond in (lambda a, b, c: c == 0, lambda a, b, c: b == 0, lambda a, b, c: a == 0,
                          lambda a, b, c: a + b + c == order)]
    return nodes, faces


def surface_mesh(E: int, order: int = 4, width: int = 64, seed: int = 0, dtype=np.float32):
    """Synthetic dG surface (lift) problem on E tetrahedra of degree `order` (N = 35 and 4 x 15
    face nodes for order 4).

    The elements form a periodic-free strip of columns: face 0 of element e meets face 1 of
    e + 1 (face nodes in reverse order), face 2 meets face 3 of e + width (same order); a face
    whose neighbour would fall outside [0, E) is a boundary face whose exterior trace is the
    element's own node (zero jump).  Returns (L, fmask, vmapP, s, u):
    L (N, 4 Nfp) ~ U[-1, 1); fmask (4 Nfp,) int32; vmapP (E, 4 Nfp) int32 into u.ravel();
    s (E, 4) ~ U[0.5, 2) per-face scale; u (E, N) ~ N(0, 1); drawn in the order L, s, u.
    """
    nodes, faces = tet_nodes(order)
    N, Nfp = len(nodes), len(faces[0])
    fmask = np.array([k for f in faces for k in f], dtype=np.int32)
    M = 4 * Nfp
    e = np.arange(E, dtype=np.int64)[:, None]
    p = np.arange(Nfp, dtype=np.int64)[None, :]
    vmapP = np.empty((E, M), dtype=np.int64)
    for f, (off, fn, rev) in enumerate(((1, 1, True), (-1, 0, True), (width, 3, False), (-width, 2, False))):
        nb = e + off
        q = (Nfp - 1 - p) if rev else p
        exterior = nb * N + fmask[fn * Nfp + q]
        interior = e * N + fmask[f * Nfp + p]
        inside = (nb >= 0) & (nb < E)
        vmapP[:, f * Nfp:(f + 1) * Nfp] = np.where(inside, exterior, interior)
    if E * N >= 2 ** 31:
        raise ValueError("vmapP holds int32 indices")
    rng = np.random.default_rng(seed)
    L = rng.uniform(-1.0, 1.0, size=(N, M))
    s = rng.uniform(0.5, 2.0, size=(E, 4))
    u = rng.standard_normal(size=(E, N))
    return _round(L, dtype), fmask, vmapP.astype(np.int32), _round(s, dtype), _round(u, dtype)


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
