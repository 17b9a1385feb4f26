"""Pins for the CPU FP64 oracle: checks against things other than the oracle itself.

Contraction (the loop domain + sum instruction of Section 2.1, dG FEM volume of
Table 1): hand-worked tables, numpy's einsum as an independent library routine,
closed forms (identity, permutation, rank one, zero), exact integer arithmetic,
linearity, and the layout change of Section 2.4.3 (node-major is the transpose).
A set of planted mistakes (transposed operand, dropped term, wrong sign, wrong
index) must each fail at least one of these checks.

bf16 rounding and split: torch's nearest-even bfloat16 conversion, hand values
at ties, and the exactness of the three-term split.

Cost model: a hand-worked network, central finite differences of the loss, and
Adam's closed form under a constant gradient.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- contraction

def _load_hand():
    with open(os.path.join(GOLDEN, "contract_hand.json")) as fh:
        return json.load(fh)["cases"]


def _pin_failures(fn):
    """Run every contraction pin against ``fn(D, u, layout)``; return failing pin names."""
    fails = []
    for case in _load_hand():
        D = np.array(case["D"], dtype=np.float64)
        u = np.array(case["u"], dtype=np.float64)
        if not np.array_equal(fn(D, u, "elem"), np.array(case["out"], dtype=np.float64)):
            fails.append("hand")
    rng = np.random.default_rng(11)
    E, N, F = 37, 9, 3
    D = rng.uniform(-1, 1, size=(F, N, N))
    u = rng.standard_normal((E, N))
    ref = np.einsum("fij,ej->fei", D, u)
    if not np.allclose(fn(D, u, "elem"), ref, rtol=1e-13, atol=1e-13):
        fails.append("einsum")
    I = np.broadcast_to(np.eye(N), (1, N, N))
    if not np.array_equal(fn(I, u, "elem")[0], u):
        fails.append("identity")
    perm = rng.permutation(N)
    P = np.zeros((1, N, N))
    P[0, np.arange(N), perm] = 1.0          # (P u)_i = u_{perm[i]}
    if not np.array_equal(fn(P, u, "elem")[0], u[:, perm]):
        fails.append("permutation")
    a = rng.standard_normal(N)
    b = rng.standard_normal(N)
    R1 = np.outer(a, b)[None]
    if not np.allclose(fn(R1, u, "elem")[0], (u @ b)[:, None] * a[None, :], rtol=1e-12, atol=1e-12):
        fails.append("rank_one")
    if np.any(fn(np.zeros((2, N, N)), u, "elem") != 0.0):
        fails.append("zero")
    Di = rng.integers(-8, 9, size=(F, N, N))
    ui = rng.integers(-8, 9, size=(E, N))
    exact = np.einsum("fij,ej->fei", Di.astype(np.int64), ui.astype(np.int64))
    if not np.array_equal(fn(Di.astype(np.float64), ui.astype(np.float64), "elem"), exact.astype(np.float64)):
        fails.append("integer_exact")
    v = rng.standard_normal((E, N))
    lhs = fn(D, 2.0 * u - 3.0 * v, "elem")
    rhs = 2.0 * fn(D, u, "elem") - 3.0 * fn(D, v, "elem")
    if not np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12):
        fails.append("linear_u")
    if not np.array_equal(fn(D, np.ascontiguousarray(u.T), "node"),
                          np.ascontiguousarray(fn(D, u, "elem").transpose(0, 2, 1))):
        fails.append("node_major")
    return fails


def test_oracle_passes_every_pin():
    assert _pin_failures(oracle.contract) == []


def _mutant(kind):
    def fn(D, u, layout):
        D = np.asarray(D, dtype=np.float64)
        u = np.asarray(u, dtype=np.float64)
        if layout == "node":
            u = u.T
        F, N, _ = D.shape
        E = u.shape[0]
        out = np.zeros((F, E, N))
        for f in range(F):
            for e in range(E):
                for i in range(N):
                    acc = 0.0
                    jr = range(N - 1) if kind == "drop_last_term" else range(N)
                    for j in jr:
                        d = D[f, j, i] if kind == "transpose_D" else D[f, i, j]
                        x = u[e, i] if kind == "u_index_i" else u[e, j]
                        acc = acc - d * x if (kind == "sign" and j == N - 1) else acc + d * x
                    out[f, e, i] = acc
        if layout == "node":
            out = out.transpose(0, 2, 1)
        return out
    return fn


@pytest.mark.parametrize("kind", ["transpose_D", "drop_last_term", "sign", "u_index_i"])
def test_pins_catch_planted_mistakes(kind):
    assert _pin_failures(_mutant(kind)), f"no pin caught the planted mistake {kind}"


def test_correct_python_loop_nest_passes_pins():
    # The same loop nest without a planted mistake passes, so the mutants fail for their mistake.
    assert _pin_failures(_mutant("none")) == []


def test_empty_and_degenerate_shapes():
    D = np.ones((2, 3, 3))
    assert oracle.contract(D, np.zeros((0, 3))).shape == (2, 0, 3)
    assert oracle.contract(D, np.zeros((3, 0)), "node").shape == (2, 3, 0)
    out = oracle.contract(np.full((1, 1, 1), 3.0), np.array([[2.0], [-1.0]]))
    assert np.array_equal(out, np.array([[[6.0], [-3.0]]]))


def test_contract_rows_matches_full():
    D, u = synth.operands(300, 7, 2, np.float32, seed=3)
    rows = np.array([0, 5, 299, 17])
    full = oracle.contract(D, u)
    assert np.array_equal(oracle.contract_rows(D, u, rows), full[:, rows, :])
    unm = synth.to_node_major(u)
    assert np.array_equal(oracle.contract_rows(D, unm, rows, "node"), full[:, rows, :])


def test_threads_do_not_change_result():
    D, u = synth.operands(1000, 13, 3, np.float32, seed=4)
    assert np.array_equal(oracle.contract(D, u, threads=1), oracle.contract(D, u, threads=4))


def test_rel_fro_error_closed_form():
    ref = np.array([3.0, 4.0])
    assert oracle.rel_fro_error(ref, ref) == 0.0
    assert abs(oracle.rel_fro_error(ref + np.array([0.3, 0.4]), ref) - 0.1) < 1e-15


# ------------------------------------------------------------------ bf16 pins

def test_bf16_round_matches_torch_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32),
        (rng.standard_normal(2000) * 1e-30).astype(np.float32),
        (rng.standard_normal(2000) * 1e30).astype(np.float32),
        np.array([0.0, -0.0, 1.0, np.float32(3.4e38), 1e-45, -1e-40, np.inf, -np.inf], np.float32),
    ])
    # exact ties: upper half even and odd, lower half 0x8000
    bits = rng.integers(0, 1 << 15, size=4000, dtype=np.uint32) << 16 | 0x8000
    bits |= rng.integers(0x30, 0x4f, size=4000, dtype=np.uint32) << 24
    x = np.concatenate([x, bits.view(np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.bf16_round(x), ref, equal_nan=True)


def test_bf16_round_hand_values():
    one = np.float32(1.0)
    x = np.array([one + np.float32(2.0 ** -8),        # tie between 1 and 1+2^-7 -> even (1)
                  one + np.float32(3 * 2.0 ** -8),    # tie between 1+2^-7 and 1+2^-6 -> even (1+2^-6)
                  one + np.float32(2.0 ** -8 + 2.0 ** -20),  # just above the tie -> up
                  np.float32(-1.5)], dtype=np.float32)
    y = oracle.bf16_round(x)
    assert y.tolist() == [1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -1.5]


def test_bf16_split3_exact_and_terms_are_bf16():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    x = (rng.standard_normal(50000) * 10.0 ** rng.uniform(-6, 6, 50000)).astype(np.float32)
    hi, mid, lo = oracle.bf16_split3(x)
    assert np.array_equal(hi.astype(np.float64) + mid + lo, x.astype(np.float64))
    for t in (hi, mid, lo):
        assert np.array_equal(oracle.bf16_round(t), t)
    # the same split through torch's conversion (differences are exact in float32)
    tx = torch.from_numpy(x)
    th = tx.to(torch.bfloat16).float()
    tm = (tx - th).to(torch.bfloat16).float()
    tl = (tx - th - tm).to(torch.bfloat16).float()
    assert np.array_equal(th.numpy(), hi) and np.array_equal(tm.numpy(), mid) and np.array_equal(tl.numpy(), lo)
    # magnitudes fall by at least 2^8 per term
    nz = hi != 0
    assert np.all(np.abs(mid[nz]) <= np.abs(hi[nz]) * 2.0 ** -8)


def test_bf16x3_all_nine_products_equal_exact_contraction():
    D, u = synth.operands(200, 11, 2, np.float32, seed=7, scale_exp=3.0)
    allpairs = [(a, b) for a in range(3) for b in range(3)]
    full = oracle.contract_bf16x3(D, u, pairs=allpairs)
    ref = oracle.contract(D, u)
    assert oracle.rel_fro_error(full, ref) < 1e-15
    kept = oracle.contract_bf16x3(D, u)
    assert oracle.rel_fro_error(kept, ref) < 2.0 ** -22
    plain = oracle.contract_bf16(D, u)
    err = oracle.rel_fro_error(plain, ref)
    assert 1e-4 < err < 1e-2   # bf16 operand rounding shows up at about 2^-8


def _bf16_pin_failures(fn):
    """Check ``fn(D, u)`` (the plain BF16 path's target) against a route that shares no
    code with the oracle: torch's nearest-even bfloat16 conversion of BOTH operands, then
    numpy's einsum in float64.  Returns the failing check names."""
    torch = pytest.importorskip("torch")
    fails = []
    for seed, scale in ((21, None), (22, 3.0)):
        D, u = synth.operands(97, 13, 3, np.float32, seed=seed, scale_exp=scale)
        Db = torch.from_numpy(D).to(torch.bfloat16).double().numpy()
        ub = torch.from_numpy(u).to(torch.bfloat16).double().numpy()
        want = np.einsum("fij,ej->fei", Db, ub)
        got = np.asarray(fn(D, u), dtype=np.float64)
        # products of bfloat16 values are exact in float64; two summation orders of
        # N = 13 terms differ by at most 2 N 2^-53 sum_j |D_ij u_j|
        den = np.einsum("fij,ej->fei", np.abs(Db), np.abs(ub))
        if got.shape != want.shape or not np.all(np.abs(got - want) <= 2 * 13 * 2.0 ** -53 * den):
            fails.append(f"torch_bf16_einsum_seed{seed}")
    return fails


def test_contract_bf16_matches_torch_rounding_and_einsum():
    assert _bf16_pin_failures(oracle.contract_bf16) == []


@pytest.mark.parametrize("kind", ["round_u_only", "round_D_only", "round_neither", "truncate"])
def test_bf16_pin_catches_planted_mistakes(kind):
    def chop(x):  # round toward zero to bfloat16 (a plausible wrong rounding mode)
        b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32) & np.uint32(0xFFFF0000)
        return b.view(np.float32)

    def fn(D, u):
        if kind == "round_u_only":
            return oracle.contract(D, oracle.bf16_round(u))
        if kind == "round_D_only":
            return oracle.contract(oracle.bf16_round(D), u)
        if kind == "round_neither":
            return oracle.contract(D, u)
        return oracle.contract(chop(D), chop(u))
    assert _bf16_pin_failures(fn), f"the bf16 pin missed the planted mistake {kind}"


def test_integer_inputs_are_bf16_exact():
    D, u = synth.integer_operands(64, 33, 2, seed=8)
    ref = oracle.contract(D, u)
    assert np.array_equal(oracle.contract_bf16(D, u), ref)
    assert np.array_equal(oracle.contract_bf16x3(D, u), ref)


# --------------------------------------------------------------- MLP pins

def test_mlp_hand_network():
    with open(os.path.join(GOLDEN, "mlp_hand.json")) as fh:
        g = json.load(fh)
    pr = g["params"]
    p = np.array([pr[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")])
    assert oracle.mlp_param_count(1, 1) == 8
    x = np.array([[c["x"]] for c in g["cases"]])
    y = oracle.mlp_forward(p, x, H=1)
    assert y.tolist() == [c["y"] for c in g["cases"]]
    gc = g["grad_case"]
    loss, grad = oracle.mlp_loss_grad(p, np.array([[gc["x"]]]), np.array([gc["t"]]), H=1)
    assert loss == gc["loss"]
    want = np.array([gc["grad"][k] for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")])
    assert np.array_equal(grad, want)


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(9)
    din, H, B = 6, 64, 16
    n = oracle.mlp_param_count(din, H)
    assert n == H * din + H + 2 * (H * H + H) + H + 1
    p = rng.uniform(-1, 1, n) * np.sqrt(6.0 / 64)
    x = rng.standard_normal((B, din))
    t = rng.standard_normal(B)
    loss, g = oracle.mlp_loss_grad(p, x, t)
    assert abs(loss - np.mean((oracle.mlp_forward(p, x) - t) ** 2)) < 1e-12
    idx = rng.choice(n, 200, replace=False)
    h = 1e-6
    fd = np.empty(idx.size)
    for k, q in enumerate(idx):
        pp = p.copy(); pp[q] += h
        pm = p.copy(); pm[q] -= h
        fd[k] = (oracle.mlp_loss_grad(pp, x, t)[0] - oracle.mlp_loss_grad(pm, x, t)[0]) / (2 * h)
    assert np.linalg.norm(fd - g[idx]) / np.linalg.norm(g[idx]) < 1e-6


def test_adam_constant_gradient_closed_form():
    # With a constant gradient the bias-corrected moments are g and g^2 exactly,
    # so every step moves p by lr * g / (|g| + eps).
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.zeros(4); m = np.zeros(4); v = np.zeros(4)
    lr, eps = 1e-3, 1e-8
    for t in range(1, 6):
        oracle.adam_step(p, g, m, v, t, lr=lr, eps=eps)
    want = -5 * lr * g / (np.abs(g) + eps)
    assert np.allclose(p, want, rtol=1e-9, atol=1e-15)


# ------------------------------------------------- geometric-factor volume derivative

def _geo_pin_failures(fn):
    """Pins of out[d,e,i] = sum_f r[e,d,f] sum_j D[f,i,j] u[e,j] against ``fn(D, u, r, layout)``."""
    fails = []
    with open(os.path.join(GOLDEN, "contract_geo_hand.json")) as fh:
        g = json.load(fh)
    if not np.array_equal(fn(np.array(g["D"], float), np.array(g["u"], float), np.array(g["r"], float), "elem"),
                          np.array(g["out"], float)):
        fails.append("hand")
    rng = np.random.default_rng(31)
    E, N, F, Dd = 23, 7, 3, 2
    D = rng.uniform(-1, 1, size=(F, N, N))
    u = rng.standard_normal((E, N))
    r = rng.standard_normal((E, Dd, F))
    if not np.allclose(fn(D, u, r, "elem"), np.einsum("edf,fij,ej->dei", r, D, u), rtol=1e-13, atol=1e-13):
        fails.append("einsum")
    # r = identity per element (Dd = F): the plain contraction, exactly
    I = np.broadcast_to(np.eye(F), (E, F, F)).copy()
    if not np.array_equal(fn(D, u, I, "elem"), oracle.contract(D, u)):
        fails.append("identity_factors")
    # r[e,d,f] = c_f for d = 0 and 0 otherwise: one weighted sum of the contractions
    c = rng.standard_normal(F)
    rc = np.zeros((E, Dd, F))
    rc[:, 0, :] = c
    want = np.einsum("f,fei->ei", c, oracle.contract(D, u))
    got = fn(D, u, rc, "elem")
    if not (np.allclose(got[0], want, rtol=1e-13, atol=1e-13) and np.all(got[1] == 0)):
        fails.append("weighted_sum")
    # linear in r
    r2 = rng.standard_normal((E, Dd, F))
    if not np.allclose(fn(D, u, 2 * r - 0.5 * r2, "elem"), 2 * fn(D, u, r, "elem") - 0.5 * fn(D, u, r2, "elem"),
                       rtol=1e-12, atol=1e-12):
        fails.append("linear_r")
    # integer-valued inputs: exact
    Di, ui, ri = rng.integers(-4, 5, (F, N, N)), rng.integers(-4, 5, (E, N)), rng.integers(-3, 4, (E, Dd, F))
    if not np.array_equal(fn(Di.astype(float), ui.astype(float), ri.astype(float), "elem"),
                          np.einsum("edf,fij,ej->dei", ri, Di, ui).astype(float)):
        fails.append("integer_exact")
    # node-major layout: the transposes
    got_n = fn(D, np.ascontiguousarray(u.T), np.ascontiguousarray(r.transpose(1, 2, 0)), "node")
    if not np.array_equal(got_n, np.ascontiguousarray(fn(D, u, r, "elem").transpose(0, 2, 1))):
        fails.append("node_major")
    return fails


def test_contract_geo_passes_every_pin():
    assert _geo_pin_failures(oracle.contract_geo) == []


@pytest.mark.parametrize("kind", ["transpose_r", "drop_last_f", "transpose_D", "none"])
def test_geo_pins_catch_planted_mistakes(kind):
    def fn(D, u, r, layout):
        if layout == "node":
            u, r = u.T, r.transpose(2, 0, 1)
        F, N, _ = D.shape
        E, Dd, _ = r.shape
        out = np.zeros((Dd, E, N))
        for d in range(Dd):
            for e in range(E):
                for i in range(N):
                    acc = 0.0
                    for f in range(F - 1 if kind == "drop_last_f" else F):
                        part = sum((D[f, j, i] if kind == "transpose_D" else D[f, i, j]) * u[e, j] for j in range(N))
                        g = r[e, f, d] if (kind == "transpose_r" and f < Dd and d < F) else r[e, d, f]
                        acc += g * part
                    out[d, e, i] = acc
        return out.transpose(0, 2, 1).copy() if layout == "node" else out
    fails = _geo_pin_failures(fn)
    if kind == "none":
        assert fails == []
    else:
        assert fails, f"no pin caught the planted mistake {kind}"


def test_contract_geo_rows_matches_full():
    D, u = synth.operands(90, 6, 3, np.float32, seed=8)
    r = np.random.default_rng(2).standard_normal((90, 3, 3)).astype(np.float32)
    rows = np.array([0, 89, 41])
    full = oracle.contract_geo(D, u, r)
    assert np.array_equal(oracle.contract_geo_rows(D, u, r, rows), full[:, rows, :])
    rn = np.ascontiguousarray(r.transpose(1, 2, 0))
    assert np.array_equal(oracle.contract_geo_rows(D, synth.to_node_major(u), rn, rows, "node"), full[:, rows, :])


# ------------------------------------------------------------------- dG surface lift

def _lift_pin_failures(fn):
    """Pins of out[e,i] = sum_m L[i,m] s[e,m//Nfp] (u[e,fmask[m]] - u.flat[vmapP[e,m]]) against
    ``fn(L, fmask, vmapP, s, u)``."""
    fails = []
    with open(os.path.join(GOLDEN, "lift_hand.json")) as fh:
        g = json.load(fh)
    got = fn(np.array(g["L"], float), np.array(g["fmask"]), np.array(g["vmapP"]), np.array(g["s"], float),
             np.array(g["u"], float))
    if not np.array_equal(got, np.array(g["out"], float)):
        fails.append("hand")
    L, fmask, vmapP, s, u = synth.surface_mesh(300, order=2, width=8, seed=3, dtype=np.float64)
    E, N = u.shape
    Nfp = fmask.size // 4
    jump = u[:, fmask] - u.ravel()[vmapP]
    want = (np.repeat(s, Nfp, axis=1) * jump) @ L.T
    if not np.allclose(fn(L, fmask, vmapP, s, u), want, rtol=1e-13, atol=1e-13):
        fails.append("einsum")
    own = (np.arange(E)[:, None] * N + fmask[None, :]).astype(np.int32)  # every face a boundary face
    if np.any(fn(L, fmask, own, s, u) != 0.0):
        fails.append("boundary_zero")
    v = np.random.default_rng(1).standard_normal(u.shape)
    if not np.allclose(fn(L, fmask, vmapP, s, 2 * u - v), 2 * fn(L, fmask, vmapP, s, u) - fn(L, fmask, vmapP, s, v),
                       rtol=1e-12, atol=1e-12):
        fails.append("linear_u")
    # a constant field has no jumps anywhere
    if np.any(fn(L, fmask, vmapP, s, np.full(u.shape, 3.25)) != 0.0):
        fails.append("constant_field")
    Li = np.random.default_rng(2).integers(-3, 4, L.shape).astype(float)
    si = np.random.default_rng(3).integers(1, 4, s.shape).astype(float)
    ui = np.random.default_rng(4).integers(-8, 9, u.shape).astype(float)
    wanti = (np.repeat(si, Nfp, axis=1) * (ui[:, fmask] - ui.ravel()[vmapP])) @ Li.T
    if not np.array_equal(fn(Li, fmask, vmapP, si, ui), wanti):
        fails.append("integer_exact")
    return fails


def test_lift_passes_every_pin():
    assert _lift_pin_failures(oracle.lift) == []


@pytest.mark.parametrize("kind", ["sign", "face_index", "transpose_L", "none"])
def test_lift_pins_catch_planted_mistakes(kind):
    def fn(L, fmask, vmapP, s, u):
        E, N = u.shape
        M = L.shape[1]
        Nf = s.shape[1]
        Nfp = M // Nf
        uf = u.ravel()
        out = np.zeros((E, N))
        for e in range(E):
            for m in range(M):
                jump = u[e, fmask[m]] - uf[vmapP[e, m]]
                if kind == "sign":
                    jump = -jump
                f = m % Nf if kind == "face_index" else m // Nfp
                flux = s[e, f] * jump
                for i in range(N):
                    lim = L[m % N, (i * Nfp + m) % M] if kind == "transpose_L" else L[i, m]
                    out[e, i] += lim * flux
        return out
    fails = _lift_pin_failures(fn)
    assert (fails == []) if kind == "none" else fails, kind


def test_surface_mesh_is_consistent():
    """Every interior face-node pair is matched both ways; boundary faces point at the element."""
    L, fmask, vmapP, s, u = synth.surface_mesh(500, order=4, width=16, seed=0)
    E, N = u.shape
    M = fmask.size
    assert N == 35 and M == 60
    src = (np.arange(E)[:, None] * N + fmask[None, :]).ravel()
    dst = vmapP.ravel().astype(np.int64)
    pairs = set(zip(src.tolist(), dst.tolist()))
    for a, b in list(pairs)[:5000]:
        assert (b, a) in pairs or a == b
    nodes, faces = synth.tet_nodes(4)
    assert all(len(f) == 15 for f in faces) and len(nodes) == 35
