"""Learned variant picker: features, exhaustive-autotuning data, MLP training and regret.

The paper's premise (Section 1) is that the controlling program picks the code
transformations per target and per workload. Here the choice is made two ways:
  * exhaustively: lc_autotune times every valid descriptor (the judge of regret);
  * by a small MLP cost model (3 hidden ReLU layers of 64) that predicts log run time
    from problem and descriptor features; its training and inference run in the
    library's own CUDA kernels (lc_mlp_loss_grad, lc_mlp_adam_step, lc_mlp_forward); an
    ensemble of three such networks, trained apart, averages their predictions.

regret(shape) = t(picked) / t(best) - 1, where best is the exhaustive autotuner's winner;
on held-out shapes the pick, the best and the default descriptor are re-timed together in
a fresh interleaved pass (a pick equal to the best has regret 0; a re-timed pick faster
than the best counts as 0).  Features and the pick itself are the library's
(lc_variant_features, lc_pick_variant): this module only collects timings, trains the
network with the library's kernels and reports.

Running ``python -m paper_1405_7470_gb300.picker --out results.json`` on a GPU runs the
whole experiment on the 600 seeded shapes (first 500 train, last 100 held out).
Training: three networks (seeds 0, 1, 2), each Adam, 1000 epochs of 512-sample
minibatches, learning rate 3e-3 decayed on a cosine schedule.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import lc

PATHS = ("fp32", "bf16", "bf16x3")
LAYOUTS = ("elem", "node")
DIN = 32  # feature count (the library's limit)


def features(shape: dict, v) -> np.ndarray:
    """The cost model's inputs for (problem, descriptor): lc_variant_features (the same code
    lc_pick_variant uses); every entry is O(1)."""
    vv = _variant_from_dict(v) if isinstance(v, dict) else v
    return lc.variant_features(kernel_for(shape["F"]), shape["E"], shape["N"], shape["F"], shape["layout"],
                               shape["path"], vv)


_KERNELS = {}


def kernel_for(F: int):
    """One kernel handle per operator count (the single-operator form for F = 1)."""
    if F not in _KERNELS:
        _KERNELS[F] = lc.Kernel() if F > 1 else lc.Kernel("{ [e,i,j]: 0<=e<E and 0<=i,j<N }",
                                                          "out[e,i] = sum(j, D[i,j]*u[e,j])")
    return _KERNELS[F]


def _variant_from_dict(d: dict):
    return lc.Variant(**d)


def he_uniform(din: int, seed: int) -> np.ndarray:
    """Initial parameters: He-uniform weights U(-sqrt(6/fan_in), +), zero biases."""
    rng = np.random.default_rng(seed)
    H = 64
    parts = [rng.uniform(-1, 1, H * din) * math.sqrt(6.0 / din), np.zeros(H),
             rng.uniform(-1, 1, H * H) * math.sqrt(6.0 / H), np.zeros(H),
             rng.uniform(-1, 1, H * H) * math.sqrt(6.0 / H), np.zeros(H),
             rng.uniform(-1, 1, H) * math.sqrt(6.0 / H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


class ProblemPool:
    """Device buffers reused across shapes (sized for the largest one); seeded data."""

    def __init__(self, max_u: int, max_out: int, max_d: int):
        import torch
        self.u = torch.empty(max_u, dtype=torch.float32, device="cuda")
        self.out = torch.empty(max_out, dtype=torch.float32, device="cuda")
        self.D = torch.empty(max_d, dtype=torch.float32, device="cuda")

    def problem(self, shape: dict, seed: int):
        import torch
        E, N, F = shape["E"], shape["N"], shape["F"]
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        u = self.u[:E * N]
        u.normal_(generator=g)
        D = self.D[:F * N * N]
        D.uniform_(-1, 1, generator=g)
        out = self.out[:F * E * N]
        if shape["layout"] == "node":
            return D.view(F, N, N), u.view(N, E), out.view(F, N, E)
        return D.view(F, N, N), u.view(E, N), out.view(F, E, N)


def collect(shapes, reps: int = 3, seed: int = 0, log=None):
    """Autotune every shape; returns per-shape records with all candidate timings."""
    import torch
    kernel = lc.Kernel()
    max_u = max(s["E"] * s["N"] for s in shapes)
    max_out = max(s["E"] * s["N"] * s["F"] for s in shapes)
    max_d = max(s["F"] * s["N"] ** 2 for s in shapes)
    pool = ProblemPool(max_u, max_out, max_d)
    stream = torch.cuda.Stream()
    recs = []
    for k, sh in enumerate(shapes):
        D, u, out = pool.problem(sh, seed * 100003 + k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            res = lc.autotune(kernel, D, u, out, sh["layout"], sh["path"], reps=reps, stream=stream)
        tune_s = time.perf_counter() - t0
        vd = lc.variant_default(kernel, sh["E"], sh["N"], sh["F"], sh["layout"], sh["path"])
        # the default descriptor, timed the same way
        with torch.cuda.stream(stream):
            for _ in range(1):
                lc.contract(kernel, vd, D, u, out, stream=stream)
            ts = []
            for _ in range(reps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lc.contract(kernel, vd, D, u, out, stream=stream)
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
        recs.append(dict(shape=sh, cands=[(ms, lc.variant_dict(v)) for ms, v in res], tune_s=tune_s,
                         default=(float(np.median(ts)), lc.variant_dict(vd))))
        if log and k % 50 == 0:
            log(f"shape {k}: {sh} best {res[0][0]:.4f} ms of {len(res)} candidates ({tune_s:.2f} s)")
    if lc.device_error() != 0:
        raise RuntimeError("device error word set during autotuning")
    return recs


def dataset(recs):
    X, y = [], []
    for r in recs:
        for ms, vd in r["cands"]:
            X.append(features(r["shape"], vd))
            y.append(math.log(max(ms, 1e-4)))
    return np.stack(X), np.asarray(y, dtype=np.float32)


def train(X: np.ndarray, y: np.ndarray, epochs: int = 1000, batch: int = 512, lr: float = 3e-3, seed: int = 0,
          log=None):
    """Adam on the library's MLP kernels with a cosine-decayed learning rate (epoch e uses
    lr * (1 + cos(pi e / epochs)) / 2); returns (params tensor, loss history)."""
    import torch
    n, din = X.shape
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    params = torch.from_numpy(he_uniform(din, seed)).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    import ctypes
    wsb = ctypes.c_size_t(0)
    lc.check(lc.load().lc_mlp_workspace_size(din, ctypes.byref(wsb)), "lc_mlp_workspace_size")
    ws = torch.empty(wsb.value // 4 + 4, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    step, hist = 0, []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        lr_ep = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            xb, yb = Xd.index_select(0, idx), yd.index_select(0, idx)
            loss, grad = lc.mlp_loss_grad(params, xb, yb, workspace=ws)
            step += 1
            lc.mlp_adam_step(params, grad, m, v, step, lr=lr_ep)
        if ep % 100 == 0 or ep == epochs - 1:
            full, _ = lc.mlp_loss_grad(params, Xd, yd)
            hist.append((ep, float(full)))
            if log:
                log(f"epoch {ep}: train mse(log t) {float(full):.4f}")
    return params, hist


def train_ensemble(X: np.ndarray, y: np.ndarray, models: int = 3, epochs: int = 1000, seed: int = 0, log=None,
                   **kw):
    """`models` networks trained apart (seeds seed, seed + 1, ...: initialisation and minibatch
    order); returns (params [models][P], loss histories)."""
    import torch
    ps, hs = [], []
    for q in range(models):
        p, h = train(X, y, epochs=epochs, seed=seed + q, log=log, **kw)
        ps.append(p)
        hs.append(h)
    return torch.stack(ps), hs


def pick(params, shape: dict, workspace=None):
    """The trained network's (or ensemble's, params [models][P]) descriptor for a shape, chosen
    by the library (lc_pick_variant / lc_pick_variant_ensemble)."""
    v, _ = lc.pick_variant(kernel_for(shape["F"]), shape["E"], shape["N"], shape["F"], shape["layout"],
                           shape["path"], params, workspace=workspace)
    return lc.variant_dict(v)


def regret_stats(r):
    r = np.asarray(r)
    return dict(geomean=float(np.exp(np.mean(np.log1p(r))) - 1), median=float(np.median(r)),
                p90=float(np.percentile(r, 90)), max=float(np.max(r)), mean=float(np.mean(r)))


def retime(pool, shape: dict, seed: int, variants, reps: int = 5, rounds: int = 3, stream=None):
    """Fresh timings of several descriptors on one problem: `rounds` interleaved passes over
    the descriptors, each the median of `reps` CUDA-event-timed launches after a warm-up;
    returns each descriptor's median over the rounds (ms)."""
    import torch
    kernel = kernel_for(shape["F"])
    D, u, out = pool.problem(shape, seed)
    stream = stream or torch.cuda.Stream()
    vs = [_variant_from_dict(d) for d in variants]
    times = [[] for _ in vs]
    with torch.cuda.stream(stream):
        for v in vs:
            lc.contract(kernel, v, D, u, out, stream=stream)
        for _ in range(rounds):
            for q, v in enumerate(vs):
                ts = []
                for _ in range(reps):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    lc.contract(kernel, v, D, u, out, stream=stream)
                    b.record(stream)
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                times[q].append(float(np.median(ts)))
    return [float(np.median(t)) for t in times]


def evaluate(params, recs, pool=None, seeds=None, reps: int = 5, rounds: int = 3):
    """Regret of the network's pick and of the default descriptor against the exhaustive best.

    With `pool` (and each record's problem seed in `seeds`) the pick, the best and the
    default are re-timed together on the same problem; otherwise the autotuning pass's times
    are used.  A pick equal to the best has regret 0; re-timed regrets are clamped at 0."""
    mlp, dflt, pick_s, same = [], [], [], 0
    ws = None
    for k, rec in enumerate(recs):
        best_v = rec["cands"][0][1]
        t0 = time.perf_counter()
        pv = pick(params, rec["shape"], workspace=ws)
        pick_s.append(time.perf_counter() - t0)
        dv = rec["default"][1]
        if pool is None:
            tbl = {json.dumps(vd, sort_keys=True): ms for ms, vd in rec["cands"]}
            t_best = rec["cands"][0][0]
            t_pick = tbl.get(json.dumps(pv, sort_keys=True), float("nan"))
            t_def = rec["default"][0]
        else:
            t_pick, t_best, t_def = retime(pool, rec["shape"], seeds[k], [pv, best_v, dv], reps=reps, rounds=rounds)
        same += pv == best_v
        mlp.append(0.0 if pv == best_v else max(t_pick / t_best - 1.0, 0.0))
        dflt.append(0.0 if dv == best_v else max(t_def / t_best - 1.0, 0.0))
    return dict(mlp=regret_stats(mlp), default=regret_stats(dflt), pick_wall_s_mean=float(np.mean(pick_s)),
                picks_equal_best=same, shapes=len(recs), mlp_per_shape=mlp, default_per_shape=dflt,
                retimed=pool is not None)


def by_path(recs, ev):
    """Held-out regrets grouped by the requested path; reduced-precision requests that the
    library serves with FP32 kernels (no tensor-core candidate) form their own groups."""
    groups = {}
    for rec, m, d in zip(recs, ev["mlp_per_shape"], ev["default_per_shape"]):
        path = rec["shape"]["path"]
        tensor = any(v.get("engine") == "tcgen05" for _, v in rec["cands"])
        key = path if (path == "fp32" or tensor) else path + " served by FP32"
        g = groups.setdefault(key, ([], []))
        g[0].append(m)
        g[1].append(d)
    return {k: dict(shapes=len(m), mlp=regret_stats(m), default=regret_stats(d)) for k, (m, d) in groups.items()}


def make_pool(shapes):
    return ProblemPool(max(s["E"] * s["N"] for s in shapes), max(s["E"] * s["N"] * s["F"] for s in shapes),
                       max(s["F"] * s["N"] ** 2 for s in shapes))


def run_experiment(out_path: str, n_shapes: int = 600, n_train: int = 500, reps: int = 3, epochs: int = 1000,
                   seed: int = 0, models: int = 3):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    log = lambda s: print(s, flush=True)
    shapes = synth.picker_shapes(seed, n_shapes)
    t0 = time.perf_counter()
    recs = collect(shapes, reps=reps, seed=seed, log=log)
    tune_total = time.perf_counter() - t0
    tr, te = recs[:n_train], recs[n_train:]
    X, y = dataset(tr)
    t1 = time.perf_counter()
    params, hists = train_ensemble(X, y, models=models, epochs=epochs, seed=seed, log=log)
    hist = hists[0]
    train_s = time.perf_counter() - t1
    pool = make_pool(shapes[n_train:])
    t2 = time.perf_counter()
    ev_te = evaluate(params, te, pool=pool, seeds=[seed * 100003 + k for k in range(n_train, n_shapes)])
    retime_s = time.perf_counter() - t2
    ev_te_pass = evaluate(params, te)
    ev_tr = evaluate(params, tr)
    res = dict(n_shapes=n_shapes, n_train=n_train, samples=int(len(y)), epochs=epochs, models=models,
               autotune_wall_s=tune_total, autotune_wall_s_per_shape=float(np.mean([r["tune_s"] for r in recs])),
               train_wall_s=train_s, retime_wall_s=retime_s, loss_history=hist, heldout=ev_te,
               heldout_by_path=by_path(te, ev_te),
               heldout_from_tuning_pass=dict(mlp=ev_te_pass["mlp"], default=ev_te_pass["default"]),
               train_fit=dict(mlp=ev_tr["mlp"]),
               candidates_per_shape=float(np.mean([len(r["cands"]) for r in recs])))
    with open(out_path, "w") as fh:
        json.dump(dict(summary=res, records=recs), fh)
    log(json.dumps({k: v for k, v in res.items() if k not in ("loss_history",)}, default=str)[:3000])
    return res


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="picker_results.json")
    ap.add_argument("--shapes", type=int, default=600)
    ap.add_argument("--train", type=int, default=500)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=1000)
    ap.add_argument("--models", type=int, default=3)
    a = ap.parse_args()
    lc.load()
    run_experiment(a.out, a.shapes, a.train, a.reps, a.epochs, models=a.models)
