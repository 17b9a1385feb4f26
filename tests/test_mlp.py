"""Cost-model network: the library's CUDA forward / backward / Adam kernels against the
CPU FP64 oracle (which is itself pinned by finite differences and closed forms), and
the picker's host-side feature code."""

import numpy as np
import pytest

import oracle
import synth
from paper_1405_7470_gb300 import picker


def test_features_are_deterministic_and_bounded():
    sh = dict(E=1 << 21, N=35, F=3, path="bf16x3", layout="elem")
    v = dict(engine="tcgen05", layout="elem", precision="bf16x3", tile_e=128, elems_per_thread=1, split_i=0,
             unroll=2, prefetch_smem=1, tail_free=0, stages=3, ctas_per_sm=0, out_buffers=0)
    x = picker.features(sh, v)
    assert x.shape == (picker.DIN,) and x.dtype == np.float32
    assert np.array_equal(x, picker.features(sh, v))
    assert np.all(np.abs(x) <= 2.0)
    from paper_1405_7470_gb300 import lc
    for s in synth.picker_shapes(0, 50):
        for c in lc.enumerate_variants(picker.kernel_for(s["F"]), s["E"], s["N"], s["F"], s["layout"], s["path"]):
            x = picker.features(s, c)
            assert np.all(np.isfinite(x)) and np.all(np.abs(np.delete(x, 27)) <= 4.0)  # 27: column blocks / 8
    # a descriptor that is not valid for the problem has no features
    with pytest.raises(lc.LcError):
        picker.features(dict(E=1000, N=300, F=3, path="bf16x3", layout="elem"), v)


def test_he_uniform_init_is_seeded():
    a, b = picker.he_uniform(24, 3), picker.he_uniform(24, 3)
    assert np.array_equal(a, b) and a.size == oracle.mlp_param_count(24)
    assert not np.array_equal(a, picker.he_uniform(24, 4))


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


def _problem(seed, n=300, din=24):
    rng = np.random.default_rng(seed)
    p = picker.he_uniform(din, seed) + rng.normal(0, 0.05, oracle.mlp_param_count(din)).astype(np.float32)
    X = rng.uniform(-1, 1, (n, din)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    return p, X, t


@pytest.mark.gpu
def test_forward_matches_oracle(lc):
    import torch
    p, X, _ = _problem(1)
    y = lc.mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    ref = oracle.mlp_forward(p, X)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.gpu
def test_loss_gradient_matches_oracle(lc):
    import torch
    for seed, n, din in ((2, 300, 24), (3, 7, 5), (4, 1, 32)):
        p, X, t = _problem(seed, n, din)
        loss, g = lc.mlp_loss_grad(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
        rl, rg = oracle.mlp_loss_grad(p, X, t)
        assert abs(float(loss) - rl) / rl < 1e-5
        g = g.cpu().numpy()
        assert np.linalg.norm(g - rg) / np.linalg.norm(rg) < 1e-4


@pytest.mark.gpu
def test_adam_step_matches_oracle(lc):
    import torch
    rng = np.random.default_rng(5)
    n = 5000
    p = rng.normal(size=n)
    m = rng.normal(size=n) * 0.1
    v = np.abs(rng.normal(size=n)) * 0.01
    g = rng.normal(size=n)
    pd, md, vd, gd = (torch.from_numpy(a.astype(np.float32)).cuda() for a in (p, m, v, g))
    lc.mlp_adam_step(pd, gd, md, vd, 7, lr=1e-3)
    oracle.adam_step(p, g, m, v, 7, lr=1e-3)
    assert np.allclose(pd.cpu().numpy(), p, rtol=1e-5, atol=1e-6)
    assert np.allclose(md.cpu().numpy(), m, rtol=1e-5, atol=1e-6)


@pytest.mark.gpu
def test_training_fits_a_smooth_target(lc):
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, (4000, 24)).astype(np.float32)
    y = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * np.abs(X[:, 3])).astype(np.float32)
    params, hist = picker.train(X, y, epochs=60, batch=256, lr=3e-3, seed=1)
    assert hist[-1][1] < 0.1 * hist[0][1]
