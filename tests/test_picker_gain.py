"""What the trained cost model gains over the method without it (GPU).

A seeded set of shapes (N ~ U{4..165}, E = floor(2^U(14, 19)), F ~ U{1..4}, every
precision path and layout) is autotuned exhaustively by the library; an ensemble of three
networks is trained on the first 400 shapes' timings by the library's own kernels; on the
40 held-out shapes the library's lc_pick_variant_ensemble chooses a descriptor, and the pick, the autotuned best and
the default descriptor (lc_variant_default: the fixed choice the method makes without a
model) are re-timed together.  The network's geo-mean regret must be below the default's.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_7470_gb300 import lc as lcmod
    lcmod.load()
    return lcmod


def test_learned_pick_beats_default_on_held_out_shapes(lc):
    from paper_1405_7470_gb300 import picker
    seed, n_train, n_test = 1, 400, 40
    shapes = synth.picker_shapes(seed, n_train + n_test, e_lo=14.0, e_hi=19.0)
    recs = picker.collect(shapes, reps=3, seed=seed)
    X, y = picker.dataset(recs[:n_train])
    params, hists = picker.train_ensemble(X, y, models=3, epochs=300, seed=seed)
    assert all(h[-1][1] < h[0][1] for h in hists)
    pool = picker.make_pool(shapes[n_train:])
    ev = picker.evaluate(params, recs[n_train:], pool=pool,
                         seeds=[seed * 100003 + k for k in range(n_train, n_train + n_test)])
    print("held-out regret, network:", ev["mlp"], "default:", ev["default"],
          "picks equal to the best:", ev["picks_equal_best"], "of", ev["shapes"])
    assert ev["retimed"] and ev["shapes"] == n_test
    assert ev["mlp"]["geomean"] < ev["default"]["geomean"]


def test_pick_is_a_valid_candidate(lc):
    """lc_pick_variant (and the ensemble form) returns one of the enumerated candidates,
    whatever the network."""
    import torch
    from paper_1405_7470_gb300 import picker
    params = torch.from_numpy(picker.he_uniform(lc.FEATURES, 3)).cuda()
    for E, N, F, layout, path in ((5000, 35, 3, "elem", "bf16x3"), (70000, 120, 2, "node", "fp32"),
                                  (1 << 16, 9, 1, "elem", "bf16")):
        kernel = picker.kernel_for(F)
        v, pred = lc.pick_variant(kernel, E, N, F, layout, path, params)
        cands = [lc.variant_dict(c) for c in lc.enumerate_variants(kernel, E, N, F, layout, path)]
        assert lc.variant_dict(v) in cands and np.isfinite(pred)
        # an ensemble of copies of one network picks what the network picks, with its prediction
        ve, pe = lc.pick_variant(kernel, E, N, F, layout, path, torch.stack([params, params, params]))
        assert lc.variant_dict(ve) == lc.variant_dict(v) and abs(pe - pred) <= 1e-5 * max(1.0, abs(pred))
        # two different networks: the mean prediction of the pick is the smallest mean
        other = torch.from_numpy(picker.he_uniform(lc.FEATURES, 4)).cuda()
        vm, pm = lc.pick_variant(kernel, E, N, F, layout, path, torch.stack([params, other]))
        assert lc.variant_dict(vm) in cands and np.isfinite(pm)
