"""Prediction with a fitted tree on raw values: distinct training values from the
encoder, raw-unit thresholds, routing of unseen samples; GPU against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2311_06952_gb300 import datagen

from gpu_helpers import ctx, to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2311_06952_gb300 import build
    build.build()
    return ctx()


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


@pytest.mark.parametrize("rb", [2, 4])
def test_encode_ex_unique_values(c, rb):
    from paper_2311_06952_gb300 import deoct
    rng = _rng(70 + rb)
    X = np.round(rng.normal(size=(5003, 6)), 2).astype(np.float32)
    X[::9, 1] = -0.0
    X[:, 5] = 4.0
    ranks, nu, uniq = deoct.deoct_encode_ex(c, to_dev(X), rb)
    nu = u32(nu)
    uq = uniq.cpu().numpy()
    for f in range(6):
        ref = np.unique(np.where(X[:, f] == 0, np.float32(0), X[:, f]))
        assert nu[f] == len(ref)
        np.testing.assert_array_equal(uq[f, : nu[f]].view(np.uint32), ref.view(np.uint32))


def test_split_values_and_predict_bit_exact(c):
    import torch
    from paper_2311_06952_gb300 import deoct
    rng = _rng(80)
    n, F, K, depth = 4000, 5, 3, 4
    X = np.round(rng.normal(size=(n, F)), 2).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    Xt = np.round(rng.normal(scale=1.5, size=(7777, F)), 3).astype(np.float32)  # unseen values
    yt = rng.integers(0, K, 7777).astype(np.uint8)
    _, nu_ref = oracle.encode(X)
    ranks, nu, uniq = deoct.deoct_encode_ex(c, to_dev(X), 2)
    for trial in range(6):
        a, th = datagen.random_population(nu_ref, 1, depth, rng, allow_nosplit=True)
        a, th = a[0], th[0]
        if trial == 0:
            th[:] = 0  # every threshold at the smallest training value
        lc = rng.integers(0, K, 1 << depth).astype(np.uint8)
        b = deoct.deoct_split_values(c, uniq, to_dev(a.astype(np.uint16)), to_dev(th))
        b_ref = oracle.split_values(X, a, th)
        np.testing.assert_array_equal(b.cpu().numpy().view(np.uint64), b_ref.view(np.uint64))
        pred, correct = deoct.deoct_predict(c, to_dev(Xt), to_dev(a.astype(np.uint16)), b, depth,
                                            to_dev(lc), y=to_dev(yt))
        p_ref = oracle.predict(Xt, a, b_ref, depth, lc)
        np.testing.assert_array_equal(pred.cpu().numpy(), p_ref)
        assert int(correct.item()) == int(np.sum(p_ref == yt))


def test_estimator_training_accuracy_is_the_loss_identity(c):
    from paper_2311_06952_gb300.estimator import MHDEOCTClassifier
    w = datagen.make_workload(0)
    clf = MHDEOCTClassifier(depth=3, horizon=2, pop=32, gens=20, cr=0.9, dither=False, seed=0,
                            warm_starts=None).fit(w["X"], w["y"])
    tr = clf.tree_
    # the oracle's errors of the fitted tree on the training set
    ranks, nu = oracle.encode(w["X"])
    a = tr["a"].astype(np.int32)[None]
    counts = oracle.eval_counts(ranks, w["y"], 2, a, tr["theta"][None], 3)
    _, err, _, _ = oracle.fitness(counts, a, len(w["y"]))
    assert clf.score(w["X"], w["y"]) == 1.0 - err[0] / len(w["y"])
    # and the oracle's own prediction of the same tree
    b_ref = oracle.split_values(w["X"], tr["a"].astype(np.int32), tr["theta"])
    np.testing.assert_array_equal(clf.predict(w["X"]),
                                  oracle.predict(w["X"], tr["a"].astype(np.int32), b_ref, 3, tr["leaf_class"]))
    # the MH tree equals the oracle's MH tree
    ref = oracle.mh(ranks, nu, w["y"], 2, depth=3, horizon=2, P=32, G=20, CR=0.9, seed=0)
    np.testing.assert_array_equal(tr["a"].astype(np.int32), ref["a"])
    np.testing.assert_array_equal(tr["theta"], ref["theta"])


def test_estimator_paper_defaults_run_and_match_oracle(c):
    """Normal preset (P=100, G=600, CR=0.1, dithered M) with both warm starts."""
    from paper_2311_06952_gb300.estimator import MHDEOCTClassifier
    w = datagen.make_workload(0, n=600)
    clf = MHDEOCTClassifier(depth=3, gens=60, seed=4).fit(w["X"], w["y"])
    ranks, nu = oracle.encode(w["X"])
    ref = oracle.mh(ranks, nu, w["y"], 2, depth=3, horizon=3, P=100, G=60, CR=0.1, seed=4, dither=True,
                    cart_seeds=True, de_seeds=True)
    np.testing.assert_array_equal(clf.tree_["a"].astype(np.int32), ref["a"])
    np.testing.assert_array_equal(clf.tree_["theta"], ref["theta"])
    np.testing.assert_array_equal(clf.tree_["leaf_class"], ref["leaf_class"])


def _oracle_tuned(X, y, K, depth, horizon, P, G, seed, n_grid=21, val_frac=1.0 / 3.0, split_seed=0):
    """The training-validation-retraining procedure of Appendix C restated on the oracle:
    alpha = cp * (n - majority count) of the set being fitted, cp on an even grid of
    [0, 1]; validation accuracy of the tree routed on raw values; ties to the larger cp."""
    perm = np.random.Generator(np.random.PCG64(split_seed)).permutation(len(y))
    nv = int(round(len(y) * val_frac))
    fit_idx, val_idx = np.sort(perm[nv:]), np.sort(perm[:nv])

    def mh(Xs, ys, alpha):
        ranks, nu = oracle.encode(Xs)
        t = oracle.mh(ranks, nu, ys, K, depth=depth, horizon=horizon, P=P, G=G, alpha=alpha, seed=seed,
                      cart_seeds=True, de_seeds=True)
        return t, oracle.split_values(Xs, t["a"], t["theta"])

    def e_root(ys):
        return len(ys) - np.bincount(ys, minlength=K).max()

    cps = np.linspace(0.0, 1.0, n_grid)
    acc = []
    for cp in cps:
        t, b = mh(X[fit_idx], y[fit_idx], float(cp * e_root(y[fit_idx])))
        pred = oracle.predict(X[val_idx], t["a"], b, depth, t["leaf_class"])
        acc.append(np.mean(pred == y[val_idx]))
    acc = np.asarray(acc)
    best = int(np.flatnonzero(acc == acc.max())[-1])
    t, _ = mh(X, y, float(cps[best] * e_root(y)))
    return cps[best], acc, t


def test_alpha_tuning_selects_what_the_oracle_selects():
    """Appendix C's procedure on a small noisy set: the GPU estimator and the oracle score
    every cp identically, pick the same one and refit the same tree."""
    from paper_2311_06952_gb300.estimator import MHDEOCTClassifier
    rng = _rng(91)
    n, F, K, depth = 1500, 5, 2, 4
    X = np.round(rng.normal(size=(n, F)), 2).astype(np.float32)
    # one planted split under 35% label noise: deeper splits only fit noise, several cp
    # values tie on validation and the largest of them must win
    y = datagen.flip_labels(datagen.planted_tree_labels(X, 1, K, rng), K, 0.35, rng)
    clf = MHDEOCTClassifier(depth=depth, horizon=2, pop=16, gens=12, cr=0.9, dither=False, seed=4,
                            warm_starts=("cart", "deoct"))
    clf.fit_tuned(X, y, K=K)
    cp, acc, tree = _oracle_tuned(X, y, K, depth, 2, 16, 12, 4)
    np.testing.assert_array_equal(clf.tuning_["val_accuracy"], acc)
    assert clf.tuning_["cp_best"] == cp
    assert cp > 0.0  # the noise makes some pruning pay on validation data
    np.testing.assert_array_equal(clf.tree_["a"].astype(np.int32), tree["a"])
    np.testing.assert_array_equal(clf.tree_["theta"], tree["theta"])
    np.testing.assert_array_equal(clf.tree_["leaf_class"], tree["leaf_class"])
