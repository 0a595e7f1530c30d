"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself or with a re-typed copy of its own
code: each test uses a second formulation (numpy.unique, routing on raw float
thresholds built from the threshold set B_p of Section 3.1, numpy's Philox
bit generator, brute force over every tree of a tiny problem, the two sides of
the loss identity at the end of Section 2).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2311_06952_gb300 import datagen

def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


# --------------------------------------------------------------------------
# Section 3.1: threshold sets / dense ranks
# --------------------------------------------------------------------------

def _numpy_ranks(X):
    X = np.where(X == 0, np.float32(0), X)  # -0.0 and +0.0 are one value
    out, nu = [], []
    for p in range(X.shape[1]):
        u, inv = np.unique(X[:, p], return_inverse=True)
        out.append(inv.astype(np.uint32))
        nu.append(len(u))
    return np.stack(out), np.array(nu, np.uint32)


@pytest.mark.parametrize("n,F,seed", [(1, 1, 0), (7, 3, 1), (1000, 8, 2), (5000, 5, 3)])
def test_encode_matches_numpy_unique(n, F, seed):
    rng = _rng(seed)
    X = np.round(rng.normal(size=(n, F)), 2).astype(np.float32)
    if n > 3:
        X[0, 0] = -0.0
        X[1, 0] = 0.0
        X[:, -1] = 3.5  # constant feature: n_p = 1
    r, nu = oracle.encode(X)
    r2, nu2 = _numpy_ranks(X)
    np.testing.assert_array_equal(nu, nu2)
    np.testing.assert_array_equal(r, r2)


def test_encode_rejects_nan():
    X = np.zeros((5, 2), np.float32)
    X[3, 1] = np.nan
    with pytest.raises(ValueError):
        oracle.encode(X)


def test_encode_workload0_tie_structure():
    w = datagen.make_workload(0)
    r, nu = oracle.encode(w["X"])
    # rounded to 3 decimals: at most 1001 distinct values per feature
    assert nu.max() <= 1001 and nu.min() > 500
    r2, nu2 = _numpy_ranks(w["X"])
    np.testing.assert_array_equal(r, r2)


# --------------------------------------------------------------------------
# Eq. aenc / Eq. benc + routing of Section 2: the rank route must equal the
# paper's route on raw values against beta_{a_t, i} of the threshold set.
# --------------------------------------------------------------------------

def _float_route_leaves(X, genes, depth):
    """Route on raw values: b_t = beta_{a_t, i}, i = floor(bhat*(n_p+1)) + 1 (Eq. benc),
    with B_p = (0, midpoints of adjacent unique values, 1) mapped back through the
    min-max scaling of Section 2 (0 -> below the minimum, 1 -> the maximum)."""
    n, F = X.shape
    B = (1 << depth) - 1
    uniq = [np.unique(np.where(X[:, p] == 0, np.float32(0), X[:, p]).astype(np.float64))
            for p in range(F)]
    leaves = np.empty((genes.shape[0], n), np.int64)
    for r, g in enumerate(genes):
        t = np.ones(n, np.int64)
        for _ in range(depth):
            go_left = np.zeros(n, bool)
            for node in range(1, B + 1):
                sel = t == node
                if not sel.any():
                    continue
                a = int(np.floor(g[node - 1]))
                if a == 0:
                    continue  # b_t = 0: nothing is below 0, all go right
                u = uniq[a - 1]
                npp = len(u)
                i = int(np.floor(np.float64(g[B + node - 1]) * (npp + 1))) + 1
                x = X[sel, a - 1].astype(np.float64)
                if i == 1:
                    beta_left = np.zeros(sel.sum(), bool)  # beta = 0: below the minimum
                elif i == npp + 1:
                    beta_left = x < u[-1]  # beta = 1: the scaled maximum
                else:
                    beta = (u[i - 2] + u[i - 1]) / 2.0  # exact for float32 inputs
                    beta_left = x < beta
                go_left[sel] = beta_left
            t = np.where(go_left, 2 * t, 2 * t + 1)
        leaves[r] = t - (B + 1)
    return leaves


@pytest.mark.parametrize("depth,seed", [(1, 0), (2, 1), (3, 2)])
def test_decode_and_route_match_float_thresholds(depth, seed):
    rng = _rng(10 + seed)
    n, F, K = 400, 4, 3
    X = np.round(rng.random((n, F)), 2).astype(np.float32)
    X[:, 2] = np.float32(0.25)  # constant feature (n_p = 1)
    y = rng.integers(0, K, n).astype(np.uint8)
    P = 40
    genes = datagen.random_genes(P, depth, F, rng)
    genes[0, :] = np.nextafter(np.float32([F + 1] * ((1 << depth) - 1) + [1.0] * ((1 << depth) - 1)),
                               np.float32(0))  # largest genes: feature F, last threshold index
    genes[1, : (1 << depth) - 1] = 0.5  # all no-split
    ranks, nu = oracle.encode(X)
    a, th = oracle.decode(genes, depth, nu)
    counts = oracle.eval_counts(ranks, y, K, a, th, depth)
    leaves = _float_route_leaves(X, genes, depth)
    L = 1 << depth
    for r in range(P):
        ref = np.zeros((L, K), np.int64)
        np.add.at(ref, (leaves[r], y), 1)
        np.testing.assert_array_equal(counts[r], ref)


def test_decode_ranges():
    rng = _rng(5)
    F = 6
    nu = np.array([1, 2, 3, 1000, 65536, 70000], np.uint32)
    genes = datagen.random_genes(5000, 2, F, rng)
    a, th = oracle.decode(genes, 2, nu)
    assert a.min() >= 0 and a.max() <= F
    assert np.all(th[a == 0] == 0)
    sel = a > 0
    assert np.all(th[sel] <= nu[a[sel] - 1] - 1)


# --------------------------------------------------------------------------
# Section 2 / 3.2: loss identity, invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_loss_identity_and_count_invariants(depth):
    rng = _rng(20 + depth)
    n, F, K = 2000, 5, 4
    X = np.round(rng.normal(size=(n, F)), 1).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    a, th = datagen.random_population(nu, 30, depth, rng, allow_nosplit=True)
    counts = oracle.eval_counts(ranks, y, K, a, th, depth)
    fit, err, spl, v = oracle.fitness(counts, a, n)
    cls = oracle.leaf_classes(counts)
    for r in range(30):
        # sum over leaves and classes is n; class totals equal the label histogram
        assert counts[r].sum() == n
        np.testing.assert_array_equal(counts[r].sum(axis=0), np.bincount(y, minlength=K))
        # left side of the loss identity: predict each sample's leaf class, count mistakes
        t = np.ones(n, np.int64)
        B = (1 << depth) - 1
        for _ in range(depth):
            at = a[r][t - 1]
            thr = th[r][t - 1]
            rk = ranks[np.maximum(at - 1, 0), np.arange(n)]
            left = (at > 0) & (rk < thr)
            t = np.where(left, 2 * t, 2 * t + 1)
        leaf_of = t - (B + 1)
        mistakes = int(np.sum(cls[r][leaf_of] != y))
        assert mistakes == err[r]
        assert spl[r] == int(np.sum(a[r] >= 1))
        assert fit[r] == float(err[r])  # alpha = 0, n_min = 1: f is the error count


def test_no_split_tree_error_is_n_minus_majority():
    rng = _rng(3)
    n, K = 777, 5
    y = rng.integers(0, K, n).astype(np.uint8)
    X = rng.random((n, 2)).astype(np.float32)
    ranks, nu = oracle.encode(X)
    for depth in (1, 2, 3):
        B = (1 << depth) - 1
        a = np.zeros((1, B), np.int32)
        th = np.zeros((1, B), np.uint32)
        counts = oracle.eval_counts(ranks, y, K, a, th, depth)
        fit, err, spl, v = oracle.fitness(counts, a, n)
        assert err[0] == n - np.bincount(y).max()
        assert spl[0] == 0
        assert counts[0, -1].sum() == n  # everything in the rightmost leaf


def test_fitness_penalties():
    # one tree, depth 1, hand-made counts: leaves with 2 and 9 samples
    counts = np.array([[[1, 1], [6, 3]]], np.uint32)
    a = np.array([[1]], np.int32)
    fit, err, spl, v = oracle.fitness(counts, a, 11, n_min=3, alpha=0.25)
    assert err[0] == 11 - 1 - 6
    assert v[0] == 1  # leaf with 2 samples < n_min = 3
    assert spl[0] == 1
    assert fit[0] == 4 + 1 + 0.25
    # an empty leaf is not penalised (n_t >= n_min * 1_N(n_t))
    counts = np.array([[[0, 0], [6, 5]]], np.uint32)
    fit, err, spl, v = oracle.fitness(counts, a, 11, n_min=3, alpha=0.0)
    assert v[0] == 0 and err[0] == 5


def test_subset_equals_materialised_subset():
    rng = _rng(4)
    n, F, K, depth = 3000, 6, 3, 3
    X = np.round(rng.random((n, F)), 2).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    a, th = datagen.random_population(nu, 20, depth, rng)
    idx = np.sort(rng.choice(n, 1234, replace=False)).astype(np.int32)
    c1 = oracle.eval_counts(ranks, y, K, a, th, depth, idx=idx)
    c2 = oracle.eval_counts(np.ascontiguousarray(ranks[:, idx]), y[idx], K, a, th, depth)
    np.testing.assert_array_equal(c1, c2)


# --------------------------------------------------------------------------
# Brute force over all trees of tiny problems
# --------------------------------------------------------------------------

def _all_depth1(nu):
    yield 0, 0
    for p in range(len(nu)):
        for t in range(int(nu[p])):
            yield p + 1, t


def test_depth1_is_brute_force_minimum_with_tie_order():
    rng = _rng(7)
    for trial in range(25):
        n = int(rng.integers(2, 14))
        F = int(rng.integers(1, 4))
        K = int(rng.integers(1, 4))
        X = rng.integers(0, 4, size=(n, F)).astype(np.float32)
        y = rng.integers(0, K, n).astype(np.uint8)
        n_min = int(rng.integers(1, 4))
        alpha = float(rng.choice([0.0, 0.5]))
        ranks, nu = oracle.encode(X)
        cands = list(_all_depth1(nu))
        a = np.array([[c[0]] for c in cands], np.int32)
        th = np.array([[c[1]] for c in cands], np.uint32)
        counts = oracle.eval_counts(ranks, y, K, a, th, 1)
        fit, _, _, _ = oracle.fitness(counts, a, n, n_min=n_min, alpha=alpha)
        first = int(np.argmin(fit))  # candidates are listed in the tie-break order
        a1, t1, f1 = oracle.depth1(ranks, nu, y, K, n_min=n_min, alpha=alpha)
        assert (a1, t1) == cands[first]
        assert f1 == fit[first]


def test_depth2_optimum_equals_split_dp():
    """min over all depth-2 trees (brute force through the evaluator) equals the
    dynamic program 'best root split + best depth-1 subtree on each side'."""
    rng = _rng(8)
    for trial in range(6):
        n = int(rng.integers(5, 11))
        F = 2
        K = 2
        X = rng.integers(0, 3, size=(n, F)).astype(np.float32)
        y = rng.integers(0, K, n).astype(np.uint8)
        ranks, nu = oracle.encode(X)
        nodes = list(_all_depth1(nu))
        trees = list(itertools.product(nodes, repeat=3))
        a = np.array([[t[0][0], t[1][0], t[2][0]] for t in trees], np.int32)
        th = np.array([[t[0][1], t[1][1], t[2][1]] for t in trees], np.uint32)
        counts = oracle.eval_counts(ranks, y, K, a, th, 2)
        _, err, _, _ = oracle.fitness(counts, a, n)
        brute = int(err.min())
        dp = None
        for (ra, rt) in nodes:
            if ra == 0:
                left = np.zeros(n, bool)
            else:
                left = ranks[ra - 1] < rt
            tot = 0
            for side in (left, ~left):
                idx = np.nonzero(side)[0].astype(np.int32)
                if len(idx) == 0:
                    continue
                _, _, f = oracle.depth1(ranks, nu, y, K, idx=idx)
                tot += int(f)
            dp = tot if dp is None else min(dp, tot)
        assert brute == dp


# --------------------------------------------------------------------------
# Philox4x64-10 vs numpy's implementation of the same published generator
# --------------------------------------------------------------------------

def _numpy_philox_block(counter, key):
    c = [int(x) for x in counter]
    # numpy increments the 256-bit counter before producing a block
    val = sum(w << (64 * i) for i, w in enumerate(c))
    val = (val - 1) % (1 << 256)
    prev = np.array([(val >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], np.uint64)
    bg = np.random.Philox(key=np.array(key, np.uint64), counter=prev)
    return bg.random_raw(4).astype(np.uint64)


@pytest.mark.parametrize("counter,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((1, 0, 0, 0), (0, 0)),
    ((5, 17, 3, 0), (0, 1)),
    ((200, 1023, 4, 0), (123456789, 77)),
    ((2**64 - 1, 2**63, 9, 0), (2**64 - 1, 2**64 - 2)),
])
def test_philox_matches_numpy(counter, key):
    ours = oracle.philox(np.array(counter, np.uint64), np.array(key, np.uint64))
    ref = _numpy_philox_block(counter, key)
    np.testing.assert_array_equal(ours, ref)


def test_draw32_layout():
    blk = oracle.philox(np.array([3, 9, 1, 0], np.uint64), np.array([11, 4], np.uint64))
    for s in range(8, 16):
        w = int(blk[(s & 7) >> 1])
        want = (w >> 32) if (s & 1) else (w & 0xFFFFFFFF)
        assert oracle.draw32(11, 4, 3, 9, s) == want


# --------------------------------------------------------------------------
# DE (Algorithm 4): invariants that hold whatever the draw conventions
# --------------------------------------------------------------------------

def test_de_trial_membership_and_distinct_indices():
    rng = _rng(9)
    F, depth, P = 5, 2, 16
    B = 3
    pop = datagen.random_genes(P, depth, F, rng)
    seen_r1 = np.zeros(P, int)
    taken_v = 0
    total = 0
    for g in range(1, 40):
        for r in range(P):
            u, r1, r2, qr = oracle.de_trial(pop, 3, g, r, F, depth, M=0.5, CR=0.3, seed=5, stream=2)
            assert len({r, r1, r2}) == 3 and 0 <= r1 < P and 0 <= r2 < P
            assert 0 <= qr < 2 * B
            seen_r1[r1] += 1
            for q in range(2 * B):
                hi = np.nextafter(np.float32(F + 1 if q < B else 1.0), np.float32(0))
                assert 0.0 <= u[q] <= hi
                if u[q] != pop[r, q]:
                    taken_v += 1
                total += 1
    # every index is drawn as r1; roughly CR of the genes come from the mutant
    assert np.all(seen_r1 > 0)
    assert 0.25 < taken_v / total < 0.55


def test_de_run_invariants():
    w = datagen.make_workload(0, n=300)
    ranks, nu = oracle.encode(w["X"])
    out = oracle.de_run(ranks, nu, w["y"], w["K"], depth=2, P=16, G=30, seed=3, history=True)
    fh = out["fit_hist"]
    assert np.all(np.diff(fh, axis=0) <= 0)  # Eq. selection: per-slot fitness never rises
    bh = out["best_fit_hist"]
    assert np.all(np.diff(bh) <= 0)  # the non-descending sequence of Section 3.3
    assert bh[-1] == out["fit"].min() == out["fit"][out["best"]]
    assert out["best"] == int(np.argmin(out["fit"]))
    # a slot either kept its vector or took a new one; both are in range
    ph = out["pop_hist"]
    B = 3
    assert np.all(ph[..., :B] >= 0) and np.all(ph[..., :B] < 9)
    assert np.all(ph[..., B:] >= 0) and np.all(ph[..., B:] < 1)
    # fitness recorded equals fitness recomputed from the final genes
    a, th = oracle.decode(out["pop"], 2, nu)
    counts = oracle.eval_counts(ranks, w["y"], w["K"], a, th, 2)
    fit, _, _, _ = oracle.fitness(counts, a, 300)
    np.testing.assert_array_equal(fit, out["fit"])


def test_de_reaches_brute_force_optimum_on_tiny_problem():
    """Statistical check (not a parity pin): DE with a generous budget finds the
    exhaustive depth-2 optimum of a tiny problem."""
    rng = _rng(12)
    n, F, K = 40, 2, 2
    X = rng.integers(0, 5, size=(n, F)).astype(np.float32)
    y = ((X[:, 0] > 1) ^ (X[:, 1] > 2)).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    nodes = list(_all_depth1(nu))
    trees = list(itertools.product(nodes, repeat=3))
    a = np.array([[t[0][0], t[1][0], t[2][0]] for t in trees], np.int32)
    th = np.array([[t[0][1], t[1][1], t[2][1]] for t in trees], np.uint32)
    _, err, _, _ = oracle.fitness(oracle.eval_counts(ranks, y, K, a, th, 2), a, n)
    hits = 0
    for seed in range(6):
        out = oracle.de_run(ranks, nu, y, K, depth=2, P=64, G=200, seed=seed)
        assert out["fit"].min() >= err.min()
        hits += int(out["fit"].min() == err.min())
    assert hits >= 4


def test_de_seeds_occupy_first_slots():
    w = datagen.make_workload(0, n=200)
    ranks, nu = oracle.encode(w["X"])
    rng = _rng(1)
    seeds = datagen.random_genes(3, 2, 8, rng)
    out = oracle.de_run(ranks, nu, w["y"], w["K"], depth=2, P=8, G=0, seeds=seeds, history=True)
    np.testing.assert_array_equal(out["pop_hist"][0, :3], seeds)


# --------------------------------------------------------------------------
# Algorithm 2 (moving horizon): special cases with a closed form
# --------------------------------------------------------------------------

def _greedy_float_tree(X, y, K, depth, n_min):
    """Greedy misclassification tree on raw values: every node takes the best
    depth-1 split (no split first, then lowest feature, then lowest threshold
    index of B_p), routed with x < beta on the float midpoints."""
    n, F = X.shape
    uniq = [np.unique(X[:, p].astype(np.float64)) for p in range(F)]
    B = (1 << depth) - 1
    a = np.zeros(B, np.int64)
    thr_idx = np.zeros(B, np.int64)
    node = np.ones(n, np.int64)
    for d in range(depth):
        for t in range(1 << d, 1 << (d + 1)):
            sel = np.nonzero(node == t)[0]
            if len(sel) <= n_min or len(np.unique(y[sel])) < 2:
                continue
            yt = y[sel]
            best = (len(sel) - np.bincount(yt, minlength=K).max(), 0, 0)
            for p in range(F):
                u = uniq[p]
                for th in range(len(u)):  # theta = th: left iff value < unique[th]
                    left = X[sel, p].astype(np.float64) < (u[th] if th > 0 else -np.inf)
                    e = len(sel) - np.bincount(yt[left], minlength=K).max() - \
                        np.bincount(yt[~left], minlength=K).max()
                    if e < best[0]:
                        best = (e, p + 1, th)
            a[t - 1], thr_idx[t - 1] = best[1], best[2]
        # move samples one level down
        nxt = node.copy()
        for t in range(1 << d, 1 << (d + 1)):
            sel = node == t
            if a[t - 1] == 0:
                left = np.zeros(sel.sum(), bool)
            else:
                u = uniq[a[t - 1] - 1]
                left = X[sel, a[t - 1] - 1].astype(np.float64) < u[thr_idx[t - 1]] if thr_idx[t - 1] > 0 \
                    else np.zeros(sel.sum(), bool)
            nxt[sel] = np.where(left, 2 * t, 2 * t + 1)
        node = nxt
    return a, thr_idx


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mh_horizon1_is_greedy_misclassification_tree(seed):
    rng = _rng(30 + seed)
    n, F, K, D = 60, 3, 3, 3
    X = rng.integers(0, 6, size=(n, F)).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    out = oracle.mh(ranks, nu, y, K, depth=D, horizon=1, P=8, G=1)
    a_ref, t_ref = _greedy_float_tree(X, y, K, D, n_min=1)
    np.testing.assert_array_equal(out["a"], a_ref)
    np.testing.assert_array_equal(out["theta"], t_ref)
    assert set(out["kind"]) <= {0, 1}


def test_mh_all_artificial_when_nmin_large_or_single_class():
    w = datagen.make_workload(0, n=100)
    ranks, nu = oracle.encode(w["X"])
    out = oracle.mh(ranks, nu, w["y"], w["K"], depth=3, horizon=2, P=8, G=2, n_min=100)
    assert np.all(out["a"] == 0) and np.all(out["theta"] == 0) and np.all(out["kind"] == 0)
    maj = np.bincount(w["y"], minlength=2).argmax()
    assert out["leaf_class"][-1] == maj and np.all(out["leaf_class"][:-1] == 0)
    y1 = np.ones(100, np.uint8)
    out = oracle.mh(ranks, nu, y1, 2, depth=3, horizon=2, P=8, G=2)
    assert np.all(out["a"] == 0) and out["leaf_class"][-1] == 1


def test_mh_root_is_deoct_root_when_horizon_covers_depth():
    w = datagen.make_workload(0, n=300)
    ranks, nu = oracle.encode(w["X"])
    out = oracle.mh(ranks, nu, w["y"], w["K"], depth=2, horizon=2, P=16, G=10, seed=4)
    de = oracle.de_run(ranks, nu, w["y"], w["K"], depth=2, P=16, G=10, seed=4, stream=1)
    a, th = oracle.decode(de["pop"][de["best"]][None, :], 2, nu)
    assert out["kind"][0] == 2
    assert out["a"][0] == a[0, 0] and out["theta"][0] == th[0, 0]
    assert out["node_fit"][0] == de["fit"][de["best"]]


# --------------------------------------------------------------------------
# Raw-unit thresholds and prediction (Section 3.1 threshold set, Section 2 routing)
# --------------------------------------------------------------------------

def test_split_values_route_training_samples_like_ranks():
    rng = _rng(61)
    n, F, K, depth = 3000, 5, 3, 3
    X = np.round(rng.normal(size=(n, F)), 2).astype(np.float32)
    X[:, 4] = -1.5
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    for trial in range(10):
        a, th = datagen.random_population(nu, 1, depth, rng, allow_nosplit=True)
        counts = oracle.eval_counts(ranks, y, K, a, th, depth)
        lc = oracle.leaf_classes(counts)[0]
        b = oracle.split_values(X, a[0], th[0])
        pred = oracle.predict(X, a[0], b, depth, lc)
        # the same samples, routed on ranks in numpy
        t = np.ones(n, np.int64)
        B = (1 << depth) - 1
        for _ in range(depth):
            at = a[0][t - 1]
            rk = ranks[np.maximum(at - 1, 0), np.arange(n)]
            t = np.where((at > 0) & (rk < th[0][t - 1]), 2 * t, 2 * t + 1)
        np.testing.assert_array_equal(pred, lc[t - (B + 1)])
        # loss identity: misclassified training samples = fitness errors
        _, err, _, _ = oracle.fitness(counts, a, n)
        assert int(np.sum(pred != y)) == int(err[0])


def test_split_values_definition():
    X = np.array([[3.0], [1.0], [2.0], [2.0], [7.0]], np.float32)
    b = oracle.split_values(X, np.array([1, 1, 1, 0]), np.array([0, 1, 3, 0], np.uint32))
    # sorted distinct values 1, 2, 3, 7
    assert list(b) == [1.0, 1.5, 5.0, 0.0]



# --------------------------------------------------------------------------
# CART warm starts (Algorithm 2): the greedy subtree
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1])
def test_greedy_tree_is_the_float_greedy_tree(seed):
    rng = _rng(90 + seed)
    n, F, K, D = 80, 3, 3, 3
    X = rng.integers(0, 6, size=(n, F)).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    a, th = oracle.greedy_tree(ranks, nu, y, K, D)
    a_ref, t_ref = _greedy_float_tree(X, y, K, D, n_min=1)
    np.testing.assert_array_equal(a, a_ref)
    np.testing.assert_array_equal(th, t_ref)
    # on a subset: the greedy tree of the materialised subset
    idx = np.sort(rng.choice(n, 50, replace=False)).astype(np.int32)
    a1, t1 = oracle.greedy_tree(ranks, nu, y, K, D, idx=idx)
    a2, t2 = _greedy_float_tree(X[idx], y[idx], K, D, n_min=1)
    # thresholds are global ranks: compare the splits through the float route instead
    np.testing.assert_array_equal(a1, a2)


def test_cart_seed_genes_decode_to_the_greedy_tree():
    w = datagen.make_workload(0, n=400)
    ranks, nu = oracle.encode(w["X"])
    out = oracle.mh(ranks, nu, w["y"], 2, depth=3, horizon=3, P=8, G=0, cart_seeds=True)
    a, th = oracle.greedy_tree(ranks, nu, w["y"], 2, 3)
    # with G = 0 the root keeps the best initial individual; the greedy tree is slot 0,
    # so the root's fitness is at most the greedy tree's fitness
    counts = oracle.eval_counts(ranks, w["y"], 2, a[None], th[None], 3)
    f, _, _, _ = oracle.fitness(counts, a[None], 400)
    assert out["node_fit"][0] <= f[0]
    assert out["kind"][0] == 2


def test_deoct_warm_start_bounds_the_root():
    """With G = 0 the root of MH keeps the best initial individual, and the full-depth
    DEOCT's root subtree is one of them (Algorithm 2, DEOCT warm start)."""
    w = datagen.make_workload(0, n=400)
    ranks, nu = oracle.encode(w["X"])
    full = oracle.de_run(ranks, nu, w["y"], 2, depth=3, P=8, G=0, seed=2, stream=0)
    a, th = oracle.decode(full["pop"][full["best"]][None], 3, nu)
    # the depth-2 subtree at the root of the full tree
    sub_a, sub_t = a[:, :3], th[:, :3]
    counts = oracle.eval_counts(ranks, w["y"], 2, sub_a, sub_t, 2)
    f, _, _, _ = oracle.fitness(counts, sub_a, 400)
    out = oracle.mh(ranks, nu, w["y"], 2, depth=3, horizon=2, P=8, G=0, seed=2, de_seeds=True)
    assert out["kind"][0] == 2 and out["node_fit"][0] <= f[0]


def test_oracle_reproduces_golden_fixtures():
    """tests/golden/ holds values written by tests/golden/make_golden.py from the oracle alone
    (the paper prints no worked numeric example): DEOCT on the tiny workload (Algorithm 4) and
    the class counts of the full population-evaluation workload (Algorithm 1).  The oracle must
    still produce them; a change here needs a change of the oracle's arithmetic that a passage of
    the paper justifies."""
    import importlib.util
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    for name, fn in (("deoct_workload0.json", mg.deoct_workload0), ("eval_workload1.json", mg.eval_workload1)):
        with open(os.path.join(here, name)) as f:
            assert fn() == json.load(f), name
