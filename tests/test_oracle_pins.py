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
# DE arithmetic (Algorithm 4, Eq. mutation, Eq. crossover, initialisation)
# restated in numpy float32 with draws from numpy's own Philox4x64-10
# --------------------------------------------------------------------------

_TWO_M24 = np.float32(2.0 ** -24)


def _np_draws(seed, stream, g, r, nslots):
    """The 32-bit draws of (g, r): block b is numpy's Philox4x64-10 at counter (g, r, b, 0)
    and key (seed, stream), split into eight halves, low half first (Reading C5)."""
    out = []
    for b in range((nslots + 7) // 8):
        for w in _numpy_philox_block((g, r, b, 0), (seed, stream)):
            out += [int(w) & 0xFFFFFFFF, int(w) >> 32]
    return out[:nslots]


def _np_u01(x):
    return np.float32(x >> 8) * _TWO_M24  # 24 bits times 2^-24: exact in float32


def _np_hi(q, B, F):
    return np.nextafter(np.float32(F + 1 if q < B else 1.0), np.float32(0))


def _np_trial(pop, best, g, r, F, B, M, CR, seed, stream, dither):
    """Eq. mutation v = s_best + M (s_r1 - s_r2), each operation rounded to float32; the clamp
    of Reading C6; Eq. crossover u_q = v_q if rand_q <= CR or q = q_rand, else s_{r,q}."""
    P, m = pop.shape
    x = _np_draws(seed, stream, g, r, 4 + m)
    r1 = (x[0] * (P - 1)) >> 32
    r1 += r1 >= r
    r2 = (x[1] * (P - 2)) >> 32
    for skip in sorted((r, r1)):
        r2 += r2 >= skip
    qrand = (x[2] * m) >> 32
    Mf = _np_u01(x[3]) if dither else np.float32(M)
    v = pop[best] + Mf * (pop[r1] - pop[r2])  # float32 arrays: one rounding per operation
    assert v.dtype == np.float32
    hi = np.array([_np_hi(q, B, F) for q in range(m)], np.float32)
    v = np.minimum(np.maximum(v, np.float32(0)), hi)
    rand = np.array([_np_u01(x[4 + q]) for q in range(m)], np.float32)
    take = (rand <= np.float32(CR)) | (np.arange(m) == qrand)
    return np.where(take, v, pop[r]), r1, r2, qrand


def _extreme_population(rng, P, B, F):
    """Genes at 0 or just below the bound half of the time, so that mutants leave the gene
    range on both sides and the clamp of Reading C6 is exercised."""
    pop = datagen.random_genes(P, int(np.log2(B + 1)), F, rng)
    hi = np.array([_np_hi(q, B, F) for q in range(2 * B)], np.float32)
    pick = rng.random(pop.shape)
    pop = np.where(pick < 0.25, np.float32(0), np.where(pick > 0.75, hi[None, :], pop))
    return pop.astype(np.float32)


@pytest.mark.parametrize("dither,CR,M", [(False, 0.9, 0.5), (False, 0.3, 0.7), (True, 0.6, 0.0),
                                         (False, 1.0, 1.3)])
def test_de_trial_equals_numpy_restatement(dither, CR, M):
    """Eq. mutation and Eq. crossover bit for bit against a numpy float32 restatement whose
    draws come from numpy's Philox (not from the oracle's draw32)."""
    rng = _rng(21)
    F, depth = 6, 3
    B = 7
    clamped_lo = clamped_hi = 0
    for P in (4, 5, 17, 64):
        pop = _extreme_population(rng, P, B, F)
        for g in (1, 2, 9, 1000):
            best = int(rng.integers(P))
            for r in range(P):
                u, r1, r2, qr = oracle.de_trial(pop, best, g, r, F, depth, M=M, CR=CR, seed=7,
                                                stream=3, dither=dither)
                want, w1, w2, wq = _np_trial(pop, best, g, r, F, B, M, CR, 7, 3, dither)
                assert (r1, r2, qr) == (w1, w2, wq)
                np.testing.assert_array_equal(u.view(np.uint32), want.view(np.uint32))
                raw = pop[best] + np.float32(M) * (pop[r1] - pop[r2])
                clamped_lo += int(np.sum(raw < 0))
                clamped_hi += int(np.sum(raw > np.array([_np_hi(q, B, F) for q in range(2 * B)])))
    if M != 0.0 and not dither:
        assert clamped_lo > 0 and clamped_hi > 0


def test_de_trial_closed_forms():
    """Facts of Eq. mutation / Eq. crossover that hold whatever the draws are: with CR = 1
    every gene is the (clamped) mutant s_best + M (s_r1 - s_r2); with CR = 0 only gene q_rand
    is (a 2^-24 draw aside); with M = 0 every gene is s_best's or s_r's."""
    rng = _rng(5)
    F, depth, P = 4, 2, 12
    B = 3
    pop = datagen.random_genes(P, depth, F, rng)
    hi = np.array([_np_hi(q, B, F) for q in range(2 * B)], np.float32)
    for g in range(1, 30):
        for r in range(P):
            best = (g + 3) % P
            u, r1, r2, qr = oracle.de_trial(pop, best, g, r, F, depth, M=0.8, CR=1.0, seed=1)
            v = pop[best] + np.float32(0.8) * (pop[r1] - pop[r2])
            np.testing.assert_array_equal(u, np.clip(v, 0, hi))
            u0, r1, r2, qr = oracle.de_trial(pop, best, g, r, F, depth, M=0.8, CR=0.0, seed=1)
            v = np.clip(pop[best] + np.float32(0.8) * (pop[r1] - pop[r2]), 0, hi)
            for q in range(2 * B):
                assert u0[q] == (v[q] if q == qr else pop[r, q])
            uz, _, _, _ = oracle.de_trial(pop, best, g, r, F, depth, M=0.0, CR=0.5, seed=1)
            assert np.all((uz == pop[best]) | (uz == pop[r]))


@pytest.mark.parametrize("S", [0, 2])
def test_de_initial_population_equals_numpy_restatement(S):
    """Initial individual r >= S (Algorithm 4): gene q = clamp(u * ub) with u the 24-bit
    uniform of draw q at generation tag 0 (numpy's Philox), ub = F + 1 for ahat, 1 for bhat."""
    w = datagen.make_workload(0, n=200)
    ranks, nu = oracle.encode(w["X"])
    F, depth, P = 8, 3, 24
    B = 7
    seeds = datagen.random_genes(S, depth, F, _rng(2)) if S else None
    out = oracle.de_run(ranks, nu, w["y"], w["K"], depth=depth, P=P, G=0, seed=11, stream=5,
                        seeds=seeds, history=True)
    init = out["pop_hist"][0]
    for r in range(P):
        if r < S:
            np.testing.assert_array_equal(init[r], seeds[r])
            continue
        x = _np_draws(11, 5, 0, r, 2 * B)
        for q in range(2 * B):
            ub = np.float32(F + 1 if q < B else 1.0)
            want = min(max(_np_u01(x[q]) * ub, np.float32(0)), _np_hi(q, B, F))
            assert init[r, q].view(np.uint32) == np.float32(want).view(np.uint32), (r, q)
    # and the genes are spread over their whole range
    a_genes = init[S:, :B].ravel() / (F + 1)
    assert 0.3 < a_genes.mean() < 0.7 and a_genes.max() > 0.8 and a_genes.min() < 0.2


@pytest.mark.parametrize("n_p", [1, 2, 3, 7, 1000, 65535, 65536, (1 << 24) - 3])
def test_node_genes_invert_eq_aenc_benc(n_p):
    """The warm-start encoding of a node (a, theta) gives genes that decode back to (a, theta)
    under Eq. aenc (a = floor(ahat)) and Eq. benc (theta = floor(bhat (n_p + 1)), restated here
    in float64), for every theta of the feature (a sample of them for 2^24 values)."""
    if n_p <= 65536:
        th = np.arange(n_p, dtype=np.uint32)
    else:
        th = np.unique(np.concatenate([np.arange(300), n_p - 1 - np.arange(300),
                                       _rng(4).integers(0, n_p, 5000)])).astype(np.uint32)
    for a in (1, 5):
        av = np.full(len(th), a, np.int32)
        ah, bh = oracle.node_genes(av, th, np.full(len(th), n_p, np.uint32))
        np.testing.assert_array_equal(np.floor(ah).astype(np.int32), av)
        dec = np.floor(bh.astype(np.float64) * (n_p + 1.0))
        np.testing.assert_array_equal(np.minimum(dec, n_p - 1), th)
        assert np.all(bh >= 0) and np.all(bh < 1)
        # the oracle's decoder agrees (depth 1 trees: [ahat, bhat])
        nu = np.full(max(a, 5), n_p, np.uint32)
        da, dt = oracle.decode(np.stack([ah, bh], axis=1), 1, nu)
        np.testing.assert_array_equal(da[:, 0], av)
        np.testing.assert_array_equal(dt[:, 0], th)
    ah, bh = oracle.node_genes(np.zeros(3, np.int32), np.zeros(3, np.uint32), np.ones(3, np.uint32))
    assert np.all(np.floor(ah) == 0) and np.all(bh == 0)  # no split stays no split


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

def _np_route_to_depth(X, uniq, a, b_idx, d):
    """BFS node (1-based) that each sample reaches after d levels of the partial tree, routing
    raw values with x < beta (beta from the threshold set B_p of Section 3.1)."""
    n = X.shape[0]
    node = np.ones(n, np.int64)
    for _ in range(d):
        left = np.zeros(n, bool)
        for t in np.unique(node):
            m = node == t
            if a[t - 1] > 0:
                p = a[t - 1] - 1
                th = b_idx[t - 1]
                beta = -np.inf if th == 0 else (uniq[p][th - 1] + uniq[p][th]) / 2
                left[m] = X[m, p].astype(np.float64) < beta
        node = np.where(left, 2 * node, 2 * node + 1)
    return node


@pytest.mark.parametrize("depth,horizon,seed,n_min", [(4, 2, 0, 1), (4, 3, 1, 1), (5, 3, 2, 12)])
def test_mh_equals_algorithm2_composed_from_pinned_steps(depth, horizon, seed, n_min):
    """Algorithm 2 restated in Python on top of the separately pinned DEOCT (de_run) and
    depth-1 search: nodes in BFS order; (X_t, Y_t) induced by routing raw values through the
    nodes fixed so far; solve iff |X_t| > n_min and two classes; D_t = min(D_MH, D - d); DEOCT
    with Philox stream t keeps its best tree's root, depth 1 is the exhaustive search; leaf
    classes by Eq. opt_c on the whole set."""
    w = datagen.make_workload(0, n=700)
    X, y, K = w["X"][:, :5], w["y"], w["K"]
    rng = _rng(seed)
    y = np.where(rng.random(len(y)) < 0.1, 1 - y, y).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    uniq = [np.unique(np.where(X[:, p] == 0, 0, X[:, p]).astype(np.float64)) for p in range(X.shape[1])]
    P, G = 8, 6
    got = oracle.mh(ranks, nu, y, K, depth, horizon, P, G, seed=seed, n_min=n_min)
    B = (1 << depth) - 1
    a = np.zeros(B, np.int64)
    th = np.zeros(B, np.int64)
    kind = np.zeros(B, np.int64)
    for t in range(1, B + 1):
        d = t.bit_length() - 1
        idx = np.nonzero(_np_route_to_depth(X, uniq, a, th, d) == t)[0].astype(np.int32)
        if not (len(idx) > n_min and len(np.unique(y[idx])) > 1):
            continue
        Dt = min(horizon, depth - d)
        if Dt >= 2:
            out = oracle.de_run(ranks, nu, y, K, depth=Dt, P=P, G=G, seed=seed, stream=t, idx=idx,
                                n_min=n_min)
            ga, gt = oracle.decode(out["pop"][out["best"]][None], Dt, nu)
            a[t - 1], th[t - 1], kind[t - 1] = ga[0, 0], gt[0, 0], 2
        else:
            a1, t1, _ = oracle.depth1(ranks, nu, y, K, idx=idx, n_min=n_min)
            a[t - 1], th[t - 1], kind[t - 1] = a1, t1, 1
    np.testing.assert_array_equal(got["kind"], kind)
    np.testing.assert_array_equal(got["a"], a)
    np.testing.assert_array_equal(got["theta"], th)
    assert (kind == 2).sum() >= 3 and (kind == 1).sum() >= 1
    leaf = _np_route_to_depth(X, uniq, a, th, depth) - (B + 1)
    cnt = np.zeros((1 << depth, K), np.int64)
    np.add.at(cnt, (leaf, y), 1)
    np.testing.assert_array_equal(got["leaf_class"], np.argmax(cnt, axis=1))


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


@pytest.mark.parametrize("cart,deo,seed", [(True, False, 3), (False, True, 4), (True, True, 5)])
def test_mh_warm_starts_equal_algorithm2_composed_from_pinned_steps(cart, deo, seed):
    """The warm starts of Algorithm 2 restated over the pinned steps: the DEOCT warm start is
    the best tree of one full-depth DEOCT (Philox stream 0) on the whole set, and node t's
    seed is its subtree at t with t's shape; the CART warm start is the greedy tree of depth
    D_t on (X_t, Y_t); both encoded by node_genes (itself pinned to decode back), the DEOCT
    seed first, then the CART seed, in the first slots of node t's DEOCT."""
    w = datagen.make_workload(0, n=600)
    X, y, K = w["X"][:, :5], w["y"], w["K"]
    rng = _rng(seed)
    y = np.where(rng.random(len(y)) < 0.1, 1 - y, y).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    uniq = [np.unique(np.where(X[:, p] == 0, 0, X[:, p]).astype(np.float64)) for p in range(X.shape[1])]
    depth, horizon, P, G = 4, 2, 8, 5
    got = oracle.mh(ranks, nu, y, K, depth, horizon, P, G, seed=seed, cart_seeds=cart, de_seeds=deo)
    B = (1 << depth) - 1
    wa = wth = None
    if deo:
        full = oracle.de_run(ranks, nu, y, K, depth=depth, P=P, G=G, seed=seed, stream=0)
        wa, wth = oracle.decode(full["pop"][full["best"]][None], depth, nu)
        wa, wth = wa[0], wth[0]

    def genes(a_, th_):
        n_p = np.array([nu[x - 1] if x > 0 else 1 for x in a_], np.uint32)
        ah, bh = oracle.node_genes(np.asarray(a_, np.int32), np.asarray(th_, np.uint32), n_p)
        return np.concatenate([ah, bh]).astype(np.float32)

    a = np.zeros(B, np.int64)
    th = np.zeros(B, np.int64)
    for t in range(1, B + 1):
        d = t.bit_length() - 1
        idx = np.nonzero(_np_route_to_depth(X, uniq, a, th, d) == t)[0].astype(np.int32)
        if not (len(idx) > 1 and len(np.unique(y[idx])) > 1):
            continue
        Dt = min(horizon, depth - d)
        if Dt >= 2:
            seeds = []
            if deo:  # the subtree at t: local level r, position j -> node (t << r) + j
                nodes = [(t << r) + j for r in range(Dt) for j in range(1 << r)]
                seeds.append(genes([wa[v - 1] for v in nodes], [wth[v - 1] for v in nodes]))
            if cart:
                ga, gt = oracle.greedy_tree(ranks, nu, y, K, Dt, idx=idx)
                seeds.append(genes(ga, gt))
            out = oracle.de_run(ranks, nu, y, K, depth=Dt, P=P, G=G, seed=seed, stream=t, idx=idx,
                                seeds=np.stack(seeds))
            dga, dgt = oracle.decode(out["pop"][out["best"]][None], Dt, nu)
            a[t - 1], th[t - 1] = dga[0, 0], dgt[0, 0]
        else:
            a1, t1, _ = oracle.depth1(ranks, nu, y, K, idx=idx)
            a[t - 1], th[t - 1] = a1, t1
    np.testing.assert_array_equal(got["a"], a)
    np.testing.assert_array_equal(got["theta"], th)
    assert (got["kind"] == 2).sum() >= 3
