"""Seeded synthetic inputs for the MH-DEOCT hot path.

This module holds data generation only -- none of the method's arithmetic (no
rank encoding, decoding, routing by ranks, counting or fitness).  Both the
CUDA path and the CPU oracle are fed from here by the tests and the bench, so
the two sides see the same bytes.

The paper measures on UCI datasets and on Bitcoin Heist, SUSY and HIGGS
(Section 5, Table 3); none of them is available here.  The generators below
stand in for them with the shapes of the paper's large-scale sets: millions of
samples, 8-30 continuous features, 2-29 classes, ties in the features, labels
from an axis-aligned tree plus uniform label noise.

Workloads (``make_workload(i)``):
  0  tiny MH/DEOCT fit: n=1000, F=8, U(0,1) rounded to 3 decimals, K=2,
     planted depth-3 tree, 5% flips; fit depth 2, P=64, G=100, M=0.5, CR=0.9.
  1  population evaluation: n=100000, F=20, 3-component isotropic Gaussian
     mixture (means ~ N(0, 4I), unit variance), K=3 = the component, 10% flips;
     256 random depth-3 candidates (feature uniform, threshold rank uniform).
  2  batched moving-horizon fit: n=1e6, F=30 (15 U(0,1) + 15 LogNormal(0,1)),
     K=4, planted depth-6 tree, 5% flips; D=8, horizon 3, P=128, G=200.
  3  large-scale DEOCT: n=1e7, F=10, U(0,1) quantised to 60000 levels, K=2,
     planted depth-4 tree, 2% flips; D=4, P=1024, G=50.
  4  serving: 500 requests, Poisson arrivals at 20/s, n log-uniform in
     [1e3, 2e6], F in [4, 60], K in [2, 10], depth in [2, 6], horizon in {2, 3},
     Gaussian-mixture features, planted-tree labels, 5% flips.
"""
from __future__ import annotations

import numpy as np

DATA_SEED_BASE = 1000


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def flip_labels(y, K, frac, rng):
    """Replace a fraction ``frac`` of labels by a uniform draw from the other K-1 classes."""
    y = y.copy()
    if K < 2 or frac <= 0:
        return y
    hit = rng.random(len(y)) < frac
    shift = rng.integers(1, K, size=int(hit.sum()))
    y[hit] = (y[hit].astype(np.int64) + shift) % K
    return y


def planted_tree_labels(X, depth, K, rng):
    """Labels of an axis-aligned depth-``depth`` tree on the raw float values.

    Each branch node splits a uniformly drawn feature at the median of the
    samples that reach it (x < median goes left); leaf classes are
    0,1,..,K-1,0,1,.. over the 2^depth leaves, shuffled.
    """
    n, F = X.shape
    node = np.ones(n, np.int64)
    for d in range(depth):
        nxt = np.empty_like(node)
        for t in range(1 << d, 1 << (d + 1)):
            sel = node == t
            f = int(rng.integers(0, F))
            if sel.any():
                thr = np.median(X[sel, f])
                left = X[sel, f] < thr
            else:
                left = np.zeros(0, bool)
            nxt[sel] = np.where(left, 2 * t, 2 * t + 1)
        node = nxt
    L = 1 << depth
    leaf_class = np.arange(L) % K
    rng.shuffle(leaf_class)
    return leaf_class[node - L].astype(np.uint8)


def gaussian_mixture(n, F, K, rng, mean_std=2.0):
    means = rng.normal(0.0, mean_std, size=(K, F))
    comp = rng.integers(0, K, size=n)
    X = means[comp] + rng.normal(0.0, 1.0, size=(n, F))
    return X.astype(np.float32), comp.astype(np.uint8)


def random_population(n_unique, P, depth, rng, allow_nosplit=False):
    """Decoded random candidates: a [P][B] in 1..F (0..F if allow_nosplit),
    theta [P][B] uniform in {0..n_p-1} of the chosen feature."""
    F = len(n_unique)
    B = (1 << depth) - 1
    lo = 0 if allow_nosplit else 1
    a = rng.integers(lo, F + 1, size=(P, B)).astype(np.int32)
    nu = np.asarray(n_unique, np.int64)
    u = rng.random((P, B))
    npick = np.where(a > 0, nu[np.maximum(a - 1, 0)], 1)
    theta = np.floor(u * npick).astype(np.int64)
    theta = np.minimum(theta, npick - 1)
    theta = np.where(a > 0, theta, 0).astype(np.uint32)
    return a, theta


def random_genes(P, depth, F, rng):
    """Uniform genes in the ranges of Section 3.1: ahat in [0, F+1), bhat in [0, 1)."""
    B = (1 << depth) - 1
    g = np.empty((P, 2 * B), np.float32)
    g[:, :B] = (rng.random((P, B)) * (F + 1)).astype(np.float32)
    g[:, B:] = rng.random((P, B)).astype(np.float32)
    hi_a = np.nextafter(np.float32(F + 1), np.float32(0))
    hi_b = np.nextafter(np.float32(1), np.float32(0))
    g[:, :B] = np.minimum(g[:, :B], hi_a)
    g[:, B:] = np.minimum(g[:, B:], hi_b)
    return g


def make_workload(i, n=None, seed=None):
    """Synthetic inputs of workload ``i`` (0..3); ``n`` overrides the sample count."""
    rng = _rng(DATA_SEED_BASE + i if seed is None else seed)
    if i == 0:
        n = 1000 if n is None else n
        F, K = 8, 2
        X = np.round(rng.random((n, F)), 3).astype(np.float32)
        y = planted_tree_labels(X, 3, K, rng)
        y = flip_labels(y, K, 0.05, rng)
        return dict(name="tiny-deoct", X=X, y=y, K=K, depth=2, horizon=2, P=64, G=100,
                    M=0.5, CR=0.9, seed=0)
    if i == 1:
        n = 100_000 if n is None else n
        F, K = 20, 3
        X, y = gaussian_mixture(n, F, K, rng)
        y = flip_labels(y, K, 0.10, rng)
        return dict(name="eval-gmm", X=X, y=y, K=K, depth=3, P=256, rank_bytes=4, pop_seed=7)
    if i == 2:
        n = 1_000_000 if n is None else n
        F, K = 30, 4
        X = np.empty((n, F), np.float32)
        X[:, :15] = rng.random((n, 15))
        X[:, 15:] = rng.lognormal(0.0, 1.0, size=(n, 15))
        y = planted_tree_labels(X, 6, K, rng)
        y = flip_labels(y, K, 0.05, rng)
        return dict(name="mh-batched", X=X, y=y, K=K, depth=8, horizon=3, P=128, G=200,
                    M=0.5, CR=0.9, seed=0, rank_bytes=4)
    if i == 3:
        n = 10_000_000 if n is None else n
        F, K = 10, 2
        X = (np.floor(rng.random((n, F)) * 60000.0) / 60000.0).astype(np.float32)
        y = planted_tree_labels(X, 4, K, rng)
        y = flip_labels(y, K, 0.02, rng)
        return dict(name="large-deoct", X=X, y=y, K=K, depth=4, P=1024, G=50, M=0.5, CR=0.9,
                    seed=0, rank_bytes=2)
    raise ValueError("workload %d has no single dataset (use serving_requests)" % i)


def serving_requests(num=500, rate=20.0, seed=DATA_SEED_BASE + 4, n_range=(1_000, 2_000_000),
                     materialize=True):
    """Request stream of the serving workload: list of dicts with arrival time and data."""
    rng = _rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=num))
    reqs = []
    for j in range(num):
        n = int(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))))
        F = int(rng.integers(4, 61))
        K = int(rng.integers(2, 11))
        D = int(rng.integers(2, 7))
        H = int(rng.integers(2, 4))
        req = dict(id=j, arrival=float(t[j]), n=n, F=F, K=K, depth=D, horizon=H,
                   data_seed=int(rng.integers(0, 2**31 - 1)))
        if materialize:
            req.update(make_request_data(req))
        reqs.append(req)
    return reqs


def make_request_data(req):
    rng = _rng(req["data_seed"])
    X, _ = gaussian_mixture(req["n"], req["F"], req["K"], rng)
    y = planted_tree_labels(X, req["depth"], req["K"], rng)
    y = flip_labels(y, req["K"], 0.05, rng)
    return dict(X=X, y=y)


# Shapes of the paper's large-scale sets (Table 3): samples, features, classes.
TABLE3_SHAPES = {"bitcoin-heist": (2_916_697, 8, 29), "susy": (5_000_000, 18, 2),
                 "higgs": (11_000_000, 28, 2)}


def table3_standin(name, seed=2000, train_frac=0.75):
    """Synthetic stand-in with the shape of one of the paper's large-scale sets:
    Gaussian-mixture features (K components), labels from a planted depth-6 tree,
    5% flips; split 75/25 into train and test as in Section 5."""
    N, F, K = TABLE3_SHAPES[name]
    rng = _rng(seed + sum(name.encode()))
    X, _ = gaussian_mixture(N, F, K, rng)
    y = planted_tree_labels(X, 6, K, rng)
    y = flip_labels(y, K, 0.05, rng)
    perm = rng.permutation(N)
    ntr = int(N * train_frac)
    tr, te = perm[:ntr], perm[ntr:]
    return dict(name=name, Xtr=X[tr], ytr=y[tr], Xte=X[te], yte=y[te], K=K)
