"""CPU oracle for the MH-DEOCT hot path (arXiv 2311.06952) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
``--impl reference`` legs may import this package.  The product library under
``paper_2311_06952_gb300/`` never imports it, and this package imports nothing
from there: the two share no code.  Inputs come from the seeded generators in
``paper_2311_06952_gb300.datagen`` (data only, none of the method's arithmetic),
passed in by the caller.

The arithmetic lives in ``deoct_oracle.c`` (plain single-threaded C, built with
``-O2 -ffp-contract=off``); this module only marshals numpy arrays into it.  Its
OpenMP twins (``encode_omp``, ``eval_counts_omp``, and the counting inside
``de_run`` / ``mh`` after ``set_threads(n > 1)``) compute the same integers on
several host cores; tests pin them bit for bit to the plain functions.
Each wrapper names the paper passage its C function follows.

Parity status per function (see the tests under ``tests/test_oracle_*.py``):
  encode, decode, eval_counts, fitness, leaf_classes, depth1 -- pinned (numpy.unique,
      float-midpoint routing of Eq. benc, brute force, the loss identity of Section 2);
  philox / draw32 -- pinned to numpy's Philox4x64-10 bit generator;
  de_trial, de_run -- Eq. mutation, Eq. crossover, the clamp and the initial
      population pinned bit for bit to a numpy float32 restatement driven by
      numpy's own Philox stream, plus closed forms (CR = 1, CR = 0, M = 0) and the
      invariants of selection; the draw-to-index maps and the clamp are readings
      of the paper (its text fixes neither), pinned as stated;
  node_genes -- decodes back to every (a, theta) under Eq. aenc / Eq. benc;
  greedy_tree -- the CART warm start: pinned to a float-threshold restatement
      (brute force over midpoints, top down);
  mh -- pinned by special cases (horizon 1 = greedy misclassification tree,
      n_min >= n, single class) and by Algorithm 2 restated in Python over the
      pinned de_run and depth1 (subsets induced on raw float thresholds), with
      and without the CART and DEOCT warm starts (restated over greedy_tree,
      de_run and node_genes);
  split_values, predict -- routing training samples on raw thresholds equals
      routing ranks; the thresholds are the midpoints of the threshold set.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "deoct_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0


def build(force: bool = False) -> str:
    """Compile ``deoct_oracle.c`` into ``oracle/liboracle.so`` with gcc."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-Wall",
               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        # the OpenMP twins (timing, full-size checks); without OpenMP they run on one thread
        r = subprocess.run(cmd[:-3] + ["-fopenmp"] + cmd[-3:], capture_output=True)
        if r.returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class DEParams(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("P", ctypes.c_int32), ("G", ctypes.c_int32),
                ("M", ctypes.c_float), ("CR", ctypes.c_float), ("alpha", ctypes.c_double),
                ("n_min", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_uint64), ("dither", ctypes.c_int32)]


class MHParams(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("horizon", ctypes.c_int32), ("P", ctypes.c_int32),
                ("G", ctypes.c_int32), ("M", ctypes.c_float), ("CR", ctypes.c_float),
                ("alpha", ctypes.c_double), ("n_min", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("dither", ctypes.c_int32), ("cart_seeds", ctypes.c_int32),
                ("de_seeds", ctypes.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_draw32.restype = ctypes.c_uint32
            _lib.orc_draw32.argtypes = [ctypes.c_uint64] * 5
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def encode(X):
    """Section 3.1 threshold sets as dense ranks: X [n][F] float32 -> (ranks [F][n] uint32, n_unique [F])."""
    X = _c(X, np.float32)
    n, F = X.shape
    ranks = np.empty((F, n), np.uint32)
    nu = np.empty(F, np.uint32)
    rc = lib().orc_encode(_p(X), ctypes.c_int64(n), ctypes.c_int32(F), _p(ranks), _p(nu))
    if rc != ORC_OK:
        raise ValueError("oracle encode failed: %d" % rc)
    return ranks, nu


def set_threads(n):
    """Threads of the OpenMP twins (encode_omp, eval_counts_omp, and the counting inside
    de_run / mh); 1 restores the plain loops.  Returns the previous setting."""
    return int(lib().orc_set_threads(ctypes.c_int(int(n))))


def host_cores():
    """Cores this process may run on (the thread count the timed oracle uses)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def encode_omp(X):
    """encode() with the features spread over the set_threads() threads (same result)."""
    X = _c(X, np.float32)
    n, F = X.shape
    ranks = np.empty((F, n), np.uint32)
    nu = np.empty(F, np.uint32)
    rc = lib().orc_encode_omp(_p(X), ctypes.c_int64(n), ctypes.c_int32(F), _p(ranks), _p(nu))
    if rc != ORC_OK:
        raise ValueError("oracle encode failed: %d" % rc)
    return ranks, nu


def eval_counts_omp(ranks, y, K, a, theta, depth, idx=None):
    """eval_counts() with (tree, sample chunk) work spread over the set_threads() threads."""
    ranks = _c(ranks, np.uint32)
    y = _c(y, np.uint8)
    a = _c(a, np.int32)
    theta = _c(theta, np.uint32)
    F, n = ranks.shape
    P = a.shape[0]
    counts = np.empty((P, 1 << depth, K), np.uint32)
    idx_arr = None if idx is None else _c(idx, np.int32)
    n_sub = n if idx is None else len(idx_arr)
    lib().orc_eval_counts_omp(_p(ranks), ctypes.c_int64(n), ctypes.c_int32(F), _p(y), ctypes.c_int32(K),
                              _p(idx_arr), ctypes.c_int64(n_sub), _p(a), _p(theta),
                              ctypes.c_int32(P), ctypes.c_int32(depth), _p(counts))
    return counts


def philox(counter, key):
    """Philox4x64-10 block (Salmon et al., SC'11) for a 4-word counter and 2-word key."""
    c = _c(counter, np.uint64)
    k = _c(key, np.uint64)
    out = np.empty(4, np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def draw32(seed, stream, g, r, s):
    return int(lib().orc_draw32(seed, stream, g, r, s))


def decode(genes, depth, n_unique):
    """Eq. aenc / Eq. benc: genes [P][2B] float32 -> (a [P][B] int32 in 0..F, theta [P][B] uint32)."""
    genes = _c(genes, np.float32)
    nu = _c(n_unique, np.uint32)
    P = genes.shape[0]
    B = (1 << depth) - 1
    assert genes.shape[1] == 2 * B
    a = np.empty((P, B), np.int32)
    th = np.empty((P, B), np.uint32)
    lib().orc_decode(_p(genes), ctypes.c_int32(P), ctypes.c_int32(depth), ctypes.c_int32(len(nu)),
                     _p(nu), _p(a), _p(th))
    return a, th


def eval_counts(ranks, y, K, a, theta, depth, idx=None):
    """Algorithm 1 class-count matrix: counts [P][2^D][K] uint32."""
    ranks = _c(ranks, np.uint32)
    y = _c(y, np.uint8)
    a = _c(a, np.int32)
    theta = _c(theta, np.uint32)
    F, n = ranks.shape
    P = a.shape[0]
    L = 1 << depth
    counts = np.empty((P, L, K), np.uint32)
    idx_arr = None if idx is None else _c(idx, np.int32)
    n_sub = n if idx is None else len(idx_arr)
    lib().orc_eval_counts(_p(ranks), ctypes.c_int64(n), ctypes.c_int32(F), _p(y), ctypes.c_int32(K),
                          _p(idx_arr), ctypes.c_int64(n_sub), _p(a), _p(theta),
                          ctypes.c_int32(P), ctypes.c_int32(depth), _p(counts))
    return counts


def fitness(counts, a, n_sub, n_min=1, alpha=0.0):
    """Section 3.2 fitness: returns (fit [P] f64, errors [P], splits [P], V [P])."""
    counts = _c(counts, np.uint32)
    a = _c(a, np.int32)
    P, L, K = counts.shape
    depth = L.bit_length() - 1
    fit = np.empty(P, np.float64)
    err = np.empty(P, np.uint32)
    spl = np.empty(P, np.uint32)
    v = np.empty(P, np.uint32)
    lib().orc_fitness(_p(counts), _p(a), ctypes.c_int32(P), ctypes.c_int32(depth), ctypes.c_int32(K),
                      ctypes.c_int64(n_sub), ctypes.c_int32(n_min), ctypes.c_double(alpha),
                      _p(fit), _p(err), _p(spl), _p(v))
    return fit, err, spl, v


def leaf_classes(counts):
    """Eq. opt_c leaf classes (lowest class on ties): [P][2^D] uint8."""
    counts = _c(counts, np.uint32)
    P, L, K = counts.shape
    out = np.empty((P, L), np.uint8)
    lib().orc_leaf_classes(_p(counts), ctypes.c_int32(P), ctypes.c_int32(L.bit_length() - 1),
                           ctypes.c_int32(K), _p(out))
    return out


def de_trial(pop, best, g, r, F, depth, M=0.5, CR=0.9, seed=0, stream=0, dither=False):
    """One trial vector (Eq. mutation + Eq. crossover) with its draws: (u, r1, r2, q_rand)."""
    pop = _c(pop, np.float32)
    P = pop.shape[0]
    B = (1 << depth) - 1
    prm = DEParams(depth, P, 0, M, CR, 0.0, 1, seed, stream, int(dither))
    u = np.empty(2 * B, np.float32)
    r1 = ctypes.c_int32()
    r2 = ctypes.c_int32()
    qr = ctypes.c_int32()
    lib().orc_de_trial(_p(pop), ctypes.c_int32(P), ctypes.c_int32(B), ctypes.c_int32(F),
                       ctypes.c_int32(best), ctypes.byref(prm), ctypes.c_int32(g), ctypes.c_int32(r),
                       _p(u), ctypes.byref(r1), ctypes.byref(r2), ctypes.byref(qr))
    return u, r1.value, r2.value, qr.value


def de_run(ranks, n_unique, y, K, depth, P, G, M=0.5, CR=0.9, alpha=0.0, n_min=1, seed=0,
           stream=0, dither=False, idx=None, seeds=None, history=False):
    """Algorithm 4 (DEOCT).  Returns dict(pop, fit, best[, best_fit_hist, pop_hist, fit_hist])."""
    ranks = _c(ranks, np.uint32)
    nu = _c(n_unique, np.uint32)
    y = _c(y, np.uint8)
    F, n = ranks.shape
    B = (1 << depth) - 1
    prm = DEParams(depth, P, G, M, CR, alpha, n_min, seed, stream, int(dither))
    idx_arr = None if idx is None else _c(idx, np.int32)
    n_sub = n if idx is None else len(idx_arr)
    seeds_arr = None if seeds is None else _c(seeds, np.float32).reshape(-1, 2 * B)
    S = 0 if seeds_arr is None else seeds_arr.shape[0]
    pop = np.empty((P, 2 * B), np.float32)
    fit = np.empty(P, np.float64)
    best = ctypes.c_int32()
    bh = np.empty(G + 1, np.float64) if history else None
    ph = np.empty((G + 1, P, 2 * B), np.float32) if history else None
    fh = np.empty((G + 1, P), np.float64) if history else None
    rc = lib().orc_de_run(_p(ranks), ctypes.c_int64(n), ctypes.c_int32(F), _p(nu), _p(y),
                          ctypes.c_int32(K), _p(idx_arr), ctypes.c_int64(n_sub), ctypes.byref(prm),
                          _p(seeds_arr), ctypes.c_int32(S), _p(pop), _p(fit), ctypes.byref(best),
                          _p(bh), _p(ph), _p(fh))
    if rc != ORC_OK:
        raise ValueError("oracle de_run failed: %d" % rc)
    out = dict(pop=pop, fit=fit, best=best.value)
    if history:
        out.update(best_fit_hist=bh, pop_hist=ph, fit_hist=fh)
    return out


def depth1(ranks, n_unique, y, K, idx=None, n_min=1, alpha=0.0):
    """Exhaustive depth-1 subtree (Algorithm 2, bottom level): (a, theta, fitness)."""
    ranks = _c(ranks, np.uint32)
    nu = _c(n_unique, np.uint32)
    y = _c(y, np.uint8)
    F, n = ranks.shape
    idx_arr = None if idx is None else _c(idx, np.int32)
    n_sub = n if idx is None else len(idx_arr)
    a = ctypes.c_int32()
    th = ctypes.c_uint32()
    f = ctypes.c_double()
    rc = lib().orc_depth1(_p(ranks), ctypes.c_int64(n), ctypes.c_int32(F), _p(nu), _p(y),
                          ctypes.c_int32(K), _p(idx_arr), ctypes.c_int64(n_sub), ctypes.c_int32(n_min),
                          ctypes.c_double(alpha), ctypes.byref(a), ctypes.byref(th), ctypes.byref(f))
    if rc != ORC_OK:
        raise ValueError("oracle depth1 failed: %d" % rc)
    return a.value, th.value, f.value


def greedy_tree(ranks, n_unique, y, K, depth, idx=None, n_min=1, alpha=0.0):
    """Greedy misclassification tree (the CART warm start of Algorithm 2): (a [B], theta [B])."""
    ranks = _c(ranks, np.uint32)
    nu = _c(n_unique, np.uint32)
    y = _c(y, np.uint8)
    F, n = ranks.shape
    B = (1 << depth) - 1
    idx_arr = None if idx is None else _c(idx, np.int32)
    n_sub = n if idx is None else len(idx_arr)
    a = np.empty(B, np.int32)
    th = np.empty(B, np.uint32)
    rc = lib().orc_greedy_tree(_p(ranks), ctypes.c_int64(n), ctypes.c_int32(F), _p(nu), _p(y),
                               ctypes.c_int32(K), _p(idx_arr), ctypes.c_int64(n_sub), ctypes.c_int32(depth),
                               ctypes.c_int32(n_min), ctypes.c_double(alpha), _p(a), _p(th))
    if rc != ORC_OK:
        raise ValueError("oracle greedy_tree failed: %d" % rc)
    return a, th


def node_genes(a, theta, n_p):
    """Genes of decoded nodes (the inverse of Eq. aenc / Eq. benc used for warm starts):
    a, theta, n_p [m] -> (ahat [m] float32, bhat [m] float32)."""
    a = _c(a, np.int32)
    theta = _c(theta, np.uint32)
    n_p = _c(n_p, np.uint32)
    m = len(a)
    ah = np.empty(m, np.float32)
    bh = np.empty(m, np.float32)
    lib().orc_node_genes(_p(a), _p(theta), _p(n_p), ctypes.c_int64(m), _p(ah), _p(bh))
    return ah, bh


def mh(ranks, n_unique, y, K, depth, horizon, P, G, M=0.5, CR=0.9, alpha=0.0, n_min=1, seed=0,
       dither=False, cart_seeds=False, de_seeds=False):
    """Algorithm 2 (moving-horizon DEOCT): dict(a, theta, leaf_class, kind, node_fit)."""
    ranks = _c(ranks, np.uint32)
    nu = _c(n_unique, np.uint32)
    y = _c(y, np.uint8)
    F, n = ranks.shape
    B = (1 << depth) - 1
    prm = MHParams(depth, horizon, P, G, M, CR, alpha, n_min, seed, int(dither), int(cart_seeds),
                   int(de_seeds))
    a = np.empty(B, np.int32)
    th = np.empty(B, np.uint32)
    lc = np.empty(1 << depth, np.uint8)
    kind = np.empty(B, np.int32)
    nf = np.empty(B, np.float64)
    rc = lib().orc_mh(_p(ranks), ctypes.c_int64(n), ctypes.c_int32(F), _p(nu), _p(y), ctypes.c_int32(K),
                      ctypes.byref(prm), _p(a), _p(th), _p(lc), _p(kind), _p(nf))
    if rc != ORC_OK:
        raise ValueError("oracle mh failed: %d" % rc)
    return dict(a=a, theta=th, leaf_class=lc, kind=kind, node_fit=nf)


def split_values(X, a, theta):
    """Raw-unit thresholds of a fitted tree (threshold set B_p of Section 3.1): b [B] float64."""
    X = _c(X, np.float32)
    a = _c(a, np.int32)
    theta = _c(theta, np.uint32)
    n, F = X.shape
    b = np.empty(len(a), np.float64)
    rc = lib().orc_split_values(_p(X), ctypes.c_int64(n), ctypes.c_int32(F), _p(a), _p(theta),
                                ctypes.c_int32(len(a)), _p(b))
    if rc != ORC_OK:
        raise ValueError("oracle split_values failed: %d" % rc)
    return b


def predict(X, a, b, depth, leaf_class):
    """Leaf class of every row of X routed on raw values (Section 2)."""
    X = _c(X, np.float32)
    a = _c(a, np.int32)
    b = _c(b, np.float64)
    lc = _c(leaf_class, np.uint8)
    m, F = X.shape
    out = np.empty(m, np.uint8)
    lib().orc_predict(_p(X), ctypes.c_int64(m), ctypes.c_int32(F), _p(a), _p(b), ctypes.c_int32(depth),
                      _p(lc), _p(out))
    return out
