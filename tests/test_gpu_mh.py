"""GPU parity of the moving-horizon driver (Algorithm 2) and the exhaustive
depth-1 search, plain per-node form and batched level form, against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2311_06952_gb300 import datagen

from gpu_helpers import ctx, gpu_dataset, to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2311_06952_gb300 import build
    build.build()
    return ctx()


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


D1_CASES = [
    # n, F, K, rank_bytes, subset, n_min, alpha, seed
    (500, 4, 2, 2, False, 1, 0.0, 0),
    (3000, 6, 3, 4, True, 1, 0.0, 1),
    (3000, 6, 5, 2, False, 40, 0.0, 2),
    (2000, 3, 4, 4, True, 5, 0.5, 3),
    (1, 2, 2, 2, False, 1, 0.0, 4),
    (40000, 8, 2, 4, False, 1, 0.0, 5),   # nearly all ranks distinct
]


@pytest.mark.parametrize("case", D1_CASES, ids=[str(x) for x in D1_CASES])
def test_depth1_search_bit_exact(c, case):
    from paper_2311_06952_gb300 import deoct
    n, F, K, rb, subset, n_min, alpha, seed = case
    rng = _rng(300 + seed)
    X = (np.round(rng.random((n, F)), 2) if seed != 5 else rng.random((n, F))).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    if n > 10:
        y[X[:, 0] < 0.3] = 0  # some structure so that splits win
    ds = gpu_dataset(c, X, y, K, rb)
    ranks, nu = oracle.encode(X)
    idx = None
    if subset:
        idx = rng.permutation(n)[: n // 2].astype(np.int32)
    a, th, f = deoct.deoct_depth1_search(c, ds, sample_idx=None if idx is None else to_dev(idx),
                                         n_min=n_min, alpha=alpha)
    ra, rth, rf = oracle.depth1(ranks, nu, y, K, idx=idx, n_min=n_min, alpha=alpha)
    assert (a, th, f) == (ra, rth, rf)


def _mh_case(name):
    if name == "w0_d3h2":
        w = datagen.make_workload(0)
        return w["X"], w["y"], w["K"], dict(depth=3, horizon=2, P=32, G=20, seed=0), 2
    if name == "w0_d2h2":
        w = datagen.make_workload(0)
        return w["X"], w["y"], w["K"], dict(depth=2, horizon=2, P=64, G=100, seed=0), 2
    if name == "w2_small":
        w = datagen.make_workload(2, n=12000)
        return w["X"], w["y"], w["K"], dict(depth=5, horizon=3, P=24, G=8, seed=3), 4
    if name == "k3_d4h3_nmin":
        rng = _rng(41)
        X = np.round(rng.random((5000, 5)), 2).astype(np.float32)
        y = datagen.planted_tree_labels(X, 3, 3, rng)
        return X, y, 3, dict(depth=4, horizon=3, P=16, G=6, seed=9, n_min=30, alpha=0.5), 2
    if name == "small_pop":
        # 6 individuals per node: every evaluator shape the batched level tries
        # has fewer than 16 trees per group (the streaming kernel)
        w = datagen.make_workload(2, n=20000)
        return w["X"], w["y"], w["K"], dict(depth=5, horizon=3, P=6, G=5, seed=5), 2
    if name == "horizon1":
        rng = _rng(42)
        X = np.round(rng.random((3000, 4)), 2).astype(np.float32)
        y = rng.integers(0, 3, 3000).astype(np.uint8)
        return X, y, 3, dict(depth=4, horizon=1, P=8, G=1, seed=0), 4
    raise KeyError(name)


@pytest.mark.parametrize("name", ["w0_d2h2", "w0_d3h2", "w2_small", "k3_d4h3_nmin", "small_pop",
                                  "horizon1"])
@pytest.mark.parametrize("batched", [False, True])
def test_moving_horizon_bit_exact(c, name, batched):
    from paper_2311_06952_gb300 import deoct
    X, y, K, kw, rb = _mh_case(name)
    ds = gpu_dataset(c, X, y, K, rb)
    ranks, nu = oracle.encode(X)
    ref = oracle.mh(ranks, nu, y, K, depth=kw["depth"], horizon=kw["horizon"], P=kw["P"], G=kw["G"],
                    seed=kw["seed"], n_min=kw.get("n_min", 1), alpha=kw.get("alpha", 0.0))
    prm = deoct.make_params(kw["depth"], kw["P"], kw["G"], seed=kw["seed"], horizon=kw["horizon"],
                            n_min=kw.get("n_min", 1), alpha=kw.get("alpha", 0.0),
                            flags=deoct.DEOCT_BATCHED if batched else 0)
    out = deoct.deoct_fit_moving_horizon(c, ds, prm)
    np.testing.assert_array_equal(out["kind"], ref["kind"])
    np.testing.assert_array_equal(out["a"].astype(np.int32), ref["a"])
    np.testing.assert_array_equal(out["theta"], ref["theta"])
    np.testing.assert_array_equal(out["node_fit"], ref["node_fit"])
    np.testing.assert_array_equal(out["leaf_class"], ref["leaf_class"])


def test_moving_horizon_special_cases(c):
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(0, n=300)
    ds = gpu_dataset(c, w["X"], w["y"], 2, 2)
    out = deoct.deoct_fit_moving_horizon(c, ds, deoct.make_params(3, 16, 3, horizon=2, n_min=300))
    assert np.all(out["a"] == 0) and np.all(out["kind"] == 0)
    ds1 = gpu_dataset(c, w["X"], np.ones(300, np.uint8), 2, 2)
    out = deoct.deoct_fit_moving_horizon(c, ds1, deoct.make_params(3, 16, 3, horizon=2,
                                                                   flags=deoct.DEOCT_BATCHED))
    assert np.all(out["a"] == 0) and out["leaf_class"][-1] == 1


@pytest.mark.slow
def test_moving_horizon_workload2_batched_equals_plain(c):
    """Batched-level moving-horizon workload shape (F=30, K=4, uint32 ranks, D=8, horizon 3) at
    reduced size: the batched and plain forms give the same tree; the oracle agrees on the
    nodes of the first levels it can afford."""
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(2, n=60000)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], 4)
    kw = dict(depth=8, horizon=3, P=32, G=10, seed=0)
    outs = []
    for flags in (0, deoct.DEOCT_BATCHED):
        prm = deoct.make_params(kw["depth"], kw["P"], kw["G"], seed=0, horizon=3, flags=flags)
        outs.append(deoct.deoct_fit_moving_horizon(c, ds, prm))
    for k in ("a", "theta", "kind", "node_fit", "leaf_class"):
        np.testing.assert_array_equal(outs[0][k], outs[1][k])
    ranks, nu = oracle.encode(w["X"])
    ref = oracle.mh(ranks, nu, w["y"], w["K"], depth=8, horizon=3, P=32, G=10, seed=0)
    np.testing.assert_array_equal(outs[1]["a"].astype(np.int32), ref["a"])
    np.testing.assert_array_equal(outs[1]["theta"], ref["theta"])
    np.testing.assert_array_equal(outs[1]["leaf_class"], ref["leaf_class"])


@pytest.mark.parametrize("name", ["w0_d3h2", "w2_small", "k3_d4h3_nmin"])
@pytest.mark.parametrize("batched", [False, True])
def test_moving_horizon_cart_seeds_bit_exact(c, name, batched):
    """CART warm starts (Algorithm 2): each DEOCT subtree starts with its greedy tree."""
    from paper_2311_06952_gb300 import deoct
    X, y, K, kw, rb = _mh_case(name)
    ds = gpu_dataset(c, X, y, K, rb)
    ranks, nu = oracle.encode(X)
    ref = oracle.mh(ranks, nu, y, K, depth=kw["depth"], horizon=kw["horizon"], P=kw["P"], G=kw["G"],
                    seed=kw["seed"], n_min=kw.get("n_min", 1), alpha=kw.get("alpha", 0.0), cart_seeds=True)
    flags = deoct.DEOCT_CART_SEEDS | (deoct.DEOCT_BATCHED if batched else 0)
    prm = deoct.make_params(kw["depth"], kw["P"], kw["G"], seed=kw["seed"], horizon=kw["horizon"],
                            n_min=kw.get("n_min", 1), alpha=kw.get("alpha", 0.0), flags=flags)
    out = deoct.deoct_fit_moving_horizon(c, ds, prm)
    for k in ("kind", "theta", "node_fit", "leaf_class"):
        np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
    np.testing.assert_array_equal(out["a"].astype(np.int32), ref["a"])


@pytest.mark.parametrize("name", ["w0_d3h2", "k3_d4h3_nmin"])
@pytest.mark.parametrize("both", [False, True])
def test_moving_horizon_deoct_seeds_bit_exact(c, name, both):
    """DEOCT warm starts (Algorithm 2): each subtree starts from the full-depth DEOCT's subtree at
    its location (and, with both flags, also from its greedy tree)."""
    from paper_2311_06952_gb300 import deoct
    X, y, K, kw, rb = _mh_case(name)
    ds = gpu_dataset(c, X, y, K, rb)
    ranks, nu = oracle.encode(X)
    ref = oracle.mh(ranks, nu, y, K, depth=kw["depth"], horizon=kw["horizon"], P=kw["P"], G=kw["G"],
                    seed=kw["seed"], n_min=kw.get("n_min", 1), alpha=kw.get("alpha", 0.0),
                    cart_seeds=both, de_seeds=True)
    flags = deoct.DEOCT_DE_SEEDS | deoct.DEOCT_BATCHED | (deoct.DEOCT_CART_SEEDS if both else 0)
    prm = deoct.make_params(kw["depth"], kw["P"], kw["G"], seed=kw["seed"], horizon=kw["horizon"],
                            n_min=kw.get("n_min", 1), alpha=kw.get("alpha", 0.0), flags=flags)
    out = deoct.deoct_fit_moving_horizon(c, ds, prm)
    for k in ("kind", "theta", "node_fit", "leaf_class"):
        np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
    np.testing.assert_array_equal(out["a"].astype(np.int32), ref["a"])


@pytest.mark.parametrize("depth,horizon,F,n_min", [(1, 2, 3, 1), (3, 5, 1, 1), (4, 2, 2, 0)])
def test_moving_horizon_edge_shapes(c, depth, horizon, F, n_min):
    """Depth 1 (a single depth-1 search), horizon beyond the depth, one feature, n_min = 0."""
    from paper_2311_06952_gb300 import deoct
    rng = _rng(600 + depth * 10 + F)
    X = np.round(rng.random((2000, F)), 2).astype(np.float32)
    y = rng.integers(0, 3, 2000).astype(np.uint8)
    ds = gpu_dataset(c, X, y, 3, 2)
    ranks, nu = oracle.encode(X)
    ref = oracle.mh(ranks, nu, y, 3, depth=depth, horizon=horizon, P=16, G=5, seed=1, n_min=n_min)
    for flags in (0, deoct.DEOCT_BATCHED):
        out = deoct.deoct_fit_moving_horizon(c, ds, deoct.make_params(depth, 16, 5, seed=1, horizon=horizon,
                                                                      n_min=n_min, flags=flags))
        np.testing.assert_array_equal(out["a"].astype(np.int32), ref["a"])
        np.testing.assert_array_equal(out["theta"], ref["theta"])
        np.testing.assert_array_equal(out["kind"], ref["kind"])
        np.testing.assert_array_equal(out["leaf_class"], ref["leaf_class"])


def test_moving_horizon_streaming_kernel_forced_bit_exact(c):
    """The batched level solve with the streaming kernel for every evaluation: same tree."""
    from paper_2311_06952_gb300 import deoct
    X, y, K, kw, rb = _mh_case("w2_small")
    ds = gpu_dataset(c, X, y, K, rb)
    ranks, nu = oracle.encode(X)
    ref = oracle.mh(ranks, nu, y, K, depth=kw["depth"], horizon=kw["horizon"], P=kw["P"], G=kw["G"],
                    seed=kw["seed"])
    prm = deoct.make_params(kw["depth"], kw["P"], kw["G"], seed=kw["seed"], horizon=kw["horizon"],
                            flags=deoct.DEOCT_BATCHED)
    try:
        c.set_eval_streaming(True)
        out = deoct.deoct_fit_moving_horizon(c, ds, prm)
    finally:
        c.set_eval_streaming(False)
    for k in ("kind", "a", "theta", "node_fit", "leaf_class"):
        np.testing.assert_array_equal(out[k].astype(ref[k].dtype), ref[k], err_msg=k)


def test_autotuned_level_solve_equals_plain_at_workload_size(c):
    """The moving-horizon workload at its full size (n = 1e6, F = 30, D = 8, horizon 3,
    P = 128, G = 200), where every level is large enough for the evaluator autotuner to time
    its candidate shapes (32-warp CTAs, tiles between the powers of two): the batched fit
    gives the plain per-node fit's tree (the plain form equals the oracle in the tests above,
    at sizes the oracle finishes)."""
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(2)
    ctx = deoct.Context(0)
    try:
        ds = gpu_dataset(ctx, w["X"], w["y"], w["K"], 4)
        outs = []
        for flags in (0, deoct.DEOCT_BATCHED):
            prm = deoct.make_params(w["depth"], w["P"], w["G"], mut_f=w["M"], cr=w["CR"], seed=w["seed"],
                                    horizon=w["horizon"], flags=flags)
            outs.append(deoct.deoct_fit_moving_horizon(ctx, ds, prm))
        for k in ("a", "theta", "kind", "node_fit", "leaf_class"):
            np.testing.assert_array_equal(outs[0][k], outs[1][k], err_msg=k)
        assert (outs[1]["kind"] == 2).sum() >= 60
    finally:
        ctx.close()
