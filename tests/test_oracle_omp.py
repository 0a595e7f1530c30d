"""The oracle's OpenMP twins against its plain single-threaded functions, bit for bit.

The twins exist to time the oracle on the host's cores and to check the full-size
workloads; they must compute exactly what the plain functions compute (integer counts,
sorts per feature), whatever the thread count or the split of the work."""
import numpy as np
import pytest

import oracle
from paper_2311_06952_gb300 import datagen


@pytest.fixture(autouse=True)
def _restore_threads():
    old = oracle.set_threads(1)
    yield
    oracle.set_threads(old)


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


@pytest.mark.parametrize("threads", [2, 3, 8])
def test_encode_omp_equals_encode(threads):
    X = datagen.make_workload(1, n=30000)["X"]
    X[::11, 3] = -0.0
    ref = oracle.encode(X)
    oracle.set_threads(threads)
    got = oracle.encode_omp(X)
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    bad = X.copy()
    bad[7, 5] = np.nan
    with pytest.raises(ValueError):
        oracle.encode_omp(bad)


@pytest.mark.parametrize("n,P,depth,K,threads,subset", [
    (200_000, 3, 3, 4, 4, False),    # more chunks than trees
    (70_000, 64, 2, 2, 3, False),    # ragged last chunk
    (1000, 1, 5, 3, 8, False),       # one item, idle threads
    (150_000, 17, 4, 5, 5, True),    # gathered subset
    (5, 9, 1, 2, 2, True),           # tiny
])
def test_eval_counts_omp_equals_eval_counts(n, P, depth, K, threads, subset):
    rng = _rng(n + P)
    X = np.round(rng.random((n, 6)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    idx = np.sort(rng.choice(n, max(1, n // 2), replace=False)).astype(np.int32) if subset else None
    ref = oracle.eval_counts(ranks, y, K, a, th, depth, idx=idx)
    oracle.set_threads(threads)
    got = oracle.eval_counts_omp(ranks, y, K, a, th, depth, idx=idx)
    np.testing.assert_array_equal(got, ref)


def test_de_run_and_mh_with_threads_equal_the_plain_oracle():
    w = datagen.make_workload(0, n=3000)
    ranks, nu = oracle.encode(w["X"])
    kw = dict(depth=3, P=16, G=8, seed=4, stream=2)
    ref = oracle.de_run(ranks, nu, w["y"], w["K"], history=True, **kw)
    ref_mh = oracle.mh(ranks, nu, w["y"], w["K"], depth=4, horizon=2, P=8, G=5, seed=1)
    oracle.set_threads(6)
    got = oracle.de_run(ranks, nu, w["y"], w["K"], history=True, **kw)
    got_mh = oracle.mh(ranks, nu, w["y"], w["K"], depth=4, horizon=2, P=8, G=5, seed=1)
    np.testing.assert_array_equal(got["pop_hist"].view(np.uint32), ref["pop_hist"].view(np.uint32))
    np.testing.assert_array_equal(got["fit_hist"], ref["fit_hist"])
    assert got["best"] == ref["best"]
    for k in ("a", "theta", "leaf_class", "kind", "node_fit"):
        np.testing.assert_array_equal(got_mh[k], ref_mh[k])
