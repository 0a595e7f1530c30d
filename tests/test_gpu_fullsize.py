"""Full-size end-to-end parity: the configurations of the measured workloads at their own
population and generation settings, checked bit for bit against the oracle run on the
host's cores (its OpenMP twins, pinned to the plain oracle in tests/test_oracle_omp.py).

  - large-scale DEOCT: n = 1e7, F = 10, uint16 ranks, K = 2, depth 4, P = 1024 -- the
    bench's exact launch configuration (the DEOCT fit whose generations replay one captured
    graph), initial evaluation + 3 generations, plus the step-by-step C-ABI form;
  - moving horizon: F = 30, K = 4, uint32 ranks, final depth 8, horizon 3, P = 128, G = 200
    (every setting of the batched-level workload but n, which is cut to what the oracle
    finishes in about a minute on the host's cores), batched and plain forms."""
import time

import numpy as np
import pytest

import oracle
from paper_2311_06952_gb300 import datagen

from gpu_helpers import ctx, gpu_dataset

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c():
    from paper_2311_06952_gb300 import build
    build.build()
    return ctx()


@pytest.fixture(scope="module")
def threads():
    old = oracle.set_threads(oracle.host_cores())
    yield oracle.host_cores()
    oracle.set_threads(old)


def test_large_deoct_full_size_first_generations(c, threads):
    import torch
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(3)
    n, F, K, D, P, G = w["X"].shape[0], w["X"].shape[1], w["K"], 4, 1024, 3
    assert n == 10_000_000
    t0 = time.perf_counter()
    ranks, nu = oracle.encode_omp(w["X"])
    ref = oracle.de_run(ranks, nu, w["y"], K, depth=D, P=P, G=G, seed=0, stream=0, history=True)
    t_oracle = time.perf_counter() - t0
    del ranks
    ds = gpu_dataset(c, w["X"], w["y"], K, 2)
    np.testing.assert_array_equal(ds.n_unique.cpu().numpy().view(np.uint32), nu)
    # the bench's path: one DEOCT fit, generations replayed from a captured graph
    prm = deoct.make_params(D, P, G, mut_f=0.5, cr=0.9, seed=0)
    pop = torch.empty((P, 2 * 15), dtype=torch.float32, device="cuda")
    a, th, f = deoct.deoct_fit_subtree(c, ds, prm, pop_out=pop)
    np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32), ref["pop"].view(np.uint32))
    assert f == ref["fit"][ref["best"]]
    a_ref, th_ref = oracle.decode(ref["pop"][ref["best"]][None], D, nu)
    np.testing.assert_array_equal(a.astype(np.int32), a_ref[0])
    np.testing.assert_array_equal(th, th_ref[0])
    # the step-by-step form: population, every fitness and the best after each generation
    pop, fit, best = deoct.deoct_de_init(c, ds, prm)
    np.testing.assert_array_equal(fit.cpu().numpy(), ref["fit_hist"][0])
    for g in range(1, G + 1):
        deoct.deoct_de_step(c, ds, prm, g, pop, fit, best)
        np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32), ref["pop_hist"][g].view(np.uint32))
        np.testing.assert_array_equal(fit.cpu().numpy(), ref["fit_hist"][g])
    assert int(best.cpu()[0]) == ref["best"]
    print("oracle on %d threads: %.1f s for %d evaluations" % (threads, t_oracle, (G + 1) * P * n))


@pytest.mark.parametrize("batched", [True, False])
def test_moving_horizon_workload_settings_bit_exact(c, threads, batched):
    from paper_2311_06952_gb300 import deoct
    n = 150_000
    w = datagen.make_workload(2, n=n)
    assert (w["depth"], w["horizon"], w["P"], w["G"], w["K"]) == (8, 3, 128, 200, 4)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], 4)
    prm = deoct.make_params(w["depth"], w["P"], w["G"], mut_f=w["M"], cr=w["CR"], seed=w["seed"],
                            horizon=w["horizon"], flags=deoct.DEOCT_BATCHED if batched else 0)
    out = deoct.deoct_fit_moving_horizon(c, ds, prm)
    ref = _mh_reference(w)
    for k in ("kind", "a", "theta", "node_fit", "leaf_class"):
        np.testing.assert_array_equal(out[k].astype(ref[k].dtype), ref[k], err_msg=k)
    assert (ref["kind"] == 2).sum() >= 40  # DEOCT solves on every level that has them


_MH_CACHE = {}


def _mh_reference(w):
    key = w["X"].shape[0]
    if key not in _MH_CACHE:
        ranks, nu = oracle.encode_omp(w["X"])
        _MH_CACHE[key] = oracle.mh(ranks, nu, w["y"], w["K"], depth=w["depth"], horizon=w["horizon"],
                                   P=w["P"], G=w["G"], M=w["M"], CR=w["CR"], seed=w["seed"])
    return _MH_CACHE[key]
