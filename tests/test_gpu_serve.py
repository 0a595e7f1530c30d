"""Serving on the GPU.

- Every served tree equals the oracle's moving-horizon tree for that request
  (Algorithm 2, same data, parameters and Philox seed) and the same request fitted
  alone, whether the requests share the engine's launches or run on their own streams.
- With the engine, launches carry the work of several requests at once.
- The library's scratch bound covers what a context really holds after a fit, and the
  server's charge never exceeds its budget."""
import numpy as np
import pytest

import oracle
from paper_2311_06952_gb300 import datagen, serve

pytestmark = pytest.mark.gpu


def _requests(num=8, seed=77, n_range=(2_000, 20_000), pop=32, gens=80):
    reqs = datagen.serving_requests(num=num, rate=200.0, seed=seed, n_range=n_range, materialize=True)
    out = []
    for r in reqs:
        out.append(serve.FitRequest(X=r["X"], y=r["y"], K=r["K"], depth=r["depth"],
                                    horizon=r["horizon"], pop=pop, gens=gens, seed=r["id"], id=r["id"],
                                    arrival=r["arrival"]))
    return out


def _oracle_tree(r):
    old = oracle.set_threads(oracle.host_cores())
    try:
        ranks, nu = oracle.encode_omp(r.X)
        return oracle.mh(ranks, nu, r.y, r.K, depth=r.depth, horizon=r.horizon, P=r.pop, G=r.gens,
                         M=r.mut_f, CR=r.cr, seed=r.seed)
    finally:
        oracle.set_threads(old)


@pytest.fixture(scope="module")
def reqs():
    from paper_2311_06952_gb300 import build
    build.build()
    rs = _requests()
    return rs, {r.id: _oracle_tree(r) for r in rs}


def _check(res, ref):
    for k in ("a", "theta", "kind", "node_fit", "leaf_class"):
        np.testing.assert_array_equal(np.asarray(getattr(res, k)).astype(ref[k].dtype), ref[k],
                                      err_msg="request %d %s" % (res.id, k))


def test_alone_equals_oracle(reqs):
    import torch
    from paper_2311_06952_gb300 import deoct
    rs, ref = reqs
    ctx = deoct.Context(0)
    stream = torch.cuda.Stream()
    for r in rs:
        with torch.cuda.stream(stream):
            out = serve.fit_on_stream(ctx, r, stream)
        for k in ("a", "theta", "kind", "node_fit", "leaf_class"):
            np.testing.assert_array_equal(out[k].astype(ref[r.id][k].dtype), ref[r.id][k])
    ctx.close()


@pytest.mark.parametrize("engine", [True, False])
def test_served_trees_equal_the_oracle_in_the_mix(reqs, engine):
    rs, ref = reqs
    budget = 64 << 30
    srv = serve.Server(budget_bytes=budget, slots=4, engine=engine)
    try:
        mixed = serve.run_trace(srv, rs)
        st = srv.engine_stats()
    finally:
        srv.close()
    assert srv.max_concurrent >= 2  # several requests were resident together
    for res in mixed:
        _check(res, ref[res.id])
        assert res.scratch_after - res.scratch_before <= res.scratch_reserve <= res.scratch_bound
    assert srv.peak_charged <= budget
    assert srv.charged == sum(srv.retained)
    if engine:
        assert st["completed"] == st["submissions"] > 0
        assert st["shared_launches"] > 0 and st["max_jobs_per_launch"] >= 2, st


def test_engine_mixes_rank_widths_depths_and_classes():
    """Requests of both rank widths, subtree depths 2 and 3 and different K, F and n in one
    engine; the first three share rank width, subtree depth and size class but not K or F,
    so their problems run in the same launches.  Each tree equals the oracle's."""
    rng = np.random.Generator(np.random.PCG64(5))
    rs = []
    for i, (n, F, K, depth, horizon, wide) in enumerate([
            (9000, 5, 2, 4, 2, False), (11000, 9, 5, 3, 2, False), (10000, 4, 3, 4, 2, False),
            (70000, 4, 3, 3, 3, True), (20000, 6, 2, 5, 3, True)]):
        X = (rng.random((n, F)) if wide else np.round(rng.random((n, F)), 3)).astype(np.float32)
        y = datagen.planted_tree_labels(X, 3, K, rng)
        rs.append(serve.FitRequest(X=X, y=y, K=K, depth=depth, horizon=horizon, pop=24, gens=60, seed=40 + i,
                                   id=i, arrival=0.0))
    srv = serve.Server(budget_bytes=64 << 30, slots=5, engine=True)
    try:
        res = serve.run_trace(srv, rs)
        st = srv.engine_stats()
    finally:
        srv.close()
    for r, q in zip(sorted(res, key=lambda x: x.id), rs):
        _check(r, _oracle_tree(q))
    assert st["max_jobs_per_launch"] >= 2


@pytest.mark.parametrize("case", [
    # n, F, K, depth, horizon, pop, flags
    (50_000, 12, 3, 6, 3, 64, "batched"),
    (30_000, 30, 7, 4, 2, 32, "plain"),
    (70_000, 5, 2, 5, 3, 40, "batched+seeds"),
    (4_000, 60, 10, 6, 3, 128, "batched"),
])
def test_scratch_bound_covers_a_fresh_context(case):
    import torch
    from paper_2311_06952_gb300 import deoct
    n, F, K, depth, horizon, pop, kind = case
    rng = np.random.Generator(np.random.PCG64(n + F))
    X = rng.random((n, F)).astype(np.float32)
    y = datagen.planted_tree_labels(X, min(depth, 4), K, rng)
    flags = 0 if kind == "plain" else deoct.DEOCT_BATCHED
    if "seeds" in kind:
        flags |= deoct.DEOCT_CART_SEEDS | deoct.DEOCT_DE_SEEDS
    prm = deoct.make_params(depth, pop, 3, horizon=horizon, flags=flags)
    ctx = deoct.Context(0)
    ds = deoct.encode_dataset(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), K, 0)
    deoct.deoct_fit_moving_horizon(ctx, ds, prm)
    held, _ = ctx.memory()
    ctx.close()
    bound = deoct.fit_scratch_bound(n, F, K, prm)
    assert held <= bound, (held, bound)
    assert held >= bound // 8  # the bound is not vacuous


def test_engine_with_warm_starts_and_dither_equals_oracle():
    """A context attached to the engine, fitting with both warm starts of Algorithm 2 and the
    dithered M of Section 3.3 (the level solves' seeds pass through the engine's problems),
    gives the oracle's tree; a second context shares the engine at the same time."""
    import threading

    import torch
    from paper_2311_06952_gb300 import deoct
    rng = np.random.Generator(np.random.PCG64(17))
    sets = []
    for n, F, K in ((6000, 6, 3), (9000, 5, 2)):
        X = np.round(rng.random((n, F)), 3).astype(np.float32)
        y = datagen.flip_labels(datagen.planted_tree_labels(X, 4, K, rng), K, 0.1, rng)
        sets.append((X, y, K))
    eng = deoct.Engine(0)
    flags = deoct.DEOCT_BATCHED | deoct.DEOCT_CART_SEEDS | deoct.DEOCT_DE_SEEDS | deoct.DEOCT_DITHER_M
    outs = [None, None]

    def fit(i):
        X, y, K = sets[i]
        ctx = deoct.Context(0)
        ctx.attach_engine(eng)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            ds = deoct.encode_dataset(ctx, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), K, 0, stream=s)
            prm = deoct.make_params(5, 16, 20, cr=0.5, seed=9 + i, horizon=3, flags=flags)
            outs[i] = deoct.deoct_fit_moving_horizon(ctx, ds, prm, stream=s)
        ctx.close()

    threads = [threading.Thread(target=fit, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    st = eng.stats()
    eng.close()
    for i, (X, y, K) in enumerate(sets):
        ranks, nu = oracle.encode(X)
        ref = oracle.mh(ranks, nu, y, K, depth=5, horizon=3, P=16, G=20, CR=0.5, seed=9 + i, dither=True,
                        cart_seeds=True, de_seeds=True)
        for k in ("kind", "a", "theta", "node_fit", "leaf_class"):
            np.testing.assert_array_equal(outs[i][k].astype(ref[k].dtype), ref[k], err_msg="set %d %s" % (i, k))
    assert st["completed"] == st["submissions"] > 0


@pytest.mark.parametrize("engine", [True, False])
def test_a_malformed_request_fails_alone(engine):
    """A request whose features hold a NaN fails with the library's invalid-input error; the
    requests around it, served by the same slots (and engine), still equal the oracle."""
    from paper_2311_06952_gb300 import deoct
    rs = _requests(num=4, seed=91, n_range=(2_000, 6_000), pop=16, gens=12)
    bad = rs[1]
    Xb = bad.X.copy()
    Xb[len(Xb) // 2, 0] = np.nan
    rs[1] = serve.FitRequest(X=Xb, y=bad.y, K=bad.K, depth=bad.depth, horizon=bad.horizon, pop=bad.pop,
                             gens=bad.gens, seed=bad.seed, id=bad.id, arrival=bad.arrival)
    srv = serve.Server(budget_bytes=32 << 30, slots=2, engine=engine)
    try:
        futs = [srv.submit(r) for r in rs]
        with pytest.raises(deoct.DeoctError) as ei:
            futs[1].result(timeout=300)
        assert ei.value.code == deoct.DEOCT_ERR_INVALID
        later = srv.submit(rs[0])  # the slot that saw the failure serves again
        good = [futs[i].result(timeout=300) for i in (0, 2, 3)] + [later.result(timeout=300)]
    finally:
        srv.close()
    for res, r in zip(good, [rs[0], rs[2], rs[3], rs[0]]):
        _check(res, _oracle_tree(r))


def test_scratch_limit_fails_cleanly_and_the_context_recovers():
    """A scratch cap below what a fit needs fails the fit with DEOCT_ERR_OOM before it
    allocates; with the cap lifted the same context fits the oracle's tree, and with the cap
    at the library's own bound the fit runs within it."""
    import torch
    from paper_2311_06952_gb300 import deoct
    r = _requests(num=1, seed=93, n_range=(20_000, 20_000), pop=16, gens=10)[0]
    ctx = deoct.Context(0)
    try:
        ctx.set_scratch_limit(1 << 20)
        with pytest.raises(deoct.DeoctError) as ei:
            out = serve.fit_on_stream(ctx, r, torch.cuda.current_stream())
        assert ei.value.code == deoct.DEOCT_ERR_OOM
        ctx.set_scratch_limit(0)
        out = serve.fit_on_stream(ctx, r, torch.cuda.current_stream())
        ref = _oracle_tree(r)
        for k in ("a", "theta", "kind", "node_fit", "leaf_class"):
            np.testing.assert_array_equal(np.asarray(out[k]).astype(ref[k].dtype), ref[k])
        ctx.release_scratch()
        bound = serve.scratch_bound(r, ctx=ctx) + ctx.memory()[0]
        ctx.set_scratch_limit(bound)
        out2 = serve.fit_on_stream(ctx, r, torch.cuda.current_stream())
        assert ctx.memory()[0] <= bound
        np.testing.assert_array_equal(np.asarray(out2["a"]), np.asarray(out["a"]))
    finally:
        ctx.close()
