"""Serving on the GPU: each request's tree is the same alone and in the mix
(exact: per-request data, parameters and Philox seeds), with requests running
concurrently on their slots' streams."""
import numpy as np
import pytest

from paper_2311_06952_gb300 import datagen, serve

pytestmark = pytest.mark.gpu


def _requests(num=8, seed=77):
    reqs = datagen.serving_requests(num=num, rate=200.0, seed=seed, n_range=(2_000, 40_000),
                                    materialize=True)
    out = []
    for r in reqs:
        out.append(serve.FitRequest(X=r["X"], y=r["y"], K=r["K"], depth=r["depth"],
                                    horizon=r["horizon"], pop=32, gens=12, seed=r["id"], id=r["id"],
                                    arrival=r["arrival"]))
    return out


def test_alone_equals_in_the_mix():
    import torch
    from paper_2311_06952_gb300 import build, deoct
    build.build()
    reqs = _requests()
    ctx = deoct.Context(0)
    stream = torch.cuda.Stream()
    alone = {}
    for r in reqs:
        with torch.cuda.stream(stream):
            alone[r.id] = serve.fit_on_stream(ctx, r, stream)
    ctx.close()
    srv = serve.Server(budget_bytes=64 << 30, slots=4)
    mixed = serve.run_trace(srv, reqs)
    srv.close()
    assert srv.max_concurrent >= 2  # work of several requests was in flight together
    for res in mixed:
        ref = alone[res.id]
        for k in ("a", "theta", "kind", "node_fit", "leaf_class"):
            np.testing.assert_array_equal(getattr(res, k), ref[k], err_msg="request %d %s" % (res.id, k))


def test_plain_and_batched_requests_agree():
    import torch
    from paper_2311_06952_gb300 import deoct
    r = _requests(num=1, seed=5)[0]
    ctx = deoct.Context(0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = serve.fit_on_stream(ctx, r, s)
        r.batched = False
        b = serve.fit_on_stream(ctx, r, s)
    ctx.close()
    for k in ("a", "theta", "kind", "node_fit", "leaf_class"):
        np.testing.assert_array_equal(a[k], b[k])
