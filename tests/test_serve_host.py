"""Serving loop host logic on CPU (no GPU): admission by slots and memory budget,
FIFO order, over-budget rejection, and latency bookkeeping."""
import threading
import time

import numpy as np
import pytest

from paper_2311_06952_gb300 import serve


def _req(i, n=1000, F=4, depth=3, arrival=0.0):
    return serve.FitRequest(X=np.zeros((n, F), np.float32), y=np.zeros(n, np.uint8), K=2, depth=depth,
                            horizon=2, pop=16, gens=2, id=i, arrival=arrival)


def _fake_fit(delay, log):
    lock = threading.Lock()
    live = [0]

    def fit(slot, req):
        with lock:
            live[0] += 1
            log.append(("start", req.id, live[0]))
        time.sleep(delay)
        with lock:
            live[0] -= 1
        B = (1 << req.depth) - 1
        return dict(a=np.zeros(B, np.uint16), theta=np.zeros(B, np.uint32),
                    leaf_class=np.zeros(B + 1, np.uint8), kind=np.zeros(B, np.int32),
                    node_fit=np.zeros(B))
    return fit


def test_slots_bound_concurrency():
    log = []
    srv = serve.Server(budget_bytes=1 << 40, slots=3, fit_fn=_fake_fit(0.05, log))
    res = serve.run_trace(srv, [_req(i) for i in range(10)])
    srv.close()
    assert sorted(r.id for r in res) == list(range(10))
    assert max(x[2] for x in log) <= 3
    assert srv.max_concurrent == 3


def _cost(req):
    return serve.input_bytes(*req.X.shape) + serve.scratch_bound(req)


def test_budget_serialises_and_fifo():
    log = []
    fp = _cost(_req(0))
    srv = serve.Server(budget_bytes=int(fp * 1.5), slots=4, fit_fn=_fake_fit(0.02, log))
    res = serve.run_trace(srv, [_req(i) for i in range(5)])
    srv.close()
    assert srv.max_concurrent == 1  # only one request fits at a time
    assert [x[1] for x in log] == list(range(5))  # admitted in arrival order
    assert srv.peak_in_use <= srv.budget
    for r in res:
        assert r.t_admit >= r.t_submit and r.t_done >= r.t_admit


def test_over_budget_request_is_rejected_not_queued():
    small = _cost(_req(1, n=10, F=1, depth=1))
    srv = serve.Server(budget_bytes=2 * small, slots=2, fit_fn=_fake_fit(0.0, []))
    fut = srv.submit(_req(0, n=100000, F=50))
    with pytest.raises(MemoryError):
        fut.result(timeout=5)
    ok = srv.submit(_req(1, n=10, F=1, depth=1))
    ok.result(timeout=5)
    srv.close()


def test_sequential_queue_latencies():
    lat = serve.sequential_queue_latencies([0.0, 0.1, 0.2], [1.0, 1.0, 1.0])
    assert np.allclose(lat, [1.0, 1.9, 2.8])
    st = serve.latency_stats([1.0, 2.0, 3.0, 4.0])
    assert st["p50_s"] == 2.5


def test_retained_scratch_is_charged_and_reused():
    """A slot keeps the scratch its request grew; the budget is charged with it, and a
    later request on that slot is charged only the growth it may still need."""
    grown = {}

    def fit(slot, req):
        B = (1 << req.depth) - 1
        grown[slot] = max(grown.get(slot, 0), serve.scratch_bound(req) // 2)  # what the fit kept
        return dict(a=np.zeros(B, np.uint16), theta=np.zeros(B, np.uint32),
                    leaf_class=np.zeros(B + 1, np.uint8), kind=np.zeros(B, np.int32),
                    node_fit=np.zeros(B), scratch_bytes=grown[slot])
    def growth(slot, req):  # what the fake fit may still grow the slot by
        return max(0, serve.scratch_bound(req) // 2 - grown.get(slot, 0))
    big = _req(0, n=20000, F=8)
    budget = _cost(big) + serve.input_bytes(20000, 8) + 1
    srv = serve.Server(budget_bytes=budget, slots=2, fit_fn=fit, growth_fn=growth)
    res = serve.run_trace(srv, [_req(i, n=20000, F=8) for i in range(4)])
    srv.close()
    assert srv.peak_charged <= budget
    # after the first request a slot holds half the bound: the next ones fit beside it
    assert srv.retained == [grown.get(0, 0), grown.get(1, 0)]
    assert srv.charged == sum(srv.retained)
    for r in res:
        assert r.scratch_after - r.scratch_before <= r.scratch_reserve
        assert r.footprint == r.inputs + (r.scratch_after - r.scratch_before)


def test_admission_prefers_the_slot_that_already_holds_scratch():
    def fit(slot, req):
        B = (1 << req.depth) - 1
        return dict(a=np.zeros(B, np.uint16), theta=np.zeros(B, np.uint32),
                    leaf_class=np.zeros(B + 1, np.uint8), kind=np.zeros(B, np.int32),
                    node_fit=np.zeros(B), scratch_bytes=serve.scratch_bound(req))
    held = {}

    def fit2(slot, req):
        out = fit(slot, req)
        held[slot] = out["scratch_bytes"]
        return out

    def growth(slot, req):
        return max(0, serve.scratch_bound(req) - held.get(slot, 0))
    r0 = _req(0, n=5000, F=6)
    budget = _cost(r0) + serve.input_bytes(5000, 6)  # room for one more request's inputs only
    srv = serve.Server(budget_bytes=budget, slots=3, fit_fn=fit2, growth_fn=growth)
    res = serve.run_trace(srv, [_req(i, n=5000, F=6, arrival=0.01 * i) for i in range(3)])
    srv.close()
    assert len({r.slot for r in res}) == 1  # every request reused the first slot's scratch
    assert srv.peak_charged <= budget


def test_a_failing_request_fails_alone():
    """A fit that raises (the library's error for bad input, say) fails its own future; the
    slot is freed, its charge returned, and the requests before and after it are served."""
    log = []
    good = _fake_fit(0.01, log)

    def fit(slot, req):
        if req.id == 3:
            raise RuntimeError("injected failure of request 3")
        return good(slot, req)

    srv = serve.Server(budget_bytes=1 << 40, slots=2, fit_fn=fit)
    futs = [srv.submit(_req(i)) for i in range(8)]
    done = []
    for i, f in enumerate(futs):
        if i == 3:
            with pytest.raises(RuntimeError, match="injected"):
                f.result(timeout=30)
        else:
            done.append(f.result(timeout=30).id)
    srv.close()
    assert done == [0, 1, 2, 4, 5, 6, 7]
    assert srv.running == 0 and srv.charged == sum(srv.retained)
    assert sorted(srv.free_slots) == [0, 1]
