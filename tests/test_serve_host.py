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


def test_budget_serialises_and_fifo():
    log = []
    fp = serve.footprint_bytes(1000, 4, 3, 16, 2)
    srv = serve.Server(budget_bytes=int(fp * 1.5), slots=4, fit_fn=_fake_fit(0.02, log))
    res = serve.run_trace(srv, [_req(i) for i in range(5)])
    srv.close()
    assert srv.max_concurrent == 1  # only one request fits at a time
    assert [x[1] for x in log] == list(range(5))  # admitted in arrival order
    assert srv.peak_in_use <= srv.budget
    for r in res:
        assert r.t_admit >= r.t_submit and r.t_done >= r.t_admit


def test_over_budget_request_is_rejected_not_queued():
    small = serve.footprint_bytes(10, 1, 1, 16, 2)
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
