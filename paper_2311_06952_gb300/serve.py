"""Continuous-batching serving loop for moving-horizon tree fitting.

Requests (a feature matrix, labels and fit parameters) arrive over time.  A
request is admitted as soon as a slot is free and its device-memory footprint
fits in what remains of the budget; it then runs on that slot's own CUDA
stream and ``deoct`` context (encode on the device, then the batched
moving-horizon fit of Algorithm 2 through the C ABI), so the kernels of all
admitted requests overlap on the GPU.  When it finishes, its memory goes back
to the budget and the next waiting request is admitted.

Every request's result depends only on its own data, parameters and Philox
seed: the same request alone or in any mix gives the same tree.
"""
from __future__ import annotations

import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


@dataclass
class FitRequest:
    X: np.ndarray                 # [n][F] float32
    y: np.ndarray                 # [n] uint8
    K: int
    depth: int
    horizon: int
    pop: int = 128
    gens: int = 200
    mut_f: float = 0.5
    cr: float = 0.9
    alpha: float = 0.0
    n_min: int = 1
    seed: int = 0
    batched: bool = True
    id: int = 0
    arrival: float = 0.0          # seconds (trace time)


@dataclass
class FitResult:
    id: int
    a: np.ndarray
    theta: np.ndarray
    leaf_class: np.ndarray
    kind: np.ndarray
    node_fit: np.ndarray
    t_submit: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    slot: int = -1
    footprint: int = 0

    @property
    def latency(self):
        return self.t_done - self.t_submit


def rank_width(n: int) -> int:
    """uint16 ranks are always enough when n <= 65536 (n_p <= n)."""
    return 2 if n <= 65536 else 4


def footprint_bytes(n: int, F: int, depth: int, pop: int, K: int) -> int:
    """Upper bound of the device memory one request holds while it runs: inputs,
    ranks, encoder scratch, moving-horizon scratch and DE state."""
    W = rank_width(n)
    ld = (n + 15) // 16 * 16
    npad = n + 16 * (1 << max(0, depth - 1)) + 64
    b = n * F * 4 + n                       # X, y
    b += F * ld * W + F * 4                 # ranks, n_unique
    b += 16 * n * F + 4 * 256 * F * (n // 2048 + 1) + 4 * F * (n // 2048 + 1)  # encoder scratch
    b += 4 * n + 8 * npad + F * npad * W + npad   # node_of, idx, pos_slot, compacted rows, labels
    b += 16 * F * npad                      # depth-1 sort keys and values
    nodes = 1 << max(0, depth - 1)
    B3, L3 = 7, 8
    b += nodes * (pop * (2 * B3 * 4 * 2 + 16 + B3 * 4 + L3 * K * 4) + 512)   # DE state per node
    return int(b * 1.1) + (8 << 20)


class Server:
    """Admission by device-memory budget, one worker per slot, overlapping streams."""

    def __init__(self, budget_bytes: int = 120 << 30, slots: int = 8, device: int = 0, fit_fn=None):
        # fit_fn(slot_state, request) -> dict replaces the GPU fit (host-logic tests)
        self.fit_fn = fit_fn
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.device = device
        self.in_use = 0
        self.cv = threading.Condition()
        self.pending = []               # FIFO of (req, future, t_submit, footprint)
        self.free_slots = list(range(self.slots))
        self.closed = False
        self.workers = []
        self.t0 = time.perf_counter()
        self.peak_in_use = 0
        self.max_concurrent = 0
        self.running = 0
        self._work = [queue.Queue() for _ in range(self.slots)]
        for s in range(self.slots):
            t = threading.Thread(target=self._worker, args=(s,), daemon=True)
            t.start()
            self.workers.append(t)
        self._admitter = threading.Thread(target=self._admit_loop, daemon=True)
        self._admitter.start()

    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, req: FitRequest) -> Future:
        fut = Future()
        fp = footprint_bytes(req.X.shape[0], req.X.shape[1], req.depth, req.pop, req.K)
        if fp > self.budget:
            fut.set_exception(MemoryError("request %d needs %d bytes, over the %d-byte budget"
                                          % (req.id, fp, self.budget)))
            return fut
        with self.cv:
            self.pending.append((req, fut, self.now(), fp))
            self.cv.notify_all()
        return fut

    def _admit_loop(self):
        while True:
            with self.cv:
                while not self.closed and not self._can_admit():
                    self.cv.wait()
                if self.closed and not self.pending:
                    return
                if not self._can_admit():
                    continue
                req, fut, ts, fp = self.pending.pop(0)
                slot = self.free_slots.pop(0)
                self.in_use += fp
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                self.running += 1
                self.max_concurrent = max(self.max_concurrent, self.running)
            self._work[slot].put((req, fut, ts, fp, self.now()))

    def _can_admit(self):
        return bool(self.pending) and bool(self.free_slots) and \
            self.in_use + self.pending[0][3] <= self.budget

    def _worker(self, slot):
        ctx = stream = None
        if self.fit_fn is None:
            import torch

            from . import deoct
            torch.cuda.set_device(self.device)
            ctx = deoct.Context(self.device)
            stream = torch.cuda.Stream(device=self.device)
        while True:
            item = self._work[slot].get()
            if item is None:
                break
            req, fut, ts, fp, ta = item
            try:
                if self.fit_fn is not None:
                    out = self.fit_fn(slot, req)
                else:
                    with torch.cuda.stream(stream):
                        out = fit_on_stream(ctx, req, stream)
                res = FitResult(req.id, out["a"], out["theta"], out["leaf_class"], out["kind"],
                                out["node_fit"], t_submit=ts, t_admit=ta, t_done=self.now(), slot=slot,
                                footprint=fp)
                fut.set_result(res)
            except Exception as e:  # the request fails, the server keeps serving
                fut.set_exception(e)
            finally:
                with self.cv:
                    self.in_use -= fp
                    self.running -= 1
                    self.free_slots.append(slot)
                    self.cv.notify_all()
        if ctx is not None:
            ctx.close()

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        self._admitter.join()
        for q in self._work:
            q.put(None)
        for t in self.workers:
            t.join()


def fit_on_stream(ctx, req: FitRequest, stream):
    """Encode a request's data on the device and fit it (moving horizon) on `stream`."""
    import torch

    from . import deoct
    Xd = torch.from_numpy(np.ascontiguousarray(req.X, np.float32)).to("cuda", non_blocking=False)
    yd = torch.from_numpy(np.ascontiguousarray(req.y, np.uint8)).to("cuda", non_blocking=False)
    ds = deoct.encode_dataset(ctx, Xd, yd, req.K, 0, stream=stream)  # width from n_p
    prm = deoct.make_params(req.depth, req.pop, req.gens, mut_f=req.mut_f, cr=req.cr, alpha=req.alpha,
                            n_min=req.n_min, seed=req.seed, horizon=req.horizon,
                            flags=deoct.DEOCT_BATCHED if req.batched else 0)
    out = deoct.deoct_fit_moving_horizon(ctx, ds, prm, stream=stream)
    return out


def run_trace(server: Server, requests, time_scale: float = 1.0):
    """Submit requests at their arrival times (scaled) and wait for all results."""
    futs = []
    t_start = server.now()
    for req in sorted(requests, key=lambda r: r.arrival):
        target = t_start + req.arrival * time_scale
        delay = target - server.now()
        if delay > 0:
            time.sleep(delay)
        futs.append(server.submit(req))
    return [f.result() for f in futs]


def latency_stats(latencies):
    lat = np.sort(np.asarray(latencies, np.float64))
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def sequential_queue_latencies(arrivals, service_times):
    """Latency of a one-at-a-time FIFO server with the given service times."""
    done = 0.0
    out = []
    for a, s in sorted(zip(arrivals, service_times)):
        start = max(a, done)
        done = start + s
        out.append(done - a)
    return out
