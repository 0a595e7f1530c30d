"""Continuous-batching serving loop for moving-horizon tree fitting.

Requests (a feature matrix, labels and fit parameters) arrive over time.  A
request is admitted as soon as a slot is free and its device memory fits in what
remains of the budget.  Its slot's host thread encodes the data on the device
and runs the batched moving-horizon fit of Algorithm 2 through the C ABI on the
slot's own context and stream.  With ``engine=True`` (the default) every slot's
context is attached to one shared ``deoct.Engine``: the DEOCT generations of all
resident requests' levels then run in shared launches, one evaluator launch and
one DE-step launch per generation for the problems of every request (continuous
batching inside the launches).  With ``engine=False`` each request runs its own
launches on its own stream and the GPU overlaps the streams.

Memory: a request holds its input arrays while it runs, and its slot's context
keeps the scratch it grew (grow-only per buffer, reused by the slot's next
requests).  The budget is charged with every slot's retained scratch, measured
after each request, plus the inputs of the running requests and, for each, the
growth its slot's scratch may still need (the library's bound of that growth for
the request's shape, given what the slot's context holds).  A request goes to the
free slot that needs the least growth.  When nothing runs and the oldest request
still does not fit, idle slots release their scratch.

Every request's result depends only on its own data, parameters and Philox seed:
the same request alone or in any mix gives the same tree.
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
    footprint: int = 0            # inputs + the slot's scratch growth (measured)
    inputs: int = 0
    scratch_before: int = 0       # the slot's scratch before and after the request
    scratch_after: int = 0
    scratch_bound: int = 0        # the library's bound for the request's shape (fresh context)
    scratch_reserve: int = 0      # growth of the slot's scratch charged at admission

    @property
    def latency(self):
        return self.t_done - self.t_submit


def input_bytes(n: int, F: int) -> int:
    """Device bytes of a request's own arrays while it runs: features, labels, the
    rank buffer of the width-choosing encoder (4-byte rows, plus the 2-byte copy kept
    when every n_p <= 65536) and n_p."""
    ld = (n + 7) // 8 * 8
    return n * F * 4 + n + F * ld * 6 + F * 4


def fit_params(req: "FitRequest"):
    from . import deoct
    return deoct.make_params(req.depth, req.pop, req.gens, mut_f=req.mut_f, cr=req.cr, alpha=req.alpha,
                             n_min=req.n_min, seed=req.seed, horizon=req.horizon,
                             flags=deoct.DEOCT_BATCHED if req.batched else 0)


def scratch_bound(req: "FitRequest", ctx=None) -> int:
    """Upper bound of the scratch a fresh context holds after fitting this request, or with
    `ctx`, of the growth of that context's scratch (the library's bound)."""
    from . import deoct
    n, F = req.X.shape
    return deoct.fit_scratch_bound(n, F, req.K, fit_params(req), ctx=ctx)


class Server:
    """Admission by device-memory budget, one worker thread per slot, shared engine."""

    def __init__(self, budget_bytes: int = 120 << 30, slots: int = 8, device: int = 0, fit_fn=None,
                 engine: bool = True, growth_fn=None):
        # fit_fn(slot, request) -> dict replaces the GPU fit (host-logic tests); it may return
        # "scratch_bytes", the slot's retained scratch after the request; growth_fn(slot,
        # request) then stands in for the library's growth bound (default: a fresh context's)
        self.fit_fn = fit_fn
        self.growth_fn = growth_fn
        self._ctx = [None] * int(slots)
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.device = device
        self.cv = threading.Condition()
        self.pending = []               # FIFO of (req, future, t_submit, inputs, bound)
        self.free_slots = []            # a slot is free once its worker is ready
        self.retained = [0] * self.slots  # scratch each slot's context holds (measured)
        self.charged = 0                # sum(retained) + running requests' inputs and reserves
        self.peak_charged = 0
        self.closed = False
        self.workers = []
        self.t0 = time.perf_counter()
        self.max_concurrent = 0
        self.running = 0
        self.engine = None
        if fit_fn is None and engine:
            from . import deoct
            self.engine = deoct.Engine(device)
        self._work = [queue.Queue() for _ in range(self.slots)]
        for s in range(self.slots):
            t = threading.Thread(target=self._worker, args=(s,), daemon=True)
            t.start()
            self.workers.append(t)
        self._admitter = threading.Thread(target=self._admit_loop, daemon=True)
        self._admitter.start()

    @property
    def peak_in_use(self):
        return self.peak_charged

    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, req: FitRequest) -> Future:
        fut = Future()
        n, F = req.X.shape
        inp, bound = input_bytes(n, F), scratch_bound(req)
        if inp + bound > self.budget:
            fut.set_exception(MemoryError("request %d needs up to %d bytes, over the %d-byte budget"
                                          % (req.id, inp + bound, self.budget)))
            return fut
        with self.cv:
            self.pending.append((req, fut, self.now(), inp, bound))
            self.cv.notify_all()
        return fut

    def _growth(self, slot, req, bound):
        if self.growth_fn is not None:
            return int(self.growth_fn(slot, req))
        if self._ctx[slot] is None:
            return bound
        return scratch_bound(req, ctx=self._ctx[slot])

    def _pick(self):
        """The free slot whose scratch needs the least growth for the oldest request, and
        what running it charges; None if it does not fit the budget now."""
        if not self.pending or not self.free_slots:
            return None
        req, _, _, inp, bound = self.pending[0]
        slot, cost = min(((s, inp + self._growth(s, req, bound)) for s in self.free_slots),
                         key=lambda x: x[1])
        if self.charged + cost > self.budget:
            return None
        return slot, cost

    def _release_idle(self):
        """Nothing runs and the oldest request does not fit: idle slots give their scratch back."""
        freed = False
        for s in self.free_slots:
            if self.retained[s] and self._ctx[s] is not None:
                self._ctx[s].release_scratch()
                held = self._ctx[s].memory()[0]
                self.charged -= self.retained[s] - held
                self.retained[s] = held
                freed = True
        return freed

    def _admit_loop(self):
        while True:
            with self.cv:
                while not self.closed and self._pick() is None:
                    if self.running == 0 and self.pending and self._release_idle():
                        continue
                    self.cv.wait()
                if self.closed and not self.pending:
                    return
                pick = self._pick()
                if pick is None:
                    continue
                slot, cost = pick
                req, fut, ts, inp, bound = self.pending.pop(0)
                self.free_slots.remove(slot)
                self.charged += cost
                self.peak_charged = max(self.peak_charged, self.charged)
                self.running += 1
                self.max_concurrent = max(self.max_concurrent, self.running)
                before = self.retained[slot]
            self._work[slot].put((req, fut, ts, inp, bound, cost, before, self.now()))

    def _worker(self, slot):
        ctx = stream = None
        if self.fit_fn is None:
            import torch

            from . import deoct
            torch.cuda.set_device(self.device)
            ctx = deoct.Context(self.device)
            if self.engine is not None:
                ctx.attach_engine(self.engine)
            stream = torch.cuda.Stream(device=self.device)
        with self.cv:
            if ctx is not None:
                self._ctx[slot] = ctx
                self.retained[slot] = ctx.memory()[0]
                self.charged += self.retained[slot]
            self.free_slots.append(slot)
            self.cv.notify_all()
        while True:
            item = self._work[slot].get()
            if item is None:
                break
            req, fut, ts, inp, bound, cost, before, ta = item
            held = before
            try:
                if self.fit_fn is not None:
                    out = self.fit_fn(slot, req)
                    held = int(out.get("scratch_bytes", before))
                else:
                    # the library holds the slot to its charge: retained scratch plus the
                    # reserve; growing past it would be DEOCT_ERR_OOM, not an overcommit
                    ctx.set_scratch_limit(before + (cost - inp))
                    try:
                        with torch.cuda.stream(stream):
                            out = fit_on_stream(ctx, req, stream)
                    finally:
                        ctx.set_scratch_limit(0)
                    held = ctx.memory()[0]
                res = FitResult(req.id, out["a"], out["theta"], out["leaf_class"], out["kind"],
                                out["node_fit"], t_submit=ts, t_admit=ta, t_done=self.now(), slot=slot,
                                footprint=inp + max(0, held - before), inputs=inp,
                                scratch_before=before, scratch_after=held, scratch_bound=bound,
                                scratch_reserve=cost - inp)
                fut.set_result(res)
            except Exception as e:  # the request fails, the server keeps serving
                fut.set_exception(e)
            finally:
                if ctx is not None:
                    held = ctx.memory()[0]  # also after a failed request
                with self.cv:
                    # the request's inputs and reserve go back; the slot's measured scratch stays
                    self.charged += (held - before) - cost
                    self.retained[slot] = held
                    self.running -= 1
                    self.free_slots.append(slot)
                    self.cv.notify_all()
        if ctx is not None:
            with self.cv:
                self._ctx[slot] = None
            ctx.close()

    def engine_stats(self):
        return None if self.engine is None else self.engine.stats()

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        self._admitter.join()
        for q in self._work:
            q.put(None)
        for t in self.workers:
            t.join()
        if self.engine is not None:
            self.engine.close()
            self.engine = None


def fit_on_stream(ctx, req: FitRequest, stream):
    """Encode a request's data on the device and fit it (moving horizon) on `stream`."""
    import torch

    from . import deoct
    Xd = torch.from_numpy(np.ascontiguousarray(req.X, np.float32)).to("cuda", non_blocking=False)
    yd = torch.from_numpy(np.ascontiguousarray(req.y, np.uint8)).to("cuda", non_blocking=False)
    ds = deoct.encode_dataset(ctx, Xd, yd, req.K, 0, stream=stream)  # width from n_p
    return deoct.deoct_fit_moving_horizon(ctx, ds, fit_params(req), stream=stream)


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
