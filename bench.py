"""Benchmark of the MH-DEOCT hot path on GB300: tree*sample evaluations per second.

Workload (the large-scale DEOCT configuration): n = 10,000,000 samples, F = 10
features U(0,1) quantised to 60,000 levels (uint16 ranks), K = 2 labels from a
planted depth-4 tree with 2% flips; one step = rank-encode the feature matrix
plus a full DEOCT fit of depth-4 trees with population 1024 and 50 generations
(Algorithm 4): (50 + 1) * 1024 * 1e7 = 5.2e11 tree*sample evaluations.  The
inputs (400 MB of features, 200 MB of ranks) are larger than the 129 MB L2,
so no flush is needed between steps.

  value  device-resident: X and y in HBM when the timed region starts.
  e2e    the same metric through the public C ABI from pinned host buffers,
         host->device copy of X, y and device->host copy of the fitted tree
         inside the timed region.

``--impl reference`` times the CPU oracle (the plain C implementation the
tests check against) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "tree*sample evals/s"
UNIT = "evals/s"
WORKLOAD = dict(workload="large-deoct: n=1e7, F=10 U(0,1) quantised to 60000 levels (uint16 ranks), "
                         "K=2 planted depth-4 tree 2% flips; step = rank encode + DEOCT depth 4, "
                         "P=1024, G=50, M=0.5, CR=0.9",
                n=10_000_000, F=10, K=2, depth=4, pop=1024, gens=50,
                l2="inputs larger than L2 (X 400 MB, ranks 200 MB); no flush")
INT32_LANES_PER_SM = 128  # Blackwell SM: 4 partitions x 32 lanes issue INT32
# DRAM bytes (read + write) of one evaluator launch on this workload, from an ncu
# capture of the evaluator on this workload; valid only for the kernel code it was
# taken on: a hash of the re-laid evaluator kernel's code in csrc/eval.cu and of the
# headers it is built from (eval_kernel.cuh, common.cuh), comments and whitespace
# left out.
EVAL_TRAFFIC = {"source_sha256_16": "4c2a85aa0dc07e19", "bytes": 212_132_864 + 3_597_568,
                # the same capture: issue rate (of 4 per SM per cycle), pipe and DRAM figures
                "ncu": {"inst_per_cycle": 3.4608, "issue_frac": 0.8652, "alu_pipe_frac": 0.8130,
                        "shared_pipe_frac": 2742440261 / 152 / (10.224672e-3 * 2.07e9),
                        "inst_per_chunk": 34.23, "dram_gbs": (212_132_864 + 3_597_568) / 10.224672e-3 / 1e9,
                        "dram_frac_of_peak": (212_132_864 + 3_597_568) / 10.224672e-3 / 1e9 / 6777.3}}


def _strip_comments(src):
    """C/C++ source without comments and with runs of whitespace collapsed: the code an
    ncu capture depends on, not its documentation."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def _eval_source_hash():
    """Key of the evaluator kernel's code and launch shape: the `eval_kernel` template and the
    shape chooser `eval_choose_config` of csrc/eval.cu, the kernel header csrc/eval_kernel.cuh
    and the device helpers of csrc/common.cuh (from its "device helpers" section on: the
    host-side context and error code above it are not the kernel's), comments and whitespace
    left out."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2311_06952_gb300", "csrc")
    ev = open(os.path.join(csrc, "eval.cu")).read()
    a = ev.index(" eval_kernel(const __grid_constant__")
    a = ev.rindex("template", 0, a)
    b = ev.index("int launch_t(", a)
    h = hashlib.sha256(_strip_comments(ev[a:b]).encode())
    # the launch shape the workload gets comes from the chooser
    a = ev.index("EvalConfig eval_choose_config(")
    b = ev.index("\n}\n", a)
    h.update(_strip_comments(ev[a:b]).encode())
    with open(os.path.join(csrc, "eval_kernel.cuh")) as fh:
        h.update(_strip_comments(fh.read()).encode())
    with open(os.path.join(csrc, "common.cuh")) as fh:
        common = fh.read()
    h.update(_strip_comments(common[common.index("// device helpers"):]).encode())
    return h.hexdigest()[:16]


def _traffic_default():
    return EVAL_TRAFFIC["bytes"] if _eval_source_hash() == EVAL_TRAFFIC["source_sha256_16"] else None


def _ncu_default():
    return EVAL_TRAFFIC["ncu"] if _eval_source_hash() == EVAL_TRAFFIC["source_sha256_16"] else None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist_setup():
    import torch
    from paper_2311_06952_gb300 import multirank
    rank, world, local = multirank.env_ranks()
    torch.cuda.set_device(local if world > 1 else 0)
    multirank.init("nccl", world)
    return rank, world, local


def _oracle_step(X, y, K, P, D, seed):
    """One bounded oracle step on host cores: rank encode + initial evaluation + one DE
    generation of the P-tree population (2 P n tree*sample evaluations)."""
    import oracle
    ranks, nu = oracle.encode_omp(X)
    oracle.de_run(ranks, nu, y, K, depth=D, P=P, G=1, seed=seed)


def _cpu_baseline(w, budget_s=15.0):
    """The oracle on the host's cores (its OpenMP twins: encode per feature, counts per
    (tree, sample chunk); bit-exact with the plain oracle): initial evaluation plus one DE
    generation of the full population on a bounded prefix of the samples."""
    import oracle
    cores = oracle.host_cores()
    old = oracle.set_threads(cores)
    try:
        P, D = w["pop"], w["depth"]
        X, y = w["X"], w["y"]
        n_try = min(len(X), 20_000 * cores)
        t0 = time.perf_counter()
        _oracle_step(X[:n_try], y[:n_try], w["K"], P, D, 0)
        dt = time.perf_counter() - t0
        n_s = int(min(len(X), max(n_try, n_try * budget_s / max(dt, 1e-3))))
        t0 = time.perf_counter()
        _oracle_step(X[:n_s], y[:n_s], w["K"], P, D, 0)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(old)
    evals = 2 * P * n_s
    return {"value": evals / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d samples of the workload: rank encode + initial evaluation + 1 DE "
                      "generation of the P=1024 depth-4 population (%d evals, %.1f s), oracle's "
                      "OpenMP twins on %d threads" % (n_s, evals, dt, cores)}


def run_reference(args):
    """Reference arm: the CPU oracle on the host's cores, rank 0 only, on bounded samples of
    the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2311_06952_gb300 import datagen
    w = dict(WORKLOAD)
    cores = oracle.host_cores()
    n_s = min(w["n"], 40_000 * cores)
    full = datagen.make_workload(3, n=n_s)
    P, D = w["pop"], w["depth"]
    times = []
    old = oracle.set_threads(cores)
    try:
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            _oracle_step(full["X"], full["y"], full["K"], P, D, it)
            dt = time.perf_counter() - t0
            if it >= args.warmup:
                times.append(dt)
    finally:
        oracle.set_threads(old)
    evals = 2 * P * n_s
    ms = 1000.0 * float(np.mean(times))
    value = evals / (ms / 1000.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(w, sample="each step: first %d samples, rank encode + initial evaluation "
                                     "+ 1 DE generation (P=1024, depth 4)" % n_s),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d samples x 1024 trees x 2 evaluations per step, oracle's "
                                       "OpenMP twins on %d threads" % (n_s, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


MH_WORKLOAD = ("mh-batched: n=1e6, F=30 (15 U(0,1) + 15 LogNormal(0,1)), K=4 planted depth-6 tree 5% "
               "flips, uint32 ranks; moving-horizon D=8, horizon 3, P=128, G=200, M=0.5, CR=0.9")


def _mh_node_counts(ranks_np, a, th, D):
    """Samples reaching each node of a fitted tree (host routing, for the work count)."""
    n = ranks_np.shape[1]
    node = np.ones(n, np.int64)
    counts = np.zeros(1 << (D + 1), np.int64)
    for d in range(D):
        cnt = np.bincount(node, minlength=1 << (D + 1))
        counts[1 << d: 1 << (d + 1)] = cnt[1 << d: 1 << (d + 1)]
        at = a[node - 1].astype(np.int64)
        tt = th[node - 1].astype(np.int64)
        rk = ranks_np[np.maximum(at - 1, 0), np.arange(n)].astype(np.int64)
        node = np.where((at > 0) & (rk < tt), 2 * node, 2 * node + 1)
    return counts


def mh_compare(args):
    """Moving-horizon training, batched level solve vs plain per-node launches, same GPU."""
    import torch
    from paper_2311_06952_gb300 import datagen, deoct
    w = datagen.make_workload(2, n=args.mh_n)
    ctx = deoct.Context(torch.cuda.current_device())
    ds = deoct.encode_dataset(ctx, torch.from_numpy(w["X"]).cuda(), torch.from_numpy(w["y"]).cuda(),
                              w["K"], 4)
    res = {}
    forms = (("batched", deoct.DEOCT_BATCHED), ("plain", 0))
    if args.mh_form != "both":
        forms = tuple(f for f in forms if f[0] == args.mh_form)
    for name, flags in forms:
        prm = deoct.make_params(w["depth"], w["P"], w["G"], mut_f=w["M"], cr=w["CR"], seed=w["seed"],
                                horizon=w["horizon"], flags=flags)
        if name == "batched":
            deoct.deoct_fit_moving_horizon(ctx, ds, prm)  # warm-up: autotuner, graph shapes
        torch.cuda.synchronize()
        ctx.reset_stats()
        t0 = time.perf_counter()
        out = deoct.deoct_fit_moving_horizon(ctx, ds, prm)
        torch.cuda.synchronize()
        res[name] = (time.perf_counter() - t0, out, ctx.stats()["launches"])
    if args.mh_form != "both":
        t, o, l = res[args.mh_form]
        ctx.close()
        return {"workload": MH_WORKLOAD, "form": args.mh_form, "seconds": t, "launches": int(l),
                "subtree_solves": int(np.sum(o["kind"] > 0)), "solves_per_s": float(np.sum(o["kind"] > 0)) / t}
    tb, ob, lb = res["batched"]
    tp, op, lp = res["plain"]
    same = all(np.array_equal(ob[k], op[k]) for k in ("a", "theta", "kind", "node_fit", "leaf_class"))
    solves = int(np.sum(ob["kind"] > 0))
    ranks_np = ds.ranks.cpu().numpy().view(np.uint32)[:, : ds.n]
    cnt = _mh_node_counts(ranks_np, ob["a"], ob["theta"], w["depth"])
    de_nodes = np.nonzero(ob["kind"] == 2)[0] + 1
    evals = int(sum((w["G"] + 1) * w["P"] * int(cnt[t]) for t in de_nodes))
    ctx.close()
    return {"workload": MH_WORKLOAD, "subtree_solves": solves,
            "de_solves": int(len(de_nodes)), "depth1_solves": int(np.sum(ob["kind"] == 1)),
            "batched_s": tb, "plain_s": tp, "batched_solves_per_s": solves / tb,
            "plain_solves_per_s": solves / tp, "speedup": tp / tb, "identical_trees": bool(same),
            "de_evals": evals, "batched_evals_per_s": evals / tb, "plain_evals_per_s": evals / tp,
            "batched_launches": int(lb), "plain_launches": int(lp)}


SERVE_WORKLOAD = ("serving: Poisson arrivals at 20 req/s, n log-uniform [1e3, 2e6], F U{4..60}, K U{2..10}, "
                  "depth U{2..6}, horizon U{2,3}, Gaussian-mixture features, planted-tree labels 5% flips, "
                  "P=128, G=200, M=0.5, CR=0.9, 120 GB budget")


def _serve_trace(raw, slots, engine):
    """Serve the trace (arrival times as generated) and return the results and the server's figures."""
    import torch
    from paper_2311_06952_gb300 import serve
    mk = lambda r: serve.FitRequest(X=r["X"], y=r["y"], K=r["K"], depth=r["depth"], horizon=r["horizon"],
                                    pop=128, gens=200, seed=r["id"], id=r["id"], arrival=r["arrival"])
    srv = serve.Server(budget_bytes=120 << 30, slots=slots, engine=engine)
    try:
        warm = [mk(r) for r in raw[:slots]]  # not timed: every slot gets its context and kernels ready
        for w in warm:
            w.arrival = 0.0
        serve.run_trace(srv, warm)
        st0 = srv.engine_stats()
        srv.max_concurrent = 0
        srv.peak_charged = srv.charged
        torch.cuda.reset_peak_memory_stats()
        t0 = srv.now()
        res = serve.run_trace(srv, [mk(r) for r in raw])
        t1 = srv.now()
        st1 = srv.engine_stats()
        held = sum(srv.retained) + torch.cuda.max_memory_reserved()
    finally:
        srv.close()
    out = {"requests": len(res), "makespan_s": t1 - t0, "throughput_rps": len(res) / (t1 - t0),
           "latency": serve.latency_stats([r.latency for r in res]), "slots": slots,
           "budget_bytes": 120 << 30, "peak_charged_bytes": srv.peak_charged,
           "device_bytes_held": int(held), "max_concurrent": srv.max_concurrent,
           "scratch_growth_within_reserve": bool(all(r.scratch_after - r.scratch_before <= r.scratch_reserve
                                                     for r in res))}
    if st1 is not None:
        out["engine"] = {k: st1[k] - st0[k] if k not in ("max_jobs_per_launch", "max_problems_per_launch")
                         else st1[k] for k in st1}
    return res, out


def serve_compare(num, slots):
    """The serving workload's first `num` requests: served with the shared engine (launches
    carrying several requests' generations), served with a stream per request, and solved
    one at a time with the plain per-node form (FIFO, same arrivals)."""
    import torch
    from paper_2311_06952_gb300 import datagen, deoct, serve
    raw = datagen.serving_requests(num=num, rate=20.0, materialize=True)  # not timed
    res_e, eng = _serve_trace(raw, slots, True)
    res_s, strm = _serve_trace(raw, slots, False)
    by_e = {r.id: r for r in res_e}
    by_s = {r.id: r for r in res_s}
    keys = ("a", "theta", "kind", "node_fit", "leaf_class")
    same = all(np.array_equal(getattr(by_e[i], k), getattr(by_s[i], k)) for i in by_e for k in keys)
    ctx = deoct.Context(0)
    stream = torch.cuda.Stream()
    service = []
    for r in raw:
        q = serve.FitRequest(X=r["X"], y=r["y"], K=r["K"], depth=r["depth"], horizon=r["horizon"], pop=128,
                             gens=200, seed=r["id"], id=r["id"], arrival=r["arrival"], batched=False)
        with torch.cuda.stream(stream):
            if r is raw[0]:
                serve.fit_on_stream(ctx, q, stream)  # warm-up
            torch.cuda.synchronize()
            ts = time.perf_counter()
            out = serve.fit_on_stream(ctx, q, stream)
            torch.cuda.synchronize()
            service.append(time.perf_counter() - ts)
        same = same and all(np.array_equal(getattr(by_e[r["id"]], k), out[k]) for k in keys)
    ctx.close()
    seq_lat = serve.sequential_queue_latencies([r["arrival"] for r in raw], service)
    seq_makespan = max(a + l for a, l in zip([r["arrival"] for r in raw], seq_lat))
    # the same requests arriving 10x faster (200 req/s): the GPU saturates and the requests'
    # work queues; served with the engine and with a stream per request
    burst = [dict(r, arrival=r["arrival"] / 10.0) for r in raw]
    res_be, beng = _serve_trace(burst, slots, True)
    res_bs, bstr = _serve_trace(burst, slots, False)
    same = same and all(np.array_equal(getattr(r, k), getattr(by_e[r.id], k)) for r in res_be + res_bs
                        for k in keys)
    return {"metric": "p50/p99 request latency and requests/s", "workload": SERVE_WORKLOAD,
            "requests": num, "served_engine": eng, "served_streams": strm,
            "sequential_plain": {"latency": serve.latency_stats(seq_lat),
                                 "throughput_rps": num / seq_makespan,
                                 "service_s_total": float(np.sum(service))},
            "engine_vs_streams": {"p99": eng["latency"]["p99_s"] / strm["latency"]["p99_s"],
                                  "p50": eng["latency"]["p50_s"] / strm["latency"]["p50_s"],
                                  "throughput": eng["throughput_rps"] / strm["throughput_rps"]},
            "burst_200rps": {"served_engine": beng, "served_streams": bstr,
                             "engine_vs_streams": {
                                 "p99": beng["latency"]["p99_s"] / bstr["latency"]["p99_s"],
                                 "p50": beng["latency"]["p50_s"] / bstr["latency"]["p50_s"],
                                 "throughput": beng["throughput_rps"] / bstr["throughput_rps"]}},
            "identical_trees_engine_streams_plain": bool(same), "data": "synthetic"}


def run_serve(args):
    """Serving workload with --serve requests (all 500: the full trace)."""
    from paper_2311_06952_gb300 import build as _build
    _build.build()
    line = dict(mode="serving", **serve_compare(args.serve, args.slots))
    print(json.dumps(line), flush=True)
    return 0


def eval_workload1(args):
    """Population-evaluation workload at full size: one evaluation of 256 random depth-3
    trees on n = 1e5 (F = 20, K = 3, uint32 ranks).  Its 8 MB of ranks fit in L2, so L2 is
    flushed (a 512 MB write) before every timed evaluation."""
    import torch
    from paper_2311_06952_gb300 import datagen, deoct
    w = datagen.make_workload(1)
    ctx = deoct.Context(torch.cuda.current_device())
    ds = deoct.encode_dataset(ctx, torch.from_numpy(w["X"]).cuda(), torch.from_numpy(w["y"]).cuda(),
                              w["K"], w["rank_bytes"])
    nu = ds.n_unique.cpu().numpy().view(np.uint32)
    a, th = datagen.random_population(nu, w["P"], w["depth"],
                                      np.random.Generator(np.random.PCG64(w["pop_seed"])))
    ad = torch.from_numpy(a.astype(np.int16)).cuda()
    td = torch.from_numpy(th.view(np.int32)).cuda()
    L = 1 << w["depth"]
    counts = torch.empty((w["P"], L, w["K"]), dtype=torch.int32, device="cuda")
    errs = torch.empty(w["P"], dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    times = []
    for it in range(args.warmup + args.steps * 4):
        flush.fill_(it & 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        deoct.deoct_eval_population(ctx, ds, ad, td, w["depth"], counts_out=counts, errors_out=errs)
        e1.record()
        torch.cuda.synchronize()
        if it >= args.warmup:
            times.append(e0.elapsed_time(e1))
    ctx.close()
    ms = float(np.median(times))
    evals = w["P"] * w["X"].shape[0]
    return {"workload": "eval-gmm: n=1e5, F=20 Gaussian mixture, K=3, 256 random depth-3 trees, "
                        "uint32 ranks, one evaluation (one launch: pack + evaluate + errors), L2 flushed",
            "ms": ms, "evals": evals, "evals_per_s": evals / (ms / 1000.0), "samples": len(times),
            "launches_per_eval": 1}


def eval_p_sweep(ctx, ranks, nu, yd, n, F, K, peaks, depth=4):
    """Where the population evaluator turns HBM-bound: one evaluation of P random depth-4
    trees on the main workload's resident ranks (n = 1e7, uint16, 200 MB: larger than L2) for
    P from 1 to 1024, timed on the evaluator launch.  Algorithmic bytes n (F w + 1) are read
    once per tree group whatever P is, so below the crossover P* = R_alu t_hbm / n (R_alu =
    the compute-bound evals/s, t_hbm = bytes / measured copy bandwidth) HBM bounds the launch."""
    import torch
    from paper_2311_06952_gb300 import datagen, deoct
    ds = deoct.DeviceDataset(ranks, 2, nu, yd, n, F, K)
    nu_h = nu.cpu().numpy().view(np.uint32)
    alg = n * (F * 2 + 1)
    rows = []
    for P in (1, 2, 4, 8, 16, 64, 256, 1024):
        a, th = datagen.random_population(nu_h, P, depth, np.random.Generator(np.random.PCG64(50 + P)))
        ad = torch.from_numpy(a.astype(np.int16)).cuda()
        td = torch.from_numpy(th.view(np.int32)).cuda()
        counts = torch.empty((P, 1 << depth, K), dtype=torch.int32, device="cuda")
        errs = torch.empty(P, dtype=torch.int32, device="cuda")
        ms = []
        for it in range(8):
            ctx.reset_stats()
            ctx.set_timing(True)
            deoct.deoct_eval_population(ctx, ds, ad, td, depth, counts_out=counts, errors_out=errs)
            torch.cuda.synchronize()
            st = ctx.stats()
            ctx.set_timing(False)
            if it >= 3:
                ms.append(st["eval_ms"] / max(1, st["eval_timed"]))
        m = float(np.median(ms))
        gbs = alg / (m / 1000.0) / 1e9
        rows.append({"P": P, "launch_ms": m, "evals_per_s": P * n / (m / 1000.0), "alg_gbs": gbs,
                     "hbm_frac": gbs / peaks["hbm_gbs"]})
    t_hbm = alg / (peaks["hbm_gbs"] * 1e9)
    r_alu = rows[-1]["evals_per_s"]
    return {"workload": "large-deoct ranks (n=1e7, F=10, uint16, K=2), P random depth-4 trees, "
                        "one evaluation launch each (fused pack + evaluate + errors)",
            "algorithmic_bytes": alg, "t_hbm_us": t_hbm * 1e6, "crossover_P": r_alu * t_hbm / n,
            "rows": rows}


def run_p_eval(args):
    """Evaluations of P random depth-4 trees on the main workload's ranks (n = --n, uint16),
    one launch each, timed on the evaluator launch; the encoder's scratch is released first,
    so little else sits on the device (the form profiled for small populations)."""
    import torch
    from paper_2311_06952_gb300 import build as _build
    from paper_2311_06952_gb300 import datagen, deoct
    _build.build()
    torch.cuda.set_device(0)
    data = datagen.make_workload(3, n=args.n)
    enc = deoct.Context(0)
    ds = deoct.encode_dataset(enc, torch.from_numpy(data["X"]).cuda(), torch.from_numpy(data["y"]).cuda(), 2, 2)
    torch.cuda.synchronize()
    enc.close()
    torch.cuda.empty_cache()
    ctx = deoct.Context(0)
    P = args.p_eval
    nu = ds.n_unique.cpu().numpy().view(np.uint32)
    a, th = datagen.random_population(nu, P, 4, np.random.Generator(np.random.PCG64(50 + P)))
    ad = torch.from_numpy(a.astype(np.int16)).cuda()
    td = torch.from_numpy(th.view(np.int32)).cuda()
    ms = []
    for it in range(args.warmup + args.steps):
        ctx.reset_stats()
        ctx.set_timing(True)
        counts, errs = deoct.deoct_eval_population(ctx, ds, ad, td, 4)
        torch.cuda.synchronize()
        st = ctx.stats()
        ctx.set_timing(False)
        if it >= args.warmup:
            ms.append(st["eval_ms"] / max(1, st["eval_timed"]))
    n, F = data["X"].shape
    m = float(np.median(ms))
    peaks, kind = _peaks()
    gbs = n * (2 * F + 1) / (m / 1000.0) / 1e9
    print(json.dumps({"mode": "p-eval", "P": P, "n": n, "launch_ms": m, "evals_per_s": P * n / (m / 1000.0),
                      "alg_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"], "peak_kind": kind,
                      "errors0": int(errs[0])}), flush=True)
    ctx.close()
    return 0


def run_stream_scan(args):
    """Single evaluations of 1 and 2 random depth-4 trees on the main workload's ranks for
    n = 1e6 .. 1e7 (L2 flushed before each launch), beside a torch reduction over the same
    number of bytes, and a line through the one-tree times: the fixed cost of a launch and
    its streaming rate."""
    import torch
    from paper_2311_06952_gb300 import build as _build
    from paper_2311_06952_gb300 import datagen, deoct
    _build.build()
    torch.cuda.set_device(0)
    ctx = deoct.Context(0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    reps = max(3, args.steps)
    rows = []
    for n in (1_000_000, 2_500_000, 5_000_000, 10_000_000):
        data = datagen.make_workload(3, n=n)
        ds = deoct.encode_dataset(ctx, torch.from_numpy(data["X"]).cuda(), torch.from_numpy(data["y"]).cuda(),
                                  2, 2)
        nu = ds.n_unique.cpu().numpy().view(np.uint32)
        F = data["X"].shape[1]
        nbytes = n * (2 * F + 1)
        row = {"n": n, "alg_bytes": nbytes}
        for P in (1, 2):
            a, th = datagen.random_population(nu, P, 4, np.random.Generator(np.random.PCG64(50 + P)))
            ad = torch.from_numpy(a.astype(np.int16)).cuda()
            td = torch.from_numpy(th.view(np.int32)).cuda()
            ms = []
            for it in range(args.warmup + reps):
                flush.fill_(it & 255)
                ctx.reset_stats()
                ctx.set_timing(True)
                deoct.deoct_eval_population(ctx, ds, ad, td, 4)
                torch.cuda.synchronize()
                st = ctx.stats()
                ctx.set_timing(False)
                if it >= args.warmup:
                    ms.append(st["eval_ms"] / max(1, st["eval_timed"]))
            row["P%d_us" % P] = 1000.0 * float(np.median(ms))
        x = torch.rand(nbytes // 4, device="cuda")
        ts = []
        for it in range(args.warmup + reps):
            flush.fill_(it & 255)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            x.sum()
            e1.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        row["torch_sum_us"] = 1000.0 * float(np.median(ts))
        rows.append(row)
        del ds, x
        torch.cuda.empty_cache()
    peaks, kind = _peaks()
    nb = np.array([r["alg_bytes"] for r in rows], dtype=np.float64)
    t1 = np.array([r["P1_us"] for r in rows])
    slope, fixed = np.polyfit(nb, t1, 1)
    rate = 1e-3 / slope  # bytes per us -> GB/s
    print(json.dumps({"mode": "stream-scan", "rows": rows, "P1_fixed_us": float(fixed),
                      "P1_stream_gbs": float(rate), "P1_stream_frac": float(rate / peaks["hbm_gbs"]),
                      "peak_kind": kind}), flush=True)
    ctx.close()
    return 0


def run_table3(args):
    """Time-to-train on synthetic sets shaped like the paper's large-scale sets (Table 3):
    MH-DEOCT in the paper's Normal mode (P=100, G=600, CR=0.1, M=rand(0,1)) with CART and DEOCT
    warm starts, horizon 2 at depth 2 and 3 otherwise, 75/25 split.  The data is synthetic,
    so the times are not comparable with the paper's, which are on the real sets."""
    import torch
    from paper_2311_06952_gb300 import build as _build
    from paper_2311_06952_gb300 import datagen
    from paper_2311_06952_gb300.estimator import MHDEOCTClassifier
    _build.build()
    rows = []
    for name in args.table3.split(","):
        d = datagen.table3_standin(name)
        for depth in (2, 4, 8):
            clf = MHDEOCTClassifier(depth=depth, preset="normal", seed=0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            clf.fit(d["Xtr"], d["ytr"], K=d["K"])
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            rows.append({"set": name, "shape": list(datagen.TABLE3_SHAPES[name]), "depth": depth,
                         "train_s": t, "train_acc": clf.score(d["Xtr"], d["ytr"]),
                         "test_acc": clf.score(d["Xte"], d["yte"])})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"mode": "table3-shapes", "settings": "Normal mode P=100 G=600 CR=0.1 dithered M, "
                      "CART + DEOCT warm starts, horizon 2 (D=2) / 3, 75/25 split, synthetic data of "
                      "the paper's Table 3 shapes", "rows": rows}), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2311_06952_gb300 import build as _build
    from paper_2311_06952_gb300 import datagen, deoct

    from paper_2311_06952_gb300 import multirank
    rank, world, local = _dist_setup()
    if rank == 0:
        _build.build()
    multirank.barrier(world)
    w = dict(WORKLOAD)
    data = datagen.make_workload(3, n=args.n)
    n, F, K = data["X"].shape[0], data["X"].shape[1], data["K"]
    P, D, G = w["pop"], w["depth"], args.gens
    stream = torch.cuda.current_stream()
    ctx = deoct.Context(torch.cuda.current_device())
    Xd = torch.from_numpy(data["X"]).cuda()
    yd = torch.from_numpy(data["y"]).cuda()
    prm = deoct.make_params(D, P, G, mut_f=0.5, cr=0.9, seed=0)
    ranks = torch.empty((F, deoct.padded_ld(n, 2)), dtype=torch.int16, device="cuda")
    nu = torch.empty(F, dtype=torch.int32, device="cuda")
    evals_per_step = (G + 1) * P * n

    def step(sid):
        deoct.deoct_encode(ctx, Xd, 2, ranks_out=ranks, n_unique_out=nu)
        ds = deoct.DeviceDataset(ranks, 2, nu, yd, n, F, K)
        return deoct.deoct_fit_subtree(ctx, ds, prm, stream_id=sid)

    for i in range(args.warmup):
        step(multirank.stream_id(rank))
    torch.cuda.synchronize()
    # the timed loop runs the path as a user gets it: per-launch timing off, so every DEOCT
    # generation is one replay of the captured CUDA graph
    ctx.reset_stats()
    ctx.set_timing(False)
    clk = ClockSampler(local) if rank == 0 else None
    if clk:
        clk.start()
    multirank.barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        res = step(multirank.stream_id(rank))
    e1.record(stream)
    torch.cuda.synchronize()
    multirank.barrier(world)
    ms_total = e0.elapsed_time(e1)
    clocks = clk.stop() if clk else None
    st = ctx.stats()
    ms_total = multirank.max_over_ranks(ms_total, world, "cuda")
    ms_step = ms_total / args.steps
    value = multirank.whole_job_rate(evals_per_step, world, ms_step / 1000.0)

    # ---- roofline pass: one more step with library-side CUDA events around every evaluator
    # launch (the launches are then issued directly, not replayed from a graph) ---------------
    ctx.reset_stats()
    ctx.set_timing(True)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    step(multirank.stream_id(rank))
    f1.record(stream)
    torch.cuda.synchronize()
    st_roof = ctx.stats()
    ctx.set_timing(False)
    ms_step_timed_launches = f0.elapsed_time(f1)

    # ---- end to end through the public API, host buffers ----------------------
    Xh = torch.from_numpy(data["X"]).pin_memory()
    yh = torch.from_numpy(data["y"]).pin_memory()
    h2d = Xh.numel() * 4 + yh.numel()
    B = (1 << D) - 1
    d2h = B * 2 + B * 4 + 8

    # every step copies its inputs host -> device and reads its fitted tree back; the copy of
    # step i + 1 runs on a copy stream while step i computes (two device buffers in turn)
    copy_stream = torch.cuda.Stream()
    bufX = [torch.empty_like(Xh, device="cuda") for _ in range(2)]
    bufY = [torch.empty_like(yh, device="cuda") for _ in range(2)]
    landed = [torch.cuda.Event() for _ in range(2)]
    # the encoder writes into caller-owned outputs, one pair per input buffer (left to
    # torch's caching allocator, the second step's fresh 200 MB block was a cudaMalloc
    # inside the timed region)
    bufR = [torch.empty((F, deoct.padded_ld(n, 2)), dtype=torch.int16, device="cuda") for _ in range(2)]
    bufN = [torch.empty(F, dtype=torch.int32, device="cuda") for _ in range(2)]

    def load(i):
        with torch.cuda.stream(copy_stream):
            bufX[i % 2].copy_(Xh, non_blocking=True)
            bufY[i % 2].copy_(yh, non_blocking=True)
            landed[i % 2].record(copy_stream)

    def e2e_steps(k, sid):
        load(0)
        for i in range(k):
            stream.wait_event(landed[i % 2])
            if i + 1 < k:
                load(i + 1)  # the previous user of this buffer (step i - 1) has finished
            deoct.deoct_encode(ctx, bufX[i % 2], 2, ranks_out=bufR[i % 2], n_unique_out=bufN[i % 2])
            ds = deoct.DeviceDataset(bufR[i % 2], 2, bufN[i % 2], bufY[i % 2], n, F, K)
            deoct.deoct_fit_subtree(ctx, ds, prm, stream_id=sid)  # host outputs (sync)

    e2e_steps(1, multirank.stream_id(rank))
    multirank.barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps(args.steps, multirank.stream_id(rank))
    torch.cuda.synchronize()
    t_e2e = multirank.max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_value = multirank.whole_job_rate(evals_per_step, world, t_e2e / args.steps)

    if rank != 0:
        return 0
    peaks, peak_kind = _peaks()
    eval_ms = st_roof["eval_ms"] / max(1, st_roof["eval_timed"])
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # per tree-sample evaluation, per level: load the node's feature and threshold, load the
    # sample's rank, compare, step to the child; then the count increment (2)
    ops_per_eval = 4 * D + 2
    ops_per_launch = ops_per_eval * P * n
    achieved = ops_per_launch / (eval_ms / 1000.0) / 1e12
    strict_ops = (2 * D + 1) * P * n  # only the comparison and the child step per level, one count
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = nsm * INT32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    bytes_per_launch = n * (F * 2 + 1)
    hbm_achieved = bytes_per_launch / (eval_ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": w, "gpu_launches": int(st["launches"]),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak,
                     "traffic": args.traffic if args.traffic is not None else (
                         _traffic_default() if args.n == WORKLOAD["n"] else None),
                     "kernel": "eval_kernel<2,4,0> (population evaluator)",
                     "ops_per_launch": ops_per_launch, "ops_per_eval": ops_per_eval,
                     "launch_ms": eval_ms, "launches_timed": int(st_roof["eval_timed"]),
                     "timing_pass": "one extra step after the timed loop, launches issued directly "
                                    "with CUDA events around each evaluator launch (%.1f ms for the "
                                    "step vs %.1f ms per graph-replayed step in the timed loop)"
                                    % (ms_step_timed_launches, ms_step),
                     "strict_view": {"ops_per_eval": 2 * D + 1, "ops_per_launch": strict_ops,
                                     "achieved": strict_ops / (eval_ms / 1000.0) / 1e12,
                                     "frac": strict_ops / (eval_ms / 1000.0) / 1e12 / peak},
                     "peak_basis": "%d SMs x %d INT32 lanes x %.0f MHz (%s max clock)" % (
                         nsm, INT32_LANES_PER_SM, sm_mhz, peak_kind),
                     "issue_view": _ncu_default() if args.n == WORKLOAD["n"] else None,
                     "hbm_view": {"achieved_gbs": hbm_achieved, "peak_gbs": peaks["hbm_gbs"],
                                  "frac": hbm_achieved / peaks["hbm_gbs"],
                                  "algorithmic_bytes_per_launch": bytes_per_launch,
                                  "peak_kind": peak_kind}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipeline": "each step's X, y copied from pinned host memory inside the timed region; "
                            "step i + 1's copy on a copy stream while step i runs; the fitted tree "
                            "read back to the host every step"},
        "clocks": clocks,
        "result": {"fitness": res[2], "train_accuracy": 1.0 - res[2] / n},
    }
    if world == 1 and not args.no_mh:
        line["p_sweep"] = eval_p_sweep(ctx, ranks, nu, yd, n, F, K, peaks)
        line["population_eval"] = eval_workload1(args)
        line["mh_batched_vs_plain"] = mh_compare(args)
    if world == 1 and args.serve_default > 0:
        del Xd, ranks
        torch.cuda.empty_cache()
        line["serving"] = serve_compare(args.serve_default, args.slots)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(dict(w, X=data["X"], y=data["y"]))
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"])
    ap.add_argument("--gens", type=int, default=WORKLOAD["gens"])
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per evaluator launch, when a capture of this kernel exists")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mh", action="store_true", help="skip the batched-vs-plain moving-horizon line")
    ap.add_argument("--mh-n", type=int, default=1_000_000)
    ap.add_argument("--serve", type=int, default=0, help="run the serving workload with this many requests")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-default", type=int, default=60,
                    help="requests of the serving trace in the default line (0: none)")
    ap.add_argument("--table3", default="", help="comma list of bitcoin-heist,susy,higgs")
    ap.add_argument("--mh-only", action="store_true", help="only the batched-vs-plain moving-horizon line")
    ap.add_argument("--mh-form", choices=["both", "batched", "plain"], default="both",
                    help="with --mh-only: time one form alone (a batched run is preceded by a warm-up fit)")
    ap.add_argument("--p-eval", type=int, default=0, help="only single evaluations of this many trees")
    ap.add_argument("--stream-scan", action="store_true",
                    help="only single evaluations of 1 and 2 trees for n = 1e6..1e7 beside a torch reduction")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.table3:
        return run_table3(args)
    if args.p_eval:
        return run_p_eval(args)
    if args.stream_scan:
        return run_stream_scan(args)
    if args.mh_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"mode": "mh-only", "mh_batched_vs_plain": mh_compare(args)}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
