"""Multi-rank host path on CPU (gloo, world size 2): ranks solve independent
problems (distinct Philox streams), exchange nothing on the data path, and the
whole-job rate divides all ranks' units by the slowest rank's time."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import oracle
    from paper_2311_06952_gb300 import datagen, multirank
    r, w, _ = multirank.env_ranks()
    multirank.init("gloo", w)
    d = datagen.make_workload(0, n=300)
    ranks, nu = oracle.encode(d["X"])
    res = oracle.de_run(ranks, nu, d["y"], d["K"], depth=2, P=16, G=5, seed=0,
                        stream=multirank.stream_id(r))
    t = 1.0 + r  # pretend rank r took 1 + r seconds
    tmax = multirank.max_over_ranks(t, w)
    rate = multirank.whole_job_rate(6 * 16 * 300, w, tmax)
    multirank.barrier(w)
    out.put((r, tmax, rate, res["pop"].tobytes()))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_independent_problems_and_max_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, pop0), (r1, t1, v1, pop1) = got
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 2.0  # both ranks see the slowest rank's time
    assert v0 == v1 == 2 * 6 * 16 * 300 / 2.0
    assert pop0 != pop1  # distinct Philox streams: independent problems


def test_single_rank_defaults():
    from paper_2311_06952_gb300 import multirank
    assert multirank.max_over_ranks(3.5, 1) == 3.5
    assert multirank.whole_job_rate(10, 1, 2.0) == 5.0
