"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integers (ranks, counts, errors) and the DE trajectory (float32 genes, double
fitness, best index) must agree bit for bit: both sides take every
float decision in the same precision with one rounding per operation.
"""
import numpy as np
import pytest

import oracle
from paper_2311_06952_gb300 import datagen

from gpu_helpers import ctx, gpu_dataset, ranks_np, to_dev, u16, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2311_06952_gb300 import build
    build.build()
    return ctx()


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


# --------------------------------------------------------------------------
# a1: rank encoder
# --------------------------------------------------------------------------

def _encode_case(name):
    rng = _rng(sum(name.encode()))
    if name == "w0":
        w = datagen.make_workload(0)
        return w["X"], 2
    if name == "w1_small":
        return datagen.make_workload(1, n=20000)["X"], 4
    if name == "w3_small":
        return datagen.make_workload(3, n=150_001)["X"], 2
    if name == "ties_signed_zero":
        X = np.round(rng.normal(size=(4097, 5)), 1).astype(np.float32)
        X[::7, 0] = -0.0
        X[::5, 0] = 0.0
        X[:, 3] = 2.0
        X[5, 4] = np.inf
        X[6, 4] = -np.inf
        return X, 2
    if name == "one_sample":
        return np.array([[3.0, -1.0]], np.float32), 4
    if name == "wide_F":
        return rng.random((3000, 131)).astype(np.float32), 4
    if name == "continuous_u32":
        return rng.lognormal(size=(70_000, 3)).astype(np.float32), 4
    raise KeyError(name)


@pytest.mark.parametrize("name", ["w0", "w1_small", "w3_small", "ties_signed_zero", "one_sample",
                                  "wide_F", "continuous_u32"])
def test_encode_bit_exact(c, name):
    X, rb = _encode_case(name)
    y = np.zeros(len(X), np.uint8)
    ds = gpu_dataset(c, X, y, 2, rb)
    r_ref, nu_ref = oracle.encode(X)
    np.testing.assert_array_equal(u32(ds.n_unique), nu_ref)
    np.testing.assert_array_equal(ranks_np(ds), r_ref)


def test_encode_rejects_nan_and_narrow_width(c):
    from paper_2311_06952_gb300 import deoct
    X = np.zeros((100, 2), np.float32)
    X[50, 1] = np.nan
    with pytest.raises(deoct.DeoctError) as e:
        gpu_dataset(c, X, np.zeros(100, np.uint8), 2, 4)
    assert e.value.code == deoct.DEOCT_ERR_INVALID
    X = np.arange(70000, dtype=np.float32)[:, None]
    with pytest.raises(deoct.DeoctError):
        gpu_dataset(c, X, np.zeros(70000, np.uint8), 2, 2)
    # the context stays usable after both errors
    X = np.arange(10, dtype=np.float32)[:, None]
    ds = gpu_dataset(c, X, np.zeros(10, np.uint8), 2, 2)
    assert u32(ds.n_unique)[0] == 10


@pytest.mark.parametrize("name,want_w", [("w3_small", 2), ("continuous_u32", 4), ("one_sample", 2),
                                         ("exactly_65536", 2), ("exactly_65537", 4)])
def test_encode_auto_width_from_n_p(c, name, want_w):
    """The automatic width is uint16 exactly when every n_p <= 65536, whatever n is; the ranks
    and the distinct values equal the oracle's."""
    import torch
    from paper_2311_06952_gb300 import deoct
    if name.startswith("exactly_"):
        m = int(name.split("_")[1])
        rng = _rng(m)
        X = np.stack([rng.permutation(np.arange(m, dtype=np.float32) / 7),
                      rng.integers(0, 5, m).astype(np.float32)], axis=1)
        X = np.concatenate([X, X[: 1000]])  # n > n_p
    else:
        X, _ = _encode_case(name)
    ranks, nu, uniq, w = deoct.deoct_encode_auto(c, to_dev(np.ascontiguousarray(X, np.float32)))
    assert w == want_w
    assert ranks.element_size() == w and ranks.shape[1] % 8 == 0
    r_ref, nu_ref = oracle.encode(X)
    np.testing.assert_array_equal(u32(nu), nu_ref)
    got = (u16(ranks) if w == 2 else u32(ranks))[:, : len(X)].astype(np.uint32)
    np.testing.assert_array_equal(got, r_ref)
    u = uniq.cpu().numpy()
    for p in range(X.shape[1]):
        np.testing.assert_array_equal(u[p, : nu_ref[p]], np.unique(np.where(X[:, p] == 0, 0, X[:, p])))


# --------------------------------------------------------------------------
# a3 + a4: evaluator
# --------------------------------------------------------------------------

EVAL_CASES = [
    # (n, F, K, depth, P, rank_bytes, subset, seed)
    (1000, 8, 2, 2, 64, 2, False, 0),
    (5001, 6, 3, 3, 40, 4, False, 1),
    (5001, 6, 3, 3, 40, 2, True, 2),
    (33, 3, 2, 1, 7, 2, False, 3),
    (1, 2, 2, 2, 5, 4, False, 4),
    (20000, 10, 4, 4, 300, 2, False, 5),   # several tree groups, K*L = 64 (2 bins per lane)
    (12345, 5, 10, 3, 50, 4, False, 6),    # K*L = 80: 3 bins per lane
    (9000, 7, 2, 5, 33, 2, False, 7),      # depth 5 ballot path
    (9000, 7, 3, 6, 20, 4, False, 8),      # depth 6: shared-atomic path
    (4000, 4, 2, 8, 9, 2, True, 9),        # depth 8, gathered subset
    (70000, 3, 5, 4, 17, 4, False, 10),
]


@pytest.mark.parametrize("case", EVAL_CASES, ids=[str(c_[:7]) for c_ in EVAL_CASES])
def test_eval_bit_exact(c, case):
    from paper_2311_06952_gb300 import deoct
    n, F, K, depth, P, rb, subset, seed = case
    rng = _rng(100 + seed)
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ds = gpu_dataset(c, X, y, K, rb)
    ranks, nu = oracle.encode(X)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    idx = None
    if subset:
        idx = np.sort(rng.choice(n, max(1, n // 3), replace=False)).astype(np.int32)
        idx = idx[rng.permutation(len(idx))]  # any order
    counts, errors = deoct.deoct_eval_population(
        c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth,
        sample_idx=None if idx is None else to_dev(idx))
    ref = oracle.eval_counts(ranks, y, K, a, th, depth, idx=idx)
    _, ref_err, _, _ = oracle.fitness(ref, a, n if idx is None else len(idx))
    np.testing.assert_array_equal(u32(counts), ref)
    np.testing.assert_array_equal(u32(errors), ref_err)


@pytest.mark.parametrize("shape", [(128, 3, 1, 1), (256, 16, 4, 3), (512, 64, 8, 7), (2048, 256, 16, 5),
                                   (8192, 1, 2, 2), (1152, 70, 32, 0), (640, 32, 32, 9), (1408, 16, 24, 0)])
def test_eval_launch_shapes_bit_exact(c, shape):
    """Persistent CTAs walking many tiles and several tree groups give the same counts, with
    tiles that are not powers of two and CTAs of up to 32 warps."""
    from paper_2311_06952_gb300 import deoct
    S, TG, warps, grid = shape
    rng = _rng(200 + S)
    n, F, K, depth, P = 23456, 6, 3, 3, 70
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    ref = oracle.eval_counts(ranks, y, K, a, th, depth)
    try:
        c.set_eval_config(S, TG, warps, grid)
        for rb in (2, 4):
            ds = gpu_dataset(c, X, y, K, rb)
            counts, _ = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth)
            np.testing.assert_array_equal(u32(counts), ref)
            idx = rng.permutation(n)[: n // 2].astype(np.int32)
            counts, _ = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth,
                                                    sample_idx=to_dev(idx))
            np.testing.assert_array_equal(u32(counts), oracle.eval_counts(ranks, y, K, a, th, depth, idx=idx))
    finally:
        c.set_eval_config(0, 0, 0, 0)


@pytest.mark.parametrize("shape", [(0, 0, 0, 0), (256, 128, 16, 0), (512, 64, 16, 7), (1024, 16, 6, 3),
                                   (128, 200, 16, 2), (768, 32, 32, 0)])
@pytest.mark.parametrize("depth,K", [(3, 4), (4, 2), (2, 30), (5, 3)])
def test_eval_streaming_kernel_large_groups_bit_exact(c, shape, depth, K):
    """The streaming kernel forced for groups of 16+ trees (shared class masks, trees split over
    the routing warps, two landing zones): same counts, both rank widths, full set and subset."""
    from paper_2311_06952_gb300 import deoct
    S, TG, warps, grid = shape
    rng = _rng(600 + S + depth * 7 + K)
    n, F, P = 30011, 7, 200
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    ref = oracle.eval_counts(ranks, y, K, a, th, depth)
    idx = np.sort(rng.choice(n, n // 3, replace=False)).astype(np.int32)
    ref_sub = oracle.eval_counts(ranks, y, K, a, th, depth, idx=idx)
    try:
        c.set_eval_streaming(True)
        c.set_eval_config(S, TG, warps, grid)
        for rb in (2, 4):
            ds = gpu_dataset(c, X, y, K, rb)
            counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth)
            np.testing.assert_array_equal(u32(counts), ref)
            counts, _ = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth,
                                                    sample_idx=to_dev(idx))
            np.testing.assert_array_equal(u32(counts), ref_sub)
    finally:
        c.set_eval_streaming(False)
        c.set_eval_config(0, 0, 0, 0)


@pytest.mark.parametrize("shape", [(0, 0, 0, 0), (128, 2, 16, 3), (1024, 8, 16, 5), (512, 1, 4, 1),
                                   (1152, 8, 32, 0)])
@pytest.mark.parametrize("depth,K", [(7, 3), (4, 29)])
def test_eval_shared_atomic_mode_shapes_bit_exact(c, shape, depth, K):
    """Many bins (2^D K > 128): warps split each tree's chunks into shared job counts."""
    from paper_2311_06952_gb300 import deoct
    S, TG, warps, grid = shape
    rng = _rng(400 + depth + K)
    n, F, P = 17001, 5, 23
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    ref = oracle.eval_counts(ranks, y, K, a, th, depth)
    try:
        c.set_eval_config(S, TG, warps, grid)
        for rb in (2, 4):
            ds = gpu_dataset(c, X, y, K, rb)
            counts, _ = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth)
            np.testing.assert_array_equal(u32(counts), ref)
    finally:
        c.set_eval_config(0, 0, 0, 0)


def test_eval_workload1_full_size(c):
    """Population-evaluation workload at its full size: n=1e5, F=20, K=3, 256 depth-3 trees."""
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(1)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], w["rank_bytes"])
    ranks, nu = oracle.encode(w["X"])
    np.testing.assert_array_equal(ranks_np(ds), ranks)
    a, th = datagen.random_population(nu, w["P"], w["depth"], _rng(w["pop_seed"]))
    counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), w["depth"])
    ref = oracle.eval_counts(ranks, w["y"], w["K"], a, th, w["depth"])
    np.testing.assert_array_equal(u32(counts), ref)


@pytest.mark.slow
def test_eval_workload3_full_size_sampled(c):
    """Large-scale workload at full size (n=1e7, 1024 depth-4 trees): every tree on the
    GPU, a sample of trees recomputed one by one by the oracle."""
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(3)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], w["rank_bytes"])
    rng = _rng(33)
    nu = u32(ds.n_unique)
    a, th = datagen.random_population(nu, w["P"], w["depth"], rng, allow_nosplit=True)
    counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), w["depth"])
    counts = u32(counts)
    # invariants on every tree
    assert np.all(counts.sum(axis=(1, 2)) == w["X"].shape[0])
    ranks = ranks_np(ds)
    pick = [0, 1, 511, 1023]
    ref = oracle.eval_counts(ranks, w["y"], w["K"], a[pick], th[pick], w["depth"])
    np.testing.assert_array_equal(counts[pick], ref)
    # and the ranks themselves against the oracle on a few features
    r_ref, nu_ref = oracle.encode(w["X"][:, :2])
    np.testing.assert_array_equal(ranks[:2], r_ref)


# --------------------------------------------------------------------------
# a2 + a5: decoding and the DE trajectory
# --------------------------------------------------------------------------

def test_decode_bit_exact(c):
    from paper_2311_06952_gb300 import deoct
    rng = _rng(5)
    X = np.round(rng.random((3000, 7)), 2).astype(np.float32)
    X[:, 6] = 1.0
    ds = gpu_dataset(c, X, np.zeros(3000, np.uint8), 2, 2)
    _, nu = oracle.encode(X)
    genes = datagen.random_genes(500, 3, 7, rng)
    genes[0] = np.nextafter(np.float32([8] * 7 + [1.0] * 7), np.float32(0))
    genes[1] = 0.0
    a, th = deoct.deoct_decode_population(c, ds, to_dev(genes), 3)
    a_ref, th_ref = oracle.decode(genes, 3, nu)
    np.testing.assert_array_equal(u16(a).astype(np.int32), a_ref)
    np.testing.assert_array_equal(u32(th), th_ref)


DE_CASES = [
    # (workload/n, depth, P, G, CR, dither, subset, K override, seed, stream)
    ("w0", 2, 64, 100, 0.9, False, False, 0, 0),
    ("w0", 3, 32, 25, 0.1, True, False, 7, 5),
    ("w0", 2, 16, 30, 0.5, False, True, 3, 9),
    ("rand_k3", 3, 24, 20, 0.9, False, False, 11, 1),
    ("w0", 2, 200, 8, 0.9, False, False, 2, 4),        # 4 threads per individual in the step
    ("rand_k3", 3, 300, 5, 0.5, True, False, 13, 6),   # 2 threads per individual
]
# alpha and n_min of the fitness (Section 3.2): 0 / 1 above; a positive alpha, a negative one
# (the step then orders fitness as doubles, not as bit patterns) and n_min > 1
ALPHA_CASES = [(0.75, 1), (-0.25, 1), (0.0, 40), (0.5, 25)]


@pytest.mark.parametrize("alpha,n_min", ALPHA_CASES)
def test_de_trajectory_alpha_nmin_bit_exact(c, alpha, n_min):
    from paper_2311_06952_gb300 import deoct
    rng = _rng(88)
    X = np.round(rng.random((3000, 5)), 2).astype(np.float32)
    y = datagen.flip_labels(datagen.planted_tree_labels(X, 3, 3, rng), 3, 0.2, rng)
    ds = gpu_dataset(c, X, y, 3, 2)
    ranks, nu = oracle.encode(X)
    P, G, depth = 40, 12, 3
    ref = oracle.de_run(ranks, nu, y, 3, depth=depth, P=P, G=G, alpha=alpha, n_min=n_min, seed=3,
                        history=True)
    prm = deoct.make_params(depth, P, G, alpha=alpha, n_min=n_min, seed=3)
    pop, fit, best = deoct.deoct_de_init(c, ds, prm)
    np.testing.assert_array_equal(fit.cpu().numpy(), ref["fit_hist"][0])
    for g in range(1, G + 1):
        deoct.deoct_de_step(c, ds, prm, g, pop, fit, best)
        np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32), ref["pop_hist"][g].view(np.uint32))
        np.testing.assert_array_equal(fit.cpu().numpy(), ref["fit_hist"][g])
    assert int(best.cpu()[0]) == ref["best"]


def test_de_resumes_from_saved_state_bit_exact(c):
    """Checkpoint and resume of a DEOCT run through the C ABI: the state is the population,
    its fitness, the best index and the generation number (the draws are Philox counters
    keyed by seed, node and generation), so a run stopped after generation 5, saved to the
    host, and continued from generation 6 by a new context on a new dataset handle ends with
    the same population, fitness and best as the run that never stopped, and as the oracle."""
    import torch
    from paper_2311_06952_gb300 import deoct
    rng = _rng(91)
    X = np.round(rng.random((4000, 6)), 2).astype(np.float32)
    y = datagen.flip_labels(datagen.planted_tree_labels(X, 3, 4, rng), 4, 0.1, rng)
    P, G, depth, K = 48, 12, 3, 4
    prm = deoct.make_params(depth, P, G, cr=0.7, seed=11, flags=deoct.DEOCT_DITHER_M)
    c1 = deoct.Context(0)
    ds1 = gpu_dataset(c1, X, y, K, 2)
    pop, fit, best = deoct.deoct_de_init(c1, ds1, prm, stream_id=5)
    for g in range(1, G + 1):
        deoct.deoct_de_step(c1, ds1, prm, g, pop, fit, best, stream_id=5)
    straight = (pop.cpu().numpy().copy(), fit.cpu().numpy().copy(), int(best.cpu()[0]))
    pop, fit, best = deoct.deoct_de_init(c1, ds1, prm, stream_id=5)
    for g in range(1, 6):
        deoct.deoct_de_step(c1, ds1, prm, g, pop, fit, best, stream_id=5)
    saved = (pop.cpu().numpy().copy(), fit.cpu().numpy().copy(), best.cpu().numpy().copy())
    c1.close()
    c2 = deoct.Context(0)
    ds2 = gpu_dataset(c2, X, y, K, 2)
    pop = torch.from_numpy(saved[0]).cuda()
    fit = torch.from_numpy(saved[1]).cuda()
    best = torch.from_numpy(saved[2]).cuda()
    for g in range(6, G + 1):
        deoct.deoct_de_step(c2, ds2, prm, g, pop, fit, best, stream_id=5)
    np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32), straight[0].view(np.uint32))
    np.testing.assert_array_equal(fit.cpu().numpy(), straight[1])
    assert int(best.cpu()[0]) == straight[2]
    c2.close()
    ranks, nu = oracle.encode(X)
    ref = oracle.de_run(ranks, nu, y, K, depth=depth, P=P, G=G, CR=0.7, seed=11, stream=5, dither=True,
                        history=True)
    np.testing.assert_array_equal(straight[0].view(np.uint32), ref["pop_hist"][G].view(np.uint32))
    assert straight[2] == ref["best"]


@pytest.mark.parametrize("case", DE_CASES, ids=[str(x[:4]) for x in DE_CASES])
def test_de_trajectory_bit_exact(c, case):
    from paper_2311_06952_gb300 import deoct
    name, depth, P, G, CR, dither, subset, seed, stream = case
    if name == "w0":
        w = datagen.make_workload(0)
        X, y, K = w["X"], w["y"], w["K"]
    else:
        rng = _rng(77)
        X = np.round(rng.random((2500, 6)), 2).astype(np.float32)
        y = rng.integers(0, 3, 2500).astype(np.uint8)
        K = 3
    ds = gpu_dataset(c, X, y, K, 2)
    ranks, nu = oracle.encode(X)
    idx = None
    if subset:
        idx = np.sort(_rng(seed).choice(len(X), len(X) // 2, replace=False)).astype(np.int32)
    ref = oracle.de_run(ranks, nu, y, K, depth=depth, P=P, G=G, CR=CR, seed=seed, stream=stream,
                        dither=dither, idx=idx, history=True)
    flags = deoct.DEOCT_DITHER_M if dither else 0
    prm = deoct.make_params(depth, P, G, cr=CR, seed=seed, flags=flags)
    sidx = None if idx is None else to_dev(idx)
    pop, fit, best = deoct.deoct_de_init(c, ds, prm, stream_id=stream, sample_idx=sidx)
    np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32), ref["pop_hist"][0].view(np.uint32))
    np.testing.assert_array_equal(fit.cpu().numpy(), ref["fit_hist"][0])
    for g in range(1, G + 1):
        deoct.deoct_de_step(c, ds, prm, g, pop, fit, best, stream_id=stream, sample_idx=sidx)
        np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32),
                                      ref["pop_hist"][g].view(np.uint32), err_msg="generation %d" % g)
        np.testing.assert_array_equal(fit.cpu().numpy(), ref["fit_hist"][g])
    assert int(best.cpu()[0]) == ref["best"]


def test_fit_subtree_matches_oracle(c):
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(0)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], 2)
    ranks, nu = oracle.encode(w["X"])
    ref = oracle.de_run(ranks, nu, w["y"], w["K"], depth=2, P=64, G=100, seed=0)
    prm = deoct.make_params(2, 64, 100, seed=0)
    import torch
    pop = torch.empty((64, 6), dtype=torch.float32, device="cuda")
    a, th, f = deoct.deoct_fit_subtree(c, ds, prm, pop_out=pop)
    a_ref, th_ref = oracle.decode(ref["pop"][ref["best"]][None], 2, nu)
    np.testing.assert_array_equal(a.astype(np.int32), a_ref[0])
    np.testing.assert_array_equal(th, th_ref[0])
    assert f == ref["fit"][ref["best"]]
    np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32), ref["pop"].view(np.uint32))


def test_fit_subtree_with_seeds(c):
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(0, n=400)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], 4)
    ranks, nu = oracle.encode(w["X"])
    seeds = datagen.random_genes(5, 2, 8, _rng(3))
    ref = oracle.de_run(ranks, nu, w["y"], w["K"], depth=2, P=16, G=12, seed=2, seeds=seeds)
    prm = deoct.make_params(2, 16, 12, seed=2)
    a, th, f = deoct.deoct_fit_subtree(c, ds, prm, seeds=to_dev(seeds))
    assert f == ref["fit"][ref["best"]]


# Populations above 256 take the split steady-state step (selection and per-CTA argmin, then
# the best and the trials, over CTAs of 32 individuals).  Fits of fewer than three generations
# issue its launches directly; longer ones replay them from the captured graph.
# (case, depth, P, G, alpha, n_min, CR, dither, subset, n_seeds, seed, stream)
WIDE_CASES = [
    ("ragged_direct", 3, 300, 2, 0.0, 1, 0.9, False, False, 0, 5, 0),   # last CTA: 12 individuals
    ("ragged_graph", 3, 300, 6, 0.5, 20, 0.7, True, True, 7, 6, 3),
    ("one_in_last", 2, 257, 5, 0.0, 1, 0.9, False, False, 0, 7, 1),    # last CTA: 1 individual
    ("neg_alpha", 4, 640, 4, -0.25, 1, 0.9, False, True, 0, 8, 2),     # doubles compared as values
    ("max_pop", 4, 4096, 3, 0.0, 1, 0.9, True, False, 0, 9, 0),        # 128 CTAs of candidates
]


@pytest.mark.parametrize("case", WIDE_CASES, ids=[x[0] for x in WIDE_CASES])
def test_fit_subtree_large_population_split_step_bit_exact(c, case):
    import torch
    from paper_2311_06952_gb300 import deoct
    name, depth, P, G, alpha, n_min, CR, dither, subset, n_seeds, seed, stream = case
    rng = _rng(300 + seed)
    n, F, K = 2500, 6, 3
    X = np.round(rng.random((n, F)), 2).astype(np.float32)
    y = datagen.flip_labels(datagen.planted_tree_labels(X, 3, K, rng), K, 0.1, rng)
    ds = gpu_dataset(c, X, y, K, 2)
    ranks, nu = oracle.encode(X)
    idx = np.sort(rng.choice(n, n // 2, replace=False)).astype(np.int32) if subset else None
    seeds = datagen.random_genes(n_seeds, depth, F, rng) if n_seeds else None
    ref = oracle.de_run(ranks, nu, y, K, depth=depth, P=P, G=G, CR=CR, alpha=alpha, n_min=n_min,
                        seed=seed, stream=stream, dither=dither, idx=idx, seeds=seeds)
    prm = deoct.make_params(depth, P, G, cr=CR, alpha=alpha, n_min=n_min, seed=seed,
                            flags=deoct.DEOCT_DITHER_M if dither else 0)
    pop = torch.empty((P, 2 * ((1 << depth) - 1)), dtype=torch.float32, device="cuda")
    a, th, f = deoct.deoct_fit_subtree(c, ds, prm, stream_id=stream, pop_out=pop,
                                       sample_idx=None if idx is None else to_dev(idx),
                                       seeds=None if seeds is None else to_dev(seeds))
    np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32), ref["pop"].view(np.uint32))
    assert f == ref["fit"][ref["best"]]
    a_ref, th_ref = oracle.decode(ref["pop"][ref["best"]][None], depth, nu)
    np.testing.assert_array_equal(a.astype(np.int32), a_ref[0])
    np.testing.assert_array_equal(th, th_ref[0])


def test_de_workload3_reduced_bit_exact(c):
    """Large-scale DE shape (F=10, K=2, depth 4, P=1024, uint16 ranks) on 60k samples, 3 generations."""
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(3, n=60_000)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], 2)
    ranks, nu = oracle.encode(w["X"])
    ref = oracle.de_run(ranks, nu, w["y"], w["K"], depth=4, P=1024, G=3, seed=0)
    prm = deoct.make_params(4, 1024, 3, seed=0)
    import torch
    pop = torch.empty((1024, 30), dtype=torch.float32, device="cuda")
    a, th, f = deoct.deoct_fit_subtree(c, ds, prm, pop_out=pop)
    np.testing.assert_array_equal(pop.cpu().numpy().view(np.uint32), ref["pop"].view(np.uint32))
    assert f == ref["fit"][ref["best"]]


def test_invalid_arguments_are_rejected(c):
    from paper_2311_06952_gb300 import deoct
    w = datagen.make_workload(0, n=100)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], 2)
    with pytest.raises(deoct.DeoctError) as e:
        deoct.deoct_fit_subtree(c, ds, deoct.make_params(2, 3, 5))  # P < 4
    assert e.value.code == deoct.DEOCT_ERR_INVALID
    with pytest.raises(deoct.DeoctError):
        deoct.deoct_fit_subtree(c, ds, deoct.make_params(11, 16, 5))  # depth > 10
    # a tree naming a feature > F is reported, not read out of bounds
    a = np.full((2, 3), 9, np.uint16)
    th = np.zeros((2, 3), np.uint32)
    deoct.deoct_eval_population(c, ds, to_dev(a), to_dev(th), 2)
    with pytest.raises(deoct.DeoctError):
        deoct.deoct_fit_subtree(c, ds, deoct.make_params(2, 16, 1))
    # and the context recovers
    deoct.deoct_fit_subtree(c, ds, deoct.make_params(2, 16, 1))


@pytest.mark.parametrize("rb,extra", [(4, 3), (2, 5), (4, 0)])
def test_eval_with_unaligned_row_stride(c, rb, extra):
    """A caller-chosen row stride that breaks 16-byte alignment takes the plain-load path."""
    import torch
    from paper_2311_06952_gb300 import deoct
    rng = _rng(500 + rb + extra)
    n, F, K, depth, P = 3001, 4, 3, 3, 30
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ld = n + extra
    dt = torch.int16 if rb == 2 else torch.int32
    ranks = torch.zeros((F, ld), dtype=dt, device="cuda")
    nu = torch.empty(F, dtype=torch.int32, device="cuda")
    deoct.deoct_encode(c, to_dev(X), rb, ranks_out=ranks, n_unique_out=nu)
    ds = deoct.DeviceDataset(ranks, rb, nu, to_dev(y), n, F, K)
    r_ref, nu_ref = oracle.encode(X)
    a, th = datagen.random_population(nu_ref, P, depth, rng, allow_nosplit=True)
    counts, _ = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth)
    np.testing.assert_array_equal(u32(counts), oracle.eval_counts(r_ref, y, K, a, th, depth))


@pytest.mark.parametrize("lab_off", [0, 1, 16])
def test_eval_is_one_launch_and_leaves_no_state(c, lab_off):
    """An evaluation of caller trees is one kernel launch: the trees are packed while the node
    tables are built, and the last CTA to finish writes errors and counts and zeroes its
    accumulator again.  Growing and shrinking shapes, both counting modes, errors-only calls,
    an invalid tree, and labels at any byte offset (bulk-copied when 16-byte aligned, else read
    with plain loads; n is not a multiple of 16) leave every next result exact."""
    import torch
    from paper_2311_06952_gb300 import deoct
    rng = _rng(777 + lab_off)
    n, F, K = 30001, 7, 3
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    base = gpu_dataset(c, X, y, K, 2)
    ybuf = torch.zeros(n + 32, dtype=torch.uint8, device="cuda")
    ybuf[lab_off:lab_off + n] = to_dev(y)
    ds = deoct.DeviceDataset(base.ranks, 2, base.n_unique, ybuf[lab_off:lab_off + n], n, F, K)
    for P, depth in [(37, 3), (300, 4), (9, 2), (300, 4), (5, 7)]:
        a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
        ref = oracle.eval_counts(ranks, y, K, a, th, depth)
        _, ref_err, _, _ = oracle.fitness(ref, a, n)
        c.reset_stats()
        counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth)
        assert c.stats()["launches"] == 1
        np.testing.assert_array_equal(u32(counts), ref)
        np.testing.assert_array_equal(u32(errors), ref_err)
        _, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth,
                                                want_counts=False)
        np.testing.assert_array_equal(u32(errors), ref_err)
    # an invalid tree is reported by the next sync call and leaves nothing behind
    bad = a.astype(np.uint16)
    bad[0, 0] = F + 2
    deoct.deoct_eval_population(c, ds, to_dev(bad), to_dev(th), depth)
    with pytest.raises(deoct.DeoctError):
        deoct.deoct_depth1_search(c, ds)
    counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth)
    np.testing.assert_array_equal(u32(counts), ref)
    np.testing.assert_array_equal(u32(errors), ref_err)


@pytest.mark.parametrize("depth,K", [(4, 2), (5, 2), (3, 5), (5, 3)])
@pytest.mark.parametrize("rb", [2, 4])
def test_eval_small_groups_streaming_bit_exact(c, depth, K, rb):
    """Groups of fewer than 16 trees run on the streaming kernel (a producer warp keeps a ring of
    landing zones filled; routing warps read the natural sample order).  P = 1, 2, 5, 15 on all
    samples and on a gathered subset; the default grid (about one tile per CTA here) and a grid
    of 7 CTAs that cycles each ring many times; 1, 2 and 3 bins per lane; two classes (whose
    masks take a shortcut when every label of a tile has landed) and more; a ragged tail."""
    from paper_2311_06952_gb300 import deoct
    rng = _rng(900 + 10 * depth + K + rb)
    n, F = 200_003, 7
    X = np.round(rng.random((n, F)), 4).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    ds = gpu_dataset(c, X, y, K, rb)
    idx = np.sort(rng.permutation(n)[: n // 3]).astype(np.int32)
    for P in (1, 2, 5, 15):
        a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
        ref = oracle.eval_counts(ranks, y, K, a, th, depth)
        ref_sub = oracle.eval_counts(ranks, y, K, a, th, depth, idx=idx)
        _, ref_err, _, _ = oracle.fitness(ref, a, n)
        for grid in (0, 7):
            try:
                c.set_eval_config(0, 0, 0, grid)
                counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)),
                                                             to_dev(th), depth)
                np.testing.assert_array_equal(u32(counts), ref)
                np.testing.assert_array_equal(u32(errors), ref_err)
                counts, _ = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th),
                                                        depth, sample_idx=to_dev(idx))
                np.testing.assert_array_equal(u32(counts), ref_sub)
            finally:
                c.set_eval_config(0, 0, 0, 0)


@pytest.mark.parametrize("depth,K", [(4, 4), (4, 8), (3, 8), (3, 16), (5, 2), (5, 4), (2, 32)])
@pytest.mark.parametrize("rb", [2, 4])
def test_eval_shared_class_bins_bit_exact(c, depth, K, rb):
    """Shapes whose bins fill whole lanes with K dividing 32 (2^D K = 32 Q, Q = 2 or 4): every
    bin of a lane has the same class and the bins differ only in their top leaf levels, so the
    evaluator ANDs the class mask and the deeper levels once per lane.  Both kernels (P = 1, 3
    and 6 stream, 24 is re-laid), both rank widths, a ragged tail."""
    from paper_2311_06952_gb300 import deoct
    rng = _rng(1300 + 10 * depth + K + rb)
    n, F = 30_011, 6
    X = np.round(rng.random((n, F)), 4).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    ds = gpu_dataset(c, X, y, K, rb)
    for P in (1, 3, 6, 24):
        a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
        ref = oracle.eval_counts(ranks, y, K, a, th, depth)
        _, ref_err, _, _ = oracle.fitness(ref, a, n)
        counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th),
                                                     depth)
        np.testing.assert_array_equal(u32(counts), ref)
        np.testing.assert_array_equal(u32(errors), ref_err)


def test_bounded_wait_timeout_is_reported_and_context_recovers(c):
    """Failure detection without a fault: a device wait on an mbarrier that nothing arrives on
    runs out after its bound, the next sync check reports DEOCT_ERR_TIMEOUT and clears the
    status word, and the context keeps evaluating correctly."""
    from paper_2311_06952_gb300 import deoct
    assert c.selftest_wait(2000) == deoct.DEOCT_ERR_TIMEOUT
    assert c.selftest_wait(1) == deoct.DEOCT_ERR_TIMEOUT
    rng = _rng(1234)
    n, F, K, depth, P = 5000, 5, 3, 3, 20
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ranks, nu = oracle.encode(X)
    ds = gpu_dataset(c, X, y, K, 2)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    counts, _ = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth)
    np.testing.assert_array_equal(u32(counts), oracle.eval_counts(ranks, y, K, a, th, depth))
    deoct.deoct_depth1_search(c, ds)  # a sync call: no status left behind


MAX_CASES = [
    # n, F, K, depth, P, rank_bytes -- each at one of the header's limits
    (3000, 256, 2, 3, 40, 4),      # F = 256 features, uint32 rows: the widest tile
    (3000, 256, 3, 2, 20, 2),      # F = 256, uint16 rows (re-laid tile)
    (5000, 4, 255, 2, 16, 2),      # K = 255 classes: shared-atomic mode, 1020 bins
    (5000, 4, 2, 10, 8, 4),        # depth 10: 1023 nodes, 2048 bins
    (2000, 3, 2, 3, 4096, 2),      # P = 4096 trees: 16 tree groups
]


@pytest.mark.parametrize("case", MAX_CASES, ids=[str(x) for x in MAX_CASES])
def test_eval_maximum_sizes_bit_exact(c, case):
    """The evaluator at the header's limits on F, K, depth and P matches the oracle."""
    from paper_2311_06952_gb300 import deoct
    n, F, K, depth, P, rb = case
    rng = _rng(1500 + F + K + depth + P)
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    ds = gpu_dataset(c, X, y, K, rb)
    ranks, nu = oracle.encode(X)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth)
    ref = oracle.eval_counts(ranks, y, K, a, th, depth)
    _, ref_err, _, _ = oracle.fitness(ref, a, n)
    np.testing.assert_array_equal(u32(counts), ref)
    np.testing.assert_array_equal(u32(errors), ref_err)


def test_encode_and_eval_at_max_samples(c):
    """n = 2^24 samples of one feature, all values distinct: ranks and thresholds reach the
    24-bit packing limit (theta up to 2^24 - 1)."""
    from paper_2311_06952_gb300 import deoct
    n = 1 << 24
    rng = _rng(1600)
    X = (rng.permutation(n).astype(np.float64) * 0.5 - 1000.0).astype(np.float32)[:, None]
    y = rng.integers(0, 2, n).astype(np.uint8)
    ds = gpu_dataset(c, X, y, 2, 4)
    ranks, nu = oracle.encode(X)
    assert int(nu[0]) == n
    np.testing.assert_array_equal(ranks_np(ds), ranks)
    a = np.ones((3, 3), np.int32)
    th = np.array([[n - 1, 5, n // 2], [0, n - 1, 1], [n // 3, n // 4, n - 2]], np.uint32)
    counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), 2)
    ref = oracle.eval_counts(ranks, y, 2, a, th, 2)
    _, ref_err, _, _ = oracle.fitness(ref, a, n)
    np.testing.assert_array_equal(u32(counts), ref)
    np.testing.assert_array_equal(u32(errors), ref_err)


def test_deoct_workload0_matches_golden_fixture(c):
    """The GPU DEOCT fit of the tiny workload reproduces the stored fixture of
    tests/golden/deoct_workload0.json (written from the oracle alone): the best tree, its
    fitness, and the final population bit for bit."""
    import hashlib
    import json
    import os
    import torch
    from paper_2311_06952_gb300 import deoct
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "deoct_workload0.json")) as f:
        gold = json.load(f)
    w = datagen.make_workload(0)
    ds = gpu_dataset(c, w["X"], w["y"], w["K"], 2)
    prm = deoct.make_params(w["depth"], w["P"], w["G"], mut_f=w["M"], cr=w["CR"], seed=w["seed"])
    B = (1 << w["depth"]) - 1
    pop = torch.empty((w["P"], 2 * B), dtype=torch.float32, device="cuda")
    a, th, fit = deoct.deoct_fit_subtree(c, ds, prm, stream_id=0, pop_out=pop)
    assert [int(x) for x in a] == gold["best_tree_a"]
    assert [int(x) for x in th] == gold["best_tree_theta"]
    assert fit == gold["best_fitness_per_generation"][-1]
    assert hashlib.sha256(pop.cpu().numpy().tobytes()).hexdigest() == gold["final_population_sha256"]


def _fuzz_case(seed):
    """A random evaluation shape: depth, classes (mostly ballot counting, 2^D K <= 128,
    sometimes shared atomics), population, rank width, data size and ties, an optional
    subset, and a forced launch shape kept within shared memory (or the automatic one)."""
    rng = _rng(9000 + seed)
    depth = int(rng.integers(1, 9))
    if depth <= 6 and rng.random() < 0.7:
        K = int(rng.integers(2, max(2, 128 >> depth) + 1))
    else:
        K = int(rng.integers(2, max(2, min(64, 4096 >> depth)) + 1))
    P = int(rng.choice([1, 2, 3, 5, 8, 13, 16, 17, 40, 64, 100, 129, 256, 300]))
    W = int(rng.choice([2, 4]))
    n = int(rng.integers(1, 30000))
    F = int(rng.integers(1, 13))
    levels = int(rng.choice([3, 50, 1000, 60000]))
    X = (np.floor(rng.random((n, F)) * levels) / levels).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    subset = bool(rng.integers(0, 2)) and n > 1
    shape = (0, 0, 0, 0)
    if rng.integers(0, 2):
        B, LK = (1 << depth) - 1, (1 << depth) * K
        tg_max = max(1, min(8192 // LK, 4096 // B))
        tg = int(rng.choice([0, 16, 32, 64, 256]))
        S = int(rng.choice([128, 256, 384, 640, 1024]))
        shape = (S, min(tg, tg_max), int(rng.choice([0, 4, 16, 32])), int(rng.choice([0, 3, 40])))
    return rng, depth, K, P, W, n, F, X, y, subset, shape


@pytest.mark.parametrize("seed", range(40))
def test_eval_random_shapes_bit_exact(c, seed):
    """Forty seeded random shapes through the one-launch evaluator (both kernels, both count
    modes, every bin map, forced and automatic launch shapes): counts and errors equal the
    oracle's."""
    from paper_2311_06952_gb300 import deoct
    rng, depth, K, P, W, n, F, X, y, subset, shape = _fuzz_case(seed)
    ranks, nu = oracle.encode(X)
    if W == 2 and int(nu.max()) > 65536:
        W = 4
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    idx = np.sort(rng.choice(n, max(1, n // 2), replace=False)).astype(np.int32) if subset else None
    ref = oracle.eval_counts(ranks, y, K, a, th, depth, idx=idx)
    _, ref_err, _, _ = oracle.fitness(ref, a, n if idx is None else len(idx))
    try:
        c.set_eval_config(*shape)
        ds = gpu_dataset(c, X, y, K, W)
        counts, errors = deoct.deoct_eval_population(c, ds, to_dev(a.astype(np.uint16)), to_dev(th), depth,
                                                     sample_idx=None if idx is None else to_dev(idx))
    finally:
        c.set_eval_config(0, 0, 0, 0)
    np.testing.assert_array_equal(u32(counts), ref, err_msg=str((depth, K, P, W, n, F, subset, shape)))
    np.testing.assert_array_equal(u32(errors), ref_err)
