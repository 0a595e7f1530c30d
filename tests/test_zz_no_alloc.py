"""deoct_eval_population_noalloc: the evaluator for callers that cannot allocate
device memory (a framework that owns all device memory, or code that must not
take cudaMalloc's device synchronisation).  Its output must equal the
allocating entry point's, call after call, although both calls share the one
fixed scratch array inside the library.

This file is collected last on purpose, so a failure here comes after every
other test has run."""
import numpy as np
import pytest

from paper_2311_06952_gb300 import datagen

from gpu_helpers import ctx, gpu_dataset, to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2311_06952_gb300 import build
    build.build()
    return ctx()


def _case(seed, n, F, K, depth, P, rb):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.round(rng.random((n, F)), 3).astype(np.float32)
    y = rng.integers(0, K, n).astype(np.uint8)
    return X, y, K, depth, P, rb, rng


def test_noalloc_matches_allocating_evaluator_on_two_calls(c):
    import torch
    from paper_2311_06952_gb300 import deoct
    for call, (seed, n, F, K, depth, P, rb) in enumerate([(1, 20000, 6, 3, 3, 200, 2),
                                                         (2, 7001, 9, 2, 4, 90, 4)]):
        X, y, K, depth, P, rb, rng = _case(seed, n, F, K, depth, P, rb)
        ds = gpu_dataset(c, X, y, K, rb)
        nu = u32(ds.n_unique)
        a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
        ad, td = to_dev(a.astype(np.uint16)), to_dev(th)
        ref_counts, ref_err = deoct.deoct_eval_population(c, ds, ad, td, depth)
        L = 1 << depth
        counts = torch.full((P, L, K), -1, dtype=torch.int32, device="cuda")
        errors = torch.full((P,), -1, dtype=torch.int32, device="cuda")
        deoct.deoct_eval_population_noalloc(ds, ad, td, depth, counts, errors)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(u32(counts), u32(ref_counts), err_msg="call %d" % call)
        np.testing.assert_array_equal(u32(errors), u32(ref_err), err_msg="call %d" % call)
        # counts kept in the library's scratch: only the error counts come back
        errors2 = torch.full((P,), -1, dtype=torch.int32, device="cuda")
        deoct.deoct_eval_population_noalloc(ds, ad, td, depth, None, errors2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(u32(errors2), u32(ref_err), err_msg="call %d (scratch counts)" % call)


@pytest.mark.parametrize("seed,n,F,K,depth,P,rb,subset", [
    (4, 30001, 7, 4, 3, 8, 2, False),     # fewer than 16 trees: the streaming kernel
    (5, 30001, 7, 4, 3, 8, 4, True),      # streaming kernel on a gathered subset
    (6, 23456, 5, 3, 4, 150, 2, True),    # re-laid kernel on a gathered subset
    (7, 5001, 3, 2, 2, 40, 4, "empty"),   # empty subset: zero counts, zero errors
])
def test_noalloc_matches_allocating_evaluator_on_subsets_and_small_populations(c, seed, n, F, K, depth,
                                                                               P, rb, subset):
    import torch
    from paper_2311_06952_gb300 import deoct
    X, y, K, depth, P, rb, rng = _case(seed, n, F, K, depth, P, rb)
    ds = gpu_dataset(c, X, y, K, rb)
    nu = u32(ds.n_unique)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    ad, td = to_dev(a.astype(np.uint16)), to_dev(th)
    idx = None
    if subset == "empty":
        idx = torch.empty(0, dtype=torch.int32, device="cuda")
    elif subset:
        idx = to_dev(np.sort(rng.choice(n, n // 3, replace=False)).astype(np.int32))
    ref_counts, ref_err = deoct.deoct_eval_population(c, ds, ad, td, depth, sample_idx=idx)
    L = 1 << depth
    for call in range(2):
        counts = torch.full((P, L, K), -1, dtype=torch.int32, device="cuda")
        errors = torch.full((P,), -1, dtype=torch.int32, device="cuda")
        deoct.deoct_eval_population_noalloc(ds, ad, td, depth, counts, errors, sample_idx=idx)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(u32(counts), u32(ref_counts), err_msg="call %d" % call)
        np.testing.assert_array_equal(u32(errors), u32(ref_err), err_msg="call %d" % call)
    if subset == "empty":
        assert not u32(ref_counts).any() and not u32(ref_err).any()


def test_noalloc_reports_device_errors_in_errors_out(c):
    """A sample index out of range or a tree naming a feature > F cannot be returned by a
    later sync call (there is no context): every error count of that call becomes 0xFFFFFFFF.
    The next valid call is unaffected (it clears the status word)."""
    import torch
    from paper_2311_06952_gb300 import deoct
    X, y, K, depth, P, rb, rng = _case(8, 9000, 4, 3, 3, 64, 2)
    ds = gpu_dataset(c, X, y, K, rb)
    nu = u32(ds.n_unique)
    a, th = datagen.random_population(nu, P, depth, rng, allow_nosplit=True)
    ad, td = to_dev(a.astype(np.uint16)), to_dev(th)
    ref_counts, ref_err = deoct.deoct_eval_population(c, ds, ad, td, depth)
    errors = torch.zeros((P,), dtype=torch.int32, device="cuda")
    bad_idx = np.arange(0, 9000, 3, dtype=np.int32)
    bad_idx[17] = 9000  # one past the last sample
    deoct.deoct_eval_population_noalloc(ds, ad, td, depth, None, errors, sample_idx=to_dev(bad_idx))
    torch.cuda.synchronize()
    assert np.all(u32(errors) == 0xFFFFFFFF)
    bad_a = a.copy()
    bad_a[5, 0] = 4 + 1  # feature index past F = 4
    errors.zero_()
    deoct.deoct_eval_population_noalloc(ds, to_dev(bad_a.astype(np.uint16)), td, depth, None, errors)
    torch.cuda.synchronize()
    assert np.all(u32(errors) == 0xFFFFFFFF)
    counts = torch.zeros_like(ref_counts)
    deoct.deoct_eval_population_noalloc(ds, ad, td, depth, counts, errors)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(u32(errors), u32(ref_err))
    np.testing.assert_array_equal(u32(counts), u32(ref_counts))


def test_noalloc_rejects_requests_beyond_its_scratch(c):
    from paper_2311_06952_gb300 import deoct
    X, y, K, depth, P, rb, rng = _case(3, 500, 4, 2, 10, 2100, 2)
    ds = gpu_dataset(c, X, y, K, rb)
    a = np.zeros((P, (1 << depth) - 1), np.uint16)
    th = np.zeros_like(a, dtype=np.uint32)
    with pytest.raises(deoct.DeoctError) as e:
        deoct.deoct_eval_population_noalloc(ds, to_dev(a), to_dev(th), depth, None, None)
    assert e.value.code == deoct.DEOCT_ERR_INVALID
    assert "scratch" in str(e.value)
    # more trees than the allocating evaluator takes, though they would fit the scratch
    d1 = 1
    P1 = 4096 * 64 + 1
    a1 = np.zeros((P1, 1), np.uint16)
    with pytest.raises(deoct.DeoctError) as e:
        deoct.deoct_eval_population_noalloc(ds, to_dev(a1), to_dev(a1.astype(np.uint32)), d1,
                                            to_dev(np.zeros((P1, 2, K), np.uint32)), None)
    assert e.value.code == deoct.DEOCT_ERR_INVALID and "out of range" in str(e.value)
