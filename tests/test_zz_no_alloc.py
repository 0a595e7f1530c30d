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
