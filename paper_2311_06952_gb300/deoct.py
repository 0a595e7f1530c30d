"""Thin ctypes binding of ``libdeoct.so`` (the C ABI of ``include/deoct.h``).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Functions keep the C names and take torch tensors (device
memory, caller-owned) or plain Python values; the stream is the current torch
CUDA stream unless one is passed.  If the library is missing or fails to load
this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libdeoct.so")

DEOCT_OK = 0
DEOCT_ERR_INVALID = -1
DEOCT_ERR_OOM = -2
DEOCT_ERR_CUDA = -3
DEOCT_ERR_TIMEOUT = -4
DEOCT_ERR_BUDGET = -5
DEOCT_DITHER_M = 0x1
DEOCT_BATCHED = 0x2
DEOCT_CART_SEEDS = 0x4
DEOCT_DE_SEEDS = 0x8

EXPORTED = [
    "deoct_create", "deoct_destroy", "deoct_last_error_string", "deoct_version",
    "deoct_set_timing", "deoct_get_stats", "deoct_reset_stats", "deoct_encode",
    "deoct_decode_population", "deoct_eval_population", "deoct_de_init", "deoct_de_step",
    "deoct_fit_subtree", "deoct_fit_moving_horizon", "deoct_depth1_search", "deoct_set_eval_config",
    "deoct_eval_population_noalloc", "deoct_encode_ex", "deoct_split_values", "deoct_predict",
    "deoct_selftest_wait", "deoct_encode_auto", "deoct_engine_create", "deoct_engine_destroy",
    "deoct_engine_attach", "deoct_engine_get_stats", "deoct_get_memory", "deoct_fit_scratch_bound",
    "deoct_release_scratch", "deoct_set_scratch_limit", "deoct_set_eval_streaming",
]
NOALLOC_SCRATCH_BYTES = 8 << 20


class DeoctError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("deoct error %d: %s" % (code, msg))
        self.code = code


class Dataset(ctypes.Structure):
    _fields_ = [("ranks", ctypes.c_void_p), ("rank_bytes", ctypes.c_int32), ("ld", ctypes.c_int64),
                ("n_unique", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("F", ctypes.c_int32), ("K", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("horizon", ctypes.c_int32), ("pop", ctypes.c_int32),
                ("gens", ctypes.c_int32), ("mut_f", ctypes.c_float), ("cr", ctypes.c_float),
                ("alpha", ctypes.c_double), ("n_min", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("eval_launches", ctypes.c_uint64),
                ("eval_ms", ctypes.c_double), ("eval_timed", ctypes.c_uint64)]


class EngineStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "submissions", "completed", "ticks", "launches", "eval_launches", "shared_launches",
        "max_jobs_per_launch", "max_problems_per_launch")]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64


def load(path: str | None = None):
    """Load libdeoct.so (build it first with ``paper_2311_06952_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise DeoctError(DEOCT_ERR_CUDA, "libdeoct.so not found at %s: run the build first" % p)
        lib = ctypes.CDLL(p)
        sig = {
            "deoct_create": [ctypes.POINTER(_vp), ctypes.c_int],
            "deoct_destroy": [_vp],
            "deoct_last_error_string": [],
            "deoct_version": [],
            "deoct_set_timing": [_vp, ctypes.c_int],
            "deoct_get_stats": [_vp, ctypes.POINTER(Stats)],
            "deoct_reset_stats": [_vp],
            "deoct_set_eval_config": [_vp, _i32, _i32, _i32, _i32],
            "deoct_selftest_wait": [_vp, _i32, _vp],
            "deoct_encode": [_vp, _vp, _i64, _i32, _i32, _vp, _i64, _vp, _vp],
            "deoct_encode_ex": [_vp, _vp, _i64, _i32, _i32, _vp, _i64, _vp, _vp, _vp],
            "deoct_encode_auto": [_vp, _vp, _i64, _i32, _vp, _i64, _vp, _vp, _vp, _vp],
            "deoct_get_memory": [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)],
            "deoct_release_scratch": [_vp],
            "deoct_set_eval_streaming": [_vp, _i32],
            "deoct_set_scratch_limit": [_vp, _u64],
            "deoct_fit_scratch_bound": [_vp, _i64, _i32, _i32, _i32, ctypes.POINTER(Params),
                                        ctypes.POINTER(_u64)],
            "deoct_engine_create": [ctypes.POINTER(_vp), _i32],
            "deoct_engine_destroy": [_vp],
            "deoct_engine_attach": [_vp, _vp],
            "deoct_engine_get_stats": [_vp, ctypes.POINTER(EngineStats)],
            "deoct_split_values": [_vp, _vp, _i64, _vp, _vp, _i32, _vp, _vp],
            "deoct_predict": [_vp, _vp, _i64, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp],
            "deoct_decode_population": [_vp, ctypes.POINTER(Dataset), _vp, _i32, _i32, _vp, _vp, _vp],
            "deoct_eval_population": [_vp, ctypes.POINTER(Dataset), _vp, _i64, _vp, _vp, _i32, _i32,
                                      _vp, _vp, _vp],
            "deoct_de_init": [_vp, ctypes.POINTER(Dataset), _vp, _i64, ctypes.POINTER(Params), _u64,
                              _vp, _i32, _vp, _vp, _vp, _vp],
            "deoct_de_step": [_vp, ctypes.POINTER(Dataset), _vp, _i64, ctypes.POINTER(Params), _u64,
                              _i32, _vp, _vp, _vp, _vp],
            "deoct_fit_subtree": [_vp, ctypes.POINTER(Dataset), _vp, _i64, ctypes.POINTER(Params), _u64,
                                  _vp, _i32, _vp, _vp, _vp, _vp, _vp],
            "deoct_fit_moving_horizon": [_vp, ctypes.POINTER(Dataset), ctypes.POINTER(Params), _vp, _vp,
                                         _vp, _vp, _vp, _vp],
            "deoct_depth1_search": [_vp, ctypes.POINTER(Dataset), _vp, _i64, _i32, ctypes.c_double,
                                    _vp, _vp, _vp, _vp],
            "deoct_eval_population_noalloc": [ctypes.POINTER(Dataset), _vp, _i64, _vp, _vp, _i32, _i32,
                                              _vp, _vp, _vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name in ("deoct_last_error_string", "deoct_version") \
                else ctypes.c_int
        _lib = lib
        return lib


class Engine:
    """Owns a ``deoct_engine``: continuous batching of the DEOCT generations of every
    attached context's batched moving-horizon level solves in shared launches."""

    def __init__(self, device: int = 0):
        h = _vp()
        _check(load().deoct_engine_create(ctypes.byref(h), device))
        self.handle = h
        self.device = device

    def stats(self):
        s = EngineStats()
        _check(load().deoct_engine_get_stats(self.handle, ctypes.byref(s)))
        return {k: int(getattr(s, k)) for k, _ in EngineStats._fields_}

    def close(self):
        if self.handle is not None:
            load().deoct_engine_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check(rc):
    if rc != DEOCT_OK:
        msg = load().deoct_last_error_string()
        raise DeoctError(rc, msg.decode() if msg else "")


def _ptr(t, itemsize=None):
    """Address of a host numpy array or a device tensor (checked: CUDA, contiguous,
    element size as the C ABI expects)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("host array must be C-contiguous")
        return t.ctypes.data_as(_vp)
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device (got %s)" % t.device)
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if itemsize is not None and t.element_size() != itemsize:
        raise ValueError("tensor element size %d, expected %d" % (t.element_size(), itemsize))
    return _vp(t.data_ptr())


_EMPTY_IDX = {}


def _idx_ptr(sample_idx):
    """Address of a sample index tensor.  An empty index (the empty subset) still needs a
    non-NULL pointer -- NULL means "all samples" in the C ABI -- but torch reports address 0
    for tensors without elements, so a one-element placeholder on the same device stands in
    (never read: the library reads no index when n_sub = 0)."""
    if sample_idx is None or sample_idx.numel() > 0:
        return _ptr(sample_idx, 4)
    import torch
    dev = sample_idx.device
    if dev not in _EMPTY_IDX:
        _EMPTY_IDX[dev] = torch.zeros(4, dtype=torch.int32, device=dev)
    return _ptr(_EMPTY_IDX[dev], 4)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream)


def version():
    return load().deoct_version().decode()


class Context:
    """Owns a ``deoct_ctx`` (device scratch, counters) on one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load()
        h = _vp()
        _check(lib.deoct_create(ctypes.byref(h), device))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle is not None:
            load().deoct_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_timing(self, enable: bool):
        _check(load().deoct_set_timing(self.handle, int(bool(enable))))

    def memory(self):
        """(device bytes, pinned host bytes) this context holds."""
        d, h = _u64(), _u64()
        _check(load().deoct_get_memory(self.handle, ctypes.byref(d), ctypes.byref(h)))
        return int(d.value), int(h.value)

    def release_scratch(self):
        """Free the context's device scratch (synchronises the device)."""
        _check(load().deoct_release_scratch(self.handle))

    def set_scratch_limit(self, nbytes: int):
        """Cap the device scratch the context may hold (0: no cap); growth past it is DEOCT_ERR_OOM."""
        _check(load().deoct_set_scratch_limit(self.handle, int(nbytes)))

    def attach_engine(self, engine):
        """Run this context's batched level solves in `engine`'s shared launches (None detaches)."""
        _check(load().deoct_engine_attach(self.handle, None if engine is None else engine.handle))
        self.engine = engine

    def stats(self):
        s = Stats()
        _check(load().deoct_get_stats(self.handle, ctypes.byref(s)))
        return dict(launches=s.launches, eval_launches=s.eval_launches, eval_ms=s.eval_ms,
                    eval_timed=s.eval_timed)

    def reset_stats(self):
        _check(load().deoct_reset_stats(self.handle))

    def selftest_wait(self, tries=1000, stream=None):
        """One warp waits on an mbarrier nothing arrives on, for `tries` tries of up
        to ~1 us; returns the status code the sync check reports (DEOCT_ERR_TIMEOUT
        when bounded waits work) and leaves the context usable."""
        return int(load().deoct_selftest_wait(self.handle, int(tries), _stream(stream)))

    def set_eval_config(self, S=0, TG=0, warps=0, grid=0):
        """Force the evaluator's launch shape (0 = automatic); results are unchanged."""
        _check(load().deoct_set_eval_config(self.handle, S, TG, warps, grid))

    def set_eval_streaming(self, on: bool):
        """Run every ballot-mode evaluation on the streaming kernel (results unchanged)."""
        _check(load().deoct_set_eval_streaming(self.handle, int(bool(on))))


class DeviceDataset:
    """A rank-encoded training set resident on the device (tensors kept alive here)."""

    def __init__(self, ranks, rank_bytes, n_unique, labels, n, F, K, ld=None):
        _ptr(ranks, rank_bytes)
        _ptr(n_unique, 4)
        _ptr(labels, 1)
        if ranks.dim() != 2 or ranks.shape[0] != F or ranks.shape[1] < n or labels.numel() < n:
            raise ValueError("ranks must be [F][ld >= n] and labels [n]")
        self.ranks, self.n_unique, self.labels = ranks, n_unique, labels
        self.rank_bytes, self.n, self.F, self.K = rank_bytes, n, F, K
        self.ld = ranks.shape[1] if ld is None else ld
        self.c = Dataset(ranks.data_ptr(), rank_bytes, self.ld, n_unique.data_ptr(), labels.data_ptr(),
                         n, F, K)


def padded_ld(n: int, rank_bytes: int) -> int:
    """Row stride that keeps every rank row 16-byte aligned (TMA staging)."""
    q = 16 // rank_bytes
    return (n + q - 1) // q * q


def deoct_encode(ctx: Context, X, rank_bytes: int, ranks_out=None, n_unique_out=None, stream=None):
    """a1: X [n][F] float32 (device) -> (ranks [F][ld], n_unique [F]); sync."""
    import torch
    n, F = X.shape
    dt = torch.int16 if rank_bytes == 2 else torch.int32
    if ranks_out is None:
        ranks_out = torch.empty((F, padded_ld(n, rank_bytes)), dtype=dt, device=X.device)
    if n_unique_out is None:
        n_unique_out = torch.empty(F, dtype=torch.int32, device=X.device)
    _check(load().deoct_encode(ctx.handle, _ptr(X, 4), n, F, rank_bytes, _ptr(ranks_out, rank_bytes),
                               ranks_out.shape[1], _ptr(n_unique_out, 4), _stream(stream)))
    return ranks_out, n_unique_out


def deoct_encode_ex(ctx: Context, X, rank_bytes: int, stream=None):
    """a1 plus the sorted distinct values: (ranks [F][ld], n_unique [F], unique [F][ld] float32)."""
    import torch
    n, F = X.shape
    dt = torch.int16 if rank_bytes == 2 else torch.int32
    ld = padded_ld(n, rank_bytes)
    ranks = torch.empty((F, ld), dtype=dt, device=X.device)
    nu = torch.empty(F, dtype=torch.int32, device=X.device)
    uniq = torch.empty((F, ld), dtype=torch.float32, device=X.device)
    _check(load().deoct_encode_ex(ctx.handle, _ptr(X), n, F, rank_bytes, _ptr(ranks), ld, _ptr(nu),
                                  _ptr(uniq), _stream(stream)))
    return ranks, nu, uniq


def deoct_encode_auto(ctx: Context, X, want_unique=True, stream=None):
    """a1 with the rank width chosen from n_p (uint16 when every n_p <= 65536):
    (ranks [F][ld], n_unique [F], unique [F][ld] float32 or None, rank_bytes); sync."""
    import torch
    n, F = X.shape
    ld = (n + 7) // 8 * 8
    buf = torch.empty(F * ld, dtype=torch.int32, device=X.device)
    nu = torch.empty(F, dtype=torch.int32, device=X.device)
    uniq = torch.empty((F, ld), dtype=torch.float32, device=X.device) if want_unique else None
    w = ctypes.c_int32()
    _check(load().deoct_encode_auto(ctx.handle, _ptr(X, 4), n, F, _ptr(buf), ld, _ptr(nu, 4),
                                    _ptr(uniq), ctypes.byref(w), _stream(stream)))
    if w.value == 2:
        # the rows were written as uint16 [F][ld] into the first half: keep only those bytes
        ranks = buf.view(torch.int16)[: F * ld].view(F, ld).clone()
    else:
        ranks = buf.view(F, ld)
    return ranks, nu, uniq, w.value


def deoct_split_values(ctx: Context, unique, a, theta, stream=None):
    """Raw-unit thresholds b [B] (float64, device) of a fitted tree (a, theta: device [B])."""
    import torch
    B = a.numel()
    b = torch.empty(B, dtype=torch.float64, device=unique.device)
    _check(load().deoct_split_values(ctx.handle, _ptr(unique), unique.shape[1], _ptr(a), _ptr(theta), B,
                                     _ptr(b), _stream(stream)))
    return b


def deoct_predict(ctx: Context, X, a, b, depth: int, leaf_class, y=None, stream=None):
    """Leaf class of every row of X [m][F] (device); with labels, also the count of correct ones."""
    import torch
    m, F = X.shape
    pred = torch.empty(m, dtype=torch.uint8, device=X.device)
    correct = torch.zeros(1, dtype=torch.int64, device=X.device) if y is not None else None
    _check(load().deoct_predict(ctx.handle, _ptr(X), m, F, _ptr(a), _ptr(b), depth, _ptr(leaf_class),
                                _ptr(y), _ptr(pred), _ptr(correct), _stream(stream)))
    return pred, correct


def encode_dataset(ctx: Context, X, y, K: int, rank_bytes: int, stream=None) -> DeviceDataset:
    """Encode X and bundle it with the labels; rank_bytes 0 picks the width from n_p."""
    if rank_bytes == 0:
        ranks, nu, _, rank_bytes = deoct_encode_auto(ctx, X, want_unique=False, stream=stream)
    else:
        ranks, nu = deoct_encode(ctx, X, rank_bytes, stream=stream)
    return DeviceDataset(ranks, rank_bytes, nu, y, X.shape[0], X.shape[1], K)


def deoct_decode_population(ctx: Context, ds: DeviceDataset, genes, depth: int, a_out=None,
                            theta_out=None, stream=None):
    import torch
    P = genes.shape[0]
    B = (1 << depth) - 1
    if a_out is None:
        a_out = torch.empty((P, B), dtype=torch.int16, device=genes.device)
    if theta_out is None:
        theta_out = torch.empty((P, B), dtype=torch.int32, device=genes.device)
    _check(load().deoct_decode_population(ctx.handle, ctypes.byref(ds.c), _ptr(genes), P, depth,
                                          _ptr(a_out), _ptr(theta_out), _stream(stream)))
    return a_out, theta_out


def deoct_eval_population(ctx: Context, ds: DeviceDataset, a, theta, depth: int, sample_idx=None,
                          counts_out=None, errors_out=None, want_counts=True, stream=None):
    import torch
    P = a.shape[0]
    L = 1 << depth
    if counts_out is None and want_counts:
        counts_out = torch.empty((P, L, ds.K), dtype=torch.int32, device=a.device)
    if errors_out is None:
        errors_out = torch.empty(P, dtype=torch.int32, device=a.device)
    n_sub = ds.n if sample_idx is None else sample_idx.numel()
    _check(load().deoct_eval_population(ctx.handle, ctypes.byref(ds.c), _idx_ptr(sample_idx), n_sub,
                                        _ptr(a, 2), _ptr(theta, 4), P, depth, _ptr(counts_out, 4),
                                        _ptr(errors_out, 4), _stream(stream)))
    return counts_out, errors_out


def fit_scratch_bound(n: int, F: int, K: int, params, rank_bytes: int = 0, ctx=None) -> int:
    """Upper bound of the device scratch a fresh context holds after encoding an n x F set
    and fitting it with deoct_fit_moving_horizon under `params`; with `ctx`, of what that
    context's scratch may still grow by (no GPU call)."""
    b = _u64()
    _check(load().deoct_fit_scratch_bound(None if ctx is None else ctx.handle, n, F, K, rank_bytes,
                                          ctypes.byref(params), ctypes.byref(b)))
    return int(b.value)


def make_params(depth, pop, gens, mut_f=0.5, cr=0.9, alpha=0.0, n_min=1, seed=0, horizon=0, flags=0):
    return Params(depth, horizon, pop, gens, mut_f, cr, alpha, n_min, flags, seed)


def deoct_de_init(ctx: Context, ds: DeviceDataset, params: Params, stream_id=0, seeds=None,
                  sample_idx=None, pop=None, fitness=None, best=None, stream=None):
    import torch
    P = params.pop
    B = (1 << params.depth) - 1
    dev = ds.ranks.device
    if pop is None:
        pop = torch.empty((P, 2 * B), dtype=torch.float32, device=dev)
    if fitness is None:
        fitness = torch.empty(P, dtype=torch.float64, device=dev)
    if best is None:
        best = torch.empty(1, dtype=torch.int32, device=dev)
    S = 0 if seeds is None else seeds.shape[0]
    n_sub = ds.n if sample_idx is None else sample_idx.numel()
    _check(load().deoct_de_init(ctx.handle, ctypes.byref(ds.c), _idx_ptr(sample_idx), n_sub,
                                ctypes.byref(params), stream_id, _ptr(seeds, 4), S, _ptr(pop, 4),
                                _ptr(fitness, 8), _ptr(best, 4), _stream(stream)))
    return pop, fitness, best


def deoct_de_step(ctx: Context, ds: DeviceDataset, params: Params, generation: int, pop, fitness,
                  best, stream_id=0, sample_idx=None, stream=None):
    n_sub = ds.n if sample_idx is None else sample_idx.numel()
    _check(load().deoct_de_step(ctx.handle, ctypes.byref(ds.c), _idx_ptr(sample_idx), n_sub,
                                ctypes.byref(params), stream_id, generation, _ptr(pop, 4), _ptr(fitness, 8),
                                _ptr(best, 4), _stream(stream)))
    return pop, fitness, best


def deoct_fit_subtree(ctx: Context, ds: DeviceDataset, params: Params, stream_id=0, seeds=None,
                      sample_idx=None, pop_out=None, stream=None):
    """DEOCT on one (sub)problem; returns (a [B] uint16, theta [B] uint32, fitness) on the host."""
    B = (1 << params.depth) - 1
    a = np.zeros(B, np.uint16)
    th = np.zeros(B, np.uint32)
    fit = ctypes.c_double()
    S = 0 if seeds is None else seeds.shape[0]
    n_sub = ds.n if sample_idx is None else sample_idx.numel()
    _check(load().deoct_fit_subtree(ctx.handle, ctypes.byref(ds.c), _idx_ptr(sample_idx), n_sub,
                                    ctypes.byref(params), stream_id, _ptr(seeds), S, _ptr(a), _ptr(th),
                                    ctypes.byref(fit), _ptr(pop_out), _stream(stream)))
    return a, th, fit.value


def deoct_fit_moving_horizon(ctx: Context, ds: DeviceDataset, params: Params, stream=None):
    """Algorithm 2; returns dict(a, theta, leaf_class, kind, node_fit) of host arrays."""
    D = params.depth
    B = (1 << D) - 1
    a = np.zeros(B, np.uint16)
    th = np.zeros(B, np.uint32)
    lc = np.zeros(1 << D, np.uint8)
    kind = np.zeros(B, np.int32)
    nf = np.zeros(B, np.float64)
    _check(load().deoct_fit_moving_horizon(ctx.handle, ctypes.byref(ds.c), ctypes.byref(params),
                                           _ptr(a), _ptr(th), _ptr(lc), _ptr(kind), _ptr(nf),
                                           _stream(stream)))
    return dict(a=a, theta=th, leaf_class=lc, kind=kind, node_fit=nf)


def deoct_depth1_search(ctx: Context, ds: DeviceDataset, sample_idx=None, n_min=1, alpha=0.0,
                        stream=None):
    a = ctypes.c_uint16()
    th = ctypes.c_uint32()
    f = ctypes.c_double()
    n_sub = ds.n if sample_idx is None else sample_idx.numel()
    _check(load().deoct_depth1_search(ctx.handle, ctypes.byref(ds.c), _idx_ptr(sample_idx), n_sub, n_min,
                                      alpha, ctypes.byref(a), ctypes.byref(th), ctypes.byref(f),
                                      _stream(stream)))
    return a.value, th.value, f.value


def deoct_eval_population_noalloc(ds: DeviceDataset, a, theta, depth: int, counts_out, errors_out,
                                  sample_idx=None, stream=None):
    """The evaluator without any device allocation (no context; fixed library
    scratch).  The caller passes every output buffer; counts_out may be None, in
    which case the counts stay in the library's scratch.  Runs on the current
    device; calls whose GPU work overlaps must be serialised by the caller."""
    P = a.shape[0]
    n_sub = ds.n if sample_idx is None else sample_idx.numel()
    _check(load().deoct_eval_population_noalloc(ctypes.byref(ds.c), _idx_ptr(sample_idx), n_sub, _ptr(a),
                                                _ptr(theta), P, depth, _ptr(counts_out), _ptr(errors_out),
                                                _stream(stream)))
    return counts_out, errors_out
