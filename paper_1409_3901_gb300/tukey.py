"""Thin ctypes binding of libtukeydepth.so (include/tukey_depth.h).

Argument marshalling only: every step of the depth computation runs in the
library's CUDA kernels.  The functions keep the C names (td_create, td_depth,
td_depth_batched, td_stream_*) and a small ``Context`` class wraps them for
numpy arrays (host pointers) and torch CUDA tensors (device pointers).

Importing this module loads the library and raises ``LibraryMissing`` if it
has not been built (``python -m paper_1409_3901_gb300.build``); there is no
fallback of any kind.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtukeydepth.so")

TD_OK = 0
TD_ERR_INVALID = -1
TD_ERR_RANGE = -2
TD_ERR_OOM = -3
TD_ERR_BUSY = -4
TD_ERR_TIMEOUT = -5
TD_ERR_CUDA = -6
TD_ERR_NOTFOUND = -7
TD_ERR_INTERNAL = -8
TD_MAX_P = 6
TD_ALG_RCOM, TD_ALG_ADIA, TD_ALG_CRITICAL = 0, 1, 2
TD_MAX_N = 2048
TD_MODE_FILTERED = 0
TD_MODE_PLAIN_EXACT = 1


class LibraryMissing(ImportError):
    pass


class TdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d)" % (msg, code))
        self.code = code


class td_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("device_pointers", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("subsets_per_warp", ctypes.c_int32),
                ("buckets_log2", ctypes.c_int32), ("early_exit", ctypes.c_int32),
                ("algorithm", ctypes.c_int32), ("unseeded", ctypes.c_int32),
                ("shard_index", ctypes.c_int64), ("shard_count", ctypes.c_int64),
                ("stream", ctypes.c_void_p)]


class td_dataset(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("p", ctypes.c_int32), ("X", ctypes.c_void_p),
                ("m", ctypes.c_int32), ("Z", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class td_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_uint64), ("skipped_dependent", ctypes.c_uint64),
                ("filtered_points", ctypes.c_uint64), ("exact_points", ctypes.c_uint64),
                ("tight_exceptions", ctypes.c_uint64), ("resolved_buckets", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("ms", ctypes.c_float),
                ("ms_sweep", ctypes.c_float), ("early_skipped", ctypes.c_uint64),
                ("adia_pops", ctypes.c_uint64), ("adia_subsets", ctypes.c_uint64),
                ("adia_union_points", ctypes.c_uint64), ("adia_fallbacks", ctypes.c_uint64),
                ("rescanned_sweeps", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TD_TUNE_MAX = 8


class td_tune_result(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("n", ctypes.c_int32), ("queries", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("spw", ctypes.c_int32 * TD_TUNE_MAX),
                ("ms", ctypes.c_float * TD_TUNE_MAX), ("ms_default", ctypes.c_float),
                ("best_spw", ctypes.c_int32), ("best_ms", ctypes.c_float)]

    def as_dict(self):
        k = self.candidates
        return {"p": self.p, "n": self.n, "queries": self.queries,
                "candidates": {int(self.spw[i]): float(self.ms[i]) for i in range(k)},
                "ms_default": self.ms_default, "best_spw": self.best_spw, "best_ms": self.best_ms}


def _load():
    if not os.path.exists(LIB_PATH):
        raise LibraryMissing("libtukeydepth.so is not built: run `python -m paper_1409_3901_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "td_coord_limit": (i64, [i32]),
        "td_create": (ctypes.c_int, [P(vp), ctypes.c_int, P(td_options)]),
        "td_set_options": (ctypes.c_int, [vp, P(td_options)]),
        "td_destroy": (ctypes.c_int, [vp]),
        "td_depth": (ctypes.c_int, [vp, vp, i32, i32, vp, i32, vp, P(td_stats)]),
        "td_depth_batched": (ctypes.c_int, [vp, P(td_dataset), i32, P(td_stats)]),
        "td_stream_create": (ctypes.c_int, [vp, ctypes.c_size_t, P(vp)]),
        "td_stream_submit": (ctypes.c_int, [vp, P(td_dataset), P(ctypes.c_uint64)]),
        "td_stream_poll": (ctypes.c_int, [vp, ctypes.c_uint64, P(ctypes.c_int)]),
        "td_stream_wait": (ctypes.c_int, [vp, ctypes.c_uint64, i64]),
        "td_stream_destroy": (ctypes.c_int, [vp]),
        "td_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "td_last_cuda_error": (ctypes.c_char_p, [vp]),
        "td_depth_noalloc": (ctypes.c_int, [vp, i32, i32, vp, i32, vp, vp]),
        "td_autotune": (ctypes.c_int, [vp, i32, i32, P(td_tune_result)]),
        "td_set_tuned": (ctypes.c_int, [vp, i32, i32, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()

# the C entry points under their own names
td_coord_limit = lib.td_coord_limit
td_create = lib.td_create
td_set_options = lib.td_set_options
td_destroy = lib.td_destroy
td_depth = lib.td_depth
td_depth_batched = lib.td_depth_batched
td_stream_create = lib.td_stream_create
td_stream_submit = lib.td_stream_submit
td_stream_poll = lib.td_stream_poll
td_stream_wait = lib.td_stream_wait
td_stream_destroy = lib.td_stream_destroy
td_strerror = lib.td_strerror
td_last_cuda_error = lib.td_last_cuda_error
td_depth_noalloc = lib.td_depth_noalloc
td_autotune = lib.td_autotune
td_set_tuned = lib.td_set_tuned
TD_NOALLOC_MAX_N = 512
TD_NOALLOC_MAX_M = 4096

EXPORTED = ["td_coord_limit", "td_create", "td_set_options", "td_destroy", "td_depth",
            "td_depth_batched", "td_stream_create", "td_stream_submit", "td_stream_poll",
            "td_stream_wait", "td_stream_destroy", "td_strerror", "td_last_cuda_error",
            "td_depth_noalloc", "td_autotune", "td_set_tuned"]


def _check(rc, ctx=None):
    if rc != TD_OK:
        msg = td_strerror(rc).decode()
        if ctx is not None and rc == TD_ERR_CUDA:
            msg += ": " + td_last_cuda_error(ctx).decode()
        raise TdError(rc, msg)


def options(mode=TD_MODE_FILTERED, device_pointers=False, use_graph=True, subsets_per_warp=0,
            buckets_log2=0, shard_index=0, shard_count=1, stream=None, early_exit=False,
            algorithm=TD_ALG_RCOM, unseeded=False):
    o = td_options()
    o.mode = mode
    o.device_pointers = 1 if device_pointers else 0
    o.use_graph = 1 if use_graph else 0
    o.subsets_per_warp = subsets_per_warp
    o.buckets_log2 = buckets_log2
    o.early_exit = 1 if early_exit else 0
    o.algorithm = algorithm
    o.unseeded = 1 if unseeded else 0
    o.shard_index = shard_index
    o.shard_count = shard_count
    o.stream = stream
    return o


def _host_i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Context:
    """One td_ctx on a CUDA device."""

    def __init__(self, device=0, **opts):
        self.ptr = ctypes.c_void_p()
        self.opts = options(**opts)
        _check(td_create(ctypes.byref(self.ptr), int(device), ctypes.byref(self.opts)))
        self.last_stats = td_stats()

    def set_options(self, **opts):
        self.opts = options(**opts)
        _check(td_set_options(self.ptr, ctypes.byref(self.opts)), self.ptr)

    def close(self):
        if self.ptr:
            td_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def depth(self, X, Z, out=None):
        """T(z) for every row z of Z.  numpy (host) arrays, or torch CUDA
        int32 tensors when the context uses device pointers."""
        st = td_stats()
        if self.opts.device_pointers:
            n, p = X.shape
            m = Z.shape[0]
            if out is None:
                import torch
                out = torch.empty(m, dtype=torch.int32, device=X.device)
            rc = td_depth(self.ptr, X.data_ptr(), n, p, Z.data_ptr(), m, out.data_ptr(), ctypes.byref(st))
        else:
            X = _host_i32(X)
            Z = _host_i32(Z).reshape(-1, X.shape[1])
            n, p = X.shape
            m = Z.shape[0]
            if out is None:
                out = np.empty(m, dtype=np.int32)
            rc = td_depth(self.ptr, X.ctypes.data, n, p, Z.ctypes.data, m, out.ctypes.data, ctypes.byref(st))
        _check(rc, self.ptr)
        self.last_stats = st
        return out

    def depth_batched(self, sets):
        """[(X, Z), ...] -> [out, ...] in one batched call (host arrays)."""
        keep = []
        arr = (td_dataset * len(sets))()
        outs = []
        for i, (X, Z) in enumerate(sets):
            if self.opts.device_pointers:
                import torch
                out = torch.empty(Z.shape[0], dtype=torch.int32, device=X.device)
                arr[i].n, arr[i].p = X.shape
                arr[i].X, arr[i].Z, arr[i].out = X.data_ptr(), Z.data_ptr(), out.data_ptr()
                arr[i].m = Z.shape[0]
            else:
                X = _host_i32(X)
                Z = _host_i32(Z).reshape(-1, X.shape[1])
                out = np.empty(Z.shape[0], dtype=np.int32)
                keep += [X, Z]
                arr[i].n, arr[i].p = X.shape
                arr[i].X, arr[i].Z, arr[i].out = X.ctypes.data, Z.ctypes.data, out.ctypes.data
                arr[i].m = Z.shape[0]
            outs.append(out)
        st = td_stats()
        _check(td_depth_batched(self.ptr, arr, len(sets), ctypes.byref(st)), self.ptr)
        self.last_stats = st
        return outs

    def autotune(self, p, n):
        """td_autotune: measure the work-tile sizes for dimension p and rows
        of about n points, keep the fastest in this context; returns the
        measurements."""
        r = td_tune_result()
        _check(td_autotune(self.ptr, int(p), int(n), ctypes.byref(r)), self.ptr)
        return r.as_dict()

    def set_tuned(self, d, octave, subsets_per_warp):
        _check(td_set_tuned(self.ptr, int(d), int(octave), int(subsets_per_warp)), self.ptr)

    def stream(self, mem_budget_bytes):
        return Stream(self, mem_budget_bytes)


def depth_sharded(X, Z, device=0, group=None, **opts):
    """T(z) for every row z of Z, with Algorithm 1's subset loop split over
    the ranks of a torch.distributed process group: rank r of W computes
    shard r of W (td_options.shard_index / shard_count: contiguous ranges of
    each query's colex subset positions) on `device`, and one all-reduce MIN
    over the ranks -- the only exchange step -- merges the shards into the
    depth, returned on every rank.  Host arrays (numpy) with a gloo group,
    or CUDA int32 tensors (device pointers) with an nccl group."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    on_device = isinstance(X, torch.Tensor) and X.is_cuda
    ctx = Context(device, shard_index=rank, shard_count=world, device_pointers=on_device, **opts)
    try:
        out = ctx.depth(X, Z)
    finally:
        ctx.close()
    t = out if on_device else torch.from_numpy(np.ascontiguousarray(out))
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return t if on_device else t.numpy()


class Stream:
    """td_stream_*: asynchronous requests with admission by memory."""

    def __init__(self, ctx, mem_budget_bytes):
        self.ctx = ctx
        self.ptr = ctypes.c_void_p()
        _check(td_stream_create(ctx.ptr, ctypes.c_size_t(int(mem_budget_bytes)), ctypes.byref(self.ptr)), ctx.ptr)
        self.pending = {}
        self.done = {}

    def submit(self, X, Z):
        """Returns a ticket, or None when admission is refused (TD_ERR_BUSY)."""
        X = _host_i32(X)
        Z = _host_i32(Z).reshape(-1, X.shape[1])
        out = np.empty(Z.shape[0], dtype=np.int32)
        d = td_dataset()
        d.n, d.p = X.shape
        d.X, d.Z, d.out, d.m = X.ctypes.data, Z.ctypes.data, out.ctypes.data, Z.shape[0]
        t = ctypes.c_uint64()
        rc = td_stream_submit(self.ptr, ctypes.byref(d), ctypes.byref(t))
        if rc == TD_ERR_BUSY:
            return None
        _check(rc, self.ctx.ptr)
        self.pending[t.value] = out
        return t.value

    def poll(self, ticket):
        """The request's outputs once it is done (the library then forgets the
        ticket), else None."""
        if ticket in self.done:
            return self.done.pop(ticket)
        done = ctypes.c_int(0)
        _check(td_stream_poll(self.ptr, ticket, ctypes.byref(done)), self.ctx.ptr)
        if not done.value:
            return None
        return self.pending.pop(ticket)

    def wait(self, ticket, timeout_us=-1):
        """The request's outputs, or raises TdError(TD_ERR_TIMEOUT)."""
        if ticket in self.done:
            return self.done.pop(ticket)
        _check(td_stream_wait(self.ptr, ticket, int(timeout_us)), self.ctx.ptr)
        return self.pending.pop(ticket)

    def close(self):
        if self.ptr:
            td_stream_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
