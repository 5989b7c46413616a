"""Python binding of libgb (include/gb.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
buffers may be given as torch CUDA tensors (their data pointer is passed) and
host buffers as numpy arrays or torch CPU tensors; the stream is a
``cudaStream_t`` handle (``torch.cuda.current_stream().cuda_stream``).  The
library itself must be built (``python -m paper_2603_02621_gb300.build``): if
``libgb.so`` is missing, loading fails loudly -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import POINTER, c_char_p, c_int, c_int32, c_int64, c_uint32, c_uint64, c_void_p

import numpy as np

from .build import LIB

GB_OK, GB_EINVAL, GB_ENOMEM, GB_ECUDA, GB_ETIMEOUT, GB_EBUSY, GB_ERANGE, GB_ECANCELED = range(8)
GB_FAULT_ALLOC, GB_FAULT_SUBMIT, GB_FAULT_CANCEL = 0, 1, 2
GB_MAX_HI = (1 << 63) - (1 << 26)      # largest hi of a range (include/gb.h)


class GbError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail or 'error'} (code {code})")
        self.code = code


class gb_config(ctypes.Structure):
    _fields_ = [("device", c_int32), ("seg_len", c_uint32), ("base_limit", c_uint64),
                ("tile_bits", c_uint32), ("cta_threads", c_uint32), ("bucket_split", c_uint32),
                ("p1", c_uint32), ("p2", c_uint32), ("cover_prefix", c_uint32), ("slab_bits", c_uint64),
                ("stream", c_void_p)]


class gb_segment_result(ctypes.Structure):
    _fields_ = [("lo", c_uint64), ("hi", c_uint64), ("n_checked", c_uint64),
                ("unresolved", c_uint64), ("max_pmin_n", c_uint64),
                ("max_pmin", c_uint32), ("hist_len", c_uint32)]


class gb_request(ctypes.Structure):
    _fields_ = [("kind", c_uint32), ("reserved", c_uint32), ("lo", c_uint64), ("hi", c_uint64)]


class gb_response(ctypes.Structure):
    _fields_ = [("status", c_int32), ("p_min", c_uint32), ("range", gb_segment_result),
                ("t_submit_us", ctypes.c_double), ("t_start_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


GB_REQ_RANGE, GB_REQ_QUERY = 0, 1


class gb_range_result(ctypes.Structure):
    _fields_ = [("n_checked", c_uint64), ("unresolved", c_uint64), ("max_pmin_n", c_uint64),
                ("max_pmin", c_uint32), ("hist_len", c_uint32), ("n_segments", c_uint32),
                ("p_final", c_uint32),
                ("hist", POINTER(c_uint64)), ("hist_cap", c_uint32),
                ("pmin", c_void_p),
                ("segs", POINTER(gb_segment_result)), ("seg_cap", c_uint32),
                ("seg_hist", POINTER(c_uint64)), ("seg_hist_stride", c_uint32),
                ("reserved", c_uint32)]


# every exported entry point of include/gb.h, with its C signature
SIGNATURES = {
    "gb_init": (c_int, [POINTER(c_void_p), POINTER(gb_config)]),
    "gb_destroy": (None, [c_void_p]),
    "gb_get_config": (c_int, [c_void_p, POINTER(gb_config)]),
    "gb_sieve_segment": (c_int, [c_void_p, c_int64, c_uint64, c_void_p, POINTER(c_uint64)]),
    "gb_prime_pi": (c_int, [c_void_p, c_uint64, POINTER(c_uint64)]),
    "gb_verify_range": (c_int, [c_void_p, c_uint64, c_uint64, c_uint32, POINTER(gb_range_result)]),
    "gb_verify_range_noalloc": (c_int, [c_void_p, c_uint64, c_uint64, c_uint32, POINTER(gb_range_result)]),
    "gb_verify_batch": (c_int, [c_void_p, POINTER(c_uint64), POINTER(c_uint64), c_uint32, c_uint32,
                                c_void_p, c_void_p, c_uint32]),
    "gb_query": (c_int, [c_void_p, c_uint64, POINTER(c_uint32)]),
    "gb_partitions": (c_int, [c_void_p, c_uint64, c_uint64, c_void_p]),
    "gb_query_batch": (c_int, [c_void_p, c_void_p, c_uint32, c_uint32, c_void_p]),
    "gb_set_config": (c_int, [c_void_p, POINTER(gb_config)]),
    "gb_init_shared": (c_int, [POINTER(c_void_p), c_void_p, c_void_p]),
    "gb_server_create": (c_int, [POINTER(c_void_p), c_void_p, c_uint32, c_uint64, c_uint32]),
    "gb_server_submit": (c_int, [c_void_p, POINTER(gb_request), POINTER(c_uint64)]),
    "gb_server_wait": (c_int, [c_void_p, c_uint64, POINTER(gb_response), c_uint32]),
    "gb_server_stats": (c_int, [c_void_p, POINTER(c_uint64), POINTER(c_uint64), POINTER(c_uint64),
                                POINTER(c_uint64)]),
    "gb_server_destroy": (None, [c_void_p]),
    "gb_server_cancel": (c_int, [c_void_p, c_uint64]),
    "gb_fault_set": (c_int, [c_char_p]),
    "gb_fault_tick": (c_int, [c_int]),
    "gb_debug_word": (c_uint32, [c_int]),
    "gb_debug_build": (c_int, []),
    "gb_tune_cache_lookup": (c_int, [c_char_p, c_char_p, POINTER(gb_config), POINTER(ctypes.c_double)]),
    "gb_tune_cache_store": (c_int, [c_char_p, c_char_p, POINTER(gb_config), ctypes.c_double]),
    "gb_autotune": (c_int, [c_void_p, POINTER(c_uint64), POINTER(c_uint64), c_uint32, c_int, c_uint32,
                            POINTER(gb_config), POINTER(ctypes.c_double)]),
    "gb_profile_enable": (c_int, [c_void_p, c_int]),
    "gb_profile_read": (c_int, [c_void_p, POINTER(ctypes.c_double), POINTER(c_uint64), POINTER(c_uint64)]),
    "gb_profile_work": (c_int, [c_void_p, POINTER(c_uint64), POINTER(c_uint64), POINTER(c_uint64)]),
    "gb_profile_kernels": (c_int, [c_void_p, POINTER(c_uint64)]),
    "gb_profile_copies": (c_int, [c_void_p, POINTER(c_uint64), POINTER(c_uint64)]),
    "gb_alloc_stats": (None, [POINTER(c_uint64), POINTER(c_uint64)]),
    "gb_bitset_bytes": (c_uint64, [c_uint64]),
    "gb_strerror": (c_char_p, [c_int]),
    "gb_last_error": (c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libgb.so (no fallback: a missing library is an error).  The
    environment variable GB_LIBRARY names another build of the same library
    (the debug build, libgb_debug.so) to load instead."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or os.environ.get("GB_LIBRARY") or LIB
        if not os.path.exists(p):
            raise ImportError(f"libgb.so not built at {p}: run python -m paper_2603_02621_gb300.build")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _check(rc: int, where: str, allow=()):
    if rc != GB_OK and rc not in allow:
        lib = load()
        raise GbError(rc, where, (lib.gb_last_error() or b"").decode() or lib.gb_strerror(rc).decode())
    return rc


def _ptr(buf) -> int:
    """Raw address of a torch tensor, numpy array or int."""
    if buf is None:
        return 0
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        return int(buf.data_ptr())
    if isinstance(buf, np.ndarray):
        return int(buf.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(buf)}")


def make_config(**kw) -> gb_config:
    c = gb_config()
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(v.cuda_stream) if hasattr(v, "cuda_stream") else int(v)
        setattr(c, k, v if v is not None else 0)
    return c


def gb_init(**kw) -> int:
    lib = load()
    cfg = make_config(**kw)
    h = c_void_p()
    _check(lib.gb_init(ctypes.byref(h), ctypes.byref(cfg)), "gb_init")
    return h.value


def gb_destroy(ctx: int) -> None:
    if ctx:
        load().gb_destroy(ctx)


def gb_get_config(ctx: int) -> dict:
    c = gb_config()
    _check(load().gb_get_config(ctx, ctypes.byref(c)), "gb_get_config")
    return {name: getattr(c, name) for name, _ in gb_config._fields_}


def gb_sieve_segment(ctx: int, A_odd: int, n_bits: int, q_bits) -> int:
    """Sieve odd numbers A_odd + 2i (i < n_bits) into the DEVICE buffer q_bits
    (>= ceil(n_bits/64) uint64 words); returns the number of primes."""
    pc = c_uint64()
    _check(load().gb_sieve_segment(ctx, A_odd, n_bits, _ptr(q_bits), ctypes.byref(pc)),
           "gb_sieve_segment")
    return pc.value


def gb_prime_pi(ctx: int, x: int) -> int:
    c = c_uint64()
    _check(load().gb_prime_pi(ctx, x, ctypes.byref(c)), "gb_prime_pi")
    return c.value


def gb_verify_range(ctx: int, lo: int, hi: int, P: int = 0, *, hist_cap: int = 0,
                    pmin=None, segs: bool = False, seg_hist_stride: int = 0,
                    allow_erange: bool = False) -> dict:
    """Verify every even n in [lo, hi).  Returns a dict with the totals, and
    'hist' (np.uint64[hist_cap]), 'segs' (structured rows), 'seg_hist'
    (np.uint64[nseg, stride]) when asked.  pmin: optional uint32 buffer of
    (hi-lo)/2 entries, host (numpy / CPU tensor) or device (CUDA tensor)."""
    return _verify(load().gb_verify_range, "gb_verify_range", ctx, lo, hi, P, hist_cap=hist_cap,
                   pmin=pmin, segs=segs, seg_hist_stride=seg_hist_stride, allow_erange=allow_erange)


def gb_verify_range_noalloc(ctx: int, lo: int, hi: int, P: int = 0, *, hist_cap: int = 0,
                            pmin=None, segs: bool = False, seg_hist_stride: int = 0,
                            allow_erange: bool = False) -> dict:
    """gb_verify_range for callers that must not allocate device memory during
    the call: one segment of at most GB_NOALLOC_MAX_N even n, scratch in a
    fixed device array of the library; pmin (if any) must be device memory."""
    return _verify(load().gb_verify_range_noalloc, "gb_verify_range_noalloc", ctx, lo, hi, P,
                   hist_cap=hist_cap, pmin=pmin, segs=segs, seg_hist_stride=seg_hist_stride,
                   allow_erange=allow_erange)


def _verify(fn, name, ctx, lo, hi, P, *, hist_cap, pmin, segs, seg_hist_stride, allow_erange):
    lib = load()
    r = gb_range_result()
    out = {}
    S = gb_get_config(ctx)["seg_len"]
    nseg = ((hi - lo) // 2 + S - 1) // S
    hist = None
    if hist_cap:
        hist = np.zeros(hist_cap, dtype=np.uint64)
        r.hist = hist.ctypes.data_as(POINTER(c_uint64))
        r.hist_cap = hist_cap
    if pmin is not None:
        r.pmin = _ptr(pmin)
    segarr = None
    if segs or seg_hist_stride:
        segarr = (gb_segment_result * nseg)()
        r.segs = segarr
        r.seg_cap = nseg
    rows = None
    if seg_hist_stride:
        rows = np.zeros((nseg, seg_hist_stride), dtype=np.uint64)
        r.seg_hist = rows.ctypes.data_as(POINTER(c_uint64))
        r.seg_hist_stride = seg_hist_stride
    rc = _check(fn(ctx, lo, hi, P, ctypes.byref(r)), name, allow=(GB_ERANGE,) if allow_erange else ())
    out.update(rc=rc, n_checked=r.n_checked, unresolved=r.unresolved, max_pmin=r.max_pmin,
               max_pmin_n=r.max_pmin_n, hist_len=r.hist_len, n_segments=r.n_segments,
               p_final=r.p_final)
    if hist is not None:
        out["hist"] = hist
    if segarr is not None:
        out["segs"] = [dict(lo=s.lo, hi=s.hi, n_checked=s.n_checked, unresolved=s.unresolved,
                            max_pmin=s.max_pmin, max_pmin_n=s.max_pmin_n, hist_len=s.hist_len)
                       for s in segarr]
    if rows is not None:
        out["seg_hist"] = rows
    return out


GB_PROF_KINDS = 5
GB_PROFILE_EVENTS = 2                  # gb_profile_enable: event times without the work counters
PROF_NAMES = ("sieve", "cover", "retry", "reduce", "large")


def gb_profile_enable(ctx: int, enable=True) -> None:
    """enable: False / 0 off, True / 1 event times and work counters,
    GB_PROFILE_EVENTS event times alone."""
    mode = GB_PROFILE_EVENTS if enable == GB_PROFILE_EVENTS and not isinstance(enable, bool) else int(bool(enable))
    _check(load().gb_profile_enable(ctx, mode), "gb_profile_enable")


def gb_profile_read(ctx: int) -> dict:
    ms = (ctypes.c_double * GB_PROF_KINDS)()
    ln = (c_uint64 * GB_PROF_KINDS)()
    un = (c_uint64 * GB_PROF_KINDS)()
    _check(load().gb_profile_read(ctx, ms, ln, un), "gb_profile_read")
    return {PROF_NAMES[k]: dict(ms=ms[k], launches=ln[k], units=un[k]) for k in range(GB_PROF_KINDS)}


def gb_profile_work(ctx: int) -> dict:
    a, b, c = c_uint64(), c_uint64(), c_uint64()
    _check(load().gb_profile_work(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "gb_profile_work")
    return dict(sieve_strikes=a.value, cover_iterations=b.value, large_strikes=c.value)


def gb_partitions(ctx: int, lo: int, hi: int, out=None):
    """r(n) for even n in [lo, hi): numpy uint32 array, or filled into `out`
    (a CUDA int32 tensor of (hi - lo) / 2 entries)."""
    count = (hi - lo) // 2
    res = None
    if out is None:
        res = np.zeros(max(count, 0), dtype=np.uint32)
        ptr = int(res.ctypes.data)
    else:
        ptr = out.data_ptr()
    _check(load().gb_partitions(ctx, lo, hi, ptr), "gb_partitions")
    return res


def gb_query(ctx: int, n: int) -> int:
    """p_min(n) (0 if no p <= the context's bound), computed on the GPU."""
    out = c_uint32()
    _check(load().gb_query(ctx, int(n), ctypes.byref(out)), "gb_query")
    return out.value


def gb_query_batch(ctx: int, ns, P: int = 0, *, out=None, allow_einval: bool = False):
    """p_min for many n: ns is a sequence / numpy array (host) or a CUDA
    tensor of int64 (device); out (optional) a CUDA int32 tensor.  Returns a
    numpy uint32 array for host output."""
    lib = load()
    if hasattr(ns, "data_ptr"):
        n_ptr, count = ns.data_ptr(), ns.numel()
        keep = None
    else:
        keep = np.ascontiguousarray(np.asarray(ns, dtype=np.uint64))
        n_ptr, count = int(keep.ctypes.data), keep.size
    res = None
    if out is None:
        res = np.zeros(count, dtype=np.uint32)
        o_ptr = int(res.ctypes.data)
    else:
        o_ptr = out.data_ptr()
    _check(lib.gb_query_batch(ctx, n_ptr, count, P, o_ptr), "gb_query_batch",
           allow=(GB_EINVAL,) if allow_einval else ())
    return res


GB_TUNE_PLAIN, GB_TUNE_BATCH = 0, 1


def gb_set_config(ctx: int, **fields) -> dict:
    """Change tunable configuration fields (see gb.h); returns the new config."""
    c = gb_config()
    _check(load().gb_get_config(ctx, ctypes.byref(c)), "gb_get_config")
    for k, v in fields.items():
        setattr(c, k, v)
    _check(load().gb_set_config(ctx, ctypes.byref(c)), "gb_set_config")
    return gb_get_config(ctx)


def gb_autotune(ctx: int, ranges, mode: int = GB_TUNE_BATCH, reps: int = 2):
    """Tune the context on a sample workload [(lo, hi), ...]; returns
    (config dict, best ms)."""
    count = len(ranges)
    lo = (c_uint64 * count)(*[int(a) for a, _ in ranges])
    hi = (c_uint64 * count)(*[int(b) for _, b in ranges])
    c = gb_config()
    ms = ctypes.c_double()
    _check(load().gb_autotune(ctx, lo, hi, count, mode, reps, ctypes.byref(c), ctypes.byref(ms)), "gb_autotune")
    return {f: getattr(c, f) for f, _ in gb_config._fields_}, ms.value


def gb_profile_kernels(ctx: int) -> int:
    n = c_uint64()
    _check(load().gb_profile_kernels(ctx, ctypes.byref(n)), "gb_profile_kernels")
    return n.value


def gb_profile_copies(ctx: int) -> dict:
    """Bytes the context's calls copied host -> device and device -> host
    since the last gb_profile_enable."""
    a, b = c_uint64(), c_uint64()
    _check(load().gb_profile_copies(ctx, ctypes.byref(a), ctypes.byref(b)), "gb_profile_copies")
    return dict(h2d=a.value, d2h=b.value)


def gb_fault_set(spec: str | None) -> None:
    """Host-side fault injection (gb.h): "kind@n[,kind@n...]", kind alloc,
    submit or cancel; None or "" clears."""
    _check(load().gb_fault_set(spec.encode() if spec else None), "gb_fault_set")


def gb_fault_tick(kind: int) -> bool:
    return bool(load().gb_fault_tick(kind))


def gb_tune_cache_lookup(path: str, key: str):
    """(config fields dict, best ms) stored for key in the autotune cache
    file, or None."""
    c = gb_config()
    ms = ctypes.c_double()
    rc = load().gb_tune_cache_lookup(path.encode(), key.encode(), ctypes.byref(c), ctypes.byref(ms))
    if rc == GB_ERANGE:
        return None
    _check(rc, "gb_tune_cache_lookup")
    return {f: getattr(c, f) for f in ("tile_bits", "bucket_split", "p1", "cover_prefix", "seg_len",
                                       "cta_threads")}, ms.value


def gb_tune_cache_store(path: str, key: str, fields: dict, best_ms: float) -> None:
    c = gb_config()
    for k, v in fields.items():
        setattr(c, k, v)
    _check(load().gb_tune_cache_store(path.encode(), key.encode(), ctypes.byref(c), best_ms), "gb_tune_cache_store")


def gb_alloc_stats() -> dict:
    """Device and pinned host allocations the library has made in this process."""
    a, b = c_uint64(), c_uint64()
    load().gb_alloc_stats(ctypes.byref(a), ctypes.byref(b))
    return dict(count=a.value, bytes=b.value)


def gb_verify_batch(ctx: int, ranges, P: int = 0, *, hist_stride: int = 0, results=None, hist=None,
                    allow_erange: bool = False) -> dict:
    """Verify many ranges [(lo, hi), ...] in one batched pass.  Returns a dict
    with 'records' (list of per-range dicts) and 'hist' (np.uint64[count,
    hist_stride]) when hist_stride > 0.  results / hist may be given as device
    buffers (torch CUDA tensors of gb_segment_result rows / uint64), in which
    case they are filled in place and not copied back."""
    lib = load()
    count = len(ranges)
    lo = (c_uint64 * count)(*[int(a) for a, _ in ranges])
    hi = (c_uint64 * count)(*[int(b) for _, b in ranges])
    recs = None
    if results is None:
        recs = (gb_segment_result * count)()
        res_ptr = ctypes.addressof(recs)
    else:
        res_ptr = _ptr(results)
    rows = None
    if hist is None and hist_stride:
        rows = np.zeros((count, hist_stride), dtype=np.uint64)
        hist_ptr = int(rows.ctypes.data)
    else:
        hist_ptr = _ptr(hist)
    rc = _check(lib.gb_verify_batch(ctx, lo, hi, count, P, res_ptr, hist_ptr, hist_stride), "gb_verify_batch",
                allow=(GB_ERANGE,) if allow_erange else ())
    out = {"rc": rc}
    if recs is not None:
        out["records"] = [dict(lo=r.lo, hi=r.hi, n_checked=r.n_checked, unresolved=r.unresolved,
                               max_pmin=r.max_pmin, max_pmin_n=r.max_pmin_n, hist_len=r.hist_len) for r in recs]
    if rows is not None:
        out["hist"] = rows
    return out


def gb_bitset_bytes(N: int) -> int:
    return int(load().gb_bitset_bytes(N))


def gb_strerror(code: int) -> str:
    return load().gb_strerror(code).decode()


def gb_last_error() -> str:
    return (load().gb_last_error() or b"").decode()


class Context:
    """Owning wrapper: ``with Context(base_limit=10**5) as g: g.verify_range(...)``."""

    def __init__(self, _handle=None, **cfg):
        self.handle = _handle if _handle is not None else gb_init(**cfg)

    def share(self, stream: int = 0) -> "Context":
        """A context sharing this one's base primes, with its own stream
        (cudaStream_t as an int, 0 = legacy default) and arenas."""
        h = c_void_p()
        _check(load().gb_init_shared(ctypes.byref(h), self.handle, stream or None), "gb_init_shared")
        return Context(_handle=h.value)

    def close(self):
        if self.handle:
            gb_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def config(self):
        return gb_get_config(self.handle)

    def sieve_segment(self, A_odd, n_bits, q_bits):
        return gb_sieve_segment(self.handle, A_odd, n_bits, q_bits)

    def prime_pi(self, x):
        return gb_prime_pi(self.handle, x)

    def verify_range(self, lo, hi, P=0, **kw):
        return gb_verify_range(self.handle, lo, hi, P, **kw)

    def verify_range_noalloc(self, lo, hi, P=0, **kw):
        return gb_verify_range_noalloc(self.handle, lo, hi, P, **kw)

    def verify_batch(self, ranges, P=0, **kw):
        return gb_verify_batch(self.handle, ranges, P, **kw)

    def partitions(self, lo, hi, out=None):
        return gb_partitions(self.handle, lo, hi, out)

    def query(self, n):
        return gb_query(self.handle, n)

    def query_batch(self, ns, P=0, **kw):
        return gb_query_batch(self.handle, ns, P, **kw)

    def set_config(self, **fields):
        return gb_set_config(self.handle, **fields)

    def autotune(self, ranges, mode=GB_TUNE_BATCH, reps=2):
        return gb_autotune(self.handle, ranges, mode, reps)


class Server:
    """Request loop with continuous batching over `lanes` GPU lanes (gb.h,
    serving).  submit() queues a range ('range', lo, hi) or a query
    ('query', n) and returns a ticket; wait(ticket) returns its response."""

    def __init__(self, ctx: "Context", lanes: int = 4, hbm_budget: int = 0, max_batch: int = 0):
        self.ctx = ctx
        h = c_void_p()
        _check(load().gb_server_create(ctypes.byref(h), ctx.handle, lanes, hbm_budget, max_batch),
               "gb_server_create")
        self.handle = h.value

    def submit(self, kind: str, a: int, b: int = 0) -> int:
        r = gb_request(GB_REQ_RANGE if kind == "range" else GB_REQ_QUERY, 0, int(a), int(b))
        t = c_uint64()
        _check(load().gb_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "gb_server_submit")
        return t.value

    def cancel(self, ticket: int) -> int:
        """Cancel a request still in its queue (GB_OK), else GB_EBUSY."""
        return _check(load().gb_server_cancel(self.handle, ticket), "gb_server_cancel", allow=(GB_EBUSY,))

    def wait(self, ticket: int, timeout_ms: int = 600000) -> dict:
        r = gb_response()
        _check(load().gb_server_wait(self.handle, ticket, ctypes.byref(r), timeout_ms), "gb_server_wait")
        g = r.range
        return dict(status=r.status, p_min=r.p_min,
                    range=dict(lo=g.lo, hi=g.hi, n_checked=g.n_checked, unresolved=g.unresolved,
                               max_pmin=g.max_pmin, max_pmin_n=g.max_pmin_n, hist_len=g.hist_len),
                    t_submit_us=r.t_submit_us, t_start_us=r.t_start_us, t_done_us=r.t_done_us)

    def stats(self) -> dict:
        v = [c_uint64() for _ in range(4)]
        _check(load().gb_server_stats(self.handle, *[ctypes.byref(x) for x in v]), "gb_server_stats")
        return dict(submitted=v[0].value, completed=v[1].value, batches=v[2].value,
                    in_flight_max_bytes=v[3].value)

    def close(self):
        if self.handle:
            load().gb_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
