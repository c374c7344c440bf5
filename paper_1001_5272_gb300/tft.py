"""Python binding of the C ABI in include/tft.h (argument marshalling only).

Every function keeps the C name and forwards to the in-tree shared library
``_lib/libtft_gb300.so``; no step of any transform runs in Python.  Device
buffers are torch CUDA tensors (any dtype whose element size is the prime's:
4 bytes for 998244353 and 2013265921, 8 bytes for 2^64 - 2^32 + 1; the bits
are the canonical residues).  Host-buffer calls take numpy arrays or CPU
tensors.  If the library is missing the import of this module still works,
but every call raises ``RuntimeError`` -- there is no fallback.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtft_gb300.so")

TFT_P998244353 = 0
TFT_P2013265921 = 1
TFT_PGOLDILOCKS = 2
PRIME_IDS = {"p998244353": 0, "p2013265921": 1, "goldilocks": 2,
             998244353: 0, 2013265921: 1, 2**64 - 2**32 + 1: 2}
MODULI = {0: 998244353, 1: 2013265921, 2: 2**64 - 2**32 + 1}
TWO_ADICITY = {0: 23, 1: 27, 2: 32}

TFT_OK, TFT_EINVAL, TFT_ERANGE, TFT_ENOMEM, TFT_ECUDA, TFT_ETIMEOUT = range(6)
TFT_CTX_HOST_STAGING = 1

_lib = None


class PolymulDesc(ctypes.Structure):
    """tft_polymul_desc: one product of a batch (device pointers)."""
    _fields_ = [("a", ctypes.c_void_p), ("na", ctypes.c_uint64),
                ("b", ctypes.c_void_p), ("nb", ctypes.c_uint64),
                ("out", ctypes.c_void_p)]


class TransformDesc(ctypes.Structure):
    """tft_transform_desc."""
    _fields_ = [("x", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class BatchParams(ctypes.Structure):
    """tft_batch_params: 0 in a field selects the library default."""
    _fields_ = [("small_log", ctypes.c_uint32), ("lr", ctypes.c_uint32),
                ("clog_plus1", ctypes.c_uint32),
                ("clog_lo_plus1", ctypes.c_uint32)]


class Request(ctypes.Structure):
    """tft_request: one served request."""
    _fields_ = [("id", ctypes.c_uint64), ("na", ctypes.c_uint64),
                ("nb", ctypes.c_uint64), ("arrival_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    """tft_server_stats."""
    _fields_ = [("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("max_batch", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("wall_s", ctypes.c_double)]


TFT_SERVE_BATCHED = 0
TFT_SERVE_ONE_BY_ONE = 1


class TFTError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"CUDA library not built: {LIB_PATH} is missing "
            "(run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    u64, u32, i32, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                         ctypes.c_void_p)
    sig = {
        "tft_ctx_create": (i32, [i32, i32, u64, u32,
                                 ctypes.POINTER(ctypes.c_void_p)]),
        "tft_ctx_destroy": (i32, [vp]),
        "tft_forward": (i32, [vp, vp, u64, u32, vp]),
        "tft_inverse": (i32, [vp, vp, u64, u32, vp]),
        "tft_polymul": (i32, [vp, vp, u64, vp, u64, vp, vp]),
        "tft_polymul_restricted": (i32, [vp, vp, u64, vp, u64, vp, vp]),
        "tft_polymul_padded": (i32, [vp, vp, u64, vp, u64, vp, vp, vp]),
        "tft_restricted_schedule": (i32, [u64, ctypes.POINTER(u64),
                                          ctypes.POINTER(u64), u32,
                                          ctypes.POINTER(u32),
                                          ctypes.POINTER(u64)]),
        "tft_forward_host": (i32, [vp, vp, u64, u32, vp]),
        "tft_inverse_host": (i32, [vp, vp, u64, u32, vp]),
        "tft_polymul_host": (i32, [vp, vp, u64, vp, u64, vp, vp]),
        "tft_footprint": (i32, [i32, u64, u32, i32,
                                ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "tft_describe_plan": (i32, [i32, u64,
                                    ctypes.POINTER(ctypes.c_int64)]),
        "tft_element_bytes": (u32, [i32]),
        "tft_last_error": (i32, [vp]),
        "tft_status_string": (ctypes.c_char_p, [i32]),
        "tft_last_cuda_error": (ctypes.c_char_p, []),
        "tft_profile_enable": (i32, [vp, i32]),
        "tft_profile_read": (i32, [vp, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(u64)]),
        "tft_kernel_name": (ctypes.c_char_p, [i32]),
        "tft_launch_count": (u64, [vp]),
        "tft_forward_noalloc": (i32, [i32, vp, u64, u32, vp]),
        "tft_calibrate": (i32, [vp, i32, u32, u32, vp, u64, vp,
                                ctypes.POINTER(u64)]),
        "tft_transform_batch": (i32, [vp, i32, ctypes.POINTER(TransformDesc),
                                      u32, vp]),
        "tft_shard_columns": (i32, [vp, i32, i32, vp, u64, u32, u32, vp, vp]),
        "tft_shard_rows": (i32, [vp, i32, vp, u64, u64, u64, vp]),
        "tft_shard_last_row": (i32, [vp, i32, vp, vp, u64, vp]),
        "tft_debug_fail_allocation": (None, [ctypes.c_int64]),
        "tft_debug_live_allocations": (ctypes.c_int64, []),
        "tft_forward_noscratch": (i32, [i32, vp, u64, u32, vp]),
        "tft_inverse_noscratch": (i32, [i32, vp, u64, u32, vp]),
        "tft_ctx_reserve_batch": (i32, [vp, u32, u64]),
        "tft_batch_work_words": (i32, [i32, ctypes.POINTER(PolymulDesc), u32,
                                       ctypes.POINTER(BatchParams),
                                       ctypes.POINTER(u64)]),
        "tft_batch_plan": (i32, [vp, ctypes.POINTER(PolymulDesc), u32,
                                 ctypes.POINTER(BatchParams)]),
        "tft_batch_run": (i32, [vp, vp]),
        "tft_polymul_batch": (i32, [vp, ctypes.POINTER(PolymulDesc), u32,
                                    ctypes.POINTER(BatchParams), vp]),
        "tft_generate": (i32, [vp, u64, u64, u32, vp, u64, vp]),
        "tft_request_bytes": (i32, [i32, u64, u64, ctypes.POINTER(BatchParams),
                                    ctypes.POINTER(u64)]),
        "tft_arena_create": (i32, [u64, u64, ctypes.POINTER(vp)]),
        "tft_arena_destroy": (i32, [vp]),
        "tft_arena_alloc": (i32, [vp, u64, ctypes.POINTER(u64)]),
        "tft_arena_free": (i32, [vp, u64]),
        "tft_arena_usage": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                  ctypes.POINTER(u64)]),
        "tft_server_create": (i32, [vp, u64, u32, ctypes.POINTER(BatchParams),
                                    ctypes.POINTER(vp)]),
        "tft_server_destroy": (i32, [vp]),
        "tft_server_replay": (i32, [vp, ctypes.POINTER(Request), u64, u64, i32,
                                    ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(vp),
                                    ctypes.POINTER(ServerStats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/tft.h that the loaded library exports."""
    L = load()
    return [n for n in _header_functions() if hasattr(L, n)]


def _header_functions():
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "tft.h")
    text = open(hdr).read()
    return re.findall(
        r"^\s*(?:tft_status|uint32_t|uint64_t|int64_t|void|const char\*)"
        r"\s+(tft_\w+)\(",
        text, flags=re.M)


def status_string(s):
    try:
        return load().tft_status_string(int(s)).decode()
    except RuntimeError:
        return str(s)


def _check(st, what):
    if st != TFT_OK:
        if st == TFT_ECUDA:
            what = f"{what} [{load().tft_last_cuda_error().decode()}]"
        raise TFTError(st, what)


def prime_id(prime):
    if isinstance(prime, int) and prime in (0, 1, 2):
        return prime
    return PRIME_IDS[prime]


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev_ptr(t, elem_bytes, what):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if t.element_size() != elem_bytes:
        raise ValueError(f"{what}: element size {t.element_size()} != "
                         f"{elem_bytes}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(arr, elem_bytes, what):
    if hasattr(arr, "data_ptr"):  # torch CPU tensor
        if arr.is_cuda or arr.element_size() != elem_bytes or \
                not arr.is_contiguous():
            raise ValueError(f"{what}: need a contiguous CPU tensor of "
                             f"{elem_bytes}-byte elements")
        return ctypes.c_void_p(arr.data_ptr()), arr.numel()
    import numpy as np
    if not isinstance(arr, np.ndarray) or arr.itemsize != elem_bytes or \
            not arr.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what}: need a C-contiguous numpy array of "
                         f"{elem_bytes}-byte elements")
    return ctypes.c_void_p(arr.ctypes.data), arr.size


class Context:
    """Owns a ``tft_ctx`` (root table, fixed scratch, product work buffer)."""

    def __init__(self, prime, device=0, max_len=1 << 20, host_staging=False):
        L = load()
        self.prime = prime_id(prime)
        self.device = device
        self.max_len = int(max_len)
        self.elem_bytes = int(L.tft_element_bytes(self.prime))
        h = ctypes.c_void_p()
        flags = TFT_CTX_HOST_STAGING if host_staging else 0
        _check(L.tft_ctx_create(self.prime, device, self.max_len, flags,
                                ctypes.byref(h)), "tft_ctx_create")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("context destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().tft_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _default_k(n):
    return max(0, (int(n) - 1).bit_length())


def tft_forward(ctx, x, k=None, stream=None):
    """In-place forward TFT of the CUDA tensor ``x`` (Algorithm 1)."""
    n = x.numel()
    k = _default_k(n) if k is None else int(k)
    _check(load().tft_forward(ctx.handle, _dev_ptr(x, ctx.elem_bytes, "x"),
                              n, k, _stream_handle(stream)), "tft_forward")
    return x


def tft_inverse(ctx, X, k=None, stream=None):
    """In-place inverse TFT of the CUDA tensor ``X`` (Algorithm 2)."""
    n = X.numel()
    k = _default_k(n) if k is None else int(k)
    _check(load().tft_inverse(ctx.handle, _dev_ptr(X, ctx.elem_bytes, "X"),
                              n, k, _stream_handle(stream)), "tft_inverse")
    return X


def tft_polymul(ctx, a, b, out, stream=None):
    """out = a * b mod p for CUDA tensors (len(out) = len(a) + len(b) - 1)."""
    if out.numel() != a.numel() + b.numel() - 1:
        raise ValueError("out must have len(a) + len(b) - 1 elements")
    _check(load().tft_polymul(ctx.handle, _dev_ptr(a, ctx.elem_bytes, "a"),
                              a.numel(), _dev_ptr(b, ctx.elem_bytes, "b"),
                              b.numel(), _dev_ptr(out, ctx.elem_bytes, "out"),
                              _stream_handle(stream)), "tft_polymul")
    return out


def tft_polymul_restricted(ctx, a, b, out, stream=None):
    """out = a * b mod p by the space-restricted product (Algorithm 3): no
    work area beyond out and the context's fixed scratch."""
    if out.numel() != a.numel() + b.numel() - 1:
        raise ValueError("out must have len(a) + len(b) - 1 elements")
    _check(load().tft_polymul_restricted(
        ctx.handle, _dev_ptr(a, ctx.elem_bytes, "a"), a.numel(),
        _dev_ptr(b, ctx.elem_bytes, "b"), b.numel(),
        _dev_ptr(out, ctx.elem_bytes, "out"), _stream_handle(stream)),
        "tft_polymul_restricted")
    return out


def tft_polymul_padded(ctx, a, b, out, scratch, stream=None):
    """out = a * b mod p through zero-padded power-of-two transforms
    (comparison path); scratch: CUDA tensor of 2 * 2^ceil(lg r) elements."""
    r = a.numel() + b.numel() - 1
    if out.numel() != r:
        raise ValueError("out must have len(a) + len(b) - 1 elements")
    N = 1 << (r - 1).bit_length()
    if scratch.numel() < 2 * N:
        raise ValueError(f"scratch needs {2 * N} elements")
    _check(load().tft_polymul_padded(
        ctx.handle, _dev_ptr(a, ctx.elem_bytes, "a"), a.numel(),
        _dev_ptr(b, ctx.elem_bytes, "b"), b.numel(),
        _dev_ptr(out, ctx.elem_bytes, "out"),
        _dev_ptr(scratch, ctx.elem_bytes, "scratch"),
        _stream_handle(stream)), "tft_polymul_padded")
    return out


def tft_restricted_schedule(r):
    """([(q, L), ...], tail_start) of the space-restricted product for an
    output of r positions (host only)."""
    q = (ctypes.c_uint64 * 64)()
    L = (ctypes.c_uint64 * 64)()
    n = ctypes.c_uint32()
    tail = ctypes.c_uint64()
    _check(load().tft_restricted_schedule(int(r), q, L, 64, ctypes.byref(n),
                                          ctypes.byref(tail)),
           "tft_restricted_schedule")
    return [(q[i], L[i]) for i in range(n.value)], tail.value


def tft_forward_host(ctx, x, k=None, stream=None):
    ptr, n = _host_ptr(x, ctx.elem_bytes, "x")
    k = _default_k(n) if k is None else int(k)
    _check(load().tft_forward_host(ctx.handle, ptr, n, k,
                                   _stream_handle(stream)), "tft_forward_host")
    return x


def tft_inverse_host(ctx, X, k=None, stream=None):
    ptr, n = _host_ptr(X, ctx.elem_bytes, "X")
    k = _default_k(n) if k is None else int(k)
    _check(load().tft_inverse_host(ctx.handle, ptr, n, k,
                                   _stream_handle(stream)), "tft_inverse_host")
    return X


def tft_polymul_host(ctx, a, b, out, stream=None):
    pa, na = _host_ptr(a, ctx.elem_bytes, "a")
    pb, nb = _host_ptr(b, ctx.elem_bytes, "b")
    po, no = _host_ptr(out, ctx.elem_bytes, "out")
    if no != na + nb - 1:
        raise ValueError("out must have len(a) + len(b) - 1 elements")
    _check(load().tft_polymul_host(ctx.handle, pa, na, pb, nb, po,
                                   _stream_handle(stream)), "tft_polymul_host")
    return out


def tft_footprint(prime, n, k=0, op=0):
    """(inplace_bytes, padded_bytes) of a transform (op=0) or product (op=1)."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().tft_footprint(prime_id(prime), int(n), int(k), int(op),
                                ctypes.byref(a), ctypes.byref(b)),
           "tft_footprint")
    return a.value, b.value


def tft_describe_plan(prime, n):
    out = (ctypes.c_int64 * 8)()
    _check(load().tft_describe_plan(prime_id(prime), int(n), out),
           "tft_describe_plan")
    keys = ("small", "l", "lr", "c", "clog", "a", "b", "row_ctas_per_sm")
    return dict(zip(keys, [int(v) for v in out]))


def tft_last_error(ctx):
    return int(load().tft_last_error(ctx.handle))


NUM_KERNEL_KINDS = 12


def kernel_name(kind):
    return load().tft_kernel_name(int(kind)).decode()


def tft_profile_enable(ctx, enable=True):
    _check(load().tft_profile_enable(ctx.handle, 1 if enable else 0),
           "tft_profile_enable")


def tft_profile_read(ctx):
    """{kernel name: (total ms, timed launches)} since the last enable."""
    ms = (ctypes.c_double * NUM_KERNEL_KINDS)()
    cnt = (ctypes.c_uint64 * NUM_KERNEL_KINDS)()
    _check(load().tft_profile_read(ctx.handle, ms, cnt), "tft_profile_read")
    return {kernel_name(k): (ms[k], int(cnt[k]))
            for k in range(NUM_KERNEL_KINDS) if cnt[k]}


def tft_launch_count(ctx):
    return int(load().tft_launch_count(ctx.handle))


def _opt_ptr(t, elem_bytes, what):
    return ctypes.c_void_p(None) if t is None else _dev_ptr(t, elem_bytes,
                                                             what)


def tft_shard_columns(ctx, inverse, which, block, n, parts, part, E=None,
                      stream=None):
    """Column step of a transform of length n held in `parts` parts, on
    part `part`'s (a + 1) x W column block (include/tft.h)."""
    _check(load().tft_shard_columns(
        ctx.handle, int(inverse), int(which),
        _dev_ptr(block, ctx.elem_bytes, "block"), int(n), int(parts),
        int(part), _opt_ptr(E, ctx.elem_bytes, "E"), _stream_handle(stream)),
        "tft_shard_columns")


def tft_shard_rows(ctx, inverse, rows, n, rho_begin, count, stream=None):
    """Row step on `count` full rows (rows rho_begin.. of the view)."""
    _check(load().tft_shard_rows(
        ctx.handle, int(inverse),
        _opt_ptr(rows if count else None, ctx.elem_bytes, "rows"), int(n),
        int(rho_begin), int(count), _stream_handle(stream)), "tft_shard_rows")


def tft_shard_last_row(ctx, inverse, row, E, n, stream=None):
    """The ragged last row from an R-word row buffer and the R-word E."""
    _check(load().tft_shard_last_row(
        ctx.handle, int(inverse), _dev_ptr(row, ctx.elem_bytes, "row"),
        _dev_ptr(E, ctx.elem_bytes, "E"), int(n), _stream_handle(stream)),
        "tft_shard_last_row")


def tft_debug_fail_allocation(n):
    """Make the library's allocation after the next n successful ones fail
    once (n < 0: off); see include/tft.h."""
    load().tft_debug_fail_allocation(int(n))


def tft_debug_live_allocations():
    return int(load().tft_debug_live_allocations())


def tft_calibrate(ctx, kind, iters, blocks, out, stream=None):
    """Launch one calibration kernel (include/tft.h); returns the number of
    operations it performs.  `out` is a device tensor of at least
    blocks * 256 * 8 bytes."""
    ops = ctypes.c_uint64(0)
    _check(load().tft_calibrate(ctx.handle, int(kind), int(iters),
                                int(blocks), ctypes.c_void_p(out.data_ptr()),
                                out.numel() * out.element_size(),
                                _stream_handle(stream), ctypes.byref(ops)),
           "tft_calibrate")
    return int(ops.value)


def tft_forward_noalloc(prime, x, k=None, stream=None):
    """In-place forward TFT without a context and without allocating device
    memory: for callers that may not call cudaMalloc (for example a serving
    loop whose memory is fully reserved up front).  The library's fixed
    128 KiB device array serves as scratch; calls that overlap on the GPU
    race on it, so order them on one stream.  Make the first call on a
    device before any stream capture (it configures the device)."""
    pid = prime_id(prime)
    n = x.numel()
    k = _default_k(n) if k is None else int(k)
    L = load()
    _check(L.tft_forward_noalloc(pid, _dev_ptr(x, int(L.tft_element_bytes(pid)),
                                               "x"),
                                 n, k, _stream_handle(stream)),
           "tft_forward_noalloc")
    return x


def _noscratch(name, prime, x, k, stream):
    pid = prime_id(prime)
    n = x.numel()
    k = _default_k(n) if k is None else int(k)
    L = load()
    _check(getattr(L, name)(pid, _dev_ptr(x, int(L.tft_element_bytes(pid)),
                                          "x"),
                            n, k, _stream_handle(stream)), name)
    return x


def tft_forward_noscratch(prime, x, k=None, stream=None):
    """In-place forward TFT (the result of tft_forward) that reads and
    writes no device memory but x: no context, no scratch, no allocation;
    the ragged last row comes from one 8-CTA cluster's shared memory."""
    return _noscratch("tft_forward_noscratch", prime, x, k, stream)


def tft_inverse_noscratch(prime, x, k=None, stream=None):
    """In-place inverse TFT (the result of tft_inverse) that reads and
    writes no device memory but x."""
    return _noscratch("tft_inverse_noscratch", prime, x, k, stream)


# ---------------------------------------------------------------------------
# Batched products
# ---------------------------------------------------------------------------

def _descs(products, elem_bytes):
    """products: sequence of (a, b, out) CUDA tensors."""
    arr = (PolymulDesc * max(1, len(products)))()
    for i, (a, b, out) in enumerate(products):
        if out.numel() != a.numel() + b.numel() - 1:
            raise ValueError(f"product {i}: out must have len(a)+len(b)-1 "
                             "elements")
        arr[i].a = _dev_ptr(a, elem_bytes, "a").value
        arr[i].na = a.numel()
        arr[i].b = _dev_ptr(b, elem_bytes, "b").value
        arr[i].nb = b.numel()
        arr[i].out = _dev_ptr(out, elem_bytes, "out").value
    return arr


def _params(params):
    if params is None:
        return None
    if isinstance(params, BatchParams):
        return ctypes.byref(params)
    p = BatchParams()
    p.small_log = int(params.get("small_log", 0))
    p.lr = int(params.get("lr", 0))
    clog = params.get("clog")
    p.clog_plus1 = 0 if clog is None else int(clog) + 1
    clog_lo = params.get("clog_lo")
    p.clog_lo_plus1 = 0 if clog_lo is None else int(clog_lo) + 1
    return ctypes.byref(p)


def tft_transform_batch(ctx, xs, inverse=False, stream=None):
    """In-place forward (or inverse) TFT of every CUDA tensor in xs."""
    arr = (TransformDesc * max(1, len(xs)))()
    for i, x in enumerate(xs):
        arr[i].x = _dev_ptr(x, ctx.elem_bytes, "x").value
        arr[i].n = x.numel()
    _check(load().tft_transform_batch(ctx.handle, 1 if inverse else 0, arr,
                                      len(xs), _stream_handle(stream)),
           "tft_transform_batch")


def tft_ctx_reserve_batch(ctx, max_products, work_words):
    _check(load().tft_ctx_reserve_batch(ctx.handle, int(max_products),
                                        int(work_words)),
           "tft_ctx_reserve_batch")


def tft_batch_work_words(prime, lengths, params=None):
    """Work-area elements a batch of (na, nb) pairs needs."""
    arr = (PolymulDesc * max(1, len(lengths)))()
    for i, (na, nb) in enumerate(lengths):
        arr[i].na, arr[i].nb = int(na), int(nb)
    w = ctypes.c_uint64()
    _check(load().tft_batch_work_words(prime_id(prime), arr, len(lengths),
                                       _params(params), ctypes.byref(w)),
           "tft_batch_work_words")
    return w.value


def tft_batch_plan(ctx, products, params=None):
    """Plan a batch of (a, b, out) CUDA tensors (uploads the tables)."""
    _check(load().tft_batch_plan(ctx.handle, _descs(products, ctx.elem_bytes),
                                 len(products), _params(params)),
           "tft_batch_plan")


def tft_batch_run(ctx, stream=None):
    """Launch the planned batch (capturable into a CUDA graph)."""
    _check(load().tft_batch_run(ctx.handle, _stream_handle(stream)),
           "tft_batch_run")


def tft_polymul_batch(ctx, products, params=None, stream=None):
    _check(load().tft_polymul_batch(ctx.handle,
                                    _descs(products, ctx.elem_bytes),
                                    len(products), _params(params),
                                    _stream_handle(stream)),
           "tft_polymul_batch")


# ---------------------------------------------------------------------------
# Served products
# ---------------------------------------------------------------------------

def tft_generate(ctx, seed, request, operand, out, stream=None):
    """Fill the CUDA tensor ``out`` with operand ``operand`` of request
    ``request`` (device generator, Philox4x32-10 reduced mod p)."""
    _check(load().tft_generate(ctx.handle, int(seed), int(request),
                               int(operand),
                               _dev_ptr(out, ctx.elem_bytes, "out"),
                               out.numel(), _stream_handle(stream)),
           "tft_generate")


def tft_request_bytes(prime, na, nb, params=None):
    v = ctypes.c_uint64()
    _check(load().tft_request_bytes(prime_id(prime), int(na), int(nb),
                                    _params(params), ctypes.byref(v)),
           "tft_request_bytes")
    return v.value


class Arena:
    """The server's first-fit arena (host bookkeeping of offsets)."""

    def __init__(self, size, align=256):
        h = ctypes.c_void_p()
        _check(load().tft_arena_create(int(size), int(align),
                                       ctypes.byref(h)), "tft_arena_create")
        self._h = h

    def alloc(self, nbytes):
        """Offset of a new range, or None when nothing fits."""
        off = ctypes.c_uint64()
        st = load().tft_arena_alloc(self._h, int(nbytes), ctypes.byref(off))
        if st == TFT_ENOMEM:
            return None
        _check(st, "tft_arena_alloc")
        return off.value

    def free(self, offset):
        _check(load().tft_arena_free(self._h, int(offset)), "tft_arena_free")

    def usage(self):
        u, p, f = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().tft_arena_usage(self._h, ctypes.byref(u),
                                      ctypes.byref(p), ctypes.byref(f)),
               "tft_arena_usage")
        return {"used": u.value, "peak": p.value, "free_ranges": f.value}

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().tft_arena_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """tft_server: continuous batching of generated requests under a device
    memory budget (or the one-by-one comparison path)."""

    def __init__(self, ctx, budget_bytes, max_batch=4096, params=None):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(load().tft_server_create(ctx.handle, int(budget_bytes),
                                        int(max_batch), _params(params),
                                        ctypes.byref(h)), "tft_server_create")
        self._h = h

    def replay(self, ids, na, nb, arrivals, seed, mode="batched", keep=None):
        """Run the requests open loop; returns (completion seconds as a
        numpy array, stats dict).  keep: optional {index: CUDA tensor of
        na + nb - 1 elements} receiving those requests' products."""
        import numpy as np
        n = len(ids)
        reqs = (Request * max(1, n))()
        for i in range(n):
            reqs[i].id = int(ids[i])
            reqs[i].na = int(na[i])
            reqs[i].nb = int(nb[i])
            reqs[i].arrival_s = float(arrivals[i])
        done = np.zeros(max(1, n), dtype=np.float64)
        keep_arr = None
        if keep:
            keep_arr = (ctypes.c_void_p * max(1, n))()
            for i, t in keep.items():
                if t.numel() != int(na[i]) + int(nb[i]) - 1:
                    raise ValueError(f"keep[{i}] has the wrong length")
                keep_arr[i] = _dev_ptr(t, self.ctx.elem_bytes, "keep").value
        st = ServerStats()
        m = TFT_SERVE_BATCHED if mode == "batched" else TFT_SERVE_ONE_BY_ONE
        _check(load().tft_server_replay(
            self._h, reqs, n, int(seed), m,
            done.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            keep_arr, ctypes.byref(st)), "tft_server_replay")
        stats = {k: getattr(st, k) for k, _ in ServerStats._fields_}
        return done[:n], stats

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().tft_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
