"""Python binding of the kgpu C ABI (include/kgpu.h): GB300 page crypto.

This layer only marshals arguments (torch tensors / numpy arrays -> pointers and
sizes, torch streams -> cudaStream_t) and turns negative return codes into
exceptions.  Every byte of every transform is computed by the CUDA kernels in
libkgpu.so; there is no Python or CPU fallback -- if the library cannot be built
or loaded, every call raises.

The function names are those of the C ABI.  `Context` is a small convenience
wrapper that owns a kgpu_ctx.
"""
from __future__ import annotations

import ctypes
import itertools
import threading
import traceback

from . import build as _build

ENCRYPT = 0
DECRYPT = 1
MODE_XTS = 0
MODE_CBC_DEC = 1
MODE_CBC_ENC = 2
MODE_ECB = 3
MODE_COPY = 4  # the empty service: output = input, no key; unit_size = bytes per warp-tile

_ERRORS = {
    -5: "EIO", -7: "E2BIG", -12: "ENOMEM", -14: "EFAULT", -16: "EBUSY", -19: "ENODEV", -22: "EINVAL", -2: "ENOENT",
    -110: "ETIMEDOUT", -38: "ENOSYS",
}

DISPATCH_AUTO = 0
DISPATCH_GPU = 1
DISPATCH_HOST = 2
DISPATCH_FORM = {1: "launch", 2: "ring"}

_lock = threading.Lock()
_lib = None


class KgpuError(RuntimeError):
    def __init__(self, rc: int, what: str):
        self.rc = rc
        self.code = _ERRORS.get(rc, str(rc))
        super().__init__(f"{what} failed: {self.code} ({rc})")


class KgpuRequest(ctypes.Structure):
    """kgpu_request (include/kgpu.h)."""
    _fields_ = [("mode", ctypes.c_uint32), ("dir", ctypes.c_uint32), ("key", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("len", ctypes.c_uint64), ("unit_size", ctypes.c_uint64), ("sector", ctypes.c_uint64),
                ("ivs", ctypes.c_void_p)]


class KgpuTuning(ctypes.Structure):
    """kgpu_tuning (include/kgpu.h)."""
    _fields_ = [("threads", ctypes.c_uint32), ("tile_chunks", ctypes.c_uint32), ("ctas", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {"threads": self.threads, "tile_chunks": self.tile_chunks, "ctas": self.ctas}


# numpy view of an array of kgpu_request, for building large batches cheaply
REQUEST_DTYPE = None


def request_dtype():
    global REQUEST_DTYPE
    if REQUEST_DTYPE is None:
        import numpy as np
        REQUEST_DTYPE = np.dtype([("mode", "<u4"), ("dir", "<u4"), ("key", "<u4"), ("flags", "<u4"),
                                  ("src", "<u8"), ("dst", "<u8"), ("len", "<u8"), ("unit_size", "<u8"),
                                  ("sector", "<u8"), ("ivs", "<u8")])
        assert REQUEST_DTYPE.itemsize == ctypes.sizeof(KgpuRequest)
    return REQUEST_DTYPE


class KgpuServeConfig(ctypes.Structure):
    """kgpu_serve_config (include/kgpu.h)."""
    _fields_ = [("ring_slots", ctypes.c_uint32), ("tile_chunks", ctypes.c_uint32),
                ("admit_bytes", ctypes.c_uint64), ("idle_timeout_ns", ctypes.c_uint64),
                ("lifetime_ns", ctypes.c_uint64), ("reserved", ctypes.c_uint32 * 4)]


class KgpuServeStats(ctypes.Structure):
    """kgpu_serve_stats (include/kgpu.h)."""
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("busy_refusals", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("inflight_bytes", ctypes.c_uint64), ("running", ctypes.c_uint32),
                ("last_exit", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class KgpuConfig(ctypes.Structure):
    _fields_ = [("max_keys", ctypes.c_uint32), ("ring_slots", ctypes.c_uint32),
                ("admit_bytes", ctypes.c_uint64), ("idle_timeout_ns", ctypes.c_uint64),
                ("host_dispatch", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 7)]


class KgpuCrossover(ctypes.Structure):
    """kgpu_crossover: requests shorter than bytes[mode][0: AES-128, 1: AES-256] run on the host."""
    _fields_ = [("bytes", (ctypes.c_uint64 * 2) * 4), ("form", ctypes.c_uint32), ("valid", ctypes.c_uint32)]

    def as_dict(self):
        names = ("xts", "cbc_dec", "cbc_enc", "ecb")
        return {"valid": bool(self.valid), "form": DISPATCH_FORM.get(self.form),
                "bytes": {n: {"aes128": int(self.bytes[m][0]), "aes256": int(self.bytes[m][1])}
                          for m, n in enumerate(names)}}


class KgpuDispatchPoint(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("key_bits", ctypes.c_uint32), ("bytes", ctypes.c_uint64),
                ("host_ns", ctypes.c_uint64), ("gpu_ns", ctypes.c_uint64)]


def ensure_built() -> str:
    """Build libkgpu.so in-tree if it is missing or stale; return its path."""
    return _build.build()


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded C library (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(ensure_built())
            vp, sz, u64, i32, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
            sig = {
                "kgpu_version": ([], i32),
                "kgpu_strerror": ([i32], ctypes.c_char_p),
                "kgpu_init": ([ctypes.POINTER(vp), i32, vp], i32),
                "kgpu_destroy": ([vp], i32),
                "kgpu_aes_setkey": ([vp, vp, sz, i32, ctypes.POINTER(u32)], i32),
                "kgpu_aes_delkey": ([vp, u32], i32),
                "kgpu_aes_xts_crypt": ([vp, u32, i32, vp, vp, sz, sz, u64, vp], i32),
                "kgpu_aes_cbc_decrypt": ([vp, u32, vp, vp, sz, sz, vp, vp], i32),
                "kgpu_aes_cbc_encrypt_pages": ([vp, u32, vp, vp, sz, sz, vp, vp], i32),
                "kgpu_aes_ecb_crypt": ([vp, u32, i32, vp, vp, sz, vp], i32),
                "kgpu_aes_xts_crypt_host": ([vp, u32, i32, vp, vp, sz, sz, u64, sz], i32),
                "kgpu_submit": ([vp, vp, sz, vp, ctypes.POINTER(u64), vp], i32),
                "kgpu_poll": ([vp, u64, ctypes.c_int64, vp], i32),
                "kgpu_set_tuning": ([vp, ctypes.POINTER(KgpuTuning)], i32),
                "kgpu_get_tuning": ([vp, ctypes.POINTER(KgpuTuning)], i32),
                "kgpu_autotune": ([vp, vp, sz, vp, u32, ctypes.POINTER(KgpuTuning), ctypes.POINTER(ctypes.c_float)],
                                  i32),
                "kgpu_serve_start": ([vp, vp], i32),
                "kgpu_serve_submit": ([vp, vp, ctypes.POINTER(u64)], i32),
                "kgpu_serve_submit_cb": ([vp, vp, DONE_FN, vp, ctypes.POINTER(u64)], i32),
                "kgpu_serve_poll": ([vp, u64, ctypes.c_int64, vp, vp], i32),
                "kgpu_serve_stop": ([vp, ctypes.c_int64], i32),
                "kgpu_serve_get_stats": ([vp, ctypes.POINTER(KgpuServeStats)], i32),
                "kgpu_replay_serve": ([vp, vp, vp, sz, ctypes.c_int64, vp, ctypes.POINTER(u64), vp], i32),
                "kgpu_replay_launches": ([vp, vp, vp, sz, u32, ctypes.c_int64, vp, ctypes.POINTER(u64)], i32),
                "kgpu_submit_noalloc": ([vp, vp, sz, vp, vp], i32),
                "kgpu_host_register": ([vp, vp, sz, u32], i32),
                "kgpu_poll_each": ([vp, u64, ctypes.c_int64, vp, vp], i32),
                "kgpu_serve_submit_many": ([vp, vp, sz, vp, ctypes.POINTER(sz)], i32),
                "kgpu_aes_xts_crypt_bitsliced": ([vp, u32, i32, vp, vp, sz, sz, u64, vp], i32),
                "kgpu_host_unregister": ([vp, vp], i32),
                "kgpu_crypt": ([vp, vp, u32, ctypes.c_int64, ctypes.POINTER(u32)], i32),
                "kgpu_replay_serve_stages": ([vp, vp, vp, sz, ctypes.c_int64, vp, ctypes.POINTER(u64), vp,
                                              ctypes.POINTER(ctypes.c_int64)], i32),
                "kgpu_calibrate_dispatch": ([vp, vp, sz, ctypes.POINTER(sz), ctypes.POINTER(KgpuCrossover)], i32),
                "kgpu_get_crossover": ([vp, ctypes.POINTER(KgpuCrossover)], i32),
                "kgpu_bulk_wait_timeouts": ([vp, ctypes.POINTER(u32)], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise KgpuError(rc, what)
    return rc


def _dev_buf(t):
    """(pointer, nbytes) of a contiguous uint8 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch.Tensor")
    if t.dtype != torch.uint8 or not t.is_contiguous():
        raise TypeError("expected a contiguous uint8 tensor")
    return t.data_ptr(), t.numel()


def _host_buf(a):
    """(pointer, nbytes) of a contiguous uint8 host buffer (numpy or CPU tensor)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.uint8 or not a.is_contiguous():
                raise TypeError("expected a contiguous uint8 CPU tensor")
            return a.data_ptr(), a.numel()
    except ImportError:
        pass
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.uint8 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a contiguous uint8 numpy array")
    return a.ctypes.data, a.size


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------- C-ABI mirrors

def kgpu_version() -> int:
    return lib().kgpu_version()


def kgpu_strerror(code: int) -> str:
    return lib().kgpu_strerror(code).decode()


def kgpu_init(device: int = 0, cfg: KgpuConfig | None = None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().kgpu_init(ctypes.byref(ctx), device, ctypes.byref(cfg) if cfg is not None else None),
           "kgpu_init")
    return ctx


def kgpu_destroy(ctx) -> None:
    _check(lib().kgpu_destroy(ctx), "kgpu_destroy")


def kgpu_aes_setkey(ctx, key: bytes, xts: bool) -> int:
    h = ctypes.c_uint32()
    kb = ctypes.create_string_buffer(bytes(key), len(key))
    _check(lib().kgpu_aes_setkey(ctx, kb, len(key), 1 if xts else 0, ctypes.byref(h)), "kgpu_aes_setkey")
    return h.value


def kgpu_aes_delkey(ctx, key: int) -> None:
    _check(lib().kgpu_aes_delkey(ctx, key), "kgpu_aes_delkey")


def kgpu_aes_xts_crypt(ctx, key: int, dir: int, src, dst, du_size: int, first_sector: int = 0,
                       stream=None) -> None:
    sp, n = _dev_buf(src)
    dp, m = _dev_buf(dst)
    if n != m:
        raise ValueError("src and dst sizes differ")
    _check(lib().kgpu_aes_xts_crypt(ctx, key, dir, sp, dp, n, du_size, first_sector, _stream(stream)),
           "kgpu_aes_xts_crypt")


def kgpu_aes_xts_crypt_bitsliced(ctx, key: int, dir: int, src, dst, du_size: int, first_sector: int = 0,
                                 stream=None) -> None:
    sp, n = _dev_buf(src)
    dp, m = _dev_buf(dst)
    if n != m:
        raise ValueError("src and dst sizes differ")
    _check(lib().kgpu_aes_xts_crypt_bitsliced(ctx, key, dir, sp, dp, n, du_size, first_sector, _stream(stream)),
           "kgpu_aes_xts_crypt_bitsliced")


def kgpu_aes_cbc_decrypt(ctx, key: int, src, dst, page_size: int, ivs, stream=None) -> None:
    sp, n = _dev_buf(src)
    dp, m = _dev_buf(dst)
    ip, _ = _dev_buf(ivs)
    if n != m:
        raise ValueError("src and dst sizes differ")
    _check(lib().kgpu_aes_cbc_decrypt(ctx, key, sp, dp, n, page_size, ip, _stream(stream)),
           "kgpu_aes_cbc_decrypt")


def kgpu_aes_cbc_encrypt_pages(ctx, key: int, src, dst, page_size: int, ivs, stream=None) -> None:
    sp, n = _dev_buf(src)
    dp, m = _dev_buf(dst)
    ip, _ = _dev_buf(ivs)
    if n != m:
        raise ValueError("src and dst sizes differ")
    _check(lib().kgpu_aes_cbc_encrypt_pages(ctx, key, sp, dp, n, page_size, ip, _stream(stream)),
           "kgpu_aes_cbc_encrypt_pages")


def kgpu_aes_ecb_crypt(ctx, key: int, dir: int, src, dst, stream=None) -> None:
    sp, n = _dev_buf(src)
    dp, m = _dev_buf(dst)
    if n != m:
        raise ValueError("src and dst sizes differ")
    _check(lib().kgpu_aes_ecb_crypt(ctx, key, dir, sp, dp, n, _stream(stream)), "kgpu_aes_ecb_crypt")


def kgpu_aes_xts_crypt_host(ctx, key: int, dir: int, src, dst, du_size: int, first_sector: int = 0,
                            chunk_bytes: int = 0) -> None:
    sp, n = _host_buf(src)
    dp, m = _host_buf(dst)
    if n != m:
        raise ValueError("src and dst sizes differ")
    _check(lib().kgpu_aes_xts_crypt_host(ctx, key, dir, sp, dp, n, du_size, first_sector, chunk_bytes),
           "kgpu_aes_xts_crypt_host")


def _req_array(reqs):
    """(pointer, count, keepalive) of a batch given as a numpy array of
    request_dtype() or a sequence of KgpuRequest."""
    import numpy as np
    if isinstance(reqs, np.ndarray):
        if reqs.dtype != request_dtype() or not reqs.flags["C_CONTIGUOUS"]:
            raise TypeError("request array must be contiguous with request_dtype()")
        return reqs.ctypes.data, reqs.size, reqs
    arr = (KgpuRequest * len(reqs))(*reqs)
    return ctypes.addressof(arr), len(reqs), arr


def kgpu_submit(ctx, reqs, stream=None, status=None) -> int:
    """Submit a batch; returns the ticket.  status: optional int32 numpy array
    (len n) that receives each request's validation code."""
    ptr, n, keep = _req_array(reqs)
    t = ctypes.c_uint64()
    sp = status.ctypes.data if status is not None else None
    rc = lib().kgpu_submit(ctx, ptr, n, _stream(stream), ctypes.byref(t), sp)
    del keep
    _check(rc, "kgpu_submit")
    return t.value


def kgpu_poll(ctx, ticket: int, timeout_ns: int = -1, status=None) -> int:
    """0 when complete, KGPU_ETIMEDOUT (-110) while running; raises otherwise."""
    sp = status.ctypes.data if status is not None else None
    rc = lib().kgpu_poll(ctx, ticket, timeout_ns, sp)
    if rc == -110:
        return rc
    return _check(rc, "kgpu_poll")


def kgpu_poll_each(ctx, ticket: int, n: int, timeout_ns: int = -1, status=None):
    """Wait for every request of a batch; returns (rc, done_ns) with done_ns[i]
    the CLOCK_MONOTONIC time (ns, as time.monotonic_ns()) at which request i
    was seen complete."""
    import numpy as np
    done = np.zeros(n, dtype=np.uint64)
    sp = status.ctypes.data if status is not None else None
    rc = lib().kgpu_poll_each(ctx, ticket, timeout_ns, sp, done.ctypes.data)
    if rc not in (0, -110):
        _check(rc, "kgpu_poll_each")
    return rc, done


def kgpu_set_tuning(ctx, threads=0, tile_chunks=0, ctas=0) -> None:
    t = KgpuTuning(threads, tile_chunks, ctas, 0)
    _check(lib().kgpu_set_tuning(ctx, ctypes.byref(t)), "kgpu_set_tuning")


def kgpu_get_tuning(ctx) -> dict:
    t = KgpuTuning()
    _check(lib().kgpu_get_tuning(ctx, ctypes.byref(t)), "kgpu_get_tuning")
    return t.as_dict()


def kgpu_autotune(ctx, reqs, stream=None, iters: int = 3):
    """Returns (best tuning dict, mean ms of the best)."""
    ptr, n, keep = _req_array(reqs)
    best = KgpuTuning()
    ms = ctypes.c_float()
    rc = lib().kgpu_autotune(ctx, ptr, n, _stream(stream), iters, ctypes.byref(best), ctypes.byref(ms))
    del keep
    _check(rc, "kgpu_autotune")
    return best.as_dict(), ms.value


def kgpu_crypt(ctx, req, dispatch=DISPATCH_AUTO, timeout_ns: int = -1):
    """One request, run and waited for; returns (status, ran_on) where ran_on is
    DISPATCH_GPU or DISPATCH_HOST.  A negative status is the request's error."""
    ptr, n, keep = _req_array(req)
    if n != 1:
        raise ValueError("kgpu_crypt takes one request")
    ran = ctypes.c_uint32(0)
    rc = lib().kgpu_crypt(ctx, ptr, dispatch, timeout_ns, ctypes.byref(ran))
    del keep
    return rc, ran.value


def kgpu_calibrate_dispatch(ctx, max_points: int = 128):
    """Measure the CPU/GPU crossover now; returns (crossover dict, list of points)."""
    pts = (KgpuDispatchPoint * max_points)()
    n = ctypes.c_size_t(0)
    xo = KgpuCrossover()
    _check(lib().kgpu_calibrate_dispatch(ctx, pts, max_points, ctypes.byref(n), ctypes.byref(xo)),
           "kgpu_calibrate_dispatch")
    names = ("xts", "cbc_dec", "cbc_enc", "ecb")
    points = [{"mode": names[p.mode], "key_bits": p.key_bits, "bytes": p.bytes, "host_ns": p.host_ns,
               "gpu_ns": p.gpu_ns} for p in pts[: n.value]]
    return xo.as_dict(), points


def kgpu_get_crossover(ctx) -> dict:
    xo = KgpuCrossover()
    _check(lib().kgpu_get_crossover(ctx, ctypes.byref(xo)), "kgpu_get_crossover")
    return xo.as_dict()


NOALLOC_MAX_REQUESTS = 512


def kgpu_submit_noalloc(ctx, reqs, stream=None, status=None) -> None:
    """Allocation-free batched submission (queued on `stream`; synchronise on it)."""
    ptr, n, keep = _req_array(reqs)
    sp = status.ctypes.data if status is not None else None
    rc = lib().kgpu_submit_noalloc(ctx, ptr, n, _stream(stream), sp)
    del keep
    _check(rc, "kgpu_submit_noalloc")


HOSTREG_PIN = 0
HOSTREG_PINNED = 1
REQ_SRC_HOST = 0x1
REQ_DST_HOST = 0x2
REQ_IVS_HOST = 0x4


def _host_span(buf, nbytes=None):
    """(address, bytes) of a host buffer: a CPU tensor, a numpy array, or an
    integer address with nbytes."""
    if isinstance(buf, int):
        if nbytes is None:
            raise ValueError("an address needs nbytes")
        return buf, int(nbytes)
    if hasattr(buf, "data_ptr"):
        if buf.is_cuda:
            raise ValueError("host registration takes host memory")
        return buf.data_ptr(), buf.numel() * buf.element_size()
    return buf.ctypes.data, buf.nbytes


def kgpu_host_register(ctx, buf, nbytes=None, flags=HOSTREG_PINNED) -> None:
    ptr, n = _host_span(buf, nbytes)
    _check(lib().kgpu_host_register(ctx, ptr, n, flags), "kgpu_host_register")


def kgpu_host_unregister(ctx, buf) -> None:
    ptr = buf if isinstance(buf, int) else _host_span(buf)[0]
    _check(lib().kgpu_host_unregister(ctx, ptr), "kgpu_host_unregister")


def kgpu_serve_start(ctx, ring_slots=0, tile_chunks=0, admit_bytes=0, idle_timeout_ns=0, lifetime_ns=0) -> None:
    cfg = KgpuServeConfig(ring_slots, tile_chunks, admit_bytes, idle_timeout_ns, lifetime_ns)
    _check(lib().kgpu_serve_start(ctx, ctypes.byref(cfg)), "kgpu_serve_start")


def kgpu_serve_submit(ctx, req) -> int:
    """Publish one request (a KgpuRequest or a record of request_dtype()).
    Returns the ticket; raises KgpuError (code EBUSY when refused: retry)."""
    import numpy as np
    if isinstance(req, np.ndarray) or isinstance(req, np.void):
        arr = np.ascontiguousarray(np.asarray(req, dtype=request_dtype()).reshape(1))
        ptr = arr.ctypes.data
        keep = arr
    else:
        keep = req
        ptr = ctypes.addressof(req)
    t = ctypes.c_uint64()
    rc = lib().kgpu_serve_submit(ctx, ptr, ctypes.byref(t))
    del keep
    _check(rc, "kgpu_serve_submit")
    return t.value


# kgpu_done_fn: void (*)(void *arg, kgpu_ticket ticket, int status)
DONE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int)
_done_callables = {}  # token passed as arg -> the Python callable, until it has run
_done_tokens = itertools.count(1)


def _done_trampoline(arg, ticket, status):
    fn = _done_callables.pop(arg, None)
    if fn is not None:
        try:
            fn(int(ticket), int(status))
        except BaseException:  # nothing can propagate into the library's thread
            traceback.print_exc()


_done_c = DONE_FN(_done_trampoline)


def kgpu_serve_submit_cb(ctx, req, fn) -> int:
    """Publish one request with a completion callback: fn(ticket, status) is
    called once, on the library's completion thread, when it completes (status
    0 or a negative KGPU_E* code).  Returns the ticket; raises KgpuError like
    kgpu_serve_submit, in which case fn is never called."""
    import numpy as np
    if isinstance(req, np.ndarray) or isinstance(req, np.void):
        arr = np.ascontiguousarray(np.asarray(req, dtype=request_dtype()).reshape(1))
        ptr = arr.ctypes.data
        keep = arr
    else:
        keep = req
        ptr = ctypes.addressof(req)
    token = next(_done_tokens)
    _done_callables[token] = fn
    t = ctypes.c_uint64()
    rc = lib().kgpu_serve_submit_cb(ctx, ptr, _done_c, token, ctypes.byref(t))
    del keep
    if rc not in (0, -5):  # on KGPU_EIO (-5) the request was published and fn will run
        _done_callables.pop(token, None)
    _check(rc, "kgpu_serve_submit_cb")
    return t.value


def kgpu_serve_submit_many(ctx, reqs):
    """Publish a batch of requests onto the ring in one burst; returns (rc,
    tickets of the accepted prefix).  rc is 0, or KGPU_EBUSY (-16) when the
    ring stopped the rest; other errors raise."""
    import numpy as np
    ptr, n, keep = _req_array(reqs)
    tickets = np.zeros(n, dtype=np.uint64)
    acc = ctypes.c_size_t()
    rc = lib().kgpu_serve_submit_many(ctx, ptr, n, tickets.ctypes.data, ctypes.byref(acc))
    del keep
    if rc not in (0, -16):
        _check(rc, "kgpu_serve_submit_many")
    return rc, tickets[: acc.value]


def kgpu_serve_poll(ctx, ticket: int, timeout_ns: int = -1):
    """(rc, status, (t_first_tile, t_done)) -- rc 0 when complete, -110 while pending."""
    st = ctypes.c_int()
    stamps = (ctypes.c_uint64 * 2)()
    rc = lib().kgpu_serve_poll(ctx, ticket, timeout_ns, ctypes.byref(st), stamps)
    if rc not in (0, -110):
        _check(rc, "kgpu_serve_poll")
    return rc, st.value, (stamps[0], stamps[1])


def kgpu_serve_stop(ctx, drain_timeout_ns: int = -1) -> int:
    rc = lib().kgpu_serve_stop(ctx, drain_timeout_ns)
    if rc not in (0, -110):
        _check(rc, "kgpu_serve_stop")
    return rc


def kgpu_serve_get_stats(ctx) -> dict:
    s = KgpuServeStats()
    _check(lib().kgpu_serve_get_stats(ctx, ctypes.byref(s)), "kgpu_serve_get_stats")
    return s.as_dict()


def _replay(fn, ctx, reqs, arrival_ns, extra, timeout_ns, detail=None):
    import numpy as np
    ptr, n, keep = _req_array(reqs)
    arr = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
    lat = np.zeros(n, dtype=np.uint64)
    wall = ctypes.c_uint64()
    tail = (detail.ctypes.data,) if detail is not None else ()
    rc = fn(ctx, ptr, arr.ctypes.data, n, *extra, timeout_ns, lat.ctypes.data, ctypes.byref(wall), *tail)
    del keep
    return rc, lat, wall.value


def kgpu_replay_serve(ctx, reqs, arrival_ns, timeout_ns: int = 60_000_000_000, detail=None):
    """Open-loop replay through the serving ring: (rc, latency_ns array, wall_ns).
    detail: optional uint64 array of 3*n (host wait before publish, device
    first-tile stamp, device completion stamp)."""
    import numpy as np
    if detail is None:
        detail = np.zeros(3 * (len(reqs)), dtype=np.uint64)
    return _replay(lib().kgpu_replay_serve, ctx, reqs, arrival_ns, (), timeout_ns, detail)


STAGE_NAMES = ("published", "dispatcher_took", "tiles_published", "first_tile", "completed", "seen")
STAGE_LOST = -(1 << 63)


def kgpu_replay_serve_stages(ctx, reqs, arrival_ns, timeout_ns: int = 60_000_000_000):
    """Replay through the serving ring with each request's latency split by
    stage: (rc, latency_ns, wall_ns, stages, (clock offset before, after)) where stages is
    an int64 (n, 6) array of ns since arrival (STAGE_NAMES; STAGE_LOST where a
    device stamp was lost)."""
    import numpy as np
    ptr, n, keep = _req_array(reqs)
    arr = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
    lat = np.zeros(n, dtype=np.uint64)
    stages = np.zeros((n, 6), dtype=np.int64)
    wall = ctypes.c_uint64()
    off = (ctypes.c_int64 * 2)()
    rc = lib().kgpu_replay_serve_stages(ctx, ptr, arr.ctypes.data, n, timeout_ns, lat.ctypes.data,
                                        ctypes.byref(wall), stages.ctypes.data, off)
    del keep
    return rc, lat, wall.value, stages, (off[0], off[1])


def kgpu_replay_launches(ctx, reqs, arrival_ns, nstreams: int = 8, timeout_ns: int = 60_000_000_000):
    """Open-loop replay with one kernel launch per request: (rc, latency_ns, wall_ns)."""
    return _replay(lib().kgpu_replay_launches, ctx, reqs, arrival_ns, (nstreams,), timeout_ns)


class Context:
    """Owns one kgpu_ctx on a device; methods mirror the C ABI without the ctx."""

    def __init__(self, device: int = 0, cfg: KgpuConfig | None = None):
        self.device = device
        self.handle = kgpu_init(device, cfg)

    def close(self):
        if self.handle is not None and self.handle.value:
            kgpu_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setkey(self, key: bytes, xts: bool) -> int:
        return kgpu_aes_setkey(self.handle, key, xts)

    def delkey(self, key: int) -> None:
        kgpu_aes_delkey(self.handle, key)

    def xts_crypt(self, key, dir, src, dst, du_size, first_sector=0, stream=None):
        kgpu_aes_xts_crypt(self.handle, key, dir, src, dst, du_size, first_sector, stream)

    def xts_crypt_bitsliced(self, key, dir, src, dst, du_size, first_sector=0, stream=None):
        kgpu_aes_xts_crypt_bitsliced(self.handle, key, dir, src, dst, du_size, first_sector, stream)

    def cbc_decrypt(self, key, src, dst, page_size, ivs, stream=None):
        kgpu_aes_cbc_decrypt(self.handle, key, src, dst, page_size, ivs, stream)

    def cbc_encrypt_pages(self, key, src, dst, page_size, ivs, stream=None):
        kgpu_aes_cbc_encrypt_pages(self.handle, key, src, dst, page_size, ivs, stream)

    def ecb_crypt(self, key, dir, src, dst, stream=None):
        kgpu_aes_ecb_crypt(self.handle, key, dir, src, dst, stream)

    def xts_crypt_host(self, key, dir, src, dst, du_size, first_sector=0, chunk_bytes=0):
        kgpu_aes_xts_crypt_host(self.handle, key, dir, src, dst, du_size, first_sector, chunk_bytes)

    def submit(self, reqs, stream=None, status=None) -> int:
        return kgpu_submit(self.handle, reqs, stream, status)

    def poll(self, ticket, timeout_ns=-1, status=None) -> int:
        return kgpu_poll(self.handle, ticket, timeout_ns, status)

    def set_tuning(self, threads=0, tile_chunks=0, ctas=0):
        kgpu_set_tuning(self.handle, threads, tile_chunks, ctas)

    def poll_each(self, ticket, n, timeout_ns=-1, status=None):
        return kgpu_poll_each(self.handle, ticket, n, timeout_ns, status)

    def get_tuning(self) -> dict:
        return kgpu_get_tuning(self.handle)

    def autotune(self, reqs, stream=None, iters=3):
        return kgpu_autotune(self.handle, reqs, stream, iters)

    def crypt(self, req, dispatch=DISPATCH_AUTO, timeout_ns=-1):
        return kgpu_crypt(self.handle, req, dispatch, timeout_ns)

    def calibrate_dispatch(self, max_points=128):
        return kgpu_calibrate_dispatch(self.handle, max_points)

    def crossover(self) -> dict:
        return kgpu_get_crossover(self.handle)

    def submit_noalloc(self, reqs, stream=None, status=None):
        kgpu_submit_noalloc(self.handle, reqs, stream, status)

    def host_register(self, buf, nbytes=None, flags=HOSTREG_PINNED):
        kgpu_host_register(self.handle, buf, nbytes, flags)

    def host_unregister(self, buf):
        kgpu_host_unregister(self.handle, buf)

    def serve_start(self, **kw):
        kgpu_serve_start(self.handle, **kw)

    def serve_submit_many(self, reqs):
        return kgpu_serve_submit_many(self.handle, reqs)

    def serve_submit(self, req) -> int:
        return kgpu_serve_submit(self.handle, req)

    def bulk_wait_timeouts(self) -> int:
        n = ctypes.c_uint32()
        _check(lib().kgpu_bulk_wait_timeouts(self.handle, ctypes.byref(n)), "kgpu_bulk_wait_timeouts")
        return n.value

    def serve_submit_cb(self, req, fn) -> int:
        return kgpu_serve_submit_cb(self.handle, req, fn)

    def serve_poll(self, ticket, timeout_ns=-1):
        return kgpu_serve_poll(self.handle, ticket, timeout_ns)

    def serve_stop(self, drain_timeout_ns=-1):
        return kgpu_serve_stop(self.handle, drain_timeout_ns)

    def serve_stats(self) -> dict:
        return kgpu_serve_get_stats(self.handle)

    def replay_serve(self, reqs, arrival_ns, timeout_ns=60_000_000_000, detail=None):
        return kgpu_replay_serve(self.handle, reqs, arrival_ns, timeout_ns, detail)

    def replay_serve_stages(self, reqs, arrival_ns, timeout_ns=60_000_000_000):
        return kgpu_replay_serve_stages(self.handle, reqs, arrival_ns, timeout_ns)

    def replay_launches(self, reqs, arrival_ns, nstreams=8, timeout_ns=60_000_000_000):
        return kgpu_replay_launches(self.handle, reqs, arrival_ns, nstreams, timeout_ns)
