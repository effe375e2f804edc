"""CPU oracle for the AES page-crypto path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The product library never calls it; the two share no
code.  The arithmetic lives in `aes_oracle.c` (plain C from FIPS-197, IEEE 1619
and NIST SP 800-38A); this module only compiles it with gcc on first use and
marshals numpy buffers into it.

All byte buffers are numpy uint8 arrays; results are new arrays unless `out` is
given (which may alias the input: every mode supports in-place operation).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aes_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile aes_oracle.c into oracle/_build/liboracle.so (plain gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.c_void_p
            lib.oracle_gf_mul.argtypes = [ctypes.c_uint8, ctypes.c_uint8]
            lib.oracle_gf_mul.restype = ctypes.c_uint8
            lib.oracle_gf_inv.argtypes = [ctypes.c_uint8]
            lib.oracle_gf_inv.restype = ctypes.c_uint8
            lib.oracle_sbox.argtypes = [u8p]
            lib.oracle_inv_sbox.argtypes = [u8p]
            lib.oracle_key_expansion.argtypes = [u8p, ctypes.c_int, u8p]
            lib.oracle_key_expansion.restype = ctypes.c_int
            lib.oracle_mix_column.argtypes = [u8p]
            lib.oracle_inv_mix_column.argtypes = [u8p]
            lib.oracle_block.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, u8p]
            lib.oracle_block.restype = ctypes.c_int
            lib.oracle_xts_mul_alpha.argtypes = [u8p]
            lib.oracle_xts.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_size_t,
                                       ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int]
            lib.oracle_xts.restype = ctypes.c_int
            lib.oracle_cbc.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_size_t,
                                       ctypes.c_size_t, u8p, ctypes.c_int]
            lib.oracle_cbc.restype = ctypes.c_int
            lib.oracle_ecb.argtypes = [u8p, ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_size_t,
                                       ctypes.c_int]
            lib.oracle_ecb.restype = ctypes.c_int
            _lib = lib
    return _lib


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _buf(x) -> np.ndarray:
    a = np.ascontiguousarray(np.frombuffer(x, dtype=np.uint8) if isinstance(x, (bytes, bytearray)) else x)
    if a.dtype != np.uint8:
        raise TypeError("byte buffers must be uint8")
    return a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleError(ValueError):
    pass


def _check(rc: int):
    if rc < 0:
        raise OracleError(f"oracle rejected the arguments (rc={rc})")
    return rc


# --- field and cipher pieces (FIPS-197 sections 4 and 5), exposed for pins ---

def gf_mul(a: int, b: int) -> int:
    return _load().oracle_gf_mul(a, b)


def gf_inv(a: int) -> int:
    return _load().oracle_gf_inv(a)


def sbox() -> np.ndarray:
    out = np.zeros(256, np.uint8)
    _load().oracle_sbox(_ptr(out))
    return out


def inv_sbox() -> np.ndarray:
    out = np.zeros(256, np.uint8)
    _load().oracle_inv_sbox(_ptr(out))
    return out


def key_expansion(key: bytes) -> np.ndarray:
    """FIPS-197 5.2: returns the (Nr+1)*4 words as a (4*(Nr+1), 4) byte array."""
    k = _buf(key)
    out = np.zeros(240, np.uint8)
    nr = _check(_load().oracle_key_expansion(_ptr(k), len(k), _ptr(out)))
    return out[:16 * (nr + 1)].reshape(4 * (nr + 1), 4)


def mix_column(col) -> np.ndarray:
    c = np.array(col, dtype=np.uint8).copy()
    _load().oracle_mix_column(_ptr(c))
    return c


def inv_mix_column(col) -> np.ndarray:
    c = np.array(col, dtype=np.uint8).copy()
    _load().oracle_inv_mix_column(_ptr(c))
    return c


def block(key: bytes, dir: int, blk) -> bytes:
    k = _buf(key)
    x = _buf(blk)
    assert x.size == 16
    y = np.zeros(16, np.uint8)
    _check(_load().oracle_block(_ptr(k), len(k), dir, _ptr(x), _ptr(y)))
    return y.tobytes()


def xts_mul_alpha(t) -> bytes:
    a = np.array(_buf(t), dtype=np.uint8).copy()
    _load().oracle_xts_mul_alpha(_ptr(a))
    return a.tobytes()


# --- page modes ---

def xts(key: bytes, dir: int, data, du: int, first_sector: int = 0, out=None,
        nthreads: int | None = None) -> np.ndarray:
    """IEEE 1619 XTS-AES over len(data)/du data units numbered first_sector, ...
    key = Key1 || Key2 (32 bytes: AES-128, 64 bytes: AES-256)."""
    k = _buf(key)
    src = _buf(data)
    dst = np.empty_like(src) if out is None else out
    _check(_load().oracle_xts(_ptr(k), len(k), dir, _ptr(src), _ptr(dst), src.size, du,
                              first_sector, nthreads or default_threads()))
    return dst


def cbc(key: bytes, dir: int, data, page: int, ivs, out=None, nthreads: int | None = None) -> np.ndarray:
    """NIST SP 800-38A CBC, one chain per page with its own IV (ivs: npages x 16)."""
    k = _buf(key)
    src = _buf(data)
    iv = np.ascontiguousarray(ivs, dtype=np.uint8).reshape(-1)
    if page <= 0 or src.size % page or iv.size != 16 * (src.size // page):
        raise OracleError("bad CBC geometry")
    dst = np.empty_like(src) if out is None else out
    _check(_load().oracle_cbc(_ptr(k), len(k), dir, _ptr(src), _ptr(dst), src.size, page, _ptr(iv),
                              nthreads or default_threads()))
    return dst


def ecb(key: bytes, dir: int, data, out=None, nthreads: int | None = None) -> np.ndarray:
    k = _buf(key)
    src = _buf(data)
    dst = np.empty_like(src) if out is None else out
    _check(_load().oracle_ecb(_ptr(k), len(k), dir, _ptr(src), _ptr(dst), src.size,
                              nthreads or default_threads()))
    return dst
