"""ctypes front end of synth.c (built on first use with gcc -O2 -fopenmp)."""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

KIND = dict(F32_PM1=0, F32_01=1, F64_PM1=2, I32_U20=3, F32_NORMAL=4, F32_LOGNORMAL=5, F32_SIGN=6,
            I32_IOTA=7, ZERO32=8, ZERO64=9, RAW16=10, RAW32=11, RAW64=12)
_KIND_DTYPE = {0: np.float32, 1: np.float32, 2: np.float64, 3: np.int32, 4: np.float32, 5: np.float32,
               6: np.float32, 7: np.int32, 8: np.uint32, 9: np.uint64, 10: np.uint16, 11: np.uint32,
               12: np.uint64}


def build(force=False):
    """Compile libsynth.so next to synth.c when it is missing or older than the source."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_key.restype = ctypes.c_uint64
            lib.synth_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_u64.restype = ctypes.c_uint64
            lib.synth_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_unit.restype = ctypes.c_double
            lib.synth_unit.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_fill.restype = ctypes.c_int
            lib.synth_fill.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_void_p]
            lib.synth_perm_i32.restype = None
            lib.synth_perm_i32.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            _lib = lib
    return _lib


def key(seed, stream):
    return _get().synth_key(seed & (2**64 - 1), stream & (2**64 - 1))


def u64(k, i):
    return _get().synth_u64(k, i)


def unit(k, i):
    """Uniform double in [0,1) from value i of stream k."""
    return _get().synth_unit(k, i)


def fill(kind, k, n=None, i0=0, idx=None, out=None):
    """Values of stream k for counters i0..i0+n (or the int64 array idx), as a numpy array."""
    if isinstance(kind, str):
        kind = KIND[kind]
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        n = idx.shape[0]
    if out is None:
        out = np.empty(n, dtype=_KIND_DTYPE[kind])
    assert out.flags.c_contiguous and out.nbytes == n * np.dtype(_KIND_DTYPE[kind]).itemsize
    rc = _get().synth_fill(kind, k, None if idx is None else idx.ctypes.data, i0, n, out.ctypes.data)
    if rc != 0:
        raise ValueError("unknown synth kind %r" % kind)
    return out


def perm_i32(k, n):
    out = np.empty(n, dtype=np.int32)
    _get().synth_perm_i32(k, n, out.ctypes.data)
    return out
