"""ctypes wrapper around the plain-C oracle (``oracle/alg_c.c`` and the
served workload's generator ``oracle/gen_c.c``).

Test infrastructure only.  ``build()`` compiles the C file with gcc -O2 into
``oracle/_build/liborc.so`` (git-ignored); every function takes and returns
numpy uint64 arrays (elements of Z/p stored in 64 bits whatever the prime).
ctypes releases the GIL during each call, so Python threads can run several
oracle calls on separate host cores.
"""

import ctypes
import os
import subprocess

import numpy as np

from . import field as _f

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alg_c.c")
_SRCS = [_SRC, os.path.join(_HERE, "gen_c.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liborc.so")
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force=False):
    """Compile the C oracle (gcc -O2, no architecture-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and \
            all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp] + _SRCS)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_omega.restype = ctypes.c_uint64
        L.orc_omega.argtypes = [ctypes.c_int, ctypes.c_uint64]
        L.orc_omega_k.restype = ctypes.c_uint64
        L.orc_omega_k.argtypes = [ctypes.c_int, ctypes.c_int]
        for name in ("orc_alg1_tft", "orc_alg2_itft", "orc_fft_pow2"):
            fn = getattr(L, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [ctypes.c_int, _u64p, ctypes.c_uint64]
        L.orc_tft_polymul.restype = ctypes.c_int
        L.orc_tft_polymul.argtypes = [ctypes.c_int, _u64p, ctypes.c_uint64,
                                      _u64p, ctypes.c_uint64, _u64p, _u64p]
        L.orc_schoolbook.restype = ctypes.c_int
        L.orc_schoolbook.argtypes = [ctypes.c_int, _u64p, ctypes.c_uint64,
                                     _u64p, ctypes.c_uint64, _u64p]
        L.orc_eval.restype = ctypes.c_uint64
        L.orc_eval.argtypes = [ctypes.c_int, _u64p, ctypes.c_uint64,
                               ctypes.c_uint64]
        L.orc_conv_coeff.restype = ctypes.c_uint64
        L.orc_conv_coeff.argtypes = [ctypes.c_int, _u64p, ctypes.c_uint64,
                                     _u64p, ctypes.c_uint64, ctypes.c_uint64]
        L.orc_eval_tft_points.restype = ctypes.c_int
        L.orc_eval_tft_points.argtypes = [ctypes.c_int, _u64p, ctypes.c_uint64,
                                          _u64p, ctypes.c_uint64, _u64p]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32)]
        L.orc_gen_operand.restype = ctypes.c_int
        L.orc_gen_operand.argtypes = [ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_uint64, _u64p]
        _lib = L
    return _lib


def _pid(prime):
    return _f.PRIME_BY_ID.index(_f.get(prime))


def _as_u64(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    return a


def _ptr(a):
    return a.ctypes.data_as(_u64p)


def alg1_tft(prime, x):
    X = _as_u64(x).copy()
    rc = lib().orc_alg1_tft(_pid(prime), _ptr(X), X.size)
    if rc:
        raise ValueError(f"orc_alg1_tft failed ({rc})")
    return X


def alg2_itft(prime, X_hat):
    X = _as_u64(X_hat).copy()
    rc = lib().orc_alg2_itft(_pid(prime), _ptr(X), X.size)
    if rc:
        raise ValueError(f"orc_alg2_itft failed ({rc})")
    return X


def fft_pow2(prime, x):
    X = _as_u64(x).copy()
    rc = lib().orc_fft_pow2(_pid(prime), _ptr(X), X.size)
    if rc:
        raise ValueError(f"orc_fft_pow2 failed ({rc})")
    return X


def tft_polymul(prime, a, b):
    A = _as_u64(a)
    B = _as_u64(b)
    r = A.size + B.size - 1
    out = np.zeros(r, dtype=np.uint64)
    work = np.zeros(r, dtype=np.uint64)
    rc = lib().orc_tft_polymul(_pid(prime), _ptr(A), A.size, _ptr(B), B.size,
                               _ptr(out), _ptr(work))
    if rc:
        raise ValueError(f"orc_tft_polymul failed ({rc})")
    return out


def schoolbook(prime, a, b):
    A = _as_u64(a)
    B = _as_u64(b)
    out = np.zeros(A.size + B.size - 1, dtype=np.uint64)
    rc = lib().orc_schoolbook(_pid(prime), _ptr(A), A.size, _ptr(B), B.size,
                              _ptr(out))
    if rc:
        raise ValueError(f"orc_schoolbook failed ({rc})")
    return out


def eval_at(prime, x, z):
    X = _as_u64(x)
    return int(lib().orc_eval(_pid(prime), _ptr(X), X.size, int(z)))


def eval_tft_points(prime, x, points):
    """F(omega_s) for each s in ``points`` (the definition, by Horner)."""
    X = _as_u64(x)
    S = _as_u64(points)
    out = np.zeros(S.size, dtype=np.uint64)
    rc = lib().orc_eval_tft_points(_pid(prime), _ptr(X), X.size, _ptr(S),
                                   S.size, _ptr(out))
    if rc:
        raise ValueError("orc_eval_tft_points failed")
    return out


def conv_coeff(prime, a, b, t):
    """One coefficient c_t = sum_i a_i b_{t-i} of the product (definition)."""
    A = _as_u64(a)
    B = _as_u64(b)
    return int(lib().orc_conv_coeff(_pid(prime), _ptr(A), A.size, _ptr(B),
                                    B.size, int(t)))


def omega(prime, s):
    return int(lib().orc_omega(_pid(prime), int(s)))


def omega_k(prime, k):
    return int(lib().orc_omega_k(_pid(prime), int(k)))


def philox4x32_10(counter, key):
    """The four output words of Philox4x32-10 for a 4-word counter and a
    2-word key (the generator's definition, in plain C)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def gen_operand(prime, seed, request, operand, n):
    """Operand `operand` (0 = a, 1 = b) of served request `request`: n
    residues, element i = (Philox4x32-10 output as a 128-bit integer) mod p
    with counter (i, operand, request lo, request hi), key (seed lo, hi)."""
    out = np.zeros(int(n), dtype=np.uint64)
    rc = lib().orc_gen_operand(_pid(prime), int(seed), int(request),
                               int(operand), int(n), _ptr(out))
    if rc:
        raise ValueError("orc_gen_operand failed")
    return out
