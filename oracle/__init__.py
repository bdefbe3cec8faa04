"""CPU FP64 oracle for RRS projection depths.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark load this package; the GPU product path never does.  It
shares no code with the CUDA library (``paper_2506_08262_gb300``) and does not
import it.

``build()`` compiles ``rrs_oracle.c`` with gcc into ``oracle/_build``.  The
functions below are thin ctypes wrappers; every computation happens in the C
file, whose header lists the paper passages it follows and the readings taken
where the paper is silent or garbled.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rrs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librrs_oracle.so")
_lock = threading.Lock()
_lib = None

HALFSPACE, PROJECTION, ASYM_PROJECTION = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (plain C11, FP contraction off, OpenMP over queries)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fexcess-precision=standard", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.rrs_oracle_philox.argtypes = [P, P, P]
        lib.rrs_oracle_philox.restype = None
        lib.rrs_oracle_logf.argtypes = [ctypes.c_float]
        lib.rrs_oracle_logf.restype = ctypes.c_float
        lib.rrs_oracle_sincos_qturn.argtypes = [ctypes.c_float, P, P]
        lib.rrs_oracle_sincos_qturn.restype = None
        lib.rrs_oracle_directions.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_float, P, P]
        lib.rrs_oracle_directions.restype = ctypes.c_int
        lib.rrs_oracle_sign.argtypes = [P, P, P, ctypes.c_int32]
        lib.rrs_oracle_sign.restype = ctypes.c_int
        lib.rrs_oracle_univariate.argtypes = [ctypes.c_int32, P, ctypes.c_int64, ctypes.c_int32, P, P,
                                              P, P]
        lib.rrs_oracle_univariate.restype = ctypes.c_int
        lib.rrs_oracle_rrs.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int64, P,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_uint64, P, P, P, P, P, P, P, ctypes.c_int32]
        lib.rrs_oracle_rrs.restype = ctypes.c_int
        lib.rrs_oracle_max_threads.argtypes = []
        lib.rrs_oracle_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(counter, key) -> np.ndarray:
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().rrs_oracle_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def logf(a: float) -> np.float32:
    return np.float32(_load().rrs_oracle_logf(float(np.float32(a))))


def sincos_qturn(a: float):
    s = np.zeros(1, np.float32)
    c = np.zeros(1, np.float32)
    _load().rrs_oracle_sincos_qturn(float(np.float32(a)), _ptr(s), _ptr(c))
    return s[0], c[0]


def directions(seed: int, q: int, round0: int, m: int, d: int, alpha: float,
               pole: Optional[np.ndarray] = None) -> np.ndarray:
    """The m FP32 directions of round ``round0`` (0-based) for query ``q``."""
    if pole is None:
        pole = np.zeros(d, np.float32)
        pole[0] = 1.0
    pole = np.ascontiguousarray(pole, dtype=np.float32)
    U = np.zeros((m, d), np.float32)
    rc = _load().rrs_oracle_directions(seed, q, round0, m, d, float(np.float32(alpha)), _ptr(pole), _ptr(U))
    if rc != 0:
        raise ValueError("rrs_oracle_directions: invalid arguments")
    return U


def exact_sign(u: np.ndarray, x: np.ndarray, z: np.ndarray) -> int:
    u = np.ascontiguousarray(u, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    return int(_load().rrs_oracle_sign(_ptr(u), _ptr(x), _ptr(z), u.shape[0]))


def univariate(kind: int, X: np.ndarray, z: np.ndarray, u: np.ndarray):
    """Depth of z along one direction u: (depth, halfspace count or -1)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float32)
    dep = np.zeros(1, np.float64)
    cnt = np.zeros(1, np.int64)
    rc = _load().rrs_oracle_univariate(kind, _ptr(X), X.shape[0], X.shape[1], _ptr(z), _ptr(u),
                                       _ptr(dep), _ptr(cnt))
    if rc != 0:
        raise ValueError("rrs_oracle_univariate: invalid arguments")
    return float(dep[0]), int(cnt[0])


def rrs(X: np.ndarray, Z: np.ndarray, kind: int, k: int, r: int, alpha: float, seed: int = 0,
        qidx: Optional[np.ndarray] = None, follow: Optional[np.ndarray] = None,
        nthreads: Optional[int] = None, rounds: bool = False):
    """Refined random search depth of every row of Z w.r.t. X.

    Returns a dict with ``depth`` (nq,), ``count`` (nq,), ``best`` (nq,) and,
    with ``rounds=True`` or ``follow``, the per-round ``round_min``,
    ``round_arg`` and ``round_at_follow`` arrays (nq, r).
    """
    X = np.ascontiguousarray(X, dtype=np.float64)
    Z = np.ascontiguousarray(Z, dtype=np.float64).reshape(-1, X.shape[1])
    nq = Z.shape[0]
    lib = _load()
    if nthreads is None:
        nthreads = lib.rrs_oracle_max_threads()
    depth = np.zeros(nq, np.float64)
    count = np.zeros(nq, np.int64)
    best = np.zeros(nq, np.int32)
    want = rounds or follow is not None
    rmin = np.zeros((nq, r), np.float64) if want else None
    rarg = np.zeros((nq, r), np.int32) if want else None
    rfol = np.full((nq, r), np.nan) if follow is not None else None
    q = None if qidx is None else np.ascontiguousarray(qidx, dtype=np.int64)
    f = None if follow is None else np.ascontiguousarray(follow, dtype=np.int32).reshape(nq, r)
    rc = lib.rrs_oracle_rrs(_ptr(X), X.shape[0], X.shape[1], _ptr(Z), nq, _ptr(q), kind, k, r,
                            float(alpha), seed, _ptr(f), _ptr(depth), _ptr(count), _ptr(best),
                            _ptr(rmin), _ptr(rarg), _ptr(rfol), int(nthreads))
    if rc != 0:
        raise ValueError(f"rrs_oracle_rrs failed ({rc})")
    out = {"depth": depth, "count": count, "best": best}
    if want:
        out["round_min"] = rmin
        out["round_arg"] = rarg
    if follow is not None:
        out["round_at_follow"] = rfol
    return out


def max_threads() -> int:
    return int(_load().rrs_oracle_max_threads())
