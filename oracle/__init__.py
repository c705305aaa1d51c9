"""CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The GPU library shares no code with it.

Each function wraps the plain C definition in ``oracle.c`` (compiled with gcc
on first use): multikey quicksort with index tie-break (Sec. 2.1), the direct
LCP scan (Sec. 2), the output check (App. B.1), the distinguishing prefix
size D (Sec. 2), and the per-step definitions of S^5 (Sec. 3.1): key word,
classification with equality buckets, splitter selection; plus the learned
CDF model's forward pass, loss and gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

VERIFY_CODES = {0: "ok", 1: "not a permutation", 2: "order violated",
                3: "equal strings not in index order", 4: "lcp wrong", -2: "out of memory"}


def build(force: bool = False) -> str:
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-std=gnu11",
                            _SRC, "-o", tmp, "-lm"], check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        u8p, u32p, u64p, dp = P(ctypes.c_uint8), P(ctypes.c_uint32), P(ctypes.c_uint64), P(ctypes.c_double)
        lib.oracle_sort.argtypes = [u8p, u64p, ctypes.c_uint32, u32p]
        lib.oracle_sort.restype = ctypes.c_int
        lib.oracle_sort_parallel.argtypes = [u8p, u64p, ctypes.c_uint32, u32p, u32p, ctypes.c_int]
        lib.oracle_sort_parallel.restype = ctypes.c_int
        lib.oracle_lcp_scan.argtypes = [u8p, u64p, ctypes.c_uint32, u32p, u32p]
        lib.oracle_lcp_scan.restype = None
        lib.oracle_verify.argtypes = [u8p, u64p, ctypes.c_uint32, u32p, u32p, u64p]
        lib.oracle_verify.restype = ctypes.c_int
        lib.oracle_dist_prefix.argtypes = [u8p, u64p, ctypes.c_uint32, u32p, u32p]
        lib.oracle_dist_prefix.restype = ctypes.c_uint64
        lib.oracle_key_word.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_key_word.restype = ctypes.c_uint64
        lib.oracle_classify.argtypes = [ctypes.c_uint64, u64p, ctypes.c_uint32]
        lib.oracle_classify.restype = ctypes.c_uint32
        lib.oracle_select_splitters.argtypes = [u64p, ctypes.c_int64, ctypes.c_int, u64p, u64p]
        lib.oracle_select_splitters.restype = ctypes.c_int
        lib.oracle_cdf_forward.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_cdf_forward.restype = None
        lib.oracle_cdf_loss.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_int]
        lib.oracle_cdf_loss.restype = ctypes.c_double
        lib.oracle_cdf_grad.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_int, dp]
        lib.oracle_cdf_grad.restype = None
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def sort(chars, offsets, n=None):
    """Sorted permutation (ties by original index) and LCP array."""
    lib = _load()
    chars = _c(chars, np.uint8)
    offsets = _c(offsets, np.uint64)
    n = len(offsets) if n is None else n
    perm = np.zeros(max(n, 1), dtype=np.uint32)
    lcp = np.zeros(max(n, 1), dtype=np.uint32)
    if lib.oracle_sort(_p(chars, ctypes.c_uint8), _p(offsets, ctypes.c_uint64), n,
                       _p(perm, ctypes.c_uint32)) != 0:
        raise MemoryError("oracle_sort")
    lib.oracle_lcp_scan(_p(chars, ctypes.c_uint8), _p(offsets, ctypes.c_uint64), n,
                        _p(perm, ctypes.c_uint32), _p(lcp, ctypes.c_uint32))
    return perm[:n], lcp[:n]


def sort_parallel(chars, offsets, threads: int, n=None):
    """The same (perm, lcp) as sort(), from independent ranges sorted on
    `threads` host threads (a timing baseline)."""
    lib = _load()
    chars = _c(chars, np.uint8)
    offsets = _c(offsets, np.uint64)
    n = len(offsets) if n is None else n
    perm = np.zeros(max(n, 1), dtype=np.uint32)
    lcp = np.zeros(max(n, 1), dtype=np.uint32)
    if lib.oracle_sort_parallel(_p(chars, ctypes.c_uint8), _p(offsets, ctypes.c_uint64), n,
                                _p(perm, ctypes.c_uint32), _p(lcp, ctypes.c_uint32), int(threads)) != 0:
        raise MemoryError("oracle_sort_parallel")
    return perm[:n], lcp[:n]


def lcp_scan(chars, offsets, perm):
    lib = _load()
    chars, offsets, perm = _c(chars, np.uint8), _c(offsets, np.uint64), _c(perm, np.uint32)
    n = len(perm)
    lcp = np.zeros(max(n, 1), dtype=np.uint32)
    lib.oracle_lcp_scan(_p(chars, ctypes.c_uint8), _p(offsets, ctypes.c_uint64), n,
                        _p(perm, ctypes.c_uint32), _p(lcp, ctypes.c_uint32))
    return lcp[:n]


def verify(chars, offsets, perm, lcp=None):
    """(code, first bad rank); code 0 means the answer is the unique correct one."""
    lib = _load()
    chars, offsets, perm = _c(chars, np.uint8), _c(offsets, np.uint64), _c(perm, np.uint32)
    n = len(perm)
    bad = np.zeros(1, dtype=np.uint64)
    lcp_arr = None if lcp is None else _c(lcp, np.uint32)
    lp = None if lcp_arr is None else _p(lcp_arr, ctypes.c_uint32)
    code = lib.oracle_verify(_p(chars, ctypes.c_uint8), _p(offsets, ctypes.c_uint64), n,
                             _p(perm, ctypes.c_uint32), lp, _p(bad, ctypes.c_uint64))
    return code, int(bad[0])


def dist_prefix(chars, offsets, perm, lcp) -> int:
    lib = _load()
    chars, offsets = _c(chars, np.uint8), _c(offsets, np.uint64)
    perm, lcp = _c(perm, np.uint32), _c(lcp, np.uint32)
    return int(lib.oracle_dist_prefix(_p(chars, ctypes.c_uint8), _p(offsets, ctypes.c_uint64),
                                      len(perm), _p(perm, ctypes.c_uint32), _p(lcp, ctypes.c_uint32)))


def key_word(chars, offset: int, depth: int) -> int:
    lib = _load()
    chars = _c(chars, np.uint8)
    return int(lib.oracle_key_word(_p(chars, ctypes.c_uint8), offset, depth))


def classify(key: int, splitters) -> int:
    lib = _load()
    x = _c(splitters, np.uint64)
    return int(lib.oracle_classify(key, _p(x, ctypes.c_uint64), len(x)))


def select_splitters(sorted_sample, k: int):
    """(level_order, in_order) arrays of v = 2^k - 1 splitters."""
    lib = _load()
    s = _c(sorted_sample, np.uint64)
    v = (1 << k) - 1
    level = np.zeros(v, dtype=np.uint64)
    ino = np.zeros(v, dtype=np.uint64)
    if lib.oracle_select_splitters(_p(s, ctypes.c_uint64), len(s), k, _p(level, ctypes.c_uint64),
                                   _p(ino, ctypes.c_uint64)) != 0:
        raise ValueError("bad sample or k")
    return level, ino


def cdf_forward(theta, u):
    lib = _load()
    theta, u = _c(theta, np.float64), _c(u, np.float64)
    F = np.zeros(max(len(u), 1), dtype=np.float64)
    lib.oracle_cdf_forward(_p(theta, ctypes.c_double), len(theta), _p(u, ctypes.c_double), len(u),
                           _p(F, ctypes.c_double))
    return F[:len(u)]


def cdf_loss(theta, u, y) -> float:
    lib = _load()
    theta, u, y = _c(theta, np.float64), _c(u, np.float64), _c(y, np.float64)
    return float(lib.oracle_cdf_loss(_p(theta, ctypes.c_double), len(theta), _p(u, ctypes.c_double),
                                     _p(y, ctypes.c_double), len(u)))


def cdf_grad(theta, u, y):
    lib = _load()
    theta, u, y = _c(theta, np.float64), _c(u, np.float64), _c(y, np.float64)
    g = np.zeros(len(theta), dtype=np.float64)
    lib.oracle_cdf_grad(_p(theta, ctypes.c_double), len(theta), _p(u, ctypes.c_double),
                        _p(y, ctypes.c_double), len(u), _p(g, ctypes.c_double))
    return g
