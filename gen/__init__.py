"""Seeded synthetic string workloads (shared by the oracle tests, the GPU
tests and the benchmark).

This module holds no sorting arithmetic.  It compiles ``gen.c`` with gcc on
first use (or when the source is newer than the library) and exposes:

* :func:`generate` -- one set of ``n`` zero-terminated strings of a kind
  (1 uniform, 2 url-like, 3 dna; see ``gen.c``), returned as a byte buffer
  plus ``uint64`` start offsets, with 16 bytes of zero slack at the end;
* :data:`WORKLOADS` -- the named workloads the tests and the bench use;
* :func:`generate_batch` -- many independent sets for the batched sort;
* :func:`from_list` -- pack a Python list of ``bytes`` (no NUL inside) the
  same way, for hand-written cases.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsssgen.so")
_lock = threading.Lock()
_lib = None

# named workloads: kind, number of strings, seed
WORKLOADS = {
    "uniform-100k": dict(kind=1, n=100_000, seed=1),
    "url-16m": dict(kind=2, n=16_000_000, seed=2),
    "dna-20m": dict(kind=3, n=20_000_000, seed=3),
    "url-64m": dict(kind=2, n=64_000_000, seed=4),
}

# batched workloads, 10,000 sets each, kinds uniform, seed 5:
#   sets-literal  sizes log-uniform in [100, 1,000,000]
#                 (1,092,616,105 strings, about 51 GB of characters)
#   sets-10k      sizes log-uniform in [100, 4000]: about 500M characters in
#                 all
BATCH_WORKLOADS = {
    "sets-literal": dict(num_sets=10_000, lo=100, hi=1_000_000, seed=5),
    "sets-10k": dict(num_sets=10_000, lo=100, hi=4000, seed=5),
}

SLACK = 16


def build(force: bool = False) -> str:
    """Compile gen.c into libsssgen.so next to it; return the library path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                   "-std=gnu11", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.gen_lengths.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        lib.gen_fill.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u64p,
                                 ctypes.POINTER(ctypes.c_uint8), ctypes.c_int]
        lib.gen_uniform_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_uint64, u64p]
        lib.gen_uniform_f64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_double)]
        ip = ctypes.POINTER(ctypes.c_int)
        lib.gen_batch_lengths.argtypes = [ctypes.c_uint32, ip, u64p, u64p, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        lib.gen_batch_fill.argtypes = [ctypes.c_uint32, ip, u64p, u64p, ctypes.c_uint64, u64p,
                                       ctypes.POINTER(ctypes.c_uint8), ctypes.c_int]
        for f in (lib.gen_lengths, lib.gen_fill, lib.gen_uniform_u64, lib.gen_uniform_f64,
                  lib.gen_batch_lengths, lib.gen_batch_fill):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class Strings:
    """n zero-terminated strings: string i starts at chars[offsets[i]]."""
    chars: np.ndarray     # uint8, total bytes + SLACK zero bytes
    offsets: np.ndarray   # uint64[n]
    n: int
    total: int            # bytes of all strings, terminators included (N)

    def get(self, i: int) -> bytes:
        o = int(self.offsets[i])
        e = o
        while self.chars[e] != 0:
            e += 1
        return self.chars[o:e].tobytes()


def _threads(threads):
    return threads or max(1, min(64, os.cpu_count() or 1))


def generate(kind: int, n: int, seed: int, threads: int | None = None) -> Strings:
    """n strings of the given kind, laid out back to back in input order."""
    lib = _load()
    t = _threads(threads)
    lens = np.zeros(max(n, 1), dtype=np.uint32)
    if lib.gen_lengths(kind, n, seed, _ptr(lens, ctypes.c_uint32), t) != 0:
        raise RuntimeError("gen_lengths failed")
    lens = lens[:n]
    offsets = np.zeros(max(n, 1), dtype=np.uint64)
    if n > 1:
        np.cumsum(lens[:-1], dtype=np.uint64, out=offsets[1:n])
    offsets = offsets[:n]
    total = int(lens.sum(dtype=np.uint64))
    chars = np.zeros(total + SLACK, dtype=np.uint8)
    if n and lib.gen_fill(kind, n, seed, _ptr(offsets, ctypes.c_uint64),
                          _ptr(chars, ctypes.c_uint8), t) != 0:
        raise RuntimeError("gen_fill failed")
    return Strings(chars=chars, offsets=offsets, n=n, total=total)


def workload(name: str, n: int | None = None, threads: int | None = None) -> Strings:
    """A named workload, optionally truncated to its first n strings' generator
    streams (same kind and seed, smaller count)."""
    w = WORKLOADS[name]
    return generate(w["kind"], w["n"] if n is None else n, w["seed"], threads)


def from_list(items) -> Strings:
    """Pack a list of bytes objects (no NUL inside) as zero-terminated strings."""
    n = len(items)
    lens = np.array([len(s) + 1 for s in items], dtype=np.uint64)
    offsets = np.zeros(n, dtype=np.uint64)
    if n > 1:
        offsets[1:] = np.cumsum(lens[:-1])
    total = int(lens.sum()) if n else 0
    chars = np.zeros(total + SLACK, dtype=np.uint8)
    for i, s in enumerate(items):
        if b"\x00" in s:
            raise ValueError("strings may not contain NUL")
        o = int(offsets[i])
        chars[o:o + len(s)] = np.frombuffer(s, dtype=np.uint8) if s else []
    return Strings(chars=chars, offsets=offsets, n=n, total=total)


@dataclass
class Batch:
    """Independent string sets stored back to back.  Set j holds the strings
    with global index in [set_begin[j], set_begin[j+1])."""
    strings: Strings
    set_begin: np.ndarray   # uint64[num_sets + 1]
    kinds: np.ndarray       # int32[num_sets]


def batch_sizes(num_sets: int, lo: int, hi: int, seed: int):
    """Set sizes log-uniform in [lo, hi] and kinds uniform in {1,2,3}."""
    lib = _load()
    u = np.zeros(max(num_sets, 1), dtype=np.float64)
    k = np.zeros(max(num_sets, 1), dtype=np.uint64)
    lib.gen_uniform_f64(seed, 0x7500000000000000, num_sets, _ptr(u, ctypes.c_double))
    lib.gen_uniform_u64(seed, 0x7600000000000000, num_sets, 3, _ptr(k, ctypes.c_uint64))
    a, b = math.log(lo), math.log(hi + 1)
    sizes = np.minimum(np.floor(np.exp(a + u[:num_sets] * (b - a))), hi).astype(np.int64)
    return sizes, (k[:num_sets] + 1).astype(np.int32)


def generate_batch(num_sets: int, lo: int, hi: int, seed: int, threads: int | None = None) -> Batch:
    """num_sets independent sets, sizes log-uniform in [lo, hi], kinds uniform
    in {1,2,3}; set j draws its strings from its own streams (seed
    seed * 1000003 + j); the url pools and dna model come from `seed` and are
    shared by the sets of a kind."""
    lib = _load()
    sizes, kinds = batch_sizes(num_sets, lo, hi, seed)
    sizes = np.ascontiguousarray(sizes.astype(np.uint64))
    kinds = np.ascontiguousarray(kinds.astype(np.int32))
    seeds = np.ascontiguousarray((np.uint64(seed) * np.uint64(1_000_003) + np.arange(num_sets, dtype=np.uint64)))
    n = int(sizes.sum())
    t = _threads(threads)
    lens = np.zeros(max(n, 1), dtype=np.uint32)
    if lib.gen_batch_lengths(num_sets, _ptr(kinds, ctypes.c_int), _ptr(sizes, ctypes.c_uint64),
                             _ptr(seeds, ctypes.c_uint64), seed, _ptr(lens, ctypes.c_uint32), t) != 0:
        raise RuntimeError("gen_batch_lengths failed")
    lens = lens[:n]
    offsets = np.zeros(max(n, 1), dtype=np.uint64)
    if n > 1:
        np.cumsum(lens[:-1], dtype=np.uint64, out=offsets[1:n])
    offsets = offsets[:n]
    total = int(lens.sum(dtype=np.uint64))
    chars = np.zeros(total + SLACK, dtype=np.uint8)
    if n and lib.gen_batch_fill(num_sets, _ptr(kinds, ctypes.c_int), _ptr(sizes, ctypes.c_uint64),
                                _ptr(seeds, ctypes.c_uint64), seed, _ptr(offsets, ctypes.c_uint64),
                                _ptr(chars, ctypes.c_uint8), t) != 0:
        raise RuntimeError("gen_batch_fill failed")
    set_begin = np.zeros(num_sets + 1, dtype=np.uint64)
    set_begin[1:] = np.cumsum(sizes)
    return Batch(strings=Strings(chars=chars, offsets=offsets, n=n, total=total),
                 set_begin=set_begin, kinds=kinds)


def set_strings(b: Batch, j: int) -> Strings:
    """Set j of a batch as its own Strings (offsets rebased, shared chars)."""
    lo, hi = int(b.set_begin[j]), int(b.set_begin[j + 1])
    return Strings(chars=b.strings.chars, offsets=b.strings.offsets[lo:hi], n=hi - lo, total=0)
