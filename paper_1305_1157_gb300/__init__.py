"""Python binding of libsss.so, the GB300 string sample sort library.

Thin ctypes marshalling over the C ABI declared in ``include/sss.h``: the
functions keep the C names and arguments.  Every array argument accepts a
``torch.Tensor`` (its ``data_ptr()`` is passed), a NumPy array (for host
pointers) or a raw integer address.  Streams accept a ``torch.cuda.Stream``,
a raw handle or ``None`` (the current torch stream when torch is loaded,
else the legacy default stream).  Non-zero status codes raise
:class:`SSSError` with the library's message.

All sorting work runs in the CUDA kernels of libsss.so; nothing here
computes.  If the library is missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "SSSError", "sss_sort", "sss_sort_ws", "sss_sort_noalloc", "sss_sort_host", "sss_sort_batched", "sss_sort_learned",
    "sss_workspace_size", "sss_gather_keys", "sss_build_splitters", "sss_classify", "sss_classify_equal",
    "sss_cdf_loss_grad",
    "sss_set_options", "sss_get_options", "sss_get_last_stats", "sss_get_last_timeline", "sss_last_error",
    "sss_release",
    "sss_version", "sss_options", "sss_stats", "sss_learned_stats", "load", "lib_path", "sort", "sss_autotune_batched",
]

STATUS = {0: "SSS_OK", -1: "SSS_ERR_INVALID", -2: "SSS_ERR_NOMEM", -3: "SSS_ERR_CUDA",
          -4: "SSS_ERR_TIMEOUT", -5: "SSS_ERR_TOO_LARGE", -6: "SSS_ERR_INTERNAL"}
MAX_ROUNDS_LOGGED = 64
K_CLASSES = ["init", "sample", "classify", "scan", "scatter", "plan", "base", "runs", "fixup", "learned",
             "medium", "alphabet"]


class SSSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class sss_options(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int32), ("base_threshold", ctypes.c_uint32),
                ("medium_threshold", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("cdf_segments", ctypes.c_uint32), ("cdf_steps", ctypes.c_uint32),
                ("cdf_lr", ctypes.c_float), ("profile", ctypes.c_uint32), ("graph", ctypes.c_uint32),
                ("key_bytes", ctypes.c_uint32), ("classifier", ctypes.c_uint32), ("alphabet", ctypes.c_uint32),
                ("radix", ctypes.c_uint32)]


class sss_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("base_tiles", ctypes.c_uint32),
                ("round_strings", ctypes.c_uint64), ("medium_strings", ctypes.c_uint64),
                ("base_iterations", ctypes.c_uint64), ("base_segment_hist", ctypes.c_uint32 * 8),
                ("base_strings", ctypes.c_uint64),
                ("run_strings", ctypes.c_uint64), ("learned_keys", ctypes.c_uint64),
                ("learned_misses", ctypes.c_uint64), ("refilled_strings", ctypes.c_uint64),
                ("medium_refilled_strings", ctypes.c_uint64),
                ("launches", ctypes.c_uint32), ("profiled", ctypes.c_uint32),
                ("prof_launches", ctypes.c_uint32 * len(K_CLASSES)),
                ("prof_ms", ctypes.c_double * len(K_CLASSES)),
                ("round_segments", ctypes.c_uint32 * MAX_ROUNDS_LOGGED),
                ("round_active", ctypes.c_uint32 * MAX_ROUNDS_LOGGED),
                ("alphabet_symbols", ctypes.c_uint32), ("alphabet_group", ctypes.c_uint32),
                ("learned_models", ctypes.c_uint32), ("radix_segments", ctypes.c_uint32),
                ("round_learned_keys", ctypes.c_uint64 * MAX_ROUNDS_LOGGED),
                ("round_learned_misses", ctypes.c_uint64 * MAX_ROUNDS_LOGGED)]

    def as_dict(self):
        r = self.rounds
        return {"rounds": r, "base_tiles": self.base_tiles, "round_strings": self.round_strings,
                "medium_strings": self.medium_strings, "base_iterations": self.base_iterations,
                "base_segment_hist": list(self.base_segment_hist),
                "base_strings": self.base_strings, "run_strings": self.run_strings,
                "learned_keys": self.learned_keys, "learned_misses": self.learned_misses,
                "refilled_strings": self.refilled_strings,
                "medium_refilled_strings": self.medium_refilled_strings, "launches": self.launches,
                "profile": ({K_CLASSES[i]: {"launches": self.prof_launches[i], "ms": self.prof_ms[i]}
                             for i in range(len(K_CLASSES))} if self.profiled else None),
                "round_segments": list(self.round_segments)[:min(r, MAX_ROUNDS_LOGGED)],
                "round_active": list(self.round_active)[:min(r, MAX_ROUNDS_LOGGED)],
                "alphabet_symbols": self.alphabet_symbols, "alphabet_group": self.alphabet_group,
                "learned_models": self.learned_models, "radix_segments": self.radix_segments,
                "round_learned_keys": list(self.round_learned_keys)[:min(r, MAX_ROUNDS_LOGGED)],
                "round_learned_misses": list(self.round_learned_misses)[:min(r, MAX_ROUNDS_LOGGED)]}


class sss_learned_stats(ctypes.Structure):
    _fields_ = [("proposals", ctypes.c_uint64), ("misses", ctypes.c_uint64), ("models", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("miss_rate", ctypes.c_double)]


_lib = None
lib_path = _build.LIB

_P = ctypes.c_void_p
_SIG = {
    "sss_sort": ([_P, _P, ctypes.c_uint32, _P, _P, _P], ctypes.c_int),
    "sss_workspace_size": ([ctypes.c_uint32], ctypes.c_size_t),
    "sss_sort_ws": ([_P, _P, ctypes.c_uint32, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "sss_sort_host": ([_P, ctypes.c_uint64, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "sss_sort_noalloc": ([_P, _P, ctypes.c_uint32, _P, _P, _P], ctypes.c_int),
    "sss_sort_batched": ([_P, _P, ctypes.c_uint32, _P, ctypes.c_uint32, _P, _P, _P], ctypes.c_int),
    "sss_sort_learned": ([_P, _P, ctypes.c_uint32, _P, _P, _P, ctypes.POINTER(sss_learned_stats)], ctypes.c_int),
    "sss_autotune_batched": ([_P, _P, ctypes.c_uint32, _P, ctypes.c_uint32, _P, _P, ctypes.c_char_p,
                              ctypes.POINTER(sss_options), ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "sss_gather_keys": ([_P, _P, _P, _P, ctypes.c_uint32, _P, _P], ctypes.c_int),
    "sss_build_splitters": ([_P, ctypes.c_uint32, ctypes.c_int32, _P, _P, _P], ctypes.c_int),
    "sss_classify": ([_P, ctypes.c_uint32, _P, _P, ctypes.c_int32, _P, _P], ctypes.c_int),
    "sss_classify_equal": ([_P, ctypes.c_uint32, _P, ctypes.c_int32, _P, _P], ctypes.c_int),
    "sss_cdf_loss_grad": ([_P, ctypes.c_uint32, _P, _P, ctypes.c_uint32, _P, _P, _P], ctypes.c_int),
    "sss_set_options": ([ctypes.POINTER(sss_options)], ctypes.c_int),
    "sss_get_options": ([ctypes.POINTER(sss_options)], ctypes.c_int),
    "sss_get_last_stats": ([ctypes.POINTER(sss_stats)], ctypes.c_int),
    "sss_get_last_timeline": ([ctypes.c_uint32, _P, _P, _P, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "sss_last_error": ([], ctypes.c_char_p),
    "sss_release": ([], ctypes.c_int),
    "sss_version": ([], ctypes.c_char_p),
}


def load(path: str | None = None):
    """Load libsss.so (raises OSError if it was not built)."""
    global _lib
    if _lib is None:
        p = path or lib_path
        if not os.path.exists(p):
            raise OSError(f"{p} is missing: build it with paper_1305_1157_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, (args, res) in _SIG.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def _check(rc):
    if rc != 0:
        raise SSSError(rc, load().sss_last_error().decode())


def sss_sort(chars, offsets, n, out_perm, out_lcp, stream=None):
    _check(load().sss_sort(_addr(chars), _addr(offsets), n, _addr(out_perm), _addr(out_lcp), _stream(stream)))


def sss_workspace_size(n) -> int:
    return int(load().sss_workspace_size(n))


def sss_sort_ws(chars, offsets, n, out_perm, out_lcp, workspace, workspace_bytes, stream=None):
    _check(load().sss_sort_ws(_addr(chars), _addr(offsets), n, _addr(out_perm), _addr(out_lcp),
                              _addr(workspace), workspace_bytes, _stream(stream)))


def sss_sort_noalloc(chars, offsets, n, out_perm, out_lcp, stream=None):
    """sss_sort for at most 65,536 strings without allocating: scratch is a
    static device array of the library (see include/sss.h)."""
    _check(load().sss_sort_noalloc(_addr(chars), _addr(offsets), n, _addr(out_perm), _addr(out_lcp),
                                   _stream(stream)))


def sss_sort_host(chars, chars_bytes, offsets, n, out_perm, out_lcp):
    _check(load().sss_sort_host(_addr(chars), chars_bytes, _addr(offsets), n, _addr(out_perm), _addr(out_lcp)))


def sss_sort_batched(chars, offsets, n, set_begin, num_sets, out_perm, out_lcp, stream=None):
    _check(load().sss_sort_batched(_addr(chars), _addr(offsets), n, _addr(set_begin), num_sets,
                                   _addr(out_perm), _addr(out_lcp), _stream(stream)))


def sss_autotune_batched(chars, offsets, n, set_begin, num_sets, out_perm, out_lcp, cache_path=None, stream=None):
    """Returns (sss_options chosen, milliseconds of the chosen setting)."""
    best = sss_options()
    ms = ctypes.c_double(0.0)
    path = cache_path.encode() if isinstance(cache_path, str) else cache_path
    _check(load().sss_autotune_batched(_addr(chars), _addr(offsets), n, _addr(set_begin), num_sets, _addr(out_perm),
                                       _addr(out_lcp), path, ctypes.byref(best), ctypes.byref(ms), _stream(stream)))
    return best, ms.value


def sss_sort_learned(chars, offsets, n, out_perm, out_lcp, stream=None):
    """Returns the call's sss_learned_stats."""
    st = sss_learned_stats()
    _check(load().sss_sort_learned(_addr(chars), _addr(offsets), n, _addr(out_perm), _addr(out_lcp),
                                   _stream(stream), ctypes.byref(st)))
    return st


def sss_gather_keys(chars, offsets, idx, depth, n, out_keys, stream=None):
    _check(load().sss_gather_keys(_addr(chars), _addr(offsets), _addr(idx), _addr(depth), n, _addr(out_keys),
                                  _stream(stream)))


def sss_build_splitters(sample, count, k, out_level, out_inorder, stream=None):
    _check(load().sss_build_splitters(_addr(sample), count, k, _addr(out_level), _addr(out_inorder),
                                      _stream(stream)))


def sss_classify(keys, n, level, inorder, k, out_bucket, stream=None):
    _check(load().sss_classify(_addr(keys), n, _addr(level), _addr(inorder), k, _addr(out_bucket),
                               _stream(stream)))


def sss_classify_equal(keys, n, level, k, out_bucket, stream=None):
    _check(load().sss_classify_equal(_addr(keys), n, _addr(level), k, _addr(out_bucket), _stream(stream)))


def sss_cdf_loss_grad(theta, M, u, y, S, out_loss, out_grad, stream=None):
    _check(load().sss_cdf_loss_grad(_addr(theta), M, _addr(u), _addr(y), S, _addr(out_loss), _addr(out_grad),
                                    _stream(stream)))


def sss_set_options(opt: sss_options = None, **kw):
    """Set the library options: opt (or the current options) with the
    fields named in kw replaced; unknown field names raise TypeError."""
    if opt is None:
        opt = sss_get_options()
    names = {f for f, _ in sss_options._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"sss_options has no field {k!r}")
        setattr(opt, k, v)
    _check(load().sss_set_options(ctypes.byref(opt)))


def sss_get_options() -> sss_options:
    o = sss_options()
    _check(load().sss_get_options(ctypes.byref(o)))
    return o


def sss_get_last_stats() -> sss_stats:
    s = sss_stats()
    _check(load().sss_get_last_stats(ctypes.byref(s)))
    return s


def sss_get_last_timeline():
    """[(class name, start ms, end ms)] of the last profiled host-driven call."""
    lib = load()
    cnt = ctypes.c_uint32(0)
    _check(lib.sss_get_last_timeline(0, None, None, None, ctypes.byref(cnt)))
    n = cnt.value
    cls = (ctypes.c_int32 * max(n, 1))()
    t0 = (ctypes.c_double * max(n, 1))()
    t1 = (ctypes.c_double * max(n, 1))()
    _check(lib.sss_get_last_timeline(n, cls, t0, t1, ctypes.byref(cnt)))
    return [(K_CLASSES[cls[i]], t0[i], t1[i]) for i in range(min(n, cnt.value))]


def sss_last_error() -> str:
    return load().sss_last_error().decode()


def sss_release():
    _check(load().sss_release())


def sss_version() -> str:
    return load().sss_version().decode()


def sort(chars, offsets, learned: bool = False, stream=None):
    """Sort device strings held in torch tensors: chars (uint8, cuda) and
    offsets (int64/uint64 view, cuda).  Returns (perm, lcp) as int32 cuda
    tensors holding uint32 values."""
    import torch
    n = offsets.numel()
    perm = torch.empty(n, dtype=torch.int32, device=offsets.device)
    lcp = torch.empty(n, dtype=torch.int32, device=offsets.device)
    (sss_sort_learned if learned else sss_sort)(chars, offsets, n, perm, lcp, stream)
    return perm, lcp
