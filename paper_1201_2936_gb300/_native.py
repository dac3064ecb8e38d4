"""ctypes declarations of the C ABI in include/qh.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

LIB_PATH = _build.LIB

_lock = threading.Lock()
_lib = None


class QhOpts(ctypes.Structure):
    _fields_ = [("pred_mode", ctypes.c_int32), ("loop_mode", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("block", ctypes.c_int32),
                ("max_iters", ctypes.c_int64), ("wait_ns", ctypes.c_int64),
                ("items", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("test_hold", ctypes.c_int32), ("small_cloud", ctypes.c_int32),
                ("max_facets", ctypes.c_int64)]


class QhDebugRecord(ctypes.Structure):
    _fields_ = [("failures", ctypes.c_int64), ("site", ctypes.c_int32),
                ("enabled", ctypes.c_int32), ("a", ctypes.c_uint64), ("b", ctypes.c_uint64)]


class QhResult(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("status", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("iterations", ctypes.c_int64),
                ("live_total", ctypes.c_int64), ("survivor_total", ctypes.c_int64),
                ("segments_total", ctypes.c_int64), ("filter_fallbacks", ctypes.c_int64),
                ("exact_argmax", ctypes.c_int64), ("extra", ctypes.c_int64 * 4)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("extra", "reserved0")}
        d["extra"] = list(self.extra)
        return d


RESULT_BYTES = ctypes.sizeof(QhResult)

# (name, restype, argtypes)
_vp, _i64, _sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
_POpts = ctypes.POINTER(QhOpts)
_PRes = ctypes.POINTER(QhResult)
SIGNATURES = [
    ("qh_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("qh_version", ctypes.c_char_p, []),
    ("qh_default_opts", None, [_POpts]),
    ("qh_workspace_bytes_2d", _sz, [_i64, _POpts]),
    ("qh_hull2d_async", ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp, _sz, _POpts, _vp]),
    ("qh_hull2d", ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, ctypes.POINTER(_i64), _PRes, _vp,
                                 _sz, _POpts, _vp]),
    ("qh_workspace_bytes_2d_multi", _sz, [ctypes.c_int32, _vp, _POpts]),
    ("qh_hull2d_multi_async", ctypes.c_int, [ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                             _sz, _POpts, _vp]),
    ("qh_hull2d_multi", ctypes.c_int, [ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                       _sz, _POpts, _vp]),
    ("qh_workspace_bytes_3d", _sz, [_i64, _POpts]),
    ("qh_workspace_bytes_4d", _sz, [_i64, _POpts]),
    ("qh_debug_timeline_4d", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    ("qh_debug_checks", ctypes.c_int, [ctypes.POINTER(QhDebugRecord), ctypes.c_int32]),
    ("qh_shard_block_words", _i64, [ctypes.c_int32, ctypes.c_int32]),
    ("qh_shard_local", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _i64,
                                      ctypes.c_int32, _vp, _vp]),
    ("qh_shard_pack", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32,
                                     ctypes.c_int32, _vp, _vp, _vp, _vp]),
    ("qh_shard_remap", ctypes.c_int, [ctypes.c_int32, _vp, _vp, _vp, _i64, _vp]),
    ("qh_hull4d", ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _i64, _vp, ctypes.POINTER(_i64), _vp,
                                 _i64, _vp, _i64, ctypes.POINTER(_i64), _PRes, _vp, _sz, _POpts,
                                 _vp]),
    ("qh_hull3d", ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _vp, ctypes.POINTER(_i64), _vp, _vp,
                                 ctypes.POINTER(_i64), _PRes, _vp, _sz, _POpts, _vp]),
    ("qh_debug_timeline_3d", ctypes.c_int, [_vp, _i64, _vp, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32), _vp]),
    ("qh_hull2d_noalloc", ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, ctypes.POINTER(_i64), _vp]),
    ("qh_debug_timeline_2d", ctypes.c_int, [_vp, _i64, _vp, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32), _vp]),
    ("qh_workspace_bytes_3d_batched", _sz, [_i64, ctypes.c_int32, _POpts]),
    ("qh_hull3d_batched", ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, ctypes.c_int32, _i64, _vp, _vp,
                                         _vp, _vp, _vp, _vp, _vp, _vp, _sz, _POpts, _vp]),
    ("qh_debug_phases_3d", ctypes.c_int, [_vp, _vp, _vp]),
    ("qh_segmented_workspace_bytes", _sz, [_i64, ctypes.c_int32]),
    ("qh_flag_permute", ctypes.c_int, [_vp, _vp, _i64, ctypes.c_int32, _vp, _vp, _vp, _sz, _vp]),
    ("qh_compact", ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, ctypes.POINTER(_i64), _vp, _sz, _vp]),
    ("qh_select", ctypes.c_int, [_vp, _vp, ctypes.c_int32, _i64, _vp, _vp, ctypes.POINTER(_i64),
                                 _vp, _sz, _vp]),
    ("qh_select_host_loop", ctypes.c_int, [_vp, _vp, ctypes.c_int32, _i64, _vp, _vp,
                                           ctypes.POINTER(_i64), _vp, _sz, _vp]),
    ("qh_workspace_bytes_2d_batched", _sz, [_i64, ctypes.c_int32, _POpts]),
    ("qh_hull2d_batched", ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.c_int32, _i64, _vp, _vp, _vp,
                                         _vp, _vp, _sz, _POpts, _vp]),
    ("qh_measures2d", ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp]),
    ("qh_hull2d_backward", ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.c_int32, _i64, _vp, _vp, _vp,
                                          _vp, _vp, _i64, _vp]),
    ("qh_measures3d", ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                     _vp]),
    ("qh_hull3d_backward", ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.c_int32, _i64, _vp, _vp, _vp,
                                          _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    ("qh_autotune_3d_batched", ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, ctypes.c_int32, _i64, _vp,
                                              _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                                              ctypes.c_int32, _POpts, _vp, _vp, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32), _vp]),
]


def exported_names():
    return [s[0] for s in SIGNATURES]


def lib():
    """The loaded libqh.so.  Raises if the library has not been built: there
    is no fallback implementation."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -m paper_1201_2936_gb300.build or __graft_entry__.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib
