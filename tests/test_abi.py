"""The C ABI library loads without a GPU and exports every function that
include/qh.h declares; the ctypes binding names the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(qh_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1201_2936_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert "qh_hull2d" in declared and "qh_status_str" in declared
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1201_2936_gb300 import _native
    assert set(_native.exported_names()) == _declared()


def test_status_strings_and_sizes(lib):
    from paper_1201_2936_gb300 import _native
    L = _native.lib()
    assert L.qh_status_str(0) == b"QH_OK"
    assert b"NONFINITE" in L.qh_status_str(2)
    assert L.qh_workspace_bytes_2d(-1, None) == 0
    w1 = L.qh_workspace_bytes_2d(1000, None)
    w2 = L.qh_workspace_bytes_2d(2000, None)
    assert 0 < w1 < w2
    assert ctypes.sizeof(_native.QhResult) == 96


def test_3d_facet_capacity_sizes_the_workspace(lib):
    # qh_opts.max_facets: 0 or anything at or above 6 n + 4 ncloud + 64 is the
    # worst case; below it the workspace shrinks with the facets (and, for one
    # cloud, the segment entries), never below 4 ncloud + 256 facets; negative
    # is refused.  Several clouds keep one entry per point.
    from paper_1201_2936_gb300 import _native
    L = _native.lib()
    assert ctypes.sizeof(_native.QhOpts) == 56
    assert _native.QhOpts.max_facets.offset == 48

    def opts(f):
        o = _native.QhOpts()
        L.qh_default_opts(ctypes.byref(o))
        o.max_facets = f
        return ctypes.byref(o)

    n = 200_000
    full = L.qh_workspace_bytes_3d(n, None)
    assert full > 0
    for f in (0, 6 * n + 68, 10 ** 12):
        assert L.qh_workspace_bytes_3d(n, opts(f)) == full
    sizes = [L.qh_workspace_bytes_3d(n, opts(f)) for f in (1, 260, 261, 50_000, 150_000)]
    assert sizes[0] == sizes[1] < sizes[2] < sizes[3] < sizes[4] < full // 3
    assert L.qh_workspace_bytes_3d(n, opts(-1)) == 0
    one = L.qh_workspace_bytes_3d_batched(n, 1, opts(150_000))
    assert sizes[4] < one < L.qh_workspace_bytes_3d_batched(n, 1, None)
    assert L.qh_workspace_bytes_3d_batched(n, 64, opts(1)) == \
        L.qh_workspace_bytes_3d_batched(n, 64, opts(4 * 64 + 256))


def test_host_side_argument_errors(lib):
    from paper_1201_2936_gb300 import _native
    L = _native.lib()
    res = ctypes.c_void_p(16)
    # negative n, bad stride, null workspace: rejected before any device work
    assert L.qh_hull2d_async(None, None, -1, 1, None, res, ctypes.c_void_p(256), 1 << 20, None, None) == 1
    assert L.qh_hull2d_async(ctypes.c_void_p(256), ctypes.c_void_p(256), 10, 0, ctypes.c_void_p(256),
                             res, ctypes.c_void_p(256), 1 << 20, None, None) == 1
    assert L.qh_hull2d_async(ctypes.c_void_p(256), ctypes.c_void_p(256), 10, 1, ctypes.c_void_p(256),
                             res, None, 1 << 20, None, None) == 1
    # workspace too small
    assert L.qh_hull2d_async(ctypes.c_void_p(256), ctypes.c_void_p(256), 10, 1, ctypes.c_void_p(256),
                             res, ctypes.c_void_p(256), 16, None, None) == 4


def test_single_cloud_workspace_covers_the_persistent_kernel(lib):
    # the persistent loop of qh_hull2d runs the several-cloud kernel with one
    # cloud: the single-cloud size covers that layout, and the fixed scratch of
    # qh_hull2d_noalloc covers its largest call
    from paper_1201_2936_gb300 import _native
    L = _native.lib()
    one = ctypes.c_int64 * 1
    for n in (0, 1, 2, 1000, 4097, 131072, 1 << 24):
        assert L.qh_workspace_bytes_2d(n, None) >= L.qh_workspace_bytes_2d_multi(1, one(n), None) > 0
    assert L.qh_workspace_bytes_2d(131072, None) <= 32 << 20
    # one byte short of the size is refused before any device work
    need = L.qh_workspace_bytes_2d(10, None)
    res = ctypes.c_void_p(16)
    assert L.qh_hull2d_async(ctypes.c_void_p(256), ctypes.c_void_p(256), 10, 1, ctypes.c_void_p(256),
                             res, ctypes.c_void_p(256), need - 1, None, None) == 4
