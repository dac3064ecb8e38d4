"""The no-alloc 2D entry point (fixed device scratch, no workspace argument)
gives the same hull, index for index, as the workspace entry point, on two
calls in a row; n above its limit is refused.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1201_2936_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1201_2936_gb300 import build, _native
    build.build()
    return _native.lib()


def _with_workspace(L, X, Y, n):
    ws = torch.empty(L.qh_workspace_bytes_2d(n, None), dtype=torch.uint8, device="cuda")
    out = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    st = L.qh_hull2d(X.data_ptr(), Y.data_ptr(), n, 1, out.data_ptr(), ctypes.byref(cnt), None,
                     ws.data_ptr(), ws.numel(), None, None)
    assert st == 0
    return out[: cnt.value].cpu().numpy()


def _noalloc(L, X, Y, n):
    out = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    st = L.qh_hull2d_noalloc(X.data_ptr(), Y.data_ptr(), n, 1, out.data_ptr(), ctypes.byref(cnt),
                             None)
    assert st == 0
    return out[: cnt.value].cpu().numpy()


def test_noalloc_matches_workspace_entry_point(lib):
    cases = [w.circle_jitter(131072, 5, 1e-4), w.uniform_disk(70001, 6)]
    for x, y in cases:   # two calls in a row share the fixed scratch
        n = len(x)
        X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        want = _with_workspace(lib, X, Y, n)
        got = _noalloc(lib, X, Y, n)
        assert got.tolist() == want.tolist()
        assert len(got) > 2


def test_noalloc_refuses_too_many_points(lib):
    n = 131073
    X = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    st = lib.qh_hull2d_noalloc(X.data_ptr(), X.data_ptr(), n, 1, out.data_ptr(), ctypes.byref(cnt),
                               None)
    assert st == 1  # QH_ERR_INVALID_ARG
