"""The no-alloc 2D entry point (fixed device scratch, no workspace argument),
for callers that cannot allocate device memory while they run.

It gives the same hull, index for index, as the workspace entry point and as
the oracle, on calls in a row that share the fixed scratch; the calls leave
the device's free memory and PyTorch's reserved memory unchanged; n = 0 and
interleaved xy input (the other bulk-copy form of the first pass) work; n
above the limit is refused.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1201_2936_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1201_2936_gb300 import build, _native
    build.build()
    oracle.build()
    return _native.lib()


def _with_workspace(L, xp, yp, n, stride):
    ws = torch.empty(L.qh_workspace_bytes_2d(n, None), dtype=torch.uint8, device="cuda")
    out = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    st = L.qh_hull2d(xp, yp, n, stride, out.data_ptr(), ctypes.byref(cnt), None,
                     ws.data_ptr(), ws.numel(), None, None)
    assert st == 0
    return out[: cnt.value].cpu().numpy()


def _noalloc(L, xp, yp, n, stride, out):
    cnt = ctypes.c_int64(-1)
    st = L.qh_hull2d_noalloc(xp, yp, n, stride, out.data_ptr(), ctypes.byref(cnt), None)
    assert st == 0
    return cnt.value


def test_noalloc_matches_workspace_entry_point_and_oracle(lib):
    cases = [w.circle_jitter(131072, 5, 1e-4), w.uniform_disk(70001, 6)]
    out = torch.empty(131072, dtype=torch.int32, device="cuda")
    for x, y in cases:   # calls in a row share the fixed scratch
        n = len(x)
        X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        want = _with_workspace(lib, X.data_ptr(), Y.data_ptr(), n, 1)
        _noalloc(lib, X.data_ptr(), Y.data_ptr(), n, 1, out)  # first call (module set-up)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        res0 = torch.cuda.memory_reserved()
        cnt = _noalloc(lib, X.data_ptr(), Y.data_ptr(), n, 1, out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0 and torch.cuda.memory_reserved() == res0
        got = out[:cnt].cpu().numpy()
        assert got.tolist() == want.tolist()
        assert got.tolist() == oracle.hull2d(x, y).tolist()
        assert len(got) > 2


def test_noalloc_interleaved_xy_and_empty(lib):
    x, y = w.uniform_square(100_003, 7)
    P = torch.from_numpy(np.stack([x, y], axis=1).copy()).cuda()  # [n, 2]: stride 2
    out = torch.empty(P.shape[0], dtype=torch.int32, device="cuda")
    n = P.shape[0]
    cnt = _noalloc(lib, P.data_ptr(), P.data_ptr() + 4, n, 2, out)
    got = out[:cnt].cpu().numpy()
    assert got.tolist() == oracle.hull2d(x, y).tolist()
    assert got.tolist() == _with_workspace(lib, P.data_ptr(), P.data_ptr() + 4, n, 2).tolist()
    assert _noalloc(lib, P.data_ptr(), P.data_ptr() + 4, 0, 2, out) == 0


def test_noalloc_refuses_too_many_points(lib):
    n = 131073
    X = torch.zeros(n, dtype=torch.float32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    st = lib.qh_hull2d_noalloc(X.data_ptr(), X.data_ptr(), n, 1, out.data_ptr(), ctypes.byref(cnt),
                               None)
    assert st == 1  # QH_ERR_INVALID_ARG
