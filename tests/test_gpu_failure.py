"""Failure detection on the GPU, without a fault: the iteration cap, the
bounded grid-barrier wait and the 3D facet capacity are made to run out on
purpose, the call reports QH_ERR_NO_CONVERGENCE, QH_ERR_TIMEOUT or
QH_ERR_CAPACITY through the C ABI, the context stays usable, and the same
workspace then gives the oracle's hull.

The wait is made to run out by the test hook qh_opts.test_hold: CTA 0 of the
persistent kernel does not arrive at its first grid barrier, so that round
never completes (a flag that nothing sets) and every CTA gives up after
wait_ns.  Nothing here traps, hangs or touches memory out of bounds."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1201_2936_gb300 import workloads as w

pytestmark = pytest.mark.gpu

QH_ERR_CAPACITY = 5
QH_ERR_TIMEOUT = 6
QH_ERR_NO_CONVERGENCE = 7
WAIT_NS = 20_000_000  # 20 ms: every CTA's wait on the held barrier ends after this


@pytest.fixture(scope="module")
def qh():
    from paper_1201_2936_gb300 import build
    build.build()
    oracle.build()
    import paper_1201_2936_gb300 as q
    return q


def _hull2d(qh, X, Y, ws, opts):
    lib = qh._native.lib()
    n = X.numel()
    out = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    res = qh.QhResult()
    buf = ws.get(qh.workspace_bytes_2d(n, opts))
    st = lib.qh_hull2d(X.data_ptr(), Y.data_ptr(), n, 1, out.data_ptr(), ctypes.byref(cnt),
                       ctypes.byref(res), buf.data_ptr(), buf.numel(), ctypes.byref(opts), None)
    return st, res, out[: cnt.value].cpu().numpy()


def _hull3d(qh, X, Y, Z, ws, opts):
    lib = qh._native.lib()
    n = X.numel()
    verts = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    foff = torch.empty(2 * n + 2, dtype=torch.int32, device="cuda")
    fidx = torch.empty(max(6 * n, 1), dtype=torch.int32, device="cuda")
    nv, nf = ctypes.c_int64(0), ctypes.c_int64(0)
    res = qh.QhResult()
    buf = ws.get(qh.workspace_bytes_3d(n, opts))
    st = lib.qh_hull3d(X.data_ptr(), Y.data_ptr(), Z.data_ptr(), n, 1, verts.data_ptr(),
                       ctypes.byref(nv), foff.data_ptr(), fidx.data_ptr(), ctypes.byref(nf),
                       ctypes.byref(res), buf.data_ptr(), buf.numel(), ctypes.byref(opts), None)
    if st != 0:
        return st, res, None, None
    off = foff[: nf.value + 1].cpu().numpy()
    idx = fidx.cpu().numpy()
    faces = [idx[off[i]:off[i + 1]].tolist() for i in range(nf.value)]
    return st, res, verts[: nv.value].cpu().numpy().tolist(), faces


def _cuda(*a):
    return [torch.from_numpy(np.ascontiguousarray(c, dtype=np.float32)).cuda() for c in a]


@pytest.mark.parametrize("loop", ["persistent", "host"])
def test_2d_iteration_cap(qh, loop):
    x, y = w.uniform_disk(200_000, 4101)
    X, Y = _cuda(x, y)
    ws = qh.Workspace()
    st, res, _ = _hull2d(qh, X, Y, ws, qh.make_opts("f32", loop, max_iters=1))
    assert st == QH_ERR_NO_CONVERGENCE and res.status == QH_ERR_NO_CONVERGENCE
    # the same workspace, default limits: the oracle's hull
    st, res, got = _hull2d(qh, X, Y, ws, qh.make_opts("f32", loop))
    assert st == 0
    assert got.tolist() == oracle.hull2d(x, y).tolist()


def test_3d_iteration_cap(qh):
    x, y, z = w.uniform_ball(100_000, 4102)
    X, Y, Z = _cuda(x, y, z)
    ws = qh.Workspace()
    st, res, _, _ = _hull3d(qh, X, Y, Z, ws, qh.make_opts("f32", max_iters=1))
    assert st == QH_ERR_NO_CONVERGENCE and res.status == QH_ERR_NO_CONVERGENCE
    st, res, v, f = _hull3d(qh, X, Y, Z, ws, qh.make_opts("f32"))
    assert st == 0
    want_v, want_f = oracle.hull3d(x, y, z)
    assert v == want_v.tolist() and f == [t.tolist() for t in want_f]


@pytest.mark.parametrize("pred", ["f32", "f64"])
def test_3d_facet_capacity(qh, pred):
    # qh_opts.max_facets: a capacity that holds every facet the run creates
    # gives the oracle's hull in a quarter of the worst-case workspace; one
    # that does not (raised to its floor of 260 facets) stops the run with
    # QH_ERR_CAPACITY, and the same workspace then serves a full run
    x, y, z = w.uniform_ball(200_000, 4105)
    X, Y, Z = _cuda(x, y, z)
    n = len(x)
    fit = qh.make_opts(pred, max_facets=150_000)
    assert qh.workspace_bytes_3d(n, fit) < qh.workspace_bytes_3d(n, qh.make_opts(pred)) // 3
    want_v, want_f = oracle.hull3d(x, y, z)
    want = (want_v.tolist(), [t.tolist() for t in want_f])
    ws = qh.Workspace()
    st, res, v, f = _hull3d(qh, X, Y, Z, ws, fit)
    assert st == 0 and (v, f) == want
    for _ in range(2):
        st, res, _, _ = _hull3d(qh, X, Y, Z, ws, qh.make_opts(pred, max_facets=1))
        assert st == QH_ERR_CAPACITY and res.status == QH_ERR_CAPACITY
    torch.cuda.synchronize()
    st, res, v, f = _hull3d(qh, X, Y, Z, ws, fit)
    assert st == 0 and (v, f) == want


def test_2d_grid_barrier_wait_runs_out(qh):
    x, y = w.circle_jitter(300_000, 4103, 1e-4)
    X, Y = _cuda(x, y)
    ws = qh.Workspace()
    for _ in range(2):  # twice: the held barrier leaves nothing behind
        st, res, _ = _hull2d(qh, X, Y, ws,
                             qh.make_opts("f32", "persistent", wait_ns=WAIT_NS, test_hold=1))
        assert st == QH_ERR_TIMEOUT and res.status == QH_ERR_TIMEOUT
    torch.cuda.synchronize()  # the context is still usable
    st, res, got = _hull2d(qh, X, Y, ws, qh.make_opts("f32", "persistent"))
    assert st == 0
    assert got.tolist() == oracle.hull2d(x, y).tolist()


def test_3d_grid_barrier_wait_runs_out(qh):
    x, y, z = w.uniform_ball(200_000, 4104)
    X, Y, Z = _cuda(x, y, z)
    ws = qh.Workspace()
    for _ in range(2):
        st, res, _, _ = _hull3d(qh, X, Y, Z, ws,
                                qh.make_opts("f32", wait_ns=WAIT_NS, test_hold=1))
        assert st == QH_ERR_TIMEOUT and res.status == QH_ERR_TIMEOUT
    torch.cuda.synchronize()
    st, res, v, f = _hull3d(qh, X, Y, Z, ws, qh.make_opts("f32"))
    assert st == 0
    want_v, want_f = oracle.hull3d(x, y, z)
    assert v == want_v.tolist() and f == [t.tolist() for t in want_f]
