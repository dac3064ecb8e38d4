"""Child process of test_gpu_debug_checks: with QH_DEBUG_BUILD=1 in its
environment it builds and loads the checked library, runs small 2D (single,
several-cloud, interleaved, host loop) and 3D (single, batched) cases against
the oracle and prints the device-check record as one JSON line."""
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1201_2936_gb300 import build  # noqa: E402
from paper_1201_2936_gb300 import workloads as w  # noqa: E402


def main():
    assert build.DEBUG, "QH_DEBUG_BUILD=1 expected"
    build.build()
    oracle.build()
    import paper_1201_2936_gb300 as qh
    qh.debug_checks(reset=True)
    ok = []
    # 2D: single cloud (separate arrays, both loops), interleaved, several clouds
    for gen, n in (("square", 100_000), ("disk", 300_001), ("circle", 50_000)):
        x, y = getattr(w, {"square": "uniform_square", "disk": "uniform_disk",
                           "circle": "circle_jitter"}[gen])(n, 900 + n)
        want = oracle.hull2d(x, y).tolist()
        X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ok.append(qh.hull2d(X, Y).cpu().tolist() == want)
        ok.append(qh.hull2d(X, Y, loop="host").cpu().tolist() == want)
        P = torch.from_numpy(np.stack([x, y], axis=1).copy()).cuda()
        ok.append(qh.hull2d(P).cpu().tolist() == want)
    clouds = [w.uniform_disk(70_001, 11), w.uniform_square(20_000, 12), w.circle_jitter(5_000, 13)]
    T = [(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()) for x, y in clouds]
    got = qh.hull2d_multi(T)
    ok.append([g.cpu().tolist() for g in got] == [oracle.hull2d(x, y).tolist() for x, y in clouds])
    # 3D: one cloud and a small batch
    x, y, z = w.uniform_ball(60_000, 21)
    v, f = oracle.hull3d(x, y, z)
    gv, off, idx = qh.hull3d(*(torch.from_numpy(c).cuda() for c in (x, y, z)))
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    faces = [idx[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    ok.append(gv.cpu().tolist() == v.tolist() and faces == [t.tolist() for t in f])
    x, y, z, off = w.batched_clouds_3d(64, 22, nmin=16, nmax=4096)
    want = [(st, v.tolist(), [t.tolist() for t in fs]) for st, v, fs in
            oracle.hull3d_batched(x, y, z, off)]
    outs = qh.hull3d_batched(torch.from_numpy(np.stack([x, y, z])).cuda(),
                             cloud_off=torch.from_numpy(off).cuda())
    verts, cvo, foff, fidx, cfo, cst = (t.cpu().numpy() for t in outs)
    got = [(int(cst[c]), verts[cvo[c]:cvo[c + 1]].tolist(),
            [fidx[foff[i]:foff[i + 1]].tolist() for i in range(cfo[c], cfo[c + 1])])
           for c in range(len(cst))]
    ok.append(got == want)
    rec = qh.debug_checks()
    torch.cuda.synchronize()
    print(json.dumps({"parity": ok, "record": rec}))


if __name__ == "__main__":
    main()
