"""The checked build (-DQH_DEBUG=1): device-side alignment and bounds checks
of every bulk copy, mbarrier, point scatter, tile-map segment index, hull
slot and vector load.  Small 2D and 3D cases run on it in a child process
(its own library build) and must equal the oracle with no failed check."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_clean():
    env = dict(os.environ, QH_DEBUG_BUILD="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_checks_child.py")],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
    out = json.loads(line)
    assert out["record"]["enabled"]
    assert out["record"]["failures"] == 0, out["record"]
    assert all(out["parity"]), out["parity"]


def test_default_build_has_no_checks():
    from paper_1201_2936_gb300 import build
    build.build()
    import paper_1201_2936_gb300 as qh
    with pytest.raises(qh.QHError) as ei:
        qh.debug_checks()
    assert ei.value.status == 9
