"""The checked build (libccdyk_checked.so, CCD_CHECKED) on the GPU: the sweep
kernels test every offset they use and would report CC_ERR_BOUNDS; on valid
inputs they must report nothing and give the normal results.  Runs in a child
process, since a process loads one of the two libraries (CCDYK_CHECKED=1)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np
import oracle
import paper_1901_10084_gb300 as cc
from paper_1901_10084_gb300 import _native
from instances import chung_lu, planted_partition, random_dissimilarity
assert _native.lib_path().endswith("libccdyk_checked.so")

def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1.0))

for n, tile, weighted in ((61, 16, True), (97, 32, False), (150, 8, True)):
    d, w, _ = chung_lu(n, 2.5, 8.0, seed=n, weights=(0.5, 2.0) if weighted else None)
    o = oracle.State(n, d, w, 0.2)
    for _ in range(3):
        o.sweep(2, tile)
    with cc.Solver(n, d, w, tile=tile, interleave=False) as s:
        s.set_state(o.x, o.f, o.ytri, o.ypair)
        s.sweep(1)
        o.sweep(2, tile)
        x, f = s.get_x()
        yt, yp = s.get_duals()
        s.check()
    assert rel(x, o.x) <= 1e-12 and rel(yt, o.ytri) <= 1e-12
    res = []
    for store in ("dense", "sparse"):
        with cc.Solver(n, d, w, tile=tile, store=store, pool_entries=64) as s:
            s.sweep(5)
            s.check()
            res.append(s.get_x()[0])
    assert np.array_equal(res[0], res[1])
dl, wl = random_dissimilarity(40, 3)
ol = oracle.State(40, dl, wl, problem="l2")
ol.sweep(2, 8)
with cc.Solver(40, dl, wl, problem="l2", tile=8, exact=True, interleave=False) as s:
    s.sweep(1)
    assert np.array_equal(s.get_x()[0], ol.x)
inst = [(n, *planted_partition(n, 3, 0.7, 0.1, seed=n)[:2]) for n in (40, 77, 120)]
with cc.Batch(inst, tile=16) as b:
    b.sweep(4)
    for i in range(3):
        b.instance(i).check()
print("CHECKED-OK")
"""


def test_checked_build_reports_no_bounds_error_on_valid_work():
    env = dict(os.environ, CCDYK_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "CHECKED-OK" in r.stdout
