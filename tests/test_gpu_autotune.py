"""The plan autotuner of the pass march: it times the plans on the context's own data at
the first solve, keeps the fastest, and reads/writes the cache file named by
PFT_AUTOTUNE_CACHE.  Any plan computes the same solve (FP32 tolerance 2e-5)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1204_5434_gb300 import pft
from paper_1204_5434_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _solve(autotune, prec=pft.PFT_FP32_MIXED, n=(64, 64, 64), Ns=20):
    w = wl.GYR64.with_(n=n, Ns=Ns)
    wp, wm = wl.fields(w)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, pft.PFT_SCFT_REAL, prec, autotune=autotune) as s:
        s.set_fields(wp, wm)
        s.solve()
        obs = s.observables()
        phiA, _ = s.densities()
        plan = pft.pft_get_plan(s.h)
    return obs, phiA, plan


def test_autotuned_plan_computes_the_same_solve():
    o0, p0, plan0 = _solve(0)
    o1, p1, plan1 = _solve(1)
    assert plan0 == (2, 1)
    # any plan the autotuner may pick at 64^3 FP32 real: pencil passes, plane kernel, the
    # separable march on the plane kernel (x-kernel variants 2, 18) or on pencils (line
    # variants 3, 19, 35, 51)
    assert plan1[0] in (0, 1, 2, 18, 3, 19, 35, 51) and plan1[1] in (0, 1)
    assert abs(o1["Q"].real - o0["Q"].real) <= 2e-5 * o0["Q"].real
    assert np.max(np.abs(p1 - p0)) <= 2e-5


def test_fp64_has_no_plane_plan():
    _, _, plan = _solve(1, prec=pft.PFT_FP64, n=(32, 32, 32), Ns=8)
    assert plan[0] in (0, 3)


_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
from paper_1204_5434_gb300 import pft, workloads as wl
w = wl.GYR64.with_(Ns=12)
wp, wm = wl.fields(w)
with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, pft.PFT_SCFT_REAL, pft.PFT_FP32_MIXED, autotune=1) as s:
    s.set_fields(wp, wm)
    s.solve()
    s.observables()
    print("PLAN", *pft.pft_get_plan(s.h))
"""


def _child(path):
    env = dict(os.environ, PFT_AUTOTUNE_CACHE=str(path))
    out = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("PLAN")][-1]
    return tuple(int(v) for v in line.split()[1:])


def test_plan_cache_file_is_written_and_read(tmp_path):
    path = tmp_path / "plans.txt"
    plan = _child(path)
    lines = path.read_text().splitlines()
    key = "64x64x64/real/fp32/Ns12"
    assert any(ln.split()[0] == key and tuple(int(v) for v in ln.split()[1:3]) == plan for ln in lines), lines
    # a cached entry is used as given (here: the plan that is not the default)
    path.write_text(f"{key} 0 0 1.0\n")
    assert _child(path) == (0, 0)
