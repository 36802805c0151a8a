"""Complex Langevin over 1000 steps on the 64^3 diblock workload (Euler-Maruyama, Eq. 9,
real Gaussian noise of Eq. 10 from the device Philox stream with the key and instance
the oracle used): the FP64 (IEEE and double-float march) and FP32-mixed GPU trajectories
against the FP64 oracle trajectory stored by tests/golden/make_cl64_drift.py.

Checked: the first steps follow the oracle step for step (identical noise; FP64 to
1e-10 relative in H, FP32-mixed to 1e-5), and over steps 100..1000 the running means of
Re H, Re mean(phiA^2) and Re mean(phiA phiB) agree with the oracle's within 5 standard
errors (block averages of 100 steps; the trajectories are chaotic, so later steps are
compared statistically).  The drift table is printed."""
import json
import os

import numpy as np
import pytest

from paper_1204_5434_gb300 import pft
from paper_1204_5434_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cl64_drift_oracle.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _run(prec, ref, steps, plan=None):
    w = wl.CL64
    wp, wm = wl.fields(w)
    rec = {"H": [], "m2A": [], "mAB": []}
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, pft.PFT_CL_COMPLEX, prec, seed=ref["noise_seed"],
                    instance=ref["noise_instance"]) as s:
        if plan is not None:
            pft.pft_set_plan(s.h, plan, 1)
        s.set_fields(wp, wm)
        for k in range(steps + 1):
            s.solve()
            obs = s.observables()
            phiA, phiB = s.densities()
            rec["H"].append(obs["H"])
            rec["m2A"].append(np.mean(phiA * phiA))
            rec["mAB"].append(np.mean(phiA * phiB))
            if k < steps:
                s.field_step(w.dt)
    return {k: np.asarray(v) for k, v in rec.items()}


def _blocks(x, start, size):
    x = np.real(np.asarray(x))[start:]
    nb = len(x) // size
    return x[: nb * size].reshape(nb, size).mean(axis=1)


def test_cl64_1000_steps_against_the_oracle():
    if not os.path.exists(GOLDEN):
        pytest.fail(f"{GOLDEN} is missing: run tests/golden/make_cl64_drift.py")
    with open(GOLDEN) as f:
        ref = json.load(f)
    steps = ref["steps"]
    oref = {k: np.array([complex(a, b) for a, b in ref[k]]) for k in ("H", "m2A", "mAB")}
    runs = {"FP64": _run(pft.PFT_FP64, ref, steps),
            "FP64 double-float march": _run(pft.PFT_FP64, ref, steps, plan=4),
            "FP32-mixed": _run(pft.PFT_FP32_MIXED, ref, steps)}
    # step for step at the start
    for name, tol in (("FP64", 1e-10), ("FP64 double-float march", 1e-10), ("FP32-mixed", 1e-5)):
        h = runs[name]["H"][:6]
        assert np.max(np.abs(h - oref["H"][:6]) / np.abs(oref["H"][:6])) <= tol, name
    # statistics over steps 100..steps
    lines = [f"CL 64^3, {steps} steps: running means over steps 100..{steps}, drift in block standard errors"]
    for q in ("H", "m2A", "mAB"):
        bo = _blocks(oref[q], 100, 100)
        se = max(np.std(bo, ddof=1) / np.sqrt(len(bo)), 1e-12 * abs(np.mean(bo)))
        line = f"  Re {q}: oracle {np.mean(bo):.8g} +- {se:.3g}"
        for name, r in runs.items():
            b = _blocks(r[q], 100, 100)
            d = (np.mean(b) - np.mean(bo)) / se
            line += f"; {name} {np.mean(b):.8g} ({d:+.2f} se)"
            assert abs(d) <= 5.0, (q, name, d)
        lines.append(line)
    for name, r in runs.items():
        dev = np.abs(r["H"] - oref["H"]) / np.abs(oref["H"])
        first = int(np.argmax(dev > 1e-6)) if np.any(dev > 1e-6) else None
        lines.append(f"  {name}: max relative |H - H_oracle| {dev.max():.2e}; first step above 1e-6: {first}")
    print("\n" + "\n".join(lines))
