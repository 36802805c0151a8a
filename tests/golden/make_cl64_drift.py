"""Writes cl64_drift_oracle.json: the FP64 oracle's complex Langevin trajectory of the
64^3 diblock workload (L = 8, Ns = 100, fA = 0.3, chiN = 20, C = 50, dt = 0.01, fields
homogeneous plus N(0, 0.05) from seed 2), 1000 Euler-Maruyama steps (Eq. 9 with the
real Gaussian noise of Eq. 10) driven by the Philox4x32-10 stream with key 2 and
instance 0.  Recorded before every step k = 0..999 and after the last: H, and the
second density moments mean(phiA^2) and mean(phiA phiB) over the grid (complex).
Calls only the oracle and the seeded input generator; about an hour on one core.

    python tests/golden/make_cl64_drift.py [steps]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as o  # noqa: E402
from paper_1204_5434_gb300 import workloads as wl  # noqa: E402

SEED, INSTANCE = 2, 0


def main(steps=1000):
    w = wl.CL64
    wp, wm = wl.fields(w)
    dV = float(np.prod(w.L)) / float(np.prod(w.n))
    std = o.cl_noise_std(w.dt, w.C, dV)
    rec = {"H": [], "m2A": [], "mAB": []}
    t0 = time.time()
    for k in range(steps + 1):
        sol = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.CL_COMPLEX)
        H = o.hamiltonian(wp, wm, sol.lnQ, w.chiN, w.C, w.n, w.L, o.CL_COMPLEX)
        rec["H"].append([float(np.real(H)), float(np.imag(H))])
        m2A = np.mean(sol.phiA * sol.phiA)
        mAB = np.mean(sol.phiA * sol.phiB)
        rec["m2A"].append([float(m2A.real), float(m2A.imag)])
        rec["mAB"].append([float(mAB.real), float(mAB.imag)])
        if k == steps:
            break
        ep, em = o.cl_noise(SEED, INSTANCE, k, wp.size, std)
        wp, wm = o.cl_euler_maruyama_step(wp, wm, sol.phiA, sol.phiB, w.chiN, w.dt, ep.reshape(w.n), em.reshape(w.n))
        if k % 50 == 0:
            print(f"step {k}: H = {H:.6f}  ({time.time() - t0:.0f} s)", flush=True)
    out = {"workload": w.name, "n": list(w.n), "L": list(w.L), "Ns": w.Ns, "fA": w.fA, "chiN": w.chiN, "C": w.C,
           "dt": w.dt, "fields_seed": w.seed, "noise_seed": SEED, "noise_instance": INSTANCE, "steps": steps,
           "note": "written by tests/golden/make_cl64_drift.py from the FP64 oracle", **rec}
    with open(os.path.join(HERE, "cl64_drift_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1000)
