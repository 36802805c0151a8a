"""Run a named workload from the command line: field updates through the public API with
the fields resident on the device, then one line of observables.

    python -m paper_1204_5434_gb300.run --workload gyr128 --precision fp32 \
        --steps 1 --warmup 3 [--scheme split2|rqm4] [--march auto|passes] [--adjoint]

Each update is one pft_solve (both propagators, Q, densities, H) and one explicit field
step (SCFT Euler for SCFT workloads, Euler-Maruyama with device Philox noise for complex
Langevin ones).  The warm-up updates run first, then the timed ones; the device time of
the timed updates is taken with CUDA events on the library's stream (through torch,
when it is importable).  Because the
launches of one update are fixed, an external profiler can select them by count (the
warm-up updates launch the same kernels first).
"""
from __future__ import annotations

import argparse
import json
import sys

from . import pft
from . import workloads as wl

_PREC = {"fp32": pft.PFT_FP32_MIXED, "fp64": pft.PFT_FP64}
_SCHEME = {"split2": pft.PFT_SCHEME_SPLIT2, "rqm4": pft.PFT_SCHEME_RQM4}
_MARCH = {"auto": pft.PFT_MARCH_AUTO, "passes": pft.PFT_MARCH_PASSES}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="gyr128", choices=sorted(wl.ALL))
    ap.add_argument("--precision", default="fp32", choices=sorted(_PREC))
    ap.add_argument("--scheme", default="split2", choices=sorted(_SCHEME))
    ap.add_argument("--march", default="auto", choices=sorted(_MARCH))
    ap.add_argument("--Ns", type=int, default=0, help="override the workload's contour steps")
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--no-graph", action="store_true", help="launch each solve eagerly")
    ap.add_argument("--plan", default="", help="fix the march plan as PLANE,STREAMS (pft_set_plan), e.g. 2,1")
    ap.add_argument("--adjoint", action="store_true",
                    help="after the updates, one reverse-mode adjoint of a seeded linear loss on the "
                         "densities (real SCFT diblock workloads)")
    a = ap.parse_args(argv)
    w = wl.ALL[a.workload]
    if a.Ns > 0:
        w = w.with_(Ns=a.Ns)
    kind = pft.PFT_SCFT_REAL if w.kind == wl.SCFT else pft.PFT_CL_COMPLEX
    step_kind = pft.PFT_STEP_SCFT_EULER if kind == pft.PFT_SCFT_REAL else pft.PFT_STEP_CL_EULER_MARUYAMA
    step_size = w.lam if kind == pft.PFT_SCFT_REAL else w.dt
    wp, wm = wl.fields(w)
    arch = pft.PFT_ARCH_EDWARDS if w.arch == "edwards" else pft.PFT_ARCH_DIBLOCK
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, kind, _PREC[a.precision], use_graph=not a.no_graph,
                    seed=w.seed, march=_MARCH[a.march], scheme=_SCHEME[a.scheme], arch=arch, B=w.B) as s:
        s.set_fields(wp, wm)
        h = s.h
        if a.plan:
            pl, st = (int(v) for v in a.plan.split(","))
            pft.pft_set_plan(h, pl, st)
        for _ in range(a.warmup):
            pft.pft_solve(h)
            pft.pft_field_step(h, step_kind, step_size)
        pft.pft_synchronize(h)
        try:
            import torch
            ts = torch.cuda.ExternalStream(pft.pft_get_stream(h))
            ev = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
        except (ImportError, RuntimeError):
            ts = None
        ms = None
        if ts is not None:
            ev[0].record(ts)
        for _ in range(a.steps):
            pft.pft_solve(h)
            pft.pft_field_step(h, step_kind, step_size)
        if ts is not None:
            ev[1].record(ts)
            ev[1].synchronize()
            ms = ev[0].elapsed_time(ev[1]) / max(1, a.steps)
        pft.pft_synchronize(h)
        pft.pft_solve(h)
        obs = s.observables()
        n_solve, n_field = pft.pft_launch_counts(h)
        plan_used = list(pft.pft_get_plan(h))
        adj_ms = None
        if a.adjoint:
            import time

            import numpy as np
            rng = np.random.default_rng(w.seed)
            GA, GB = rng.normal(size=w.n), rng.normal(size=w.n)
            t0 = time.perf_counter()
            s.adjoint(GA, GB)
            adj_ms = (time.perf_counter() - t0) * 1e3
    units = (1 if arch == pft.PFT_ARCH_EDWARDS else 2) * w.M * w.Ns  # propagators marched
    out = {"workload": w.name, "precision": a.precision, "scheme": a.scheme, "Ns": w.Ns, "steps": a.steps,
           "ms_per_update": ms, "units_per_s": (units / (ms * 1e-3)) if ms else None,
           "kernels_per_solve": n_solve, "kernels_per_field_step": n_field, "plan": plan_used,
           "Q": [obs["Q"].real, obs["Q"].imag], "H": [obs["H"].real, obs["H"].imag]}
    if a.adjoint:
        out["adjoint_ms_host_wall"] = adj_ms
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
