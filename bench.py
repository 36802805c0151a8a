#!/usr/bin/env python3
"""Throughput of the diblock propagator hot path on GB300 (one JSON line on stdout).

A step is one full field update of the 128^3 gyroid-seeded SCFT workload (Ns=100,
fA=0.35, chiN=18, L=8 Rg): Boltzmann factors, forward march, Q, conjugate march with
fused contour quadrature, densities, H and the explicit-Euler field update.  One
step advances 2*M*Ns grid-point contour steps (M = 128^3).  The headline path runs
the propagators and FFTs in FP32 with FP64 quadrature, reductions and field update;
the plain FP64 path is measured on the same workload and reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 (launched by torchrun) each rank runs an independent replica of the
workload (its own seed): the path has no exchange step, so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1204_5434_gb300 import workloads as wl  # noqa: E402

METRIC = "grid-pt·contour-steps/s at 128³ (FP32-mixed vs FP64), % HBM roofline"
UNIT = "grid-pt·contour-steps/s"
WORK = wl.GYR128
# Mean algorithmic bytes per unit (one grid point, one contour step, one propagator)
# with each 3D FFT on chip: forward reads q_{n-1} and B and writes q_n (2e+f); the
# conjugate step also reads the partner q and reads+writes an FP64 accumulator
# (3e+f+2a).  Mean (5e+2f+2a)/2 with e=f=4, a=8 (FP32-mixed) or e=f=a=8 (FP64), real fields.
BYTES_PER_UNIT = {"fp32": 22.0, "fp64": 36.0}
# FP64 is bound by the GB300 FP64 pipe, whose rate is measured live (pft_fma_throughput,
# a DFMA loop over every SM) as the denominator of the FP64 roofline.  Flops per unit: in the
# usual 5 N log2 N convention a length-n complex transform of two paired real lines costs
# 2.5 log2(n) flops per real point, so the separable march's forward and inverse transform
# along each of the three axes cost 5 log2(M) per point and contour step -- the same count
# as a real-to-half-spectrum 3D transform pair -- plus about 6 pointwise flops (two
# Boltzmann multiplies, the diffusion multiplies, the quadrature update).
FP64_NOMINAL_TFLOPS = 1.25
# DRAM traffic of one launch of the separable march (one contour step of one
# propagator: a plane kernel or an x kernel in turn) on the FP32 128^3 path in steady state:
# dram__bytes_read.sum + dram__bytes_write.sum averaged over 60 consecutive launches of
# the second warm-up update of the bench workload, captured with caches left as the
# previous launches left them (so each launch is charged with the write-backs its stores
# cause).  Reads are nearly nil (the field and both factors stay in L2); the writes are the
# q slices.  Valid only for the kernel sources it was taken on: null once any changes.
TRAFFIC_FP32 = {"bytes_per_contour_step": 8607257.6,
                "sources": ("paper_1204_5434_gb300/csrc/pft_sep.cuh", "paper_1204_5434_gb300/csrc/pft_sepp.cuh",
                            "paper_1204_5434_gb300/csrc/pft_plane.cuh", "paper_1204_5434_gb300/csrc/pft_tma.cuh",
                            "paper_1204_5434_gb300/csrc/pft_batch.cuh", "paper_1204_5434_gb300/csrc/pft_passes.cuh",
                            "paper_1204_5434_gb300/csrc/pft_fft.cuh", "paper_1204_5434_gb300/csrc/pft_dd.cuh"),
                "sha256": "a5c42a028a5e668d181a9e1d713064fe9e968e698dac53e4ef9fae5b65572f79"}


def _traffic_fp32():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_FP32["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return TRAFFIC_FP32["bytes_per_contour_step"] if h.hexdigest() == TRAFFIC_FP32["sha256"] else None


def fp64_flops_per_unit(M):
    return 5.0 * math.log2(M) + 6.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _max_over_ranks(torch, x, ws, device):
    """MAX of a per-rank scalar over every rank of the process group (one rank: x)."""
    if ws <= 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.p = None
        self.path = os.path.join("/tmp", f"pft_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "25"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        # the sampler takes a moment to start: wait (at most 3 s) for its first line so that
        # the samples cover the timed region that follows
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0 and self.p.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _cpu_model():
    """CPU model of this host (lscpu's model name, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


ORACLE_SAMPLE_NS = 10


def _oracle_sample(workers=None, Ns=ORACLE_SAMPLE_NS):
    """Time the FP64 oracle on a bounded sample of the workload: one complete field update
    (both marches, Q, the contour quadrature, densities, H and the explicit-Euler field
    step) on the full 128^3 grid with Ns contour steps instead of the workload's 100, so
    that a sample is seconds, not minutes.  workers=None: numpy.fft on one core (the
    oracle as it stands); workers=k: the same oracle with its transforms on k threads of
    scipy.fft.  Returns (units/s, sample description, cores)."""
    import oracle as o
    w = WORK.with_(Ns=Ns)
    wp, wm = wl.fields(w)

    def update():
        s = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
        o.hamiltonian(wp, wm, s.lnQ, w.chiN, w.C, w.n, w.L, o.SCFT_REAL)
        o.scft_euler_step(wp, wm, s.phiA, s.phiB, w.chiN, w.lam)

    def timed():
        t0 = time.perf_counter()
        update()
        return time.perf_counter() - t0
    if workers is None:
        dt = timed()
        cores, how = 1, "numpy.fft, 1 core"
    else:
        with o.fft_workers(workers):
            dt = timed()
        cores, how = workers, f"scipy.fft with {workers} workers (other oracle arithmetic on 1 core)"
    units = 2 * w.M * w.Ns
    return units / dt, (f"one complete oracle field update (solve + H + Euler step) of the 128^3 workload at "
                        f"Ns={Ns} ({dt:.1f} s; {how})"), cores


def _config(ws):
    return {"workload": WORK.name, "grid": list(WORK.n), "L": list(WORK.L), "Ns": WORK.Ns, "fA": WORK.fA,
            "chiN": WORK.chiN, "step": "solve + SCFT Euler field update (lambda=0.1)",
            "units_per_step": 2 * WORK.M * WORK.Ns, "parallelism": f"replicas x{ws}",
            "l2": "q and q-dagger histories of 101 slices each (2 x 850 MB f32) stream through HBM every step; "
                  "no flush"}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    vals = []
    for i in range(args.warmup + args.steps):
        v, sample, cores = _oracle_sample(Ns=4)
        if i >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": _cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_device(pft, torch, h, stream, steps, warmup, units_per_step):
    """Device-resident steps (inputs already in HBM): solve + field step per step."""
    for _ in range(warmup):
        pft.pft_solve(h)
        pft.pft_field_step(h, pft.PFT_STEP_SCFT_EULER, WORK.lam)
    pft.pft_synchronize(h)
    s = torch.cuda.ExternalStream(stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        pft.pft_solve(h)
        pft.pft_field_step(h, pft.PFT_STEP_SCFT_EULER, WORK.lam)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def _variable_cell(pft, torch, prec, steps, warmup, wpa, wma, lam_L=0.05):
    """Variable-cell SCFT step of the same workload: solve, exact gradients (field
    gradients from the densities, box derivative by one recompute march), explicit
    Euler field update, cell update L_a += lam_L dlnQ/dL_a."""
    s = pft.System(WORK.n, WORK.L, WORK.Ns, WORK.fA, WORK.chiN, WORK.C, pft.PFT_SCFT_REAL, prec)
    h = s.h
    pft.pft_set_fields(h, wpa, wma)
    L = list(WORK.L)

    def one():
        pft.pft_solve(h)
        _, dq = pft.pft_gradients(h)
        pft.pft_field_step(h, pft.PFT_STEP_SCFT_EULER, WORK.lam)
        for a in range(3):
            L[a] += lam_L * dq[a]
        pft.pft_set_box(h, L)
    for _ in range(warmup):
        one()
    pft.pft_synchronize(h)
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    pft.pft_synchronize(h)
    ms = (time.perf_counter() - t0) * 1e3 / steps
    s.close()
    units = 3 * WORK.M * WORK.Ns  # forward, conjugate and the recompute march of the box derivative
    return {"ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT, "units_per_step": units,
            "step": "solve + gradients (field + box) + Euler field step + cell step (lam_L=0.05)",
            "timing": "host wall clock around synchronised steps (the gradient call reads back 3 scalars)"}


def _cl(pft, torch, w, prec, steps, warmup=1, checkpoint=0, plan=None):
    """Complex Langevin field updates (solve + Euler-Maruyama step with the device Philox
    noise) of a complex-field workload, timed with CUDA events on the context stream.
    checkpoint K >= 2 keeps every K-th q slice and recomputes segments (one extra march);
    plan: (code, streams) for pft_set_plan, else the context's default."""
    s = pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, pft.PFT_CL_COMPLEX, prec, seed=w.seed, checkpoint=checkpoint)
    h = s.h
    if plan is not None:
        pft.pft_set_plan(h, *plan)
    wp, wm = wl.fields(w)
    pft.pft_set_fields(h, wp, wm)

    def one():
        pft.pft_solve(h)
        pft.pft_field_step(h, pft.PFT_STEP_CL_EULER_MARUYAMA, w.dt)
    for _ in range(warmup):
        one()
    pft.pft_synchronize(h)
    st = torch.cuda.ExternalStream(pft.pft_get_stream(h))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        one()
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    obs = pft.pft_get_observables(h)
    mem = pft.pft_memory_bytes(h)
    hist_k = pft.pft_get_checkpoint(h)
    plan_used = list(pft.pft_get_plan(h))
    s.close()
    units = 2 * w.M * w.Ns
    bpu = 44.0 if prec == pft.PFT_FP32_MIXED else 72.0
    peak, _ = _peaks()
    return {"workload": w.name, "ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT,
            "hbm_roofline_frac": bpu * units / (ms * 1e-3) / 1e9 / peak, "bytes_per_unit": bpu,
            "device_bytes": mem, "history_interval": hist_k, "plan": plan_used,
            "H_last": [obs["H"].real, obs["H"].imag]}


def _variant(pft, torch, w, prec, steps, warmup=1, scheme=0, step_kind=None, step_size=None, plan=None):
    """Field updates of a workload with another contour scheme, field-step kind or march
    plan, timed with CUDA events on the context stream (fields resident on the device)."""
    kind = pft.PFT_SCFT_REAL if w.kind == wl.SCFT else pft.PFT_CL_COMPLEX
    if step_kind is None:
        step_kind = pft.PFT_STEP_SCFT_EULER if kind == pft.PFT_SCFT_REAL else pft.PFT_STEP_CL_EULER_MARUYAMA
    if step_size is None:
        step_size = w.lam if kind == pft.PFT_SCFT_REAL else w.dt
    arch = pft.PFT_ARCH_EDWARDS if w.arch == "edwards" else pft.PFT_ARCH_DIBLOCK
    s = pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, kind, prec, seed=w.seed, scheme=scheme, arch=arch, B=w.B)
    h = s.h
    if plan is not None:
        pft.pft_set_plan(h, *plan)
    wp, wm = wl.fields(w)
    pft.pft_set_fields(h, wp, wm)

    def one():
        pft.pft_solve(h)
        pft.pft_field_step(h, step_kind, step_size)
    for _ in range(warmup):
        one()
    pft.pft_synchronize(h)
    st = torch.cuda.ExternalStream(pft.pft_get_stream(h))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        one()
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    plan_used = list(pft.pft_get_plan(h))
    s.close()
    units = (1 if arch == pft.PFT_ARCH_EDWARDS else 2) * w.M * w.Ns  # propagators marched
    return {"workload": w.name, "ms_per_step": ms, "value": units / (ms * 1e-3), "unit": UNIT, "plan": plan_used}


def _adjoint_time(pft, torch, w, prec, reps=5):
    """Reverse-mode adjoint of a density loss after one solve (device arrays): ms per call
    and, for scale, ms per solve of the same context."""
    s = pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, pft.PFT_SCFT_REAL, prec, checkpoint=1)
    h = s.h
    wp, wm = wl.fields(w)
    pft.pft_set_fields(h, wp, wm)
    pft.pft_solve(h)
    ga = torch.randn(w.n, dtype=torch.float64, device="cuda")
    gb = torch.randn(w.n, dtype=torch.float64, device="cuda")
    op = torch.empty_like(ga)
    om = torch.empty_like(gb)
    pft.pft_adjoint(h, ga, gb, op, om)
    pft.pft_synchronize(h)
    st = torch.cuda.ExternalStream(pft.pft_get_stream(h))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        pft.pft_adjoint(h, ga, gb, op, om)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    e0.record(st)
    for _ in range(reps):
        pft.pft_solve(h)
    e1.record(st)
    e1.synchronize()
    ms_solve = e0.elapsed_time(e1) / reps
    s.close()
    return {"workload": w.name, "ms_per_adjoint": ms, "ms_per_solve": ms_solve,
            "note": "gradient of a loss on (phiA, phiB) w.r.t. (W+, W-) through the discrete march"}


def _library_fft_step(torch, wpa, wma, steps=5, warmup=2):
    """Comparison arm (not the product path): the same field update written with
    torch.fft (cuFFT) R2C/C2R transforms and separate elementwise kernels, FP32
    propagators and FP64 quadrature/update, on the headline workload, replayed as a
    captured CUDA graph."""
    w = WORK
    dev = torch.device("cuda")
    n = tuple(w.n)
    Ns = w.Ns
    ds = 1.0 / Ns
    NsA = int(math.floor(w.fA * Ns + 0.5))
    f64 = torch.float64
    kx = 2 * math.pi * torch.fft.fftfreq(n[0], d=w.L[0] / n[0], device=dev, dtype=f64)
    ky = 2 * math.pi * torch.fft.fftfreq(n[1], d=w.L[1] / n[1], device=dev, dtype=f64)
    kz = 2 * math.pi * torch.fft.rfftfreq(n[2], d=w.L[2] / n[2], device=dev, dtype=f64)
    k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    D = torch.exp(-k2 * ds).to(torch.float32)
    wp = torch.from_numpy(wpa).to(dev)
    wm = torch.from_numpy(wma).to(dev)
    q = torch.empty((Ns + 1,) + n, device=dev, dtype=torch.float32)

    def step(wp, wm):
        BA = torch.exp(-(wp - wm) * (ds / 2)).float()
        BB = torch.exp(-(wp + wm) * (ds / 2)).float()
        q[0].fill_(1.0)
        for s in range(1, Ns + 1):
            B = BA if s <= NsA else BB
            q[s] = B * torch.fft.irfftn(D * torch.fft.rfftn(B * q[s - 1]), s=n)
        Q = q[Ns].double().mean()
        accA = torch.zeros(n, device=dev, dtype=f64)
        accB = torch.zeros(n, device=dev, dtype=f64)
        qd = torch.ones(n, device=dev, dtype=torch.float32)
        for m in range(0, Ns + 1):
            if m > 0:
                nb = Ns + 1 - m
                B = BA if nb <= NsA else BB
                qd = B * torch.fft.irfftn(D * torch.fft.rfftn(B * qd), s=n)
            k = Ns - m
            prod = (q[k] * qd).double()
            if NsA > 0 and k <= NsA:
                accA += (0.5 if k in (0, NsA) else 1.0) * prod
            if NsA < Ns and k >= NsA:
                accB += (0.5 if k in (NsA, Ns) else 1.0) * prod
        phiA = accA * (ds / Q)
        phiB = accB * (ds / Q)
        wp2 = wp + w.lam * (phiA + phiB - 1.0)
        wm2 = wm - w.lam * (2.0 * wm / w.chiN + phiB - phiA)
        return wp2, wm2, Q

    # warm-up on a side stream (cuFFT plans are made here, outside the capture), then one
    # field update captured as a CUDA graph and replayed: the comparison pays no Python
    # launch overhead
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(warmup):
            step(wp, wm)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        wp2, wm2, Q = step(wp, wm)
        wp.copy_(wp2)
        wm.copy_(wm2)
    graph.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    units = 2 * w.M * Ns
    out = {"kind": "torch.fft (cuFFT) R2C/C2R + torch elementwise kernels, one field update captured as a "
                   "CUDA graph and replayed", "ms_per_step": ms,
           "value": units / (ms * 1e-3), "unit": UNIT, "Q_last": float(Q)}
    del graph
    return out


def _batch(pft, prec, updates=2):
    """The uneven batch: 256 instances, grids {32,48,64}^3, Ns {50,100,200}, half SCFT
    and half CL; graph-captured batched launches against one launch sequence per instance."""
    descs = wl.batch_instances()
    inst = [dict(n=d.n, L=d.L, Ns=d.Ns, fA=d.fA, chiN=d.chiN, C=d.C,
                 kind=pft.PFT_SCFT_REAL if d.kind == wl.SCFT else pft.PFT_CL_COMPLEX, seed=d.seed) for d in descs]
    out = {}
    for mode_name, mode in (("graphed", pft.PFT_BATCH_GRAPHED), ("per_instance", pft.PFT_BATCH_PER_INSTANCE),
                            ("graphed_autotuned", pft.PFT_BATCH_GRAPHED)):
        b = pft.pft_batch_create(inst, prec)
        try:
            for i, d in enumerate(descs):
                wp, wm = wl.sinusoid_fields(d)
                pft.pft_batch_set_fields(b, i, wp, wm)
            if mode_name == "graphed_autotuned":
                pft.pft_batch_autotune(b)
                out["plans"] = [pft.pft_batch_class_info(b, k) for k in range(pft.pft_batch_info(b)["classes"])]
            pft.pft_batch_run(b, 1, 0.1, 0.01, mode)
            pft.pft_batch_synchronize(b)
            t0 = time.perf_counter()
            pft.pft_batch_run(b, updates, 0.1, 0.01, mode)
            pft.pft_batch_synchronize(b)
            ms = (time.perf_counter() - t0) * 1e3 / updates
            info = pft.pft_batch_info(b)
            out[mode_name] = {"ms_per_update": ms, "value": info["units_per_update"] / (ms * 1e-3)}
            out["units_per_update"] = info["units_per_update"]
            out["classes"] = info["classes"]
            if mode == pft.PFT_BATCH_GRAPHED:
                out[mode_name]["launches_per_update"] = info["launches"]
        finally:
            pft.pft_batch_destroy(b)
    out["unit"] = UNIT
    out["instances"] = len(descs)
    out["graphed_over_per_instance"] = out["graphed"]["value"] / out["per_instance"]["value"]
    # algorithmic roofline of the batch: 22 B per unit for a real (SCFT) instance, 44 B for
    # a complex (CL) one, FP32-mixed, over the graphed update time
    bpu = {wl.SCFT: 22.0, wl.CL: 44.0}
    algo_bytes = sum(2 * d.M * d.Ns * bpu[d.kind] for d in descs)
    peak, src = _peaks()
    for k in ("graphed", "graphed_autotuned"):
        gbs = algo_bytes / (out[k]["ms_per_update"] * 1e-3) / 1e9
        out[k]["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                              "peak_source": f"{src} hbm_gbs", "algorithmic_bytes_per_update": algo_bytes}
    return out


def run(args):
    import torch

    from paper_1204_5434_gb300 import pft
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    peak, peak_src = _peaks()
    wpa, wma = wl.fields(WORK.with_(seed=WORK.seed + rank))
    units_per_step = 2 * WORK.M * WORK.Ns
    res = {}
    for prec_name, prec in (("fp32", pft.PFT_FP32_MIXED), ("fp64", pft.PFT_FP64)):
        sys_ = pft.System(WORK.n, WORK.L, WORK.Ns, WORK.fA, WORK.chiN, WORK.C, pft.PFT_SCFT_REAL, prec,
                          seed=1000 + rank)
        h = sys_.h
        stream = pft.pft_get_stream(h)
        dwp = torch.from_numpy(wpa).cuda()
        dwm = torch.from_numpy(wma).cuda()
        torch.cuda.synchronize()
        pft.pft_set_fields(h, dwp, dwm)
        steps = args.steps if prec_name == "fp32" else max(3, args.steps // 2)
        clocks = Clocks(local)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks.start()
        ms = _time_device(pft, torch, h, stream, steps, args.warmup, units_per_step)
        ck = clocks.stop()
        torch.cuda.synchronize()
        ms = _max_over_ranks(torch, ms, ws, "cuda")
        if ws > 1:
            torch.distributed.barrier()
        value = ws * units_per_step / (ms * 1e-3)
        # kernels per timed step: the nodes of the solve graph plus the field update
        n_solve, n_field = pft.pft_launch_counts(h)
        launches = n_solve + n_field if n_solve >= 0 else None
        # per-kernel device times of one eager step (events between launches)
        prof = pft.pft_profile_step(h, pft.PFT_STEP_SCFT_EULER, WORK.lam)
        # end-to-end through the public API with pinned host buffers
        hp = torch.from_numpy(wpa).pin_memory()
        hm = torch.from_numpy(wma).pin_memory()
        op = torch.empty_like(hp).pin_memory()
        om = torch.empty_like(hm).pin_memory()
        e2e_steps = max(2, steps // 2)
        for _ in range(1):
            pft.pft_set_fields(h, hp, hm)
            pft.pft_solve(h)
            pft.pft_field_step(h, pft.PFT_STEP_SCFT_EULER, WORK.lam)
            pft.pft_get_fields(h, op, om)
            pft.pft_get_observables(h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            pft.pft_set_fields(h, hp, hm)
            pft.pft_solve(h)
            pft.pft_field_step(h, pft.PFT_STEP_SCFT_EULER, WORK.lam)
            pft.pft_get_fields(h, op, om)
        pft.pft_synchronize(h)
        e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
        e2e_ms = _max_over_ranks(torch, e2e_ms, ws, "cuda")
        sys_.close()
        del dwp, dwm
        torch.cuda.empty_cache()
        bpu = BYTES_PER_UNIT[prec_name]
        # the contour step (plane kernel and x pass) over the timed region: units/s from
        # the event-timed graph replays, which include the quadrature and pointwise kernels
        step_ms = ms / (2 * WORK.Ns)
        achieved = bpu * WORK.M / (step_ms * 1e-3) / 1e9
        top = max(prof["kinds"].items(), key=lambda kv: kv[1]["ms"])
        if prec_name == "fp32":
            roof = {"bound": "hbm", "kernel": "separable march: y/z plane kernel and x kernel in turn, one launch a "
                                              "contour step, both propagators on two streams",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)", "bytes_per_unit": bpu,
                    "units_per_launch": WORK.M, "step_us": step_ms * 1e3, "traffic": _traffic_fp32(),
                    "traffic_note": "ncu dram read + write bytes per launch (one contour step of one "
                                    "propagator) in steady state, caches not flushed between launches; the "
                                    "field and both factors stay in L2, the writes are the q slices"}
        else:
            fpu = fp64_flops_per_unit(WORK.M)
            tf = fpu * WORK.M / (step_ms * 1e-3) / 1e12
            dfma = pft.pft_fma_throughput(pft.PFT_FP64)
            roof = {"bound": "alu", "kernel": "separable march on pencils: a y launch and an x or z launch per contour step; FP64 pipe",
                    "achieved": tf, "peak": dfma, "unit": "TFLOP/s", "frac": tf / dfma,
                    "peak_source": f"measured DFMA throughput of this GPU (pft_fma_throughput; nominal "
                                   f"{FP64_NOMINAL_TFLOPS} TFLOP/s)",
                    "flops_per_unit": fpu, "units_per_launch": WORK.M, "step_us": step_ms * 1e3,
                    "hbm_achieved_GBps": achieved, "hbm_frac": achieved / peak, "traffic": None}
        res[prec_name] = {
            "value": value, "ms_per_step": ms, "clocks": ck, "launches_per_step": launches,
            "roofline": roof,
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                            "share": round(v["ms"] / prof["total_ms"], 4) if prof["total_ms"] else None,
                            "logical_GBps": round(v["bytes_per_launch"] * v["launches"] / (v["ms"] * 1e-3) / 1e9, 1)
                            if v["ms"] > 0 and v["bytes_per_launch"] > 0 else None}
                        for k, v in prof["kinds"].items() if v["launches"]},
            "kernels_note": "device time per kernel class of one eager solve (events between launches, "
                            "two-member launches on one stream); logical_GBps counts every byte each launch "
                            "addresses, including spectrum round trips that L2 serves -- it is not DRAM "
                            "throughput",
            "top_kernel": top[0],
            "e2e": {"value": ws * units_per_step / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": 2 * WORK.M * 8, "d2h_bytes_per_step": 2 * WORK.M * 8},
        }
    vc = _variable_cell(pft, torch, pft.PFT_FP32_MIXED, max(2, args.steps // 3), 1, wpa, wma)
    cl = {"cl64_fp32": _cl(pft, torch, wl.CL64, pft.PFT_FP32_MIXED, 10),
          "cl64_fp64": _cl(pft, torch, wl.CL64, pft.PFT_FP64, 3),
          "cl256_fp32": _cl(pft, torch, wl.CL256, pft.PFT_FP32_MIXED, 3),
          "cl256_fp64": _cl(pft, torch, wl.CL256, pft.PFT_FP64, 1),
          # FP64 contexts with the double-float march (plan 4): FP64 history, quadrature and
          # update, the march's arithmetic as pairs of floats on the FP32 pipe
          "cl64_fp64_double_float": _cl(pft, torch, wl.CL64, pft.PFT_FP64, 5, plan=(4, 1)),
          "cl256_fp64_double_float": _cl(pft, torch, wl.CL256, pft.PFT_FP64, 1, plan=(4, 1)),
          "cl256_fp32_checkpoint14": _cl(pft, torch, wl.CL256, pft.PFT_FP32_MIXED, 2, checkpoint=14)}
    torch.cuda.empty_cache()
    variants = {
        # the paper's 4th-order scheme (three split steps per contour step): units are
        # 4th-order contour steps
        "rqm4_fp32": dict(_variant(pft, torch, WORK, pft.PFT_FP32_MIXED, 5, scheme=pft.PFT_SCHEME_RQM4),
                          scheme="RQM4 (Eq. 13), Simpson quadrature"),
        "rqm4_fp64": dict(_variant(pft, torch, WORK, pft.PFT_FP64, 2, scheme=pft.PFT_SCHEME_RQM4),
                          scheme="RQM4 (Eq. 13), Simpson quadrature"),
        # semi-implicit field steps (Eq. 11): one FP64 transform pair per update on top
        "sis_scft_fp32": dict(_variant(pft, torch, WORK, pft.PFT_FP32_MIXED, 10, step_kind=pft.PFT_STEP_SCFT_SIS),
                              step="solve + semi-implicit SCFT step (lambda=0.1)"),
        "sis_cl64_fp32": dict(_variant(pft, torch, wl.CL64, pft.PFT_FP32_MIXED, 10, step_kind=pft.PFT_STEP_CL_SIS),
                              step="solve + semi-implicit complex Langevin step"),
        # Edwards homopolymer model: one reversible chain (q-dagger = q), one march per solve
        "edwards_scft128_fp32": _variant(pft, torch, wl.EDW128, pft.PFT_FP32_MIXED, 10),
        "edwards_cl128_fp32": _variant(pft, torch, wl.EDWCL128, pft.PFT_FP32_MIXED, 10),
        "adjoint_fp32": _adjoint_time(pft, torch, WORK, pft.PFT_FP32_MIXED),
        # the FP64 line's workload with the double-float march (plan 4, two-member launches)
        "fp64_double_float": _variant(pft, torch, WORK, pft.PFT_FP64, max(3, args.steps // 4), warmup=2, plan=(4, 0)),
    }
    ddv = variants["fp64_double_float"]
    ddv["fp64_equivalent_TFLOPs"] = fp64_flops_per_unit(WORK.M) * ddv["value"] / 1e12
    ddv["over_measured_dfma_peak"] = ddv["fp64_equivalent_TFLOPs"] / pft.pft_fma_throughput(pft.PFT_FP64)
    ddv["speedup_over_ieee_fp64"] = res["fp64"]["ms_per_step"] / ddv["ms_per_step"]
    ddv["note"] = ("FP64 context, march in double-float arithmetic (value = hi + lo of two floats, about 48 "
                   "significant bits, FP32 pipe); FP64 history, quadrature, reductions and update; parity "
                   "against the FP64 oracle at the FP64 tolerances (tests/test_gpu_double_float.py)")
    torch.cuda.empty_cache()
    lib_fft = _library_fft_step(torch, wpa, wma)
    torch.cuda.empty_cache()
    batch = _batch(pft, pft.PFT_FP32_MIXED)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    cpu_v, cpu_sample, cpu_cores = _oracle_sample()
    ncpu = os.cpu_count() or 1
    cpu_all_v, cpu_all_sample, _ = _oracle_sample(workers=ncpu)
    main = res["fp32"]
    fp64 = res["fp64"]
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "precision": "f32 propagators/FFTs, f64 quadrature/reductions/update",
        "data": "synthetic",
        "config": _config(ws),
        "roofline": main["roofline"], "kernels": main["kernels"],
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cpu_cores, "kind": "oracle", "sample": cpu_sample,
                         "cpu_model": _cpu_model(),
                         "all_cores": {"value": cpu_all_v, "unit": UNIT, "cores": ncpu, "sample": cpu_all_sample}},
        "e2e": main["e2e"],
        "gpu_launches": main["launches_per_step"] * args.steps if main["launches_per_step"] else None,
        "gpu_launches_per_step": main["launches_per_step"], "clocks": main["clocks"],
        "fp64": {"value": fp64["value"], "ms_per_step": fp64["ms_per_step"], "roofline": fp64["roofline"],
                 "kernels": fp64["kernels"], "e2e": fp64["e2e"], "clocks": fp64["clocks"],
                 "note": "FP64 FFTs are bound by the GB300 FP64 pipe (about 1.2 TFLOP/s measured)"},
        "fp32_over_fp64": main["value"] / fp64["value"],
        "variable_cell": vc,
        "batch": batch,
        "complex_langevin": cl,
        "library_fft_comparison": dict(lib_fft, ours_over_library=main["value"] / lib_fft["value"]),
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    from paper_1204_5434_gb300 import build
    build.build()
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
