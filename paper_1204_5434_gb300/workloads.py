"""Seeded synthetic inputs for the diblock workloads (shared by tests, bench and smoke).

This module only draws fields and states workload parameters; it holds none of the
method's arithmetic.  All fields are float64 (SCFT, Wick-rotated real W+ and W-) or
complex128 (complex Langevin omega+ and omega-), row-major [x][y][z], from
``numpy.random.default_rng(seed)``.  "N(0, s)" means an i.i.d. normal draw with
standard deviation s per grid point.  The parameter sets follow the paper's own
workloads: a lamellar SCFT seed (cos along x), a gyroid level-set seed for 3D SCFT,
and homogeneous complex Langevin starts (the paper's LAM, GYR and CL examples).
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

SCFT = "scft"
CL = "cl"


@dataclass(frozen=True)
class Workload:
    name: str
    n: tuple
    L: tuple
    Ns: int
    fA: float
    chiN: float
    C: float
    kind: str            # "scft" (real W+/W-) or "cl" (complex omega+/omega-)
    seed: int
    seed_kind: str       # "lam", "gyroid", "homogeneous"
    amp: float           # amplitude of the periodic part of W-
    noise: float         # std of the i.i.d. normal part
    lam: float = 0.1     # SCFT relaxation step
    dt: float = 0.01     # CL time step
    steps: int = 1
    arch: str = "diblock"  # "diblock" or "edwards" (homopolymer in implicit solvent, one field)
    B: float = 0.0       # Edwards excluded-volume parameter

    @property
    def M(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _coords(n, L):
    return [np.arange(n[a]) * (L[a] / n[a]) for a in range(3)]


def fields(wl: Workload):
    """(wp, wm) for the workload: real float64 in SCFT mode, complex128 in CL mode."""
    rng = np.random.default_rng(wl.seed)
    n = tuple(int(v) for v in wl.n)
    x, y, z = _coords(n, wl.L)
    if wl.seed_kind == "lam":
        wm = np.broadcast_to((wl.amp * np.cos(2 * np.pi * x / wl.L[0]))[:, None, None], n).copy()
        wm += rng.normal(0.0, wl.noise, n)
        wp = np.zeros(n)
    elif wl.seed_kind == "gyroid":
        X = (2 * np.pi * x / wl.L[0])[:, None, None]
        Y = (2 * np.pi * y / wl.L[1])[None, :, None]
        Z = (2 * np.pi * z / wl.L[2])[None, None, :]
        G = np.sin(X) * np.cos(Y) + np.sin(Y) * np.cos(Z) + np.sin(Z) * np.cos(X)
        wm = wl.amp * G + rng.normal(0.0, wl.noise, n)
        wp = rng.normal(0.0, wl.noise, n)
    elif wl.seed_kind == "homogeneous":
        # homogeneous melt start: omega- at chiN (2 fA - 1)/2, omega+ at 0, plus noise
        wp = rng.normal(0.0, wl.noise, n)
        wm = wl.chiN * (2 * wl.fA - 1) / 2 + rng.normal(0.0, wl.noise, n)
    elif wl.seed_kind == "edwards_saddle":
        # homogeneous mean-field saddle of the Edwards model, W = i omega = C/B, plus noise;
        # the second field is unused (zeros)
        wp = wl.C / wl.B + rng.normal(0.0, wl.noise, n)
        wm = np.zeros(n)
        if wl.kind == CL:
            return (-1j * wp).astype(np.complex128), wm.astype(np.complex128)
    elif wl.seed_kind == "random":
        wp = rng.normal(0.0, wl.noise, n)
        wm = rng.normal(0.0, wl.amp, n)
    else:
        raise ValueError(wl.seed_kind)
    if wl.kind == CL:
        return wp.astype(np.complex128), wm.astype(np.complex128)
    return np.ascontiguousarray(wp, dtype=np.float64), np.ascontiguousarray(wm, dtype=np.float64)


# The paper's workload shapes, at the sizes this library is exercised on.
LAM32 = Workload("lamellar SCFT 32^3, L=4, Ns=64, fA=0.5, chiN=15", (32, 32, 32), (4.0, 4.0, 4.0),
                 64, 0.5, 15.0, 1.0, SCFT, 1, "lam", 5.0, 0.1, lam=0.1, steps=50)
CL64 = Workload("complex Langevin 64^3, L=8, Ns=100, fA=0.3, chiN=20, C=50", (64, 64, 64), (8.0, 8.0, 8.0),
                100, 0.3, 20.0, 50.0, CL, 2, "homogeneous", 0.0, 0.05, dt=0.01, steps=1000)
GYR64 = Workload("gyroid-seeded SCFT 64^3, L=8, Ns=100, fA=0.35, chiN=18", (64, 64, 64), (8.0, 8.0, 8.0),
                 100, 0.35, 18.0, 1.0, SCFT, 4, "gyroid", 4.0, 0.1, lam=0.1, steps=200)
GYR128 = GYR64.with_(name="gyroid-seeded SCFT 128^3, L=8, Ns=100, fA=0.35, chiN=18", n=(128, 128, 128))
CL256 = Workload("complex Langevin 256^3, L=16, Ns=200, fA=0.5, chiN=14, C=100", (256, 256, 256), (16.0, 16.0, 16.0),
                 200, 0.5, 14.0, 100.0, CL, 5, "homogeneous", 0.0, 0.05, dt=0.005, steps=200)
CL128 = CL64.with_(name="complex Langevin 128^3, L=8, Ns=100, fA=0.3, chiN=20, C=50", n=(128, 128, 128))

# Edwards homopolymer solution (Eq. 2): SCFT and complex Langevin around the homogeneous saddle
EDW128 = Workload("Edwards homopolymer SCFT 128^3, L=8, Ns=100, B=1, C=20", (128, 128, 128), (8.0, 8.0, 8.0),
                  100, 1.0, 1.0, 20.0, SCFT, 6, "edwards_saddle", 0.0, 0.1, lam=0.1, arch="edwards", B=1.0)
EDWCL128 = EDW128.with_(name="Edwards homopolymer CL 128^3, L=8, Ns=100, B=1, C=20", kind=CL, dt=0.01)

ALL = {"lam32": LAM32, "cl64": CL64, "gyr64": GYR64, "gyr128": GYR128, "cl128": CL128, "cl256": CL256,
       "edw128": EDW128, "edwcl128": EDWCL128}


def batch_instances(count: int = 256, seed: int = 3):
    """Uneven batch of independent instances: grids from {32^3, 48^3, 64^3}, Ns from
    {50, 100, 200}, L = n/8 Rg, fA ~ U[0.25, 0.5], chiN ~ U[12, 25]; the first half SCFT
    (real fields), the second half CL (complex).  W- is a sum of four random low-k
    sinusoids with amplitudes U(0, 2) plus N(0, 0.1); W+ is N(0, 0.1)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nn = int(rng.choice([32, 48, 64]))
        Ns = int(rng.choice([50, 100, 200]))
        fA = float(rng.uniform(0.25, 0.5))
        chiN = float(rng.uniform(12, 25))
        kind = SCFT if i < count // 2 else CL
        wl = Workload(f"batch[{i}]", (nn, nn, nn), (nn / 8.0,) * 3, Ns, fA, chiN, 50.0 if kind == CL else 1.0,
                      kind, int(rng.integers(1 << 31)), "sinusoids", 0.0, 0.1, lam=0.1, dt=0.01)
        out.append(wl)
    return out


def sinusoid_fields(wl: Workload):
    """Fields of one batch instance (see ``batch_instances``)."""
    rng = np.random.default_rng(wl.seed)
    n = tuple(int(v) for v in wl.n)
    x, y, z = _coords(n, wl.L)
    wm = np.zeros(n)
    for _ in range(4):
        m = rng.integers(-2, 3, size=3)
        a = rng.uniform(0, 2)
        th = rng.uniform(0, 2 * np.pi)
        ph = (2 * np.pi * (m[0] * x[:, None, None] / wl.L[0] + m[1] * y[None, :, None] / wl.L[1]
                           + m[2] * z[None, None, :] / wl.L[2]) + th)
        wm += a * np.cos(ph)
    wm += rng.normal(0.0, 0.1, n)
    wp = rng.normal(0.0, 0.1, n)
    if wl.kind == CL:
        return wp.astype(np.complex128), wm.astype(np.complex128)
    return wp, wm
