"""The large complex Langevin workload's code path (256-point complex pencils) against the
FP64 oracle.

The complex Langevin 256^3 workload (L=16, fA=0.5, chiN=14, C=100; Eqs. 5, 8 and 13 with
complex fields) runs no plane kernel: its complex z transforms of length 256 (the fused
z-inverse / z-forward pencils), its x pass of length 256 and, at 256^3, its y passes all
take the pencil kernels.  These tests drive exactly the plan the bench times in both
precisions -- the separable march on pencils (a y launch and an x or z launch per contour
step; in FP32 the x and z kernels stage the Boltzmann factor's tile in shared memory) -- with two chains,
full history (or every K-th slice) -- on seeded complex fields and compare Q, H, phiA,
phiB and propagator slices element by element with the oracle.

Tolerances as in test_gpu_parity: FP64 relative 1e-12 on Q, 1e-10 max-abs on phi, 1e-12
(relative to the slice maximum) on propagator slices; FP32-mixed 2e-5 on each.  H is
checked through the intensive h = H/(C V), absolutely (FP64 1e-12, FP32 2e-5): from the
homogeneous start of this workload H is a near-cancellation of its two terms in Eq. 3
(|H| ~ 0.006 against terms ~ 2.5, with Q ~ 1 and lnQ ~ 1e-4), so a relative bound on H
itself would ask for more digits than Q carries.
"""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft
from paper_1204_5434_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64, FP32 = pft.PFT_FP64, pft.PFT_FP32_MIXED
CL = pft.PFT_CL_COMPLEX
TOL = {FP64: dict(Q=1e-12, H=1e-12, phi=1e-10, q=1e-12), FP32: dict(Q=2e-5, h=2e-5, phi=2e-5, q=2e-5)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _complex_fields(w, seed):
    """The workload's homogeneous start plus an imaginary part N(0, 0.05) on both fields,
    so that every complex product of the march is exercised."""
    wp, wm = wl.fields(w)
    rng = np.random.default_rng(seed)
    return wp + 1j * rng.normal(0, 0.05, w.n), wm + 1j * rng.normal(0, 0.05, w.n)


def _rel(a, b):
    return abs(a - b) / abs(b)


def _check(w, prec, K, wp, wm):
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.CL_COMPLEX)
    Href = o.hamiltonian(wp, wm, ref.lnQ, w.chiN, w.C, w.n, w.L, o.CL_COMPLEX)
    t = TOL[prec]
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, CL, prec, seed=w.seed, checkpoint=K) as s:
        # the plan the bench's complex Langevin 256^3 line runs (the separable march on
        # pencils), two chains on two streams
        assert pft.pft_get_plan(s.h) == (3, 1)
        assert pft.pft_get_checkpoint(s.h) == (1 if K in (0, 1) else K)
        s.set_fields(wp, wm)
        s.solve()
        obs = s.observables()
        phiA, phiB = s.densities()
        eq = 0.0
        slices = [(0, w.Ns), (1, w.Ns)] + ([(0, 1), (2, 1)] if K in (0, 1) else [])
        for which, k in slices:
            g = s.propagator(which, k)
            hist = ref.q if which == 0 else ref.qd
            e = np.max(np.abs(g - hist[k])) / np.max(np.abs(hist[k]))
            eq = max(eq, e)
            assert e <= t["q"], (which, k, e)
    eQ = _rel(obs["Q"], ref.Q)
    ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
    V = float(np.prod(w.L))
    eH = abs(obs["H"] - Href) / (w.C * V)
    print(f"\nCL {w.n} Ns={w.Ns} prec={prec} K={K}: Q rel {eQ:.2e} H {eH:.2e} phi abs {ephi:.2e} "
          f"slices rel {eq:.2e}")
    assert eQ <= t["Q"] and ephi <= t["phi"]
    assert eH <= (1e-12 if prec == FP64 else t["h"])


@pytest.mark.parametrize("K", [1, 2])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_cl_256_pencils_match_oracle(prec, K):
    """256 x 16 x 256 complex fields, Ns = 4: the complex 256-point z and x pencils of the
    large workload, with the full history and with every second slice kept (the
    conjugate march recomputes the dropped ones)."""
    w = wl.CL256.with_(n=(256, 16, 256), L=(16.0, 1.0, 16.0), Ns=4)
    wp, wm = _complex_fields(w, 501)
    _check(w, prec, K, wp, wm)


def test_cl_256cubed_fp32_matches_oracle():
    """The full 256^3 grid in FP32-mixed (Ns = 2 keeps the oracle's histories to a few GB):
    the same kernels, grid and plan as the timed complex Langevin 256^3 update."""
    w = wl.CL256.with_(Ns=2)
    wp, wm = _complex_fields(w, 502)
    _check(w, FP32, 0, wp, wm)
