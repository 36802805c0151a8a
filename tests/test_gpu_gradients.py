"""GPU parity of the exact gradients (field gradients and box derivative / stress)
against the FP64 oracle, and the two identities that pin them on the GPU path itself:
delta lnQ / delta w = -phi/V (finite differences of the GPU's own lnQ) and dlnQ/dL_a
against finite differences of the GPU's lnQ in the box length."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft
from paper_1204_5434_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
FP64, FP32 = pft.PFT_FP64, pft.PFT_FP32_MIXED
SCFT = pft.PFT_SCFT_REAL


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _fields(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.3, n), rng.normal(0, 1.0, n)


def fd5(f, h):
    return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)


# FP64 with its default plan and with the double-float march (plan 4) producing the histories
@pytest.mark.parametrize("prec,tol,plan", [(FP64, 1e-9, None), (FP64, 1e-9, 4), (FP32, 2e-4, None)])
@pytest.mark.parametrize("n,L,Ns,fA", [((16, 12, 8), (4.0, 3.0, 2.0), 20, 0.35), ((12, 24, 16), (3.0, 6.0, 4.0), 16, 0.5)])
def test_gradients_match_oracle(n, L, Ns, fA, prec, tol, plan):
    chiN, C = 18.0, 2.0
    wp, wm = _fields(n, 31)
    ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    H = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, o.SCFT_REAL)
    gq = o.dlnQ_dL(ref, n, L)
    gH = o.dH_dL(H, ref, C, n, L)
    gp, gm = o.dH_dfields(wp, wm, ref, chiN, C, n, L, o.SCFT_REAL)
    with pft.System(n, L, Ns, fA, chiN, C, SCFT, prec) as s:
        if plan is not None:
            pft.pft_set_plan(s.h, plan, 1)
        s.set_fields(wp, wm)
        s.solve()
        a, b, dL, dq = s.gradients()
    err_q = max(abs(dq[i] - gq[i]) / max(abs(gq[i]), 1e-300) for i in range(3))
    err_H = max(abs(dL[i] - gH[i]) / abs(gH[i]) for i in range(3))
    print(f"\nstress prec={prec}: dlnQ/dL rel {err_q:.2e}, dH/dL rel {err_H:.2e}")
    assert err_q <= tol, (dq, gq)
    assert err_H <= tol, (dL, gH)
    ft = 1e-12 if prec == FP64 else 2e-5
    assert np.max(np.abs(a - gp)) <= ft * C * np.prod(L) / np.prod(n) * 10
    assert np.max(np.abs(b - gm)) <= ft * C * np.prod(L) / np.prod(n) * 10


def test_density_identity_on_gpu():
    """d lnQ / d W+_j = -(phiA+phiB)_j / M using the GPU's own lnQ (FP64)."""
    n, L, Ns, fA = (8, 8, 12), (2.0, 2.0, 3.0), 16, 0.35
    wp, wm = _fields(n, 32)
    with pft.System(n, L, Ns, fA, 15.0, 1.0, SCFT, FP64) as s:
        s.set_fields(wp, wm)
        s.solve()
        phiA, phiB = s.densities()

        def lnQ_at(dwp, dwm):
            s.set_fields(wp + dwp, wm + dwm)
            s.solve()
            return s.observables()["lnQ"].real
        # round-off floor of the five-point difference: about 18 ulps of lnQ (~4e-16
        # each for |lnQ| ~ 1) divided by 12 h = 1.2e-2, i.e. ~6e-13 absolute
        fd_floor = 1e-12
        for j in (5, 300, 700):
            idx = np.unravel_index(j, n)
            e = np.zeros(n)
            e[idx] = 1.0
            fp = fd5(lambda h: lnQ_at(h * e, 0 * e), 1e-3)
            fm = fd5(lambda h: lnQ_at(0 * e, h * e), 1e-3)
            M = wp.size
            assert abs(fp + (phiA + phiB)[idx] / M) <= 1e-9 * abs((phiA + phiB)[idx] / M) + fd_floor
            assert abs(fm - (phiA - phiB)[idx] / M) <= 1e-9 * abs((phiA - phiB)[idx] / M) + fd_floor


def test_stress_identity_on_gpu():
    """dlnQ/dL_a from pft_gradients against finite differences of the GPU's lnQ in L_a."""
    n, L, Ns, fA = (16, 8, 12), (4.0, 2.5, 3.0), 16, 0.35
    wp, wm = _fields(n, 33)
    with pft.System(n, L, Ns, fA, 15.0, 1.0, SCFT, FP64) as s:
        s.set_fields(wp, wm)
        s.solve()
        _, _, _, dq = s.gradients(want_fields=False)
        for a in range(3):
            def f(h):
                Lh = list(L)
                Lh[a] += h
                s.set_box(Lh)
                s.solve()
                return s.observables()["lnQ"].real
            fd = fd5(f, 1e-3)
            assert abs(fd - dq[a]) <= 1e-8 * abs(dq[a]), (a, fd, dq[a])
            s.set_box(L)


def test_variable_cell_relaxation_lowers_h():
    """A few steps of the gyroid-seeded 64^3 variable-cell SCFT (fields by explicit Euler,
    box by L_a += lam_L dlnQ/dL_a) against the oracle's identical loop."""
    w = wl.GYR64.with_(n=(32, 32, 32), Ns=40)
    wp, wm = wl.fields(w)
    L = np.array(w.L)
    lamL = 0.05
    with pft.System(w.n, tuple(L), w.Ns, w.fA, w.chiN, w.C, SCFT, FP64) as s:
        s.set_fields(wp, wm)
        for it in range(3):
            s.solve()
            _, _, _, dq = s.gradients(want_fields=False)
            ref = o.solve(wp, wm, w.n, tuple(L), w.Ns, w.fA, o.SCFT_REAL)
            gq = o.dlnQ_dL(ref, w.n, tuple(L))
            assert np.max(np.abs(np.array(dq) - gq) / np.abs(gq)) <= 1e-9
            s.field_step(w.lam)
            wp, wm = o.scft_euler_step(wp, wm, ref.phiA, ref.phiB, w.chiN, w.lam)
            L = L + lamL * np.array(dq)
            s.set_box(tuple(L))
        gp, gm = s.get_fields()
    assert np.max(np.abs(gm - wm)) <= 1e-10


def test_box_derivative_on_the_plane_kernel_64cubed_fp32():
    """64^3 FP32-mixed: the forward spectra of the box derivative come from the plane
    kernel's first step (z and y forward in one kernel) -- against the oracle."""
    w = wl.GYR64.with_(Ns=12)
    wp, wm = wl.fields(w)
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    gq = o.dlnQ_dL(ref, w.n, w.L)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, FP32) as s:
        s.set_fields(wp, wm)
        s.solve()
        assert pft.pft_get_plan(s.h)[0] >= 1
        _, _, _, dq = s.gradients(want_fields=False)
    err = max(abs(dq[i] - gq[i]) / abs(gq[i]) for i in range(3))
    print(f"\nbox derivative 64^3 FP32 (plane path) rel err {err:.2e}")
    assert err <= 2e-4


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_box_derivative_128cubed_matches_oracle(prec):
    """128^3 gyroid workload, Ns = 10: dlnQ/dL_a in both precisions against the oracle's
    dlnQ_dL (FP32-mixed: the forward spectra from the plane kernel)."""
    w = wl.GYR128.with_(Ns=10)
    wp, wm = wl.fields(w)
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    gq = o.dlnQ_dL(ref, w.n, w.L)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, prec) as s:
        s.set_fields(wp, wm)
        s.solve()
        if prec == FP32:
            assert pft.pft_get_plan(s.h)[0] >= 1
        dq = s.gradients(want_fields=False)[3]
    err = max(abs(dq[i] - gq[i]) / abs(gq[i]) for i in range(3))
    print(f"\nbox derivative 128^3 prec={prec} vs oracle: rel err {err:.2e}")
    assert err <= (1e-9 if prec == FP64 else 2e-4)
