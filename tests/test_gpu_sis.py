"""GPU parity of the semi-implicit field steps (Eq. 11) against the oracle: the W+ / omega+
increment is transformed (FP64), divided by 1 + a g_D(k) with the whole-chain Debye
function, and transformed back; the exchange field takes its linear term implicitly.
Tolerances: FP64 fields 1e-12 (SCFT) and 1e-10 (CL, as for the Euler-Maruyama step);
FP32-mixed 1e-5 on the fields (the densities carry ~1e-6, times the step size)."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu

FP64, FP32 = pft.PFT_FP64, pft.PFT_FP32_MIXED
SCFT, CL = pft.PFT_SCFT_REAL, pft.PFT_CL_COMPLEX


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _fields(n, kind, seed, amp_p=0.3, amp_m=1.0):
    rng = np.random.default_rng(seed)
    wp = rng.normal(0, amp_p, n)
    wm = rng.normal(0, amp_m, n)
    if kind == CL:
        wp = wp + 1j * rng.normal(0, amp_p, n)
        wm = wm + 1j * rng.normal(0, 0.3 * amp_m, n)
    return wp, wm


CASES = [((16, 12, 8), (4.0, 3.0, 2.0), 16, 0.4), ((12, 12, 12), (3.0, 3.0, 3.0), 13, 0.5),
         ((48, 4, 6), (6.0, 1.0, 1.5), 10, 0.6), ((64, 64, 64), (8.0, 8.0, 8.0), 20, 0.35)]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("lam", [0.1, 2.0])
@pytest.mark.parametrize("case", CASES)
def test_scft_sis_step_matches_oracle(case, lam, prec):
    n, L, Ns, fA = case
    chiN = 15.0
    wp, wm = _fields(n, SCFT, 80 + Ns)
    ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    ep, em = o.scft_sis_step(wp, wm, ref.phiA, ref.phiB, chiN, lam, n, L)
    with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, prec) as s:
        s.set_fields(wp, wm)
        s.solve()
        s.field_step(lam, semi_implicit=True)
        gp, gm = s.get_fields()
        s.solve()
        obs = s.observables()
    tol = 1e-12 if prec == FP64 else 1e-5
    assert np.max(np.abs(gp - ep)) <= tol * max(1.0, lam), np.max(np.abs(gp - ep))
    assert np.max(np.abs(gm - em)) <= tol * max(1.0, lam), np.max(np.abs(gm - em))
    # the next solve sees the new fields (Boltzmann factors rebuilt in the step)
    ref2 = o.solve(ep, em, n, L, Ns, fA, o.SCFT_REAL)
    assert abs(obs["Q"].real - ref2.Q) <= (1e-12 if prec == FP64 else 2e-5) * ref2.Q


def test_cl_sis_steps_with_supplied_noise_match_oracle():
    n, L, Ns, fA, chiN, C, dt = (16, 8, 12), (4.0, 2.0, 3.0), 12, 0.3, 20.0, 50.0, 0.05
    wp, wm = _fields(n, CL, 22, 0.05, 0.2)
    wm = wm + chiN * (2 * fA - 1) / 2
    dV = np.prod(L) / np.prod(n)
    std = o.cl_noise_std(dt, C, dV)
    rng = np.random.default_rng(7)
    with pft.System(n, L, Ns, fA, chiN, C, CL, FP64) as s:
        s.set_fields(wp, wm)
        for it in range(3):
            s.solve()
            ref = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
            obs = s.observables()
            Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, o.CL_COMPLEX)
            assert abs(obs["H"] - Href) <= 1e-12 * abs(Href)
            ep = std * rng.normal(size=n)
            em = std * rng.normal(size=n)
            s.field_step(dt, ep, em, semi_implicit=True)
            wp, wm = o.cl_sis_step(wp, wm, ref.phiA, ref.phiB, chiN, dt, ep, em, n, L)
            gp, gm = s.get_fields()
            assert np.max(np.abs(gp - wp)) <= 1e-10 and np.max(np.abs(gm - wm)) <= 1e-10


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_cl_sis_step_with_device_philox_matches_oracle_generator(prec):
    n, L, Ns, fA, chiN, C, dt = (8, 8, 16), (2.0, 2.0, 4.0), 10, 0.3, 20.0, 50.0, 0.05
    wp, wm = _fields(n, CL, 23, 0.05, 0.2)
    seed, inst = 0x1234_5678_9ABC, 5
    dV = np.prod(L) / np.prod(n)
    std = o.cl_noise_std(dt, C, dV)
    with pft.System(n, L, Ns, fA, chiN, C, CL, prec, seed=seed, instance=inst) as s:
        s.set_fields(wp, wm)
        for step in range(2):
            s.solve()
            ref = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
            s.field_step(dt, semi_implicit=True)
            ep, em = o.cl_noise(seed, inst, step, wp.size, std)
            wp, wm = o.cl_sis_step(wp, wm, ref.phiA, ref.phiB, chiN, dt, ep.reshape(n), em.reshape(n), n, L)
            gp, gm = s.get_fields()
            tol = 1e-10 if prec == FP64 else 1e-5
            assert np.max(np.abs(gp - wp)) <= tol and np.max(np.abs(gm - wm)) <= tol


def test_scft_sis_relaxation_trajectory_matches_oracle():
    n, L, Ns, fA, chiN, lam = (16, 12, 8), (4.0, 3.0, 2.0), 16, 0.4, 15.0, 1.0
    wp, wm = _fields(n, SCFT, 24)
    with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, FP64) as s:
        s.set_fields(wp, wm)
        for it in range(5):
            s.solve()
            ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
            s.field_step(lam, semi_implicit=True)
            wp, wm = o.scft_sis_step(wp, wm, ref.phiA, ref.phiB, chiN, lam, n, L)
        gp, gm = s.get_fields()
    assert np.max(np.abs(gp - wp)) <= 1e-11 and np.max(np.abs(gm - wm)) <= 1e-11


def test_sis_relaxes_where_explicit_euler_grows():
    """Disordered melt (fA = 1/2, chiN = 10) with a long-wave W+ perturbation and lam = 5:
    the explicit step multiplies the k = 2 pi/L mode by |1 - lam g_D| = 1.55 per step,
    the semi-implicit step by 1/(1 + lam g_D) = 0.28 (g_D = 0.51)."""
    n, L, Ns, fA, chiN, lam = (32, 32, 32), (4.0, 4.0, 4.0), 32, 0.5, 10.0, 5.0
    x = np.arange(32) * 4.0 / 32
    wp0 = np.broadcast_to(0.1 * np.cos(2 * np.pi * x / 4.0)[:, None, None], n).copy()
    wm0 = 0.05 * np.random.default_rng(1).normal(size=n)
    norms = {}
    for sis in (False, True):
        with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, FP64) as s:
            s.set_fields(wp0, wm0)
            f = []
            for it in range(6):
                s.solve()
                obs = s.observables()
                f.append(obs["force_p_rms"])
                s.field_step(lam, semi_implicit=sis)
            norms[sis] = f
    assert norms[False][-1] > 2.0 * norms[False][0], norms[False]
    assert norms[True][-1] < 0.1 * norms[True][0], norms[True]


def test_sis_refuses_mismatched_kinds():
    n = (8, 8, 8)
    wp, wm = _fields(n, SCFT, 3)
    with pft.System(n, (2.0, 2.0, 2.0), 8, 0.5, 15.0, 1.0, SCFT, FP64) as s:
        s.set_fields(wp, wm)
        s.solve()
        with pytest.raises(pft.PftError) as ei:
            pft.pft_field_step(s.h, pft.PFT_STEP_CL_SIS, 0.1)
        assert ei.value.status == pft.PFT_ERR_ARG
