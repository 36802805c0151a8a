"""GPU parity of the reverse-mode adjoint (gradient of a loss on the densities with respect
to W+ and W-, through the discrete march) against the oracle's adjoint, which is pinned by
finite differences.  Tolerances relative to the largest gradient entry: FP64 1e-11, FP32-
mixed 1e-4 (two adjoint marches of Ns steps in FP32, ~1e-6 per step)."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu
FP64, FP32 = pft.PFT_FP64, pft.PFT_FP32_MIXED
SCFT = pft.PFT_SCFT_REAL


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _fields(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.3, n), rng.normal(0, 1.0, n), rng


CASES = [((16, 12, 8), (4.0, 3.0, 2.0), 20, 0.35), ((12, 12, 12), (3.0, 3.0, 3.0), 13, 0.5),
         ((48, 4, 6), (6.0, 1.0, 1.5), 10, 0.6), ((64, 64, 64), (8.0, 8.0, 8.0), 16, 0.35)]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("loss", ["linear", "quadratic"])
@pytest.mark.parametrize("case", CASES)
def test_adjoint_matches_oracle(case, loss, prec):
    n, L, Ns, fA = case
    wp, wm, rng = _fields(n, 60 + Ns)
    with pft.System(n, L, Ns, fA, 15.0, 1.0, SCFT, prec, checkpoint=1) as s:
        s.set_fields(wp, wm)
        s.solve()
        phiA, phiB = s.densities()
        if loss == "linear":
            GA, GB = rng.normal(size=n), rng.normal(size=n)
        else:
            t = rng.uniform(0.2, 0.6, n)
            GA, GB = phiA - t, np.zeros(n)
        gp, gm = s.adjoint(GA, GB)
    ep, em = o.adjoint_field_gradient(wp, wm, n, L, Ns, fA, GA, GB)
    scale = max(np.max(np.abs(ep)), np.max(np.abs(em)))
    tol = 1e-11 if prec == FP64 else 1e-4
    err = max(np.max(np.abs(gp - ep)), np.max(np.abs(gm - em))) / scale
    print(f"\nadjoint {n} Ns={Ns} {loss} prec={prec}: rel err {err:.2e}")
    assert err <= tol


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_adjoint_of_the_sum_rules_vanishes(prec):
    n, L, Ns, fA = (16, 12, 8), (4.0, 3.0, 2.0), 20, 0.35
    wp, wm, _ = _fields(n, 3)
    with pft.System(n, L, Ns, fA, 15.0, 1.0, SCFT, prec) as s:
        s.set_fields(wp, wm)
        s.solve()
        gp, gm = s.adjoint(np.ones(n), np.ones(n))
        gp2, gm2 = s.adjoint(np.ones(n), np.zeros(n))
    tol = 1e-13 if prec == FP64 else 2e-6
    for g in (gp, gm, gp2, gm2):
        assert np.max(np.abs(g)) <= tol, np.max(np.abs(g))


def test_adjoint_matches_finite_differences_of_the_gpu_solve():
    n, L, Ns, fA = (8, 8, 12), (2.0, 2.0, 3.0), 16, 0.35
    wp, wm, rng = _fields(n, 4)
    UA, UB = rng.normal(size=n), rng.normal(size=n)
    with pft.System(n, L, Ns, fA, 15.0, 1.0, SCFT, FP64) as s:
        def loss(a, b):
            s.set_fields(a, b)
            s.solve()
            pa, pb = s.densities()
            return float(np.sum(UA * pa + UB * pb))
        loss(wp, wm)
        gp, gm = s.adjoint(UA, UB)
        h = 1e-4
        for idx in [(1, 2, 3), (5, 0, 7)]:
            for which, g in ((0, gp), (1, gm)):
                def f(d, idx=idx, which=which):
                    a, b = wp.copy(), wm.copy()
                    (a if which == 0 else b)[idx] += d
                    return loss(a, b)
                fd = (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)
                assert abs(fd - g[idx]) <= 1e-8 * max(1.0, abs(g[idx])), (idx, which, fd, g[idx])


def test_adjoint_refuses_what_it_does_not_cover():
    n = (16, 16, 16)
    wp, wm, _ = _fields(n, 5)
    for kw in (dict(scheme=pft.PFT_SCHEME_RQM4), dict(checkpoint=4)):
        with pft.System(n, (4.0, 4.0, 4.0), 8, 0.5, 15.0, 1.0, SCFT, FP64, **kw) as s:
            s.set_fields(wp, wm)
            s.solve()
            with pytest.raises(pft.PftError) as ei:
                s.adjoint(np.ones(n), np.ones(n))
            assert ei.value.status == pft.PFT_ERR_UNSUPPORTED
    with pft.System(n, (4.0, 4.0, 4.0), 8, 0.5, 15.0, 1.0, pft.PFT_CL_COMPLEX, FP64) as s:
        s.set_fields(wp.astype(complex), wm.astype(complex))
        s.solve()
        with pytest.raises(pft.PftError) as ei:
            s.adjoint(np.ones(n), np.ones(n))
        assert ei.value.status == pft.PFT_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec,plan", [(FP64, None), (FP32, None), (FP32, 1)])
def test_adjoint_128cubed_matches_oracle(prec, plan):
    """128^3 gyroid workload, Ns = 20, a linear loss: the FP32-mixed adjoint on the
    separable march (the default: both adjoint marches store their histories, one pass
    forms the gradient) and on the plane kernel (plan 1: the fused adjoint step), FP64 on
    the pencil passes; all against the oracle's adjoint_field_gradient over every point."""
    from paper_1204_5434_gb300 import workloads as wl
    w = wl.GYR128.with_(Ns=20)
    wp, wm = wl.fields(w)
    rng = np.random.default_rng(12)
    GA, GB = rng.normal(size=w.n), rng.normal(size=w.n)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, prec, checkpoint=1) as s:
        if plan is not None:
            pft.pft_set_plan(s.h, plan, 1)
        s.set_fields(wp, wm)
        s.solve()
        gp, gm = s.adjoint(GA, GB)
        if prec == FP32:
            assert pft.pft_get_plan(s.h)[0] == (2 if plan is None else plan)
    ep, em = o.adjoint_field_gradient(wp, wm, w.n, w.L, w.Ns, w.fA, GA, GB)
    scale = max(np.max(np.abs(ep)), np.max(np.abs(em)))
    err = max(np.max(np.abs(gp - ep)), np.max(np.abs(gm - em))) / scale
    print(f"\nadjoint 128^3 Ns=20 prec={prec} plan={plan} vs oracle: rel err {err:.2e}")
    assert err <= (1e-11 if prec == FP64 else 1e-4)
