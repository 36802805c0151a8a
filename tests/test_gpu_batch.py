"""Batches of independent systems of uneven grid and contour sizes (SCFT and complex
Langevin mixed), advanced by batched launches captured in one CUDA graph, against the
FP64 oracle run instance by instance, and against the library's own one-launch-sequence-
per-instance mode."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu
SCFT, CL = pft.PFT_SCFT_REAL, pft.PFT_CL_COMPLEX


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


DESCS = [
    dict(n=(16, 16, 16), L=(3.0, 3.0, 3.0), Ns=10, fA=0.4, chiN=15.0, C=1.0, kind=SCFT, seed=11),
    dict(n=(24, 24, 24), L=(4.0, 4.0, 4.0), Ns=14, fA=0.3, chiN=20.0, C=50.0, kind=CL, seed=12),
    dict(n=(16, 16, 16), L=(3.0, 3.0, 3.0), Ns=20, fA=0.25, chiN=18.0, C=50.0, kind=CL, seed=13),
    dict(n=(12, 12, 12), L=(2.0, 2.0, 2.0), Ns=7, fA=0.5, chiN=12.0, C=1.0, kind=SCFT, seed=14),
    dict(n=(16, 16, 16), L=(3.0, 3.0, 3.0), Ns=15, fA=0.45, chiN=14.0, C=1.0, kind=SCFT, seed=15),
    dict(n=(24, 24, 24), L=(4.0, 4.0, 4.0), Ns=9, fA=0.35, chiN=16.0, C=1.0, kind=SCFT, seed=16),
    dict(n=(24, 24, 24), L=(4.0, 4.0, 4.0), Ns=11, fA=0.3, chiN=20.0, C=50.0, kind=CL, seed=17),
]
LAM, DT = 0.1, 0.01


def _fields(d, seed):
    rng = np.random.default_rng(seed)
    n = d["n"]
    wp = rng.normal(0, 0.2, n)
    wm = rng.normal(0, 1.0, n)
    if d["kind"] == CL:
        return wp.astype(complex), (wm + d["chiN"] * (2 * d["fA"] - 1) / 2).astype(complex)
    return wp, wm


def _make(prec, descs=DESCS):
    b = pft.pft_batch_create(descs, prec)
    fields = []
    for i, d in enumerate(descs):
        wp, wm = _fields(d, 100 + i)
        pft.pft_batch_set_fields(b, i, wp, wm)
        fields.append((wp, wm))
    return b, fields


def _oracle_updates(d, i, wp, wm, updates):
    kind = o.SCFT_REAL if d["kind"] == SCFT else o.CL_COMPLEX
    M = int(np.prod(d["n"]))
    dV = float(np.prod(d["L"])) / M
    for u in range(updates):
        s = o.solve(wp, wm, d["n"], d["L"], d["Ns"], d["fA"], kind)
        H = o.hamiltonian(wp, wm, s.lnQ, d["chiN"], d["C"], d["n"], d["L"], kind)
        if kind == o.SCFT_REAL:
            wp, wm = o.scft_euler_step(wp, wm, s.phiA, s.phiB, d["chiN"], LAM)
        else:
            std = o.cl_noise_std(DT, d["C"], dV)
            ep, em = o.cl_noise(d["seed"], i, u, M, std)
            wp, wm = o.cl_euler_maruyama_step(wp, wm, s.phiA, s.phiB, d["chiN"], DT, ep.reshape(d["n"]),
                                              em.reshape(d["n"]))
    return wp, wm, s, H


def test_batch_graphed_matches_oracle_fp64():
    b, fields = _make(pft.PFT_FP64)
    try:
        pft.pft_batch_run(b, 2, LAM, DT, pft.PFT_BATCH_GRAPHED)
        info = pft.pft_batch_info(b)
        assert info["classes"] == 5
        assert info["units_per_update"] == sum(2 * np.prod(d["n"]) * d["Ns"] for d in DESCS)
        for i, d in enumerate(DESCS):
            wp, wm, s, H = _oracle_updates(d, i, *fields[i], 2)
            dt = np.float64 if d["kind"] == SCFT else np.complex128
            gp = np.empty(d["n"], dt)
            gm = np.empty(d["n"], dt)
            pft.pft_batch_get_fields(b, i, gp, gm)
            obs = pft.pft_batch_get_observables(b, i)
            assert np.max(np.abs(gp - wp)) <= 1e-11 and np.max(np.abs(gm - wm)) <= 1e-11, i
            Hg = obs["H"] if d["kind"] == CL else obs["H"].real
            assert abs(Hg - H) <= 1e-11 * abs(H), (i, Hg, H)
            assert obs["step"] == 2
    finally:
        pft.pft_batch_destroy(b)


@pytest.mark.parametrize("prec", [pft.PFT_FP64, pft.PFT_FP32_MIXED])
def test_batch_graphed_plan0_equals_per_instance(prec):
    """Plan 0 (one march after the other, fused quadrature) is the per-instance arithmetic
    exactly, so the graphed batch reproduces the per-instance mode bit for bit."""
    res = []
    for mode in (pft.PFT_BATCH_GRAPHED, pft.PFT_BATCH_PER_INSTANCE):
        b, _ = _make(prec)
        try:
            pft.pft_batch_set_plan(b, -1, 0)
            pft.pft_batch_run(b, 3, LAM, DT, mode)
            out = []
            for i, d in enumerate(DESCS):
                dt = np.float64 if d["kind"] == SCFT else np.complex128
                gp = np.empty(d["n"], dt)
                gm = np.empty(d["n"], dt)
                pft.pft_batch_get_fields(b, i, gp, gm)
                out.append((gp, gm, pft.pft_batch_get_observables(b, i)["Q"]))
            res.append(out)
        finally:
            pft.pft_batch_destroy(b)
    for a, c in zip(*res):
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]) and a[2] == c[2]


# One member per class of the timed 256-instance batch (grids 32^3, 48^3, 64^3; real SCFT
# and complex CL fields; Ns from {50, 100, 200}); the 64^3 classes run on the batched plane
# kernels under plan 1.
BENCH_CLASSES = [
    dict(n=(32, 32, 32), L=(4.0, 4.0, 4.0), Ns=200, fA=0.3, chiN=14.0, C=1.0, kind=SCFT, seed=21),
    dict(n=(48, 48, 48), L=(6.0, 6.0, 6.0), Ns=100, fA=0.45, chiN=22.0, C=1.0, kind=SCFT, seed=22),
    dict(n=(64, 64, 64), L=(8.0, 8.0, 8.0), Ns=50, fA=0.27, chiN=17.0, C=1.0, kind=SCFT, seed=23),
    dict(n=(32, 32, 32), L=(4.0, 4.0, 4.0), Ns=50, fA=0.5, chiN=24.0, C=50.0, kind=CL, seed=24),
    dict(n=(48, 48, 48), L=(6.0, 6.0, 6.0), Ns=200, fA=0.38, chiN=12.5, C=50.0, kind=CL, seed=25),
    dict(n=(64, 64, 64), L=(8.0, 8.0, 8.0), Ns=100, fA=0.33, chiN=19.0, C=50.0, kind=CL, seed=26),
]


@pytest.mark.parametrize("plan", [1, 2, 3, 19, 35, 51])
def test_batch_fp32_classes_of_the_timed_batch_match_oracle(plan):
    """FP32-mixed batch with one member per class of the timed batch, graph-captured, in
    plan 1 (both marches per launch; plane kernels for the 64^3 classes), plan 2 (the
    separable march on the plane and x kernels for the 64^3 classes, plan 1 elsewhere),
    plan 3 (the separable march on pencils for every class), plan 19 (plan 3 with
    register lines for the 32^3 and 48^3 classes), plan 35 (plan 3 with 32-line tiles) or
    plan 51 (plan 3 with twice the elements a thread in 32-line tiles): each member's Q, phiA,
    phiB and fields after one update against the FP64 oracle.  FP32 tolerances of the
    single-context path (relative 2e-5 on Q, absolute 2e-5 on phi) scaled by the
    random-walk growth of the rounding error over 2 Ns <= 400 transform pairs (x sqrt 2)."""
    b, fields = _make(pft.PFT_FP32_MIXED, BENCH_CLASSES)
    try:
        info = pft.pft_batch_info(b)
        assert info["classes"] == 6
        pft.pft_batch_set_plan(b, -1, plan)
        plans = [pft.pft_batch_class_info(b, k)["plan"] for k in range(info["classes"])]
        assert plans.count(plan) == {2: 2, 19: 4}.get(plan, 6), plans
        pft.pft_batch_run(b, 1, LAM, DT, pft.PFT_BATCH_GRAPHED)
        for i, d in enumerate(BENCH_CLASSES):
            wp, wm, s, H = _oracle_updates(d, i, *fields[i], 1)
            dt = np.float64 if d["kind"] == SCFT else np.complex128
            gp, gm = np.empty(d["n"], dt), np.empty(d["n"], dt)
            pA, pB = np.empty(d["n"], dt), np.empty(d["n"], dt)
            pft.pft_batch_get_fields(b, i, gp, gm)
            pft.pft_batch_get_densities(b, i, pA, pB)
            obs = pft.pft_batch_get_observables(b, i)
            Q = obs["Q"] if d["kind"] == CL else obs["Q"].real
            eQ = abs(Q - s.Q) / abs(s.Q)
            ephi = max(np.max(np.abs(pA - s.phiA)), np.max(np.abs(pB - s.phiB)))
            ew = max(np.max(np.abs(gp - wp)), np.max(np.abs(gm - wm)))
            print(f"\nbatch FP32 plan {plan} member {i} {d['n']} Ns={d['Ns']} kind={d['kind']}: Q rel {eQ:.2e} "
                  f"phi abs {ephi:.2e} fields abs {ew:.2e}")
            assert eQ <= 3e-5 and ephi <= 3e-5 and ew <= 1e-5, i
        pft.pft_batch_synchronize(b)
    finally:
        pft.pft_batch_destroy(b)


def test_batch_rejects_bad_members():
    with pytest.raises(pft.PftError) as e:
        pft.pft_batch_create([dict(n=(128, 16, 16), L=(1, 1, 1), Ns=4, fA=0.5, chiN=10.0, C=1.0, kind=SCFT)])
    assert e.value.status == pft.PFT_ERR_SHAPE
    b = pft.pft_batch_create(DESCS[:2])
    try:
        with pytest.raises(pft.PftError) as e:
            pft.pft_batch_run(b, 1, LAM, DT)
        assert e.value.status == pft.PFT_ERR_STATE
    finally:
        pft.pft_batch_destroy(b)


@pytest.mark.parametrize("prec", [pft.PFT_FP64, pft.PFT_FP32_MIXED])
def test_batch_plans_agree_and_autotune_picks_one(prec):
    """Plan 1 (both marches per launch, post-march quadrature) against plan 0 after three
    updates: the propagators are the same arithmetic, the FP64 quadrature sums run in
    another order (FP64: 1e-12 on fields; FP32: 1e-5, the FP32 Boltzmann factors of
    fields differing in the last FP64 bits may round apart).  The autotuner then picks a
    plan per class and the run continues from the same state."""
    out = {}
    for plan in (0, 1, 3):
        b, _ = _make(prec)
        try:
            pft.pft_batch_set_plan(b, -1, plan)
            pft.pft_batch_run(b, 3, LAM, DT, pft.PFT_BATCH_GRAPHED)
            res = []
            for i, d in enumerate(DESCS):
                dt = np.float64 if d["kind"] == SCFT else np.complex128
                gp = np.empty(d["n"], dt)
                gm = np.empty(d["n"], dt)
                pft.pft_batch_get_fields(b, i, gp, gm)
                res.append((gp, gm))
            out[plan] = res
            if plan == 1:
                pft.pft_batch_autotune(b)
                info = pft.pft_batch_info(b)
                for k in range(info["classes"]):
                    ci = pft.pft_batch_class_info(b, k)
                    tuned = [v for v in ci["tuned_ms"] if v > 0]
                    assert ci["plan"] in (0, 1, 2, 3, 19, 35, 51) and ci["tuned_ms"][0] > 0 and ci["tuned_ms"][1] > 0
                    assert ci["tuned_ms"][{19: 4, 35: 5, 51: 6}.get(ci["plan"], ci["plan"])] == min(tuned)
                pft.pft_batch_run(b, 1, LAM, DT, pft.PFT_BATCH_GRAPHED)
                pft.pft_batch_synchronize(b)
        finally:
            pft.pft_batch_destroy(b)
    tol = 1e-12 if prec == pft.PFT_FP64 else 1e-5
    for other in (1, 3):
        for (a0, b0), (a1, b1) in zip(out[0], out[other]):
            assert np.max(np.abs(a0 - a1)) <= tol and np.max(np.abs(b0 - b1)) <= tol
