"""The separable march (plan 2): the diffusion operator of Eq. 13 applied as three 1D
periodic Gaussian convolutions in alternating axis order, one launch per contour step
(plane kernel and x kernel in turn), against the FP64 oracle and against the plane-kernel
plan.  FP32-mixed tolerances as in test_gpu_parity: relative 2e-5 on Q, absolute 2e-5 on
phi; propagator slices relative to the slice maximum 2e-5 (1e-4 at 128^3, where the
maximum is taken over 2,097,152 points: see test_gyroid_128cubed_full_size)."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft
from paper_1204_5434_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
FP32, FP64 = pft.PFT_FP32_MIXED, pft.PFT_FP64
SCFT, CL = pft.PFT_SCFT_REAL, pft.PFT_CL_COMPLEX


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _solve(w, plan, streams, wp, wm):
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, FP32) as s:
        pft.pft_set_plan(s.h, plan, streams)
        s.set_fields(wp, wm)
        s.solve()
        s.solve()  # the replayed graph
        assert pft.pft_get_plan(s.h) == (plan, streams)
        obs = s.observables()
        phiA, phiB = s.densities()
        q = {k: s.propagator(0, k) for k in sorted({1, 2, w.Ns // 2, w.Ns - 1, w.Ns}) if 1 <= k <= w.Ns}
        qd = {k: s.propagator(2, k) for k in sorted({1, w.Ns - 1, w.Ns}) if 1 <= k <= w.Ns}
    return obs, phiA, phiB, q, qd


# 128^3 with even and odd Ns (the last launch a plane or an x kernel), 64^3 with one and
# two steps and a junction inside the march, uneven box lengths
CASES = [
    (wl.GYR128.with_(Ns=20), 1, 1e-4),
    (wl.GYR128.with_(Ns=9), 1, 1e-4, 18),  # the x kernel's alternative plan
    (wl.GYR64.with_(n=(64, 64, 64), Ns=4), 0, 2e-5, 18),
    (wl.GYR128.with_(Ns=7), 0, 1e-4),
    (wl.GYR64.with_(Ns=1, fA=0.5), 1, 2e-5),
    (wl.GYR64.with_(Ns=2, fA=0.5), 0, 2e-5),
    (wl.GYR64.with_(Ns=9, fA=0.35, L=(7.0, 8.0, 9.5)), 1, 2e-5),
    (wl.GYR64.with_(n=(128, 64, 64), L=(16.0, 8.0, 8.0), Ns=12), 1, 2e-5),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_separable_march_matches_oracle(case):
    w, streams, qtol = CASES[case][:3]
    code = CASES[case][3] if len(CASES[case]) > 3 else 2
    wp, wm = wl.fields(w)
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    obs, phiA, phiB, q, qd = _solve(w, code, streams, wp, wm)
    eQ = abs(obs["Q"].real - ref.Q) / ref.Q
    ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
    eq = max(np.max(np.abs(v - ref.q[k])) / np.max(np.abs(ref.q[k])) for k, v in q.items())
    eqd = max(np.max(np.abs(v - ref.qd[k])) / np.max(np.abs(ref.qd[k])) for k, v in qd.items())
    print(f"\nseparable {w.n} Ns={w.Ns} plan={code} streams={streams}: Q rel {eQ:.2e} phi abs {ephi:.2e} "
          f"q {eq:.2e} qd {eqd:.2e}")
    assert eQ <= 2e-5 and ephi <= 2e-5 and eq <= qtol and eqd <= qtol


def test_separable_march_agrees_with_the_plane_kernel_plan():
    w = wl.GYR128.with_(Ns=30)
    wp, wm = wl.fields(w)
    a = _solve(w, 2, 1, wp, wm)
    b = _solve(w, 1, 1, wp, wm)
    assert abs(a[0]["Q"].real - b[0]["Q"].real) <= 2e-5 * b[0]["Q"].real
    assert np.max(np.abs(a[1] - b[1])) <= 2e-5 and np.max(np.abs(a[2] - b[2])) <= 2e-5


def test_separable_plan_is_refused_where_it_does_not_apply():
    for n, kind, prec in (((64, 64, 64), SCFT, FP64), ((128, 128, 128), CL, FP32), ((32, 32, 32), SCFT, FP32),
                          ((64, 32, 64), SCFT, FP32), ((32, 64, 64), CL, FP32)):
        with pft.System(n, (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, kind, prec) as s:
            with pytest.raises(pft.PftError) as e:
                pft.pft_set_plan(s.h, 2, 1)
            assert e.value.status == pft.PFT_ERR_UNSUPPORTED
    with pft.System((64, 64, 64), (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, SCFT, FP32) as s:
        with pytest.raises(pft.PftError) as e:
            pft.pft_set_plan(s.h, 2, 2)
        assert e.value.status == pft.PFT_ERR_ARG


# ------------------------------------------------- separable march on pencils (plan 3)
PCASES = [
    # complex Langevin fields: the 64^3 workload's grid, 256-point pencils, ragged sizes
    ((64, 64, 64), (8.0, 8.0, 8.0), 12, 0.3, CL, FP32, 1),
    ((256, 16, 256), (16.0, 1.0, 16.0), 4, 0.5, CL, FP32, 1),
    ((12, 48, 24), (3.0, 6.0, 4.0), 9, 0.4, CL, FP64, 0),
    ((16, 12, 96), (4.0, 3.0, 9.0), 7, 0.35, CL, FP64, 1),
    # real fields: batch-class sizes and ragged ones, both precisions, one- and two-step chains
    ((32, 32, 32), (4.0, 4.0, 4.0), 10, 0.3, SCFT, FP32, 1),
    ((48, 48, 48), (6.0, 6.0, 6.0), 2, 0.5, SCFT, FP32, 0),
    ((24, 6, 48), (4.0, 1.5, 6.0), 1, 0.5, SCFT, FP64, 1),
    ((128, 128, 128), (8.0, 8.0, 8.0), 6, 0.35, SCFT, FP64, 1),
    ((8, 12, 16), (2.0, 3.0, 4.0), 13, 0.6, SCFT, FP64, 0),
    # FP32 tiles that are partly outside the grid (the x and z kernels then read B_s from
    # global memory instead of staging the tile): 36 x lines in tiles of 16; 24 z pencils of
    # 256 points in tiles of 16
    ((12, 6, 12), (3.0, 1.5, 3.0), 5, 0.4, SCFT, FP32, 1),
    ((6, 4, 256), (1.5, 1.0, 16.0), 3, 0.5, CL, FP32, 0),
]
PTOL = {FP64: dict(Q=1e-12, phi=1e-10, q=1e-12), FP32: dict(Q=2e-5, phi=2e-5, q=2e-5)}


def _pfields(n, kind, seed):
    rng = np.random.default_rng(seed)
    wp = rng.normal(0, 0.3, n)
    wm = rng.normal(0, 1.0, n)
    if kind == CL:
        wp = wp + 1j * rng.normal(0, 0.3, n)
        wm = wm + 1j * rng.normal(0, 0.3, n)
    return wp, wm


@pytest.mark.parametrize("case", range(len(PCASES)))
def test_separable_pencil_march_matches_oracle(case):
    n, L, Ns, fA, kind, prec, streams = PCASES[case]
    wp, wm = _pfields(n, kind, 300 + case)
    okind = o.SCFT_REAL if kind == SCFT else o.CL_COMPLEX
    ref = o.solve(wp, wm, n, L, Ns, fA, okind)
    t = PTOL[prec]
    with pft.System(n, L, Ns, fA, 17.0, 2.0, kind, prec) as s:
        pft.pft_set_plan(s.h, 3, streams)
        s.set_fields(wp, wm)
        s.solve()
        s.solve()
        assert pft.pft_get_plan(s.h) == (3, streams)
        obs = s.observables()
        phiA, phiB = s.densities()
        eq = 0.0
        for which, k in ((0, 1), (0, Ns), (2, 1), (2, Ns)):
            g = s.propagator(which, k)
            hist = ref.q if which == 0 else ref.qd
            eq = max(eq, np.max(np.abs(g - hist[k])) / np.max(np.abs(hist[k])))
    Q = obs["Q"] if kind == CL else obs["Q"].real
    eQ = abs(Q - ref.Q) / abs(ref.Q)
    ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
    print(f"\nseparable pencils {n} Ns={Ns} kind={kind} prec={prec}: Q rel {eQ:.2e} phi abs {ephi:.2e} "
          f"slices {eq:.2e}")
    assert eQ <= t["Q"] and ephi <= t["phi"] and eq <= t["q"]


# register lines (code 19): FP32 x and y lines of at most 48 points in one thread each
RCASES = [
    ((32, 32, 32), (4.0, 4.0, 4.0), 10, 0.3, SCFT, 1),
    ((48, 48, 48), (6.0, 6.0, 6.0), 7, 0.45, SCFT, 0),
    ((48, 32, 64), (6.0, 4.0, 8.0), 5, 0.5, SCFT, 1),
    ((32, 32, 32), (4.0, 4.0, 4.0), 9, 0.5, CL, 1),
    ((48, 48, 48), (6.0, 6.0, 6.0), 4, 0.38, CL, 0),
    ((24, 12, 16), (3.0, 2.0, 4.0), 13, 0.4, CL, 1),
]


@pytest.mark.parametrize("case", range(len(RCASES)))
def test_register_lines_match_oracle(case):
    n, L, Ns, fA, kind, streams = RCASES[case]
    wp, wm = _pfields(n, kind, 400 + case)
    okind = o.SCFT_REAL if kind == SCFT else o.CL_COMPLEX
    ref = o.solve(wp, wm, n, L, Ns, fA, okind)
    with pft.System(n, L, Ns, fA, 17.0, 2.0, kind, FP32) as s:
        pft.pft_set_plan(s.h, 19, streams)
        s.set_fields(wp, wm)
        s.solve()
        s.solve()
        assert pft.pft_get_plan(s.h) == (19, streams)
        obs = s.observables()
        phiA, phiB = s.densities()
        eq = 0.0
        for which, k in ((0, 1), (0, Ns), (2, 1), (2, Ns)):
            g = s.propagator(which, k)
            hist = ref.q if which == 0 else ref.qd
            eq = max(eq, np.max(np.abs(g - hist[k])) / np.max(np.abs(hist[k])))
    Q = obs["Q"] if kind == CL else obs["Q"].real
    eQ = abs(Q - ref.Q) / abs(ref.Q)
    ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
    print(f"\nregister lines {n} Ns={Ns} kind={kind}: Q rel {eQ:.2e} phi abs {ephi:.2e} slices {eq:.2e}")
    assert eQ <= 2e-5 and ephi <= 2e-5 and eq <= 2e-5


def test_register_lines_are_refused_where_they_do_not_apply():
    for n, prec in (((64, 32, 32), FP32), ((32, 64, 32), FP32), ((32, 32, 32), FP64)):
        with pft.System(n, (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, SCFT, prec) as s:
            with pytest.raises(pft.PftError) as e:
                pft.pft_set_plan(s.h, 19, 1)
            assert e.value.status == pft.PFT_ERR_UNSUPPORTED


# line variants 35 (32-line tiles; FP32, any grid) and 51 (twice the elements a thread,
# another radix order, 32-line tiles; FP32 x and y lines of 32, 48 or 64 points)
WCASES = [
    ((32, 32, 32), (4.0, 4.0, 4.0), 10, 0.3, SCFT, 1),
    ((48, 48, 48), (6.0, 6.0, 6.0), 7, 0.45, SCFT, 0),
    ((64, 48, 24), (8.0, 6.0, 3.0), 5, 0.5, SCFT, 1),
    ((32, 64, 16), (4.0, 8.0, 2.0), 9, 0.5, CL, 1),
    ((48, 32, 48), (6.0, 4.0, 6.0), 4, 0.38, CL, 0),
    ((64, 64, 64), (8.0, 8.0, 8.0), 1, 0.4, CL, 1),
    # 256-, 192- and 128-point x lines, a 96-point y line, ragged tile grids (12 x 6 and
    # 128 x 6 x 12: 36 x lines, not whole 16-line tiles)
    ((256, 16, 128), (16.0, 1.0, 8.0), 3, 0.5, CL, 1),
    ((128, 96, 64), (8.0, 6.0, 4.0), 4, 0.35, SCFT, 0),
    ((12, 6, 12), (3.0, 1.5, 3.0), 5, 0.4, SCFT, 1),
    ((192, 8, 16), (12.0, 1.0, 2.0), 6, 0.45, SCFT, 1),
    ((128, 6, 12), (8.0, 1.5, 3.0), 2, 0.5, CL, 0),
    ((256, 8, 32), (16.0, 1.0, 4.0), 1, 0.5, SCFT, 1),
]


def _variant_applies(code, n):
    if code == 51:
        return all(a in (32, 48, 64) for a in n[:2])
    return True


@pytest.mark.parametrize("code", [35, 51])
@pytest.mark.parametrize("case", range(len(WCASES)))
def test_line_variants_match_oracle(case, code):
    n, L, Ns, fA, kind, streams = WCASES[case]
    if not _variant_applies(code, n):
        pytest.skip(f"line variant {code} does not apply to {n}")
    wp, wm = _pfields(n, kind, 500 + case)
    okind = o.SCFT_REAL if kind == SCFT else o.CL_COMPLEX
    ref = o.solve(wp, wm, n, L, Ns, fA, okind)
    with pft.System(n, L, Ns, fA, 17.0, 2.0, kind, FP32) as s:
        pft.pft_set_plan(s.h, code, streams)
        s.set_fields(wp, wm)
        s.solve()
        s.solve()
        assert pft.pft_get_plan(s.h) == (code, streams)
        obs = s.observables()
        phiA, phiB = s.densities()
        eq = 0.0
        for which, k in ((0, 1), (0, Ns), (2, 1), (2, Ns)):
            g = s.propagator(which, k)
            hist = ref.q if which == 0 else ref.qd
            eq = max(eq, np.max(np.abs(g - hist[k])) / np.max(np.abs(hist[k])))
    Q = obs["Q"] if kind == CL else obs["Q"].real
    eQ = abs(Q - ref.Q) / abs(ref.Q)
    ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
    print(f"\nline variant {code} {n} Ns={Ns} kind={kind}: Q rel {eQ:.2e} phi abs {ephi:.2e} slices {eq:.2e}")
    assert eQ <= 2e-5 and ephi <= 2e-5 and eq <= 2e-5


def test_line_variants_are_refused_where_they_do_not_apply():
    for n, prec, codes in (((128, 32, 32), FP32, (51,)), ((32, 96, 32), FP32, (51,)), ((32, 32, 32), FP64, (35, 51))):
        with pft.System(n, (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, SCFT, prec) as s:
            for code in codes:
                with pytest.raises(pft.PftError) as e:
                    pft.pft_set_plan(s.h, code, 1)
                assert e.value.status == pft.PFT_ERR_UNSUPPORTED
    with pft.System((32, 32, 32), (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, SCFT, FP32) as s:
        for code in (67, 34, 50):
            with pytest.raises(pft.PftError) as e:
                pft.pft_set_plan(s.h, code, 1)
            assert e.value.status == pft.PFT_ERR_ARG


def test_default_plans():
    for n, kind, prec, plan in (((64, 64, 64), CL, FP32, 2), ((32, 32, 32), SCFT, FP32, 3),
                                ((64, 64, 64), SCFT, FP64, 3), ((256, 16, 256), CL, FP64, 3),
                                ((256, 16, 256), CL, FP32, 3), ((128, 128, 128), SCFT, FP32, 2)):
        with pft.System(n, (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, kind, prec) as s:
            assert pft.pft_get_plan(s.h) == (plan, 1), (n, kind, prec)
    with pft.System((64, 64, 64), (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, SCFT, FP32) as s:
        assert pft.pft_get_plan(s.h) == (2, 1)
        with pytest.raises(pft.PftError) as e:
            pft.pft_set_plan(s.h, 5, 1)
        assert e.value.status == pft.PFT_ERR_ARG
        with pytest.raises(pft.PftError) as e:  # double-float arithmetic: FP64 contexts only
            pft.pft_set_plan(s.h, 4, 1)
        assert e.value.status == pft.PFT_ERR_UNSUPPORTED
