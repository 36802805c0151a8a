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
    (wl.GYR128.with_(Ns=7), 0, 1e-4),
    (wl.GYR64.with_(Ns=1, fA=0.5), 1, 2e-5),
    (wl.GYR64.with_(Ns=2, fA=0.5), 0, 2e-5),
    (wl.GYR64.with_(Ns=9, fA=0.35, L=(7.0, 8.0, 9.5)), 1, 2e-5),
    (wl.GYR64.with_(n=(128, 64, 64), L=(16.0, 8.0, 8.0), Ns=12), 1, 2e-5),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_separable_march_matches_oracle(case):
    w, streams, qtol = CASES[case]
    wp, wm = wl.fields(w)
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    obs, phiA, phiB, q, qd = _solve(w, 2, streams, wp, wm)
    eQ = abs(obs["Q"].real - ref.Q) / ref.Q
    ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
    eq = max(np.max(np.abs(v - ref.q[k])) / np.max(np.abs(ref.q[k])) for k, v in q.items())
    eqd = max(np.max(np.abs(v - ref.qd[k])) / np.max(np.abs(ref.qd[k])) for k, v in qd.items())
    print(f"\nseparable {w.n} Ns={w.Ns} streams={streams}: Q rel {eQ:.2e} phi abs {ephi:.2e} "
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
    for n, kind, prec in (((64, 64, 64), SCFT, FP64), ((64, 64, 64), CL, FP32), ((32, 32, 32), SCFT, FP32),
                          ((64, 32, 64), SCFT, FP32)):
        with pft.System(n, (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, kind, prec) as s:
            with pytest.raises(pft.PftError) as e:
                pft.pft_set_plan(s.h, 2, 1)
            assert e.value.status == pft.PFT_ERR_UNSUPPORTED
    with pft.System((64, 64, 64), (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, SCFT, FP32) as s:
        with pytest.raises(pft.PftError) as e:
            pft.pft_set_plan(s.h, 3, 1)
        assert e.value.status == pft.PFT_ERR_ARG
