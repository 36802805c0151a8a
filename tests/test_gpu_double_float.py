"""The double-float march (plan 4 of an FP64 context) against the FP64 oracle, at the
unchanged FP64 tolerances.

Plan 4 runs the separable pencil march of Eq. 13 (Kx Ky Kz with alternating axis order,
the Boltzmann factors between) with every transform, diffusion and Boltzmann product in
double-float arithmetic: each value the unevaluated sum of two floats, about 48
significant bits, on the FP32 pipe.  q_0, the stored q_s, the quadrature of Eq. 8 and
everything after the march stay FP64.  Double-float rounding (about 2^-48 per operation
instead of 2^-53) puts the propagator error near 1e-14 instead of 1e-15: still two orders
below the FP64 bounds of test_gpu_parity, which this plan has to meet as they stand --
relative 1e-12 on Q and on propagator slices (relative to the slice maximum), 1e-10
max-abs on phi.  H is checked through h = H/(C V), absolutely to 1e-12: the field term of
Eq. 3 is FP64 on both sides, so the error of h is that of lnQ, whereas H itself can be a
near-cancellation of its two terms (random fields), where a relative bound would ask for
more digits than Q carries.
"""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft
from paper_1204_5434_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
FP64 = pft.PFT_FP64
SCFT, CL = pft.PFT_SCFT_REAL, pft.PFT_CL_COMPLEX
TOL = dict(Q=1e-12, h=1e-12, phi=1e-10, q=1e-12)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _fields(n, kind, seed, sp=0.3, sm=1.0):
    rng = np.random.default_rng(seed)
    wp = rng.normal(0, sp, n)
    wm = rng.normal(0, sm, n)
    if kind == CL:
        wp = wp + 1j * rng.normal(0, sp, n)
        wm = wm + 1j * rng.normal(0, sp, n)
    return wp, wm


def _check(n, L, Ns, fA, chiN, C, kind, streams, wp, wm, slices=None):
    okind = o.SCFT_REAL if kind == SCFT else o.CL_COMPLEX
    ref = o.solve(wp, wm, n, L, Ns, fA, okind)
    Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, okind)
    with pft.System(n, L, Ns, fA, chiN, C, kind, FP64) as s:
        pft.pft_set_plan(s.h, 4, streams)
        s.set_fields(wp, wm)
        s.solve()
        s.solve()  # the replayed graph
        assert pft.pft_get_plan(s.h) == (4, streams)
        obs = s.observables()
        phiA, phiB = s.densities()
        eq = 0.0
        for which, k in slices or ((0, 1), (0, Ns // 2), (0, Ns), (2, 1), (2, Ns)):
            if k < 1:
                continue
            g = s.propagator(which, k)
            hist = ref.q if which == 0 else ref.qd
            eq = max(eq, np.max(np.abs(g - hist[k])) / np.max(np.abs(hist[k])))
    Q = obs["Q"] if kind == CL else obs["Q"].real
    eQ = abs(Q - ref.Q) / abs(ref.Q)
    ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
    eh = abs(obs["H"] - Href) / (C * float(np.prod(L)))
    print(f"\ndouble-float {n} Ns={Ns} kind={kind} streams={streams}: Q rel {eQ:.2e} h {eh:.2e} "
          f"phi abs {ephi:.2e} slices {eq:.2e}")
    assert eQ <= TOL["Q"] and eh <= TOL["h"] and ephi <= TOL["phi"] and eq <= TOL["q"]


# complex and real fields; 8 to 256 points an axis, unequal and non-power-of-two extents;
# one- and two-step chains; both stream layouts
CASES = [
    ((64, 64, 64), (8.0, 8.0, 8.0), 20, 0.35, SCFT, 1),
    ((64, 64, 64), (8.0, 8.0, 8.0), 100, 0.3, CL, 0),
    ((12, 48, 24), (3.0, 6.0, 4.0), 9, 0.4, CL, 1),
    ((16, 12, 96), (4.0, 3.0, 9.0), 7, 0.35, CL, 0),
    ((256, 16, 256), (16.0, 1.0, 16.0), 4, 0.5, CL, 1),
    ((8, 12, 16), (2.0, 3.0, 4.0), 13, 0.6, SCFT, 0),
    ((24, 6, 48), (4.0, 1.5, 6.0), 1, 0.5, SCFT, 1),
    ((48, 48, 48), (6.0, 6.0, 6.0), 2, 0.5, SCFT, 0),
    ((128, 32, 192), (8.0, 2.0, 12.0), 11, 0.3, SCFT, 1),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_double_float_march_matches_oracle(case):
    n, L, Ns, fA, kind, streams = CASES[case]
    wp, wm = _fields(n, kind, 900 + case)
    _check(n, L, Ns, fA, 17.0, 2.0, kind, streams, wp, wm)


def test_double_float_gyroid_128cubed_full_size():
    """The bench's FP64 workload (gyroid SCFT 128^3, Ns = 100) over the full arrays."""
    w = wl.GYR128
    wp, wm = wl.fields(w)
    _check(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, 1, wp, wm,
           slices=[(0, k) for k in (1, 35, 36, 50, 99, 100)] + [(2, k) for k in (1, 64, 65, 100)])


def test_double_float_plan_is_refused_where_it_does_not_apply():
    with pft.System((64, 64, 64), (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, SCFT, pft.PFT_FP32_MIXED) as s:
        with pytest.raises(pft.PftError) as e:
            pft.pft_set_plan(s.h, 4, 1)
        assert e.value.status == pft.PFT_ERR_UNSUPPORTED
    with pft.System((64, 64, 64), (4.0, 4.0, 4.0), 4, 0.5, 15.0, 1.0, SCFT, FP64) as s:
        assert pft.pft_get_plan(s.h) == (3, 1)  # IEEE FP64 stays the default
