"""The complex-field plane kernel (FP32-mixed complex Langevin fields with ny = nz = 64:
y and z transforms of one x-plane in one CTA, complex Boltzmann factors) against the
oracle: Q, H, phiA, phiB and propagator slices of one solve, a few Euler-Maruyama steps
with caller noise, and the block junction, a one-step chain and x extents other than
64.  Tolerances as for the FP32-mixed pass march: relative 2e-5 on Q and on propagator
slices, absolute 2e-5 on phi and on h = H/(C V), 1e-5 on the fields after the steps."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu

FP32 = pft.PFT_FP32_MIXED
CL = pft.PFT_CL_COMPLEX


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _fields(n, seed, amp_p=0.1, amp_m=0.6):
    rng = np.random.default_rng(seed)
    wp = amp_p * (rng.normal(size=n) + 1j * rng.normal(size=n))
    wm = amp_m * rng.normal(size=n) + 1j * 0.3 * amp_m * rng.normal(size=n)
    return wp, wm


CASES = [((64, 64, 64), (8.0, 8.0, 8.0), 16, 0.3), ((16, 64, 64), (2.0, 8.0, 8.0), 7, 0.5),
         ((48, 64, 64), (6.0, 8.0, 8.0), 1, 0.5)]


@pytest.mark.parametrize("case", CASES)
def test_plane_kernel_solve_matches_oracle(case):
    n, L, Ns, fA = case
    chiN, C = 20.0, 50.0
    wp, wm = _fields(n, 40 + Ns)
    ref = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
    Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, o.CL_COMPLEX)
    with pft.System(n, L, Ns, fA, chiN, C, CL, FP32) as s:
        pft.pft_set_plan(s.h, 1, 1)  # the 3D plane kernel (plan 2 where nx allows is the default)
        s.set_fields(wp, wm)
        s.solve()
        assert pft.pft_get_plan(s.h) == (1, 1)
        obs = s.observables()
        phiA, phiB = s.densities()
        assert abs(obs["Q"] - ref.Q) <= 2e-5 * abs(ref.Q)
        assert abs(obs["H"] - Href) / (C * float(np.prod(L))) <= 2e-5
        assert np.max(np.abs(phiA - ref.phiA)) <= 2e-5
        assert np.max(np.abs(phiB - ref.phiB)) <= 2e-5
        for k in sorted({1, Ns // 2, Ns}):
            q = s.propagator(0, k)
            assert np.max(np.abs(q - ref.q[k])) <= 2e-5 * np.max(np.abs(ref.q[k]))


def test_plane_kernel_cl_steps_with_caller_noise():
    n, L, Ns, fA, chiN, C, dt = (32, 64, 64), (4.0, 8.0, 8.0), 10, 0.3, 20.0, 50.0, 0.01
    wp, wm = _fields(n, 7, 0.05, 0.2)
    wm = wm + chiN * (2 * fA - 1) / 2
    dV = np.prod(L) / np.prod(n)
    std = o.cl_noise_std(dt, C, dV)
    rng = np.random.default_rng(9)
    with pft.System(n, L, Ns, fA, chiN, C, CL, FP32) as s:
        s.set_fields(wp, wm)
        for _ in range(3):
            s.solve()
            assert pft.pft_get_plan(s.h)[0] == 1
            ref = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
            ep = std * rng.normal(size=n)
            em = std * rng.normal(size=n)
            s.field_step(dt, ep, em)
            wp, wm = o.cl_euler_maruyama_step(wp, wm, ref.phiA, ref.phiB, chiN, dt, ep, em)
            gp, gm = s.get_fields()
            assert np.max(np.abs(gp - wp)) <= 1e-5 and np.max(np.abs(gm - wm)) <= 1e-5


def test_other_complex_grids_take_the_separable_pencil_march():
    # no plane kernel for these complex grids: the default is the separable march on pencils
    for n in ((64, 32, 64), (64, 64, 32), (32, 128, 128)):
        with pft.System(n, (4.0, 4.0, 4.0), 4, 0.5, 20.0, 50.0, CL, FP32) as s:
            s.set_fields(*_fields(n, 3))
            s.solve()
            assert pft.pft_get_plan(s.h)[0] == 3, n


@pytest.mark.parametrize("n,Ns,streams,code", [((64, 64, 64), 16, 1, 2), ((128, 64, 64), 7, 0, 2), ((64, 64, 64), 2, 1, 2),
                                               ((64, 64, 64), 5, 1, 18)])
def test_complex_separable_march_matches_oracle(n, Ns, streams, code):
    """The separable march for complex fields (the default at CL 64^3): complex column and
    row lines of the 64 x 64 planes, complex x-lines, against the oracle."""
    L, fA, chiN, C = (n[0] / 8.0, 8.0, 8.0), 0.3, 20.0, 50.0
    wp, wm = _fields(n, 70 + Ns)
    ref = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
    Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, o.CL_COMPLEX)
    with pft.System(n, L, Ns, fA, chiN, C, CL, FP32) as s:
        if streams == 1:
            assert pft.pft_get_plan(s.h) == (2, 1)
        pft.pft_set_plan(s.h, code, streams)
        s.set_fields(wp, wm)
        s.solve()
        s.solve()
        obs = s.observables()
        phiA, phiB = s.densities()
        eq = max(np.max(np.abs(s.propagator(w, k) - (ref.q if w == 0 else ref.qd)[k]))
                 / np.max(np.abs((ref.q if w == 0 else ref.qd)[k])) for w, k in ((0, 1), (0, Ns), (2, 1), (2, Ns)))
    eQ = abs(obs["Q"] - ref.Q) / abs(ref.Q)
    ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
    print(f"\ncomplex separable {n} Ns={Ns}: Q rel {eQ:.2e} phi abs {ephi:.2e} slices {eq:.2e}")
    assert eQ <= 2e-5 and ephi <= 2e-5 and eq <= 2e-5
    assert abs(obs["H"] - Href) / (C * float(np.prod(L))) <= 2e-5
