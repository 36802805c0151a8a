"""GPU parity of the Edwards homopolymer model (Eq. 2: one field, q-dagger = q, one march)
against the oracle.  Tolerances as for the diblock solve: FP64 relative 1e-12 on Q and H,
1e-10 absolute on phi, 1e-12 relative on propagator slices; FP32-mixed 2e-5 (Q, phi,
h = H/(C V))."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu

FP64, FP32 = pft.PFT_FP64, pft.PFT_FP32_MIXED
SCFT, CL = pft.PFT_SCFT_REAL, pft.PFT_CL_COMPLEX
OKIND = {SCFT: o.SCFT_REAL, CL: o.CL_COMPLEX}
EDW = pft.PFT_ARCH_EDWARDS


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _field(n, kind, seed, amp=0.5):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, amp, n)
    if kind == CL:
        w = w + 1j * rng.normal(0, 0.5 * amp, n)
    return w


def _rel(a, b):
    return abs(a - b) / abs(b)


def _system(n, L, Ns, kind, prec, B=2.0, C=5.0, **kw):
    return pft.System(n, L, Ns, 0.5, 1.0, C, kind, prec, arch=EDW, B=B, **kw)


CASES = [((16, 12, 8), (4.0, 3.0, 2.0), 20), ((12, 12, 12), (3.0, 3.0, 3.0), 13), ((48, 4, 6), (6.0, 1.0, 1.5), 10),
         ((64, 64, 64), (8.0, 8.0, 8.0), 16), ((8, 8, 8), (2.0, 2.0, 2.0), 1)]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("kind", [SCFT, CL])
@pytest.mark.parametrize("case", CASES)
def test_edwards_solve_matches_oracle(case, kind, prec):
    n, L, Ns = case
    B, C = 2.0, 5.0
    w = _field(n, kind, 90 + Ns)
    ref = o.edwards_solve(w, n, L, Ns, OKIND[kind])
    Href = o.edwards_hamiltonian(w, ref.lnQ, B, C, n, L, OKIND[kind])
    with _system(n, L, Ns, kind, prec, B, C) as s:
        s.set_fields(w)
        s.solve()
        obs = s.observables()
        phi, phiB = s.densities()
        Q = obs["Q"] if kind == CL else obs["Q"].real
        H = obs["H"] if kind == CL else obs["H"].real
        t = 1e-12 if prec == FP64 else 2e-5
        assert _rel(Q, ref.Q) <= t
        if prec == FP64:
            assert _rel(H, Href) <= 1e-12
        else:
            assert abs(H - Href) / (C * float(np.prod(L))) <= 2e-5
        assert np.max(np.abs(phi - ref.phi)) <= (1e-10 if prec == FP64 else 2e-5)
        assert np.max(np.abs(phiB)) == 0.0
        for k in sorted({0, 1, Ns}):
            q = s.propagator(0, k)
            assert np.max(np.abs(q - ref.q[k])) <= t * np.max(np.abs(ref.q[k]))
        qd = s.propagator(1, 0)  # qd_Ns = q_Ns for the reversible chain
        assert np.max(np.abs(qd - ref.q[Ns])) <= t * np.max(np.abs(ref.q[Ns]))
        assert abs(obs["phiA_mean"].real - 1.0) <= (1e-12 if prec == FP64 else 1e-6)


def test_edwards_uniform_field_closed_form():
    n, L, Ns = (8, 12, 16), (2.0, 3.0, 4.0), 20
    with _system(n, L, Ns, SCFT, FP64) as s:
        s.set_fields(np.full(n, 0.7))
        s.solve()
        obs = s.observables()
        phi, _ = s.densities()
    assert _rel(obs["Q"].real, np.exp(-0.7)) <= 1e-13
    assert np.max(np.abs(phi - 1.0)) <= 1e-13


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_edwards_scft_relaxation_matches_oracle_and_reaches_the_saddle(prec):
    n, L, Ns, B, C, lam = (16, 12, 8), (4.0, 3.0, 2.0), 16, 2.0, 5.0, 0.5
    W = 2.5 + _field(n, SCFT, 33, 0.3)
    with _system(n, L, Ns, SCFT, prec, B, C) as s:
        s.set_fields(W)
        f0 = None
        for it in range(40):
            s.solve()
            obs = s.observables()
            if it < 4:
                ref = o.edwards_solve(W, n, L, Ns, o.SCFT_REAL)
                W = o.edwards_scft_step(W, ref.phi, B, C, lam)
            if f0 is None:
                f0 = obs["force_p_rms"]
            s.field_step(lam)
            if it == 3:
                gW, _ = s.get_fields()
                assert np.max(np.abs(gW - W)) <= (1e-12 if prec == FP64 else 1e-5)
        s.solve()
        obs = s.observables()
        gW, _ = s.get_fields()
    # homogeneous saddle W* = (C/B) phi with phi = 1
    assert obs["force_p_rms"] < 1e-3 * f0
    assert np.max(np.abs(gW - C / B)) < 1e-3


def test_edwards_cl_steps_with_supplied_and_device_noise_match_oracle():
    n, L, Ns, B, C, dt = (16, 8, 12), (4.0, 2.0, 3.0), 12, 1.0, 50.0, 0.01
    w = 0.02 + _field(n, CL, 34, 0.05)
    dV = np.prod(L) / np.prod(n)
    std = o.cl_noise_std(dt, C, dV)
    rng = np.random.default_rng(8)
    seed, inst = 777, 2
    with _system(n, L, Ns, CL, FP64, B, C, seed=seed, instance=inst) as s:
        s.set_fields(w)
        for it in range(4):
            s.solve()
            ref = o.edwards_solve(w, n, L, Ns, o.CL_COMPLEX)
            obs = s.observables()
            Href = o.edwards_hamiltonian(w, ref.lnQ, B, C, n, L, o.CL_COMPLEX)
            assert abs(obs["H"] - Href) <= 1e-12 * abs(Href)
            if it < 2:
                eta = std * rng.normal(size=n)
                s.field_step(dt, eta, np.zeros(n))
            else:
                s.field_step(dt)
                eta = o.cl_noise(seed, inst, it, w.size, std)[0].reshape(n)
            w = o.edwards_cl_step(w, ref.phi, B, C, dt, eta)
            gw, _ = s.get_fields()
            assert np.max(np.abs(gw - w)) <= 1e-10


def test_edwards_128cubed_fp32_against_the_oracle():
    """128^3 (the plane-kernel path), Ns = 50: Q, H and phi at 4096 sampled points."""
    n, L, Ns, B, C = (128, 128, 128), (8.0, 8.0, 8.0), 50, 1.0, 20.0
    x = np.arange(128) * (2 * np.pi / 128)
    W = 1.0 + 0.5 * np.sin(x)[:, None, None] * np.cos(x)[None, :, None] + 0.1 * np.random.default_rng(3).normal(size=n)
    ref = o.edwards_solve(W, n, L, Ns, o.SCFT_REAL)
    Href = o.edwards_hamiltonian(W, ref.lnQ, B, C, n, L, o.SCFT_REAL)
    with _system(n, L, Ns, SCFT, FP32, B, C) as s:
        s.set_fields(W)
        s.solve()
        obs = s.observables()
        phi, _ = s.densities()
    idx = np.random.default_rng(4).choice(phi.size, 4096, replace=False)
    assert _rel(obs["Q"].real, ref.Q) <= 2e-5
    assert abs(obs["H"].real - Href) / (C * float(np.prod(L))) <= 2e-5
    assert np.max(np.abs(phi.ravel()[idx] - ref.phi.ravel()[idx])) <= 2e-5


def test_edwards_refuses_what_it_does_not_implement():
    n, L = (64, 64, 64), (8.0, 8.0, 8.0)
    for kw in (dict(scheme=pft.PFT_SCHEME_RQM4), dict(checkpoint=4)):
        with pytest.raises(pft.PftError) as ei:
            _system(n, L, 10, SCFT, FP32, **kw)
        assert ei.value.status == pft.PFT_ERR_UNSUPPORTED
    with _system((8, 8, 8), (2.0, 2.0, 2.0), 8, SCFT, FP64) as s:
        s.set_fields(_field((8, 8, 8), SCFT, 5))
        s.solve()
        with pytest.raises(pft.PftError) as ei:
            s.gradients()
        assert ei.value.status == pft.PFT_ERR_UNSUPPORTED
        with pytest.raises(pft.PftError) as ei:
            s.field_step(0.1, semi_implicit=True)
        assert ei.value.status == pft.PFT_ERR_UNSUPPORTED
