"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties one part of the oracle to something other than the oracle itself: a
closed form, an exact invariant of the discrete scheme, a brute-force or dense-matrix
computation, the continuum (exact-in-s) limit, the linear-response (Debye) result,
or published known-answer vectors.  A plausible mistake (dropped Boltzmann half-step,
wrong quadrature weight, A/B swap, sign of the Wick rotation, transposed operand,
wrong k^2 scaling) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fd5(f, h=1e-3):
    """Five-point central difference of f at 0: truncation O(h^4), round-off ~eps/h."""
    return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)


def _rand_fields(n, kind, seed, amp_p=0.3, amp_m=1.0):
    rng = np.random.default_rng(seed)
    wp = rng.normal(0, amp_p, n)
    wm = rng.normal(0, amp_m, n)
    if kind == o.CL_COMPLEX:
        wp = wp + 1j * rng.normal(0, amp_p, n)
        wm = wm + 1j * rng.normal(0, 0.3 * amp_m, n)
    return wp, wm


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_uniform_fields_closed_form(kind):
    """Uniform fields: only the k=0 mode is excited and D(0)=1, so q_n = exp(-w n ds)
    on each block and Q = exp(-(fA wA + fB wB)) exactly (Eqs. 4, 5); phiA = fA."""
    n, L, Ns, fA = (6, 4, 8), (3.0, 2.0, 5.0), 20, 0.35
    NsA = o.n_A_steps(Ns, fA)
    fa = NsA / Ns
    if kind == o.SCFT_REAL:
        wp, wm = np.full(n, 0.7), np.full(n, -1.3)
        wA, wB = 0.7 + 1.3, 0.7 - 1.3
    else:
        wp, wm = np.full(n, 0.4 - 0.2j), np.full(n, -1.1 + 0.3j)
        wA, wB = 1j * (0.4 - 0.2j) + 1.1 - 0.3j, 1j * (0.4 - 0.2j) - 1.1 + 0.3j
    s = o.solve(wp, wm, n, L, Ns, fA, kind)
    Qx = np.exp(-(fa * wA + (1 - fa) * wB))
    assert abs(s.Q - Qx) <= 1e-13 * abs(Qx)
    for k in range(Ns + 1):
        ex = np.exp(-wA * k / Ns) if k <= NsA else np.exp(-wA * fa - wB * (k - NsA) / Ns)
        assert np.max(np.abs(s.q[k] - ex)) <= 1e-13 * abs(ex)
    assert np.max(np.abs(s.phiA - fa)) < 1e-13
    assert np.max(np.abs(s.phiB - (1 - fa))) < 1e-13


def test_hamiltonian_uniform_closed_form():
    """Eq. 3 for uniform fields: H/(C V) = W-^2/chiN - W+ + fA wA + fB wB."""
    n, L, Ns, fA, chiN, C = (4, 4, 4), (2.0, 3.0, 4.0), 10, 0.3, 17.0, 2.5
    wpv, wmv = 0.25, -0.8
    s = o.solve(np.full(n, wpv), np.full(n, wmv), n, L, Ns, fA, o.SCFT_REAL)
    H = o.hamiltonian(np.full(n, wpv), np.full(n, wmv), s.lnQ, chiN, C, n, L, o.SCFT_REAL)
    fa = o.n_A_steps(Ns, fA) / Ns
    V = 24.0
    Hx = C * V * (wmv ** 2 / chiN - wpv + fa * (wpv - wmv) + (1 - fa) * (wpv + wmv))
    assert abs(H - Hx) <= 1e-13 * abs(Hx)


def test_diffusion_alone_plane_wave():
    """w = 0 and q_0 = exp(i k.x): the Laplacian eigenmode decays as exp(-k^2 s),
    so after Ns steps of ds = 1/Ns, q = exp(-k^2) exp(i k.x) exactly (Eq. 5)."""
    n, L, Ns = (8, 6, 4), (4.0, 3.0, 2.5), 16
    x = [np.arange(n[a]) * L[a] / n[a] for a in range(3)]
    m = (1, -2, 1)
    k = [2 * np.pi * m[a] / L[a] for a in range(3)]
    phase = (k[0] * x[0][:, None, None] + k[1] * x[1][None, :, None] + k[2] * x[2][None, None, :])
    q0 = np.exp(1j * phase)
    zero = np.zeros(n)
    s = o.solve(zero, zero, n, L, Ns, 0.5, o.SCFT_REAL, q0=q0, qd0=q0)
    k2 = sum(kk * kk for kk in k)
    assert np.max(np.abs(s.q[Ns] - np.exp(-k2) * q0)) < 1e-13


# ---------------------------------------------------------- exact invariants
@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_slice_invariance(kind):
    """Each split step is a (complex-)symmetric operator, so (1/M) sum q_n qd_{Ns-n}
    is the same Q at every cut of the chain."""
    n, L = (8, 6, 4), (4.0, 3.5, 2.0)
    wp, wm = _rand_fields(n, kind, 3)
    s = o.solve(wp, wm, n, L, 24, 0.4, kind)
    Qn = o.slice_partition_functions(s)
    assert np.max(np.abs(Qn - s.Q)) <= 1e-13 * abs(s.Q)


@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_sum_rules(kind):
    """With trapezoid weights per block: <phiA> = fA_eff and dV sum(phiA+phiB) = V."""
    n, L, Ns, fA = (6, 6, 6), (3.0, 3.0, 3.0), 30, 0.37
    wp, wm = _rand_fields(n, kind, 4)
    s = o.solve(wp, wm, n, L, Ns, fA, kind)
    fa = o.n_A_steps(Ns, fA) / Ns
    assert abs(s.phiA.mean() - fa) < 1e-13
    assert abs((s.phiA + s.phiB).mean() - 1.0) < 1e-13


def _perturbed(arr, idx, h):
    b = arr.copy()
    b[idx] += h
    return b


def test_density_is_exact_gradient_real():
    """dlnQ/dW+_j = -(phiA+phiB)_j/M and dlnQ/dW-_j = (phiA-phiB)_j/M hold exactly for
    the discrete 2nd-order scheme with trapezoid weights (Eq. 8 read as
    delta lnQ/delta w); a five-point difference agrees to ~1e-10 relative."""
    n, L, Ns, fA = (6, 4, 4), (3.0, 2.0, 2.0), 20, 0.35
    wp, wm = _rand_fields(n, o.SCFT_REAL, 5)
    s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    M = wp.size
    rng = np.random.default_rng(0)
    for j in rng.choice(M, 5, replace=False):
        idx = np.unravel_index(j, n)
        fdp = fd5(lambda h: o.solve(_perturbed(wp, idx, h), wm, n, L, Ns, fA, o.SCFT_REAL).lnQ)
        fdm = fd5(lambda h: o.solve(wp, _perturbed(wm, idx, h), n, L, Ns, fA, o.SCFT_REAL).lnQ)
        anp = -(s.phiA + s.phiB)[idx] / M
        anm = (s.phiA - s.phiB)[idx] / M
        assert abs(fdp - anp) <= 1e-9 * abs(anp), (fdp, anp)
        assert abs(fdm - anm) <= 1e-9 * abs(anm) + 1e-13, (fdm, anm)


def test_density_is_exact_gradient_complex():
    """Complex Langevin mapping: lnQ is holomorphic in omega, with
    dlnQ/domega+_j = -i(phiA+phiB)_j/M and dlnQ/domega-_j = (phiA-phiB)_j/M."""
    n, L, Ns, fA = (4, 4, 6), (2.0, 2.0, 3.0), 16, 0.3
    wp, wm = _rand_fields(n, o.CL_COMPLEX, 6)
    s = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
    M = wp.size
    for j in (1, 17, 50):
        idx = np.unravel_index(j, n)
        fdp = fd5(lambda h: o.solve(_perturbed(wp, idx, h), wm, n, L, Ns, fA, o.CL_COMPLEX).lnQ)
        fdm = fd5(lambda h: o.solve(wp, _perturbed(wm, idx, h), n, L, Ns, fA, o.CL_COMPLEX).lnQ)
        anp = -1j * (s.phiA + s.phiB)[idx] / M
        anm = (s.phiA - s.phiB)[idx] / M
        assert abs(fdp - anp) <= 1e-9 * abs(anp), (fdp, anp)
        assert abs(fdm - anm) <= 1e-9 * abs(anm) + 1e-13, (fdm, anm)


def test_shift_invariance():
    """A constant added to W+ shifts lnQ by -c and the field term by -c V, so H is
    unchanged (Eq. 3), and the mean W+ force vanishes."""
    n, L, Ns, fA, chiN, C = (6, 4, 4), (3.0, 2.0, 2.0), 16, 0.45, 15.0, 1.0
    wp, wm = _rand_fields(n, o.SCFT_REAL, 7)
    s1 = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    s2 = o.solve(wp + 0.73, wm, n, L, Ns, fA, o.SCFT_REAL)
    H1 = o.hamiltonian(wp, wm, s1.lnQ, chiN, C, n, L, o.SCFT_REAL)
    H2 = o.hamiltonian(wp + 0.73, wm, s2.lnQ, chiN, C, n, L, o.SCFT_REAL)
    assert abs(H1 - H2) < 1e-12 * abs(H1)
    assert abs((s1.phiA + s1.phiB - 1).mean()) < 1e-14


def test_symmetric_diblock():
    """fA = 1/2, W- odd under x -> x + L/2 and W+ even: reversing the chain and shifting
    by L/2 swaps A and B, so qd_n(x) = q_n(x + L/2) and phiA(x + L/2) = phiB(x).
    With W- = 0 the chain is symmetric and q = qd."""
    n, L, Ns = (8, 4, 4), (4.0, 2.0, 2.0), 20
    rng = np.random.default_rng(8)
    half = rng.normal(0, 1.0, (4, 4, 4))
    wm = np.concatenate([half, -half], axis=0)
    hp = rng.normal(0, 0.3, (4, 4, 4))
    wp = np.concatenate([hp, hp], axis=0)
    s = o.solve(wp, wm, n, L, Ns, 0.5, o.SCFT_REAL)
    for k in range(Ns + 1):
        assert np.max(np.abs(s.qd[k] - np.roll(s.q[k], -4, axis=0))) < 1e-13 * np.max(np.abs(s.q[k]))
    assert np.max(np.abs(np.roll(s.phiA, -4, axis=0) - s.phiB)) < 1e-13
    s0 = o.solve(wp, np.zeros(n), n, L, Ns, 0.5, o.SCFT_REAL)
    assert np.max(np.abs(s0.q - s0.qd)) < 1e-13 * np.max(np.abs(s0.q))


# --------------------------------------------------- brute force / dense / expm
def test_fft_equals_bruteforce_dft():
    """The FFT used by the oracle equals the O(M^2) DFT written out entry by entry."""
    rng = np.random.default_rng(9)
    x = rng.normal(size=(8, 8, 8)) + 1j * rng.normal(size=(8, 8, 8))
    a = np.fft.fftn(x)
    b = o.dft3_bruteforce(x)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))
    y = rng.normal(size=(4, 6, 8))
    assert np.max(np.abs(np.fft.fftn(y) - o.dft3_bruteforce(y))) < 1e-12 * 48


def test_fft_workers_changes_only_the_library():
    """The all-core timing switch (scipy.fft on several threads) computes the same DFT:
    a solve agrees with the numpy.fft one to rounding, and the default comes back after."""
    n, L, Ns, fA = (8, 12, 16), (2.0, 3.0, 4.0), 10, 0.4
    wp, wm = _rand_fields(n, o.CL_COMPLEX, 67)
    a = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
    with o.fft_workers(2):
        b = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
    c = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
    assert abs(a.Q - b.Q) <= 1e-14 * abs(a.Q) and np.max(np.abs(a.phiA - b.phiA)) <= 1e-14
    assert a.Q == c.Q and np.array_equal(a.phiA, c.phiA)


@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_march_equals_dense_matrix(kind):
    """Forward march with FFTs equals the march with the diffusion operator as the
    explicit M x M matrix F^-1 diag(D) F (8^3 grid)."""
    n, L, Ns, fA = (8, 8, 8), (4.0, 4.0, 4.0), 12, 0.5
    wp, wm = _rand_fields(n, kind, 10)
    s = o.solve(wp, wm, n, L, Ns, fA, kind)
    Dm = o.dense_propagator_matrix(n, s.D)
    if kind == o.SCFT_REAL:
        assert np.max(np.abs(Dm.imag)) < 1e-13
        Dm = Dm.real
    qd = o.forward_march_dense(s.BA, s.BB, Dm, Ns, s.NsA)
    assert np.max(np.abs(qd - s.q[Ns])) < 1e-12 * np.max(np.abs(s.q[Ns]))


def test_second_order_convergence_to_continuum():
    """Q(Ns) converges to the exact-in-s answer (dense expm of the spectral operator)
    as ds^2: successive errors at Ns = 32 .. 512 shrink by a factor that tends to 4
    (grid-scale noise makes the coarsest steps pre-asymptotic)."""
    n, L = (8, 4, 4), (4.0, 2.0, 2.0)
    xs = np.arange(8) * 4.0 / 8
    wm = np.broadcast_to(1.5 * np.cos(2 * np.pi * xs / 4.0)[:, None, None], n).copy()
    wm += 0.2 * np.random.default_rng(11).normal(size=n)
    wp = 0.1 * np.random.default_rng(12).normal(size=n)
    wA, wB = o.species_fields(wp, wm, o.SCFT_REAL)
    Qs = o.continuum_Q(wA, wB, n, L, 0.25)
    errs = [o.solve(wp, wm, n, L, Ns, 0.25, o.SCFT_REAL).Q - Qs for Ns in (32, 64, 128, 256, 512)]
    ratios = [errs[i] / errs[i + 1] for i in range(4)]
    assert all(3.4 < r < 4.1 for r in ratios), ratios
    assert 3.95 < ratios[-1] < 4.05 and 3.9 < ratios[-2] < 4.1, ratios
    assert abs(errs[-1]) < 1e-6 * abs(Qs)


def test_rpa_debye_response():
    """Weak exchange field W- = eps cos(k x): the k-mode of phiA - fA is
    eps (gAA - gAB) and that of phiB - fB is eps (gAB - gBB) (linearised density
    response with the Debye functions, as used for the semi-implicit update near
    Eq. 10), up to O(eps^3) and O(ds^2); Richardson extrapolation removes the latter."""
    eps = 1e-4
    n, L = (16, 2, 2), (5.0, 1.0, 1.0)
    fA = 0.25
    x = np.arange(16) * 5.0 / 16
    k = 2 * np.pi / 5.0
    wm = np.broadcast_to(eps * np.cos(k * x)[:, None, None], n).copy()
    wp = np.zeros(n)
    amps = []
    for Ns in (64, 128, 256):
        s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
        cA = 2 * np.mean(s.phiA[:, 0, 0] * np.cos(k * x))
        cB = 2 * np.mean(s.phiB[:, 0, 0] * np.cos(k * x))
        amps.append(np.array([cA, cB]))
    r1 = (4 * amps[1] - amps[0]) / 3
    r2 = (4 * amps[2] - amps[1]) / 3
    rr = (16 * r2 - r1) / 15
    gAA, gBB, gAB = o.debye_g(k * k, fA)
    ex = eps * np.array([gAA - gAB, gAB - gBB])
    assert np.all(np.abs(rr - ex) <= 1e-6 * np.abs(ex)), (rr, ex)


def test_debye_small_x_limits():
    """gAA -> f^2, gBB -> (1-f)^2, gAB -> f(1-f) as x -> 0 (normalisation check)."""
    gAA, gBB, gAB = o.debye_g(1e-5, 0.3)
    assert abs(gAA - 0.09) < 1e-5 and abs(gBB - 0.49) < 1e-5 and abs(gAB - 0.21) < 1e-5


# ------------------------------------------------------------- box derivative
@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_stress_matches_finite_difference(kind):
    """dlnQ/dL_a from the slice-by-slice derivative of the diffusion factor equals a
    finite difference of lnQ in L_a with the fields held fixed on the grid."""
    n, L, Ns, fA = (6, 4, 8), (3.0, 2.5, 4.0), 16, 0.35
    wp, wm = _rand_fields(n, kind, 13)
    s = o.solve(wp, wm, n, L, Ns, fA, kind)
    g = o.dlnQ_dL(s, n, L)
    for a in range(3):
        def f(h):
            Lh = list(L)
            Lh[a] += h
            return o.solve(wp, wm, n, Lh, Ns, fA, kind).lnQ
        fd = fd5(f)
        assert abs(fd - g[a]) <= 1e-9 * abs(g[a]) + 1e-12, (a, fd, g[a])


def _H_at(wp, wm, n, L, Ns, fA, chiN, C):
    return o.hamiltonian(wp, wm, o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL).lnQ, chiN, C, n, L, o.SCFT_REAL)


def test_dH_dL_matches_finite_difference():
    """dH/dL_a = H/L_a - C V dlnQ/dL_a against a finite difference of Eq. 3."""
    n, L, Ns, fA, chiN, C = (4, 6, 4), (2.0, 3.0, 2.2), 12, 0.4, 18.0, 3.0
    wp, wm = _rand_fields(n, o.SCFT_REAL, 14)
    s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    H = o.hamiltonian(wp, wm, s.lnQ, chiN, C, n, L, o.SCFT_REAL)
    g = o.dH_dL(H, s, C, n, L)
    for a in range(3):
        def f(h):
            Lh = list(L)
            Lh[a] += h
            return _H_at(wp, wm, n, Lh, Ns, fA, chiN, C)
        fd = fd5(f)
        assert abs(fd - g[a]) <= 1e-9 * abs(g[a]) + 1e-11


def test_dH_dfields_matches_finite_difference():
    """Discrete gradient of H (Eq. 3 with Eq. 7 forces times C dV) against finite
    differences of H."""
    n, L, Ns, fA, chiN, C = (4, 4, 6), (2.0, 2.0, 3.0), 12, 0.35, 18.0, 2.0
    wp, wm = _rand_fields(n, o.SCFT_REAL, 15)
    s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    gp, gm = o.dH_dfields(wp, wm, s, chiN, C, n, L, o.SCFT_REAL)
    for j in (3, 40, 77):
        idx = np.unravel_index(j, n)
        fdp = fd5(lambda h: _H_at(_perturbed(wp, idx, h), wm, n, L, Ns, fA, chiN, C))
        fdm = fd5(lambda h: _H_at(wp, _perturbed(wm, idx, h), n, L, Ns, fA, chiN, C))
        assert abs(fdp - gp[idx]) < 1e-9 * abs(gp[idx]) + 1e-10
        assert abs(fdm - gm[idx]) < 1e-9 * abs(gm[idx]) + 1e-10


# ------------------------------------------------------------- field updates
def test_homogeneous_saddle_is_fixed_point():
    """The homogeneous melt W+ = const, W- = chiN (2 fA - 1)/2 zeroes both forces of
    Eq. 7, so a relaxation step and a noise-free CL step leave it unchanged."""
    n, L, Ns, fA, chiN = (4, 4, 4), (2.0, 2.0, 2.0), 20, 0.3, 20.0
    fa = o.n_A_steps(Ns, fA) / Ns
    wp = np.full(n, 0.2)
    wm = np.full(n, chiN * (2 * fa - 1) / 2)
    s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    a, b = o.scft_euler_step(wp, wm, s.phiA, s.phiB, chiN, 0.1)
    assert np.max(np.abs(a - wp)) < 1e-14 and np.max(np.abs(b - wm)) < 1e-13
    cp, cm = wp.astype(complex), wm.astype(complex)
    s2 = o.solve(cp, cm, n, L, Ns, fA, o.CL_COMPLEX)
    z = np.zeros(n)
    a, b = o.cl_euler_maruyama_step(cp, cm, s2.phiA, s2.phiB, chiN, 0.01, z, z)
    assert np.max(np.abs(a - cp)) < 1e-14 and np.max(np.abs(b - cm)) < 1e-13


def _h_cl(wp, wm, n, L, Ns, fA, chiN, C, kind):
    s = o.solve(wp, wm, n, L, Ns, fA, kind)
    return o.hamiltonian(wp, wm, s.lnQ, chiN, C, n, L, kind), s


def test_scft_step_is_ascent_on_W_plus_and_descent_on_W_minus():
    """Direction and scale of the relaxation of Eq. 9 (Wick-rotated, force per C), pinned
    through H alone: a step along +lam dH/dW+/(C dV) changes H by +(C dV/lam)|dW+|^2 to
    first order, one along -lam dH/dW-/(C dV) by -(C dV/lam)|dW-|^2.  A flipped sign,
    a dropped 1/C or a missing dV in the step fails the ratio; H is pinned elsewhere by
    closed forms and by finite differences."""
    n, L, Ns, fA, chiN, C, lam = (6, 4, 8), (3.0, 2.0, 4.0), 12, 0.35, 16.0, 2.5, 1e-5
    wp, wm = _rand_fields(n, o.SCFT_REAL, 61)
    dV = float(np.prod(L)) / int(np.prod(n))
    H0, s = _h_cl(wp, wm, n, L, Ns, fA, chiN, C, o.SCFT_REAL)
    wpn, wmn = o.scft_euler_step(wp, wm, s.phiA, s.phiB, chiN, lam)
    dp, dm = wpn - wp, wmn - wm
    Hp = _h_cl(wpn, wm, n, L, Ns, fA, chiN, C, o.SCFT_REAL)[0]
    Hm = _h_cl(wp, wmn, n, L, Ns, fA, chiN, C, o.SCFT_REAL)[0]
    pred_p = C * dV / lam * np.sum(dp * dp)
    pred_m = -C * dV / lam * np.sum(dm * dm)
    assert Hp - H0 > 0 and Hm - H0 < 0
    assert abs((Hp - H0) / pred_p - 1) < 1e-3 and abs((Hm - H0) / pred_m - 1) < 1e-3


def test_cl_drift_is_minus_the_holomorphic_gradient():
    """Direction and scale of the noise-free complex Langevin step of Eq. 9 (lam = 1,
    force per C): H is holomorphic in the complex fields, so a drift d omega =
    -dt dH/domega/(C dV) changes H by -(C dV/dt) sum(d omega^2) (the complex square, not the
    modulus) to first order, separately for omega+ and omega-."""
    n, L, Ns, fA, chiN, C, dt = (4, 6, 4), (2.0, 3.0, 2.5), 10, 0.3, 20.0, 50.0, 1e-6
    wp, wm = _rand_fields(n, o.CL_COMPLEX, 62)
    dV = float(np.prod(L)) / int(np.prod(n))
    H0, s = _h_cl(wp, wm, n, L, Ns, fA, chiN, C, o.CL_COMPLEX)
    z = np.zeros(n)
    wpn, wmn = o.cl_euler_maruyama_step(wp, wm, s.phiA, s.phiB, chiN, dt, z, z)
    dp, dm = wpn - wp, wmn - wm
    Hp = _h_cl(wpn, wm, n, L, Ns, fA, chiN, C, o.CL_COMPLEX)[0]
    Hm = _h_cl(wp, wmn, n, L, Ns, fA, chiN, C, o.CL_COMPLEX)[0]
    for dH, d in ((Hp - H0, dp), (Hm - H0, dm)):
        pred = -C * dV / dt * np.sum(d * d)
        assert abs(dH / pred - 1) < 1e-3, (dH, pred)


def test_cl_step_without_noise_is_the_wick_rotated_scft_step():
    """omega+ = -i W+ (purely imaginary), real omega- = W- and no noise: the CL drift with
    dt = lam is the SCFT relaxation rotated back (W+ = i omega+), i.e. ascent on W+ comes
    out of the same equation of motion as descent on omega+."""
    n, L, Ns, fA, chiN, lam = (6, 4, 8), (3.0, 2.0, 4.0), 12, 0.4, 14.0, 0.3
    wp, wm = _rand_fields(n, o.SCFT_REAL, 63)
    s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    wpn, wmn = o.scft_euler_step(wp, wm, s.phiA, s.phiB, chiN, lam)
    sc = o.solve(-1j * wp, wm.astype(complex), n, L, Ns, fA, o.CL_COMPLEX)
    assert np.max(np.abs(sc.phiA - s.phiA)) < 1e-13
    z = np.zeros(n)
    cpn, cmn = o.cl_euler_maruyama_step(-1j * wp, wm.astype(complex), sc.phiA, sc.phiB, chiN, lam, z, z)
    assert np.max(np.abs(1j * cpn - wpn)) < 1e-13 and np.max(np.abs(cmn - wmn)) < 1e-13


def test_dH_dfields_matches_finite_difference_complex():
    """The CL forces times C dV are the holomorphic derivatives of H: a real increment h
    of one grid value of omega+- changes H by h dH/domega (finite differences of Eq. 3)."""
    n, L, Ns, fA, chiN, C = (4, 4, 6), (2.0, 2.0, 3.0), 10, 0.3, 20.0, 50.0
    wp, wm = _rand_fields(n, o.CL_COMPLEX, 64)
    s = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
    gp, gm = o.dH_dfields(wp, wm, s, chiN, C, n, L, o.CL_COMPLEX)

    def H(a, b):
        return _h_cl(a, b, n, L, Ns, fA, chiN, C, o.CL_COMPLEX)[0]
    for j in (5, 50, 90):
        idx = np.unravel_index(j, n)
        fdp = fd5(lambda h: H(_perturbed(wp, idx, h), wm))
        fdm = fd5(lambda h: H(wp, _perturbed(wm, idx, h)))
        assert abs(fdp - gp[idx]) < 1e-8 * abs(gp[idx]) + 1e-9
        assert abs(fdm - gm[idx]) < 1e-8 * abs(gm[idx]) + 1e-9


def test_scft_relaxation_converges_to_a_lamellar_saddle():
    """From the perturbed lamellar seed (W- = 5 cos(2 pi x/L) + noise, W+ = 0), repeated
    explicit Euler steps of Eq. 9 drive both forces of Eq. 7 to zero (a saddle point of H),
    with the lamellar order kept (the fundamental of W- stays large).  A step with either
    sign flipped runs away instead."""
    n, L, Ns, fA, chiN, lam = (16, 2, 2), (4.0, 1.0, 1.0), 32, 0.5, 15.0, 1.0
    x = np.arange(n[0]) * L[0] / n[0]
    rng = np.random.default_rng(65)
    wm = 5.0 * np.cos(2 * np.pi * x / L[0])[:, None, None] + rng.normal(0, 0.1, n)
    wp = np.zeros(n)

    def run(sgn_p, sgn_m, steps):
        a, b = wp.copy(), wm.copy()
        norms = []
        for _ in range(steps):
            with np.errstate(all="ignore"):
                s = o.solve(a, b, n, L, Ns, fA, o.SCFT_REAL)
            fp, fm = o.mean_field_forces(a, b, s.phiA, s.phiB, chiN, o.SCFT_REAL)
            norms.append(math.sqrt(np.mean(fp * fp) + np.mean(fm * fm)))
            an, bn = o.scft_euler_step(a, b, s.phiA, s.phiB, chiN, lam)
            a, b = a + sgn_p * (an - a), b + sgn_m * (bn - b)
            if not np.all(np.isfinite(b)) or np.max(np.abs(b)) > 1e3:
                norms.append(float("inf"))
                break
        return norms, b
    norms, b = run(1, 1, 300)
    assert norms[-1] < 1e-4 * norms[0]
    fund = abs(np.fft.fft(b.mean(axis=(1, 2)))[1]) / n[0]
    assert fund > 1.0
    for sp, sm in ((1, -1), (-1, 1)):
        bad, _ = run(sp, sm, 300)
        assert not bad[-1] < 1e-2 * norms[0]


def test_variable_cell_step_lowers_h():
    """The cell step of the variable-cell relaxation, L_a <- L_a - lam_L dh/dL_a with
    h = H/(C V) = <field term> - lnQ, lowers h by lam_L |dh/dL|^2 to first order (fields
    held on the grid; dlnQ/dL pinned by finite differences above)."""
    n, Ns, fA, chiN, lam_L = (6, 4, 8), 12, 0.35, 16.0, 1e-5
    L = np.array([3.0, 2.0, 4.0])
    wp, wm = _rand_fields(n, o.SCFT_REAL, 66)

    def h(Lx):
        s = o.solve(wp, wm, n, Lx, Ns, fA, o.SCFT_REAL)
        return o.hamiltonian(wp, wm, s.lnQ, chiN, 1.0, n, Lx, o.SCFT_REAL) / float(np.prod(Lx)), s
    h0, s = h(L)
    Ln = o.variable_cell_step(L, s, n, lam_L)
    h1, _ = h(Ln)
    g = -np.real(o.dlnQ_dL(s, n, L))
    pred = -lam_L * float(np.sum(g * g))
    assert h1 - h0 < 0 and abs((h1 - h0) / pred - 1) < 1e-3


# ---------------------------------------------------------------- generator
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t, 16) for t in line.split()])
    for r in rows:
        out = o.philox4x32_10(np.array([r[0:4]], dtype=np.uint32), (r[4], r[5]))[0]
        assert [int(v) for v in out] == r[6:10]


def test_philox_normals_moments():
    z = o.philox_normals(12345, 7, 3, 1, 400001)
    N = z.size
    assert abs(z.mean()) < 5 / math.sqrt(N)
    assert abs(z.var() - 1) < 5 * math.sqrt(2.0 / N)
    assert abs((z ** 4).mean() - 3) < 5 * math.sqrt(96.0 / N)
    z2 = o.philox_normals(12345, 7, 3, 0, 1000)
    z3 = o.philox_normals(12345, 7, 4, 1, 1000)
    assert abs(np.corrcoef(z[:1000], z2)[0, 1]) < 0.2 and abs(np.corrcoef(z[:1000], z3)[0, 1]) < 0.2


def test_cl_noise_variance():
    """Discrete noise variance 2 lam dt/(C dV) (below Eq. 10, force per C)."""
    std = o.cl_noise_std(0.01, 50.0, 0.5)
    assert abs(std ** 2 - 2 * 0.01 / (50.0 * 0.5)) < 1e-18
    ep, em = o.cl_noise(1, 0, 0, 200000, std)
    assert abs(ep.var() / std ** 2 - 1) < 0.02 and abs(em.var() / std ** 2 - 1) < 0.02


# ------------------------------------------------------------ RQM4 (Eq. 13)
@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_rqm4_uniform_fields_exact(kind):
    """Uniform fields: every split step multiplies by exp(-w h) exactly, so the
    Richardson combination (4 e^{-w h} - e^{-w h})/3 is exact too."""
    n, L, Ns, fA = (4, 6, 4), (2.0, 3.0, 2.0), 14, 0.4
    fa = o.n_A_steps(Ns, fA) / Ns
    if kind == o.SCFT_REAL:
        wp, wm = np.full(n, 0.3), np.full(n, -0.9)
        wA, wB = 1.2, -0.6
    else:
        wp, wm = np.full(n, 0.2 + 0.1j), np.full(n, -0.5 + 0.2j)
        wA, wB = 1j * (0.2 + 0.1j) + 0.5 - 0.2j, 1j * (0.2 + 0.1j) - 0.5 + 0.2j
    s = o.solve(wp, wm, n, L, Ns, fA, kind, scheme=o.RQM4)
    Qx = np.exp(-(fa * wA + (1 - fa) * wB))
    assert abs(s.Q - Qx) <= 1e-13 * abs(Qx)
    assert np.max(np.abs(s.phiA - fa)) < 1e-13


def test_simpson_weights_exact_for_cubics():
    """The composite rule (Simpson, 3/8 for an odd tail, trapezoid for one interval)
    integrates cubics exactly on any block [n0, n1]."""
    Ns = 17
    s = np.arange(Ns + 1) / Ns
    for n0, n1 in [(0, 17), (0, 6), (6, 17), (3, 4), (5, 5), (2, 9)]:
        c = o.simpson_weights(n0, n1, Ns + 1)
        a, b = n0 / Ns, n1 / Ns
        f = 1.0 + 2.0 * s - 3.0 * s ** 2 + 5.0 * s ** 3
        exact = (b - a) + (b ** 2 - a ** 2) - (b ** 3 - a ** 3) + 1.25 * (b ** 4 - a ** 4)
        if n1 - n0 == 1:
            continue  # the trapezoid fallback is exact only for linear functions
        assert abs(np.sum(c * f) / Ns - exact) < 1e-13


@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_rqm4_slice_invariance_and_sum_rules(kind):
    """The RQM4 step is a combination of symmetric operators, hence symmetric: Q is the
    same at every cut, and with a rule exact on constants <phiA> = fA_eff exactly."""
    n, L, Ns, fA = (6, 4, 4), (3.0, 2.0, 2.0), 15, 0.4
    wp, wm = _rand_fields(n, kind, 31)
    s = o.solve(wp, wm, n, L, Ns, fA, kind, scheme=o.RQM4)
    Qn = o.slice_partition_functions(s)
    assert np.max(np.abs(Qn - s.Q)) <= 1e-13 * abs(s.Q)
    assert abs(s.phiA.mean() - o.n_A_steps(Ns, fA) / Ns) < 1e-13
    assert abs((s.phiA + s.phiB).mean() - 1.0) < 1e-13


def test_rqm4_fourth_order_convergence_to_continuum():
    """Q(Ns) from the scheme of Eq. 13 converges to the exact-in-s answer (dense expm)
    as ds^4: error ratios for Ns = 8 .. 128 rise towards 16 (14.0, 15.0, 15.5, 15.7)."""
    n, L = (8, 4, 4), (4.0, 2.0, 2.0)
    xs = np.arange(8) * 4.0 / 8
    wm = np.broadcast_to(1.5 * np.cos(2 * np.pi * xs / 4.0)[:, None, None], n).copy()
    wp = 0.3 * np.broadcast_to(np.sin(2 * np.pi * xs / 4.0)[:, None, None], n).copy()
    wA, wB = o.species_fields(wp, wm, o.SCFT_REAL)
    Qs = o.continuum_Q(wA, wB, n, L, 0.25)
    errs = [o.solve(wp, wm, n, L, Ns, 0.25, o.SCFT_REAL, scheme=o.RQM4).Q - Qs for Ns in (8, 16, 32, 64, 128)]
    ratios = [errs[i] / errs[i + 1] for i in range(4)]
    assert all(13.5 < r < 16.5 for r in ratios), ratios
    assert ratios[-1] > 15.5 and all(ratios[i] < ratios[i + 1] for i in range(3)), ratios
    assert abs(errs[-1]) < 1e-9 * abs(Qs)


def test_rqm4_densities_are_fourth_order_gradients():
    """With RQM4 and Simpson weights phi is the lnQ gradient up to O(ds^4): the mismatch
    against a finite difference falls by ~16 when Ns doubles."""
    n, L, fA = (6, 4, 4), (3.0, 2.0, 2.0), 0.5
    wp, wm = _rand_fields(n, o.SCFT_REAL, 32, amp_p=0.2, amp_m=0.6)
    idx = (1, 2, 3)
    mism = []
    for Ns in (64, 128):
        s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL, scheme=o.RQM4)
        fd = fd5(lambda h: o.solve(wp, _perturbed(wm, idx, h), n, L, Ns, fA, o.SCFT_REAL, scheme=o.RQM4).lnQ)
        mism.append(abs(fd - (s.phiA - s.phiB)[idx] / wp.size))
    assert mism[1] < mism[0] / 12.0, mism


# ------------------------------------------------------------ SIS (Eq. 11)
def test_debye_chain_is_the_sum_of_the_block_functions():
    """g_D = g_AA + 2 g_AB + g_BB for any block split (the whole chain's Debye function)
    where the block closed forms are accurate (x >= 0.01), and the closed form evaluated
    in 50-digit arithmetic across the series/closed-form switch at small x."""
    for x in (0.01, 0.3, 2.0, 17.0):
        for f in (0.2, 0.5, 0.65):
            gAA, gBB, gAB = o.debye_g(x, f)
            assert abs(float(o.debye_chain(x)) - (gAA + 2 * gAB + gBB)) < 1e-10, (x, f)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    for x in (1e-6, 1e-3, 0.0999, 0.1001, 0.5):
        X = mpmath.mpf(x)
        ref = float(2 * (mpmath.exp(-X) + X - 1) / X ** 2)
        assert abs(float(o.debye_chain(x)) - ref) < 1e-13, x
    assert float(o.debye_chain(0.0)) == 1.0


def _cos_field(eps, n, L, k_index=1):
    x = np.arange(n[0]) * L[0] / n[0]
    k = 2 * np.pi * k_index / L[0]
    return np.broadcast_to(eps * np.cos(k * x)[:, None, None], n).copy(), x, k


@pytest.mark.parametrize("lam", [0.5, 4.0])
def test_sis_linear_response_is_the_wavevector_dependent_step(lam):
    """W+ = eps cos(k x), W- = 0, fA = 1/2: the linearised force is -g_D(k) W+, so one
    SIS step leaves the amplitude eps / (1 + lam g_D(k)) up to O(eps^2) + O(ds^2) (error
    4e-7 at Ns = 128, falling 4x per halving of ds); the explicit Euler step leaves
    eps (1 - lam g_D(k)), which grows for lam g_D > 2."""
    eps = 1e-4
    n, L = (16, 2, 2), (5.0, 1.0, 1.0)
    wp, x, k = _cos_field(eps, n, L)
    wm = np.zeros(n)
    gD = float(o.debye_chain(k * k))
    errs = []
    for Ns in (64, 128):
        s = o.solve(wp, wm, n, L, Ns, 0.5, o.SCFT_REAL)
        wpn, wmn = o.scft_sis_step(wp, wm, s.phiA, s.phiB, 15.0, lam, n, L)
        amp = 2 * np.mean(wpn[:, 0, 0] * np.cos(k * x)) / eps
        errs.append(abs(amp * (1 + lam * gD) - 1))
        assert np.max(np.abs(wmn)) < 1e-12  # fA = 1/2: no exchange-field response to W+
        wpe, _ = o.scft_euler_step(wp, wm, s.phiA, s.phiB, 15.0, lam)
        ampe = 2 * np.mean(wpe[:, 0, 0] * np.cos(k * x)) / eps
        assert abs(ampe - (1 - lam * gD)) < 1e-5
    assert errs[1] < 1e-6 and 3.0 < errs[0] / errs[1] < 5.0, errs
    if lam * gD > 2:
        assert abs(1 - lam * gD) > 1 > 1 / (1 + lam * gD)


def test_sis_leaves_the_homogeneous_saddle_fixed():
    """At the homogeneous saddle (W+ uniform, W- = chiN (2 fA_eff - 1)/2) both forces
    vanish and the SIS step changes nothing (SCFT and CL forms)."""
    n, L, Ns, fA, chiN = (6, 4, 8), (3.0, 2.0, 4.0), 20, 0.35, 12.0
    fa = o.n_A_steps(Ns, fA) / Ns
    wp = np.full(n, 0.4)
    wm = np.full(n, chiN * (2 * fa - 1) / 2)
    s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    wpn, wmn = o.scft_sis_step(wp, wm, s.phiA, s.phiB, chiN, 0.7, n, L)
    assert np.max(np.abs(wpn - wp)) < 1e-13 and np.max(np.abs(wmn - wm)) < 1e-13
    z = np.zeros(n)
    cpn, cmn = o.cl_sis_step(-1j * wp, wm.astype(complex), s.phiA, s.phiB, chiN, 0.7, z, z, n, L)
    assert np.max(np.abs(cpn + 1j * wp)) < 1e-13 and np.max(np.abs(cmn - wm)) < 1e-13


def test_cl_sis_without_noise_is_the_wick_rotated_scft_sis():
    """With omega+ = -i W+ (purely imaginary), real omega- and no noise, the CL SIS step
    with dt = lam is the SCFT SIS step rotated back (W+ = i omega+)."""
    n, L, Ns, fA, chiN, lam = (6, 4, 8), (3.0, 2.0, 4.0), 12, 0.4, 14.0, 0.3
    wp, wm = _rand_fields(n, o.SCFT_REAL, 41)
    s = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    wpn, wmn = o.scft_sis_step(wp, wm, s.phiA, s.phiB, chiN, lam, n, L)
    z = np.zeros(n)
    cpn, cmn = o.cl_sis_step(-1j * wp, wm.astype(complex), s.phiA, s.phiB, chiN, lam, z, z, n, L)
    assert np.max(np.abs(1j * cpn - wpn)) < 1e-13 and np.max(np.abs(cmn - wmn)) < 1e-13


def test_cl_sis_filters_the_noise_with_the_same_factor():
    """Eq. 11 puts the noise on the same side as the force, so at a saddle a plane-wave
    noise eta+ = a cos(k x) moves omega+ by a cos(k x) / (1 + dt g_D(k)), and eta- moves
    omega- by eta- / (1 + 2 dt/chiN)."""
    n, L, Ns, fA, chiN, dt = (16, 2, 2), (5.0, 1.0, 1.0), 16, 0.5, 10.0, 0.8
    wp = np.zeros(n, complex)
    wm = np.zeros(n, complex)
    s = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
    eta, x, k = _cos_field(0.3, n, L, k_index=2)
    gD = float(o.debye_chain(k * k))
    cpn, cmn = o.cl_sis_step(wp, wm, s.phiA, s.phiB, chiN, dt, eta, eta, n, L)
    assert np.max(np.abs(cpn - eta / (1 + dt * gD))) < 1e-13
    assert np.max(np.abs(cmn - eta / (1 + 2 * dt / chiN))) < 1e-13


# ------------------------------------------------------- Edwards homopolymer (Eq. 2)
@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_edwards_uniform_field_closed_form(kind):
    """Uniform field: q_n = exp(-w n ds), Q = exp(-w), phi = 1 exactly."""
    n, L, Ns = (4, 6, 4), (2.0, 3.0, 2.0), 14
    w = np.full(n, 0.7) if kind == o.SCFT_REAL else np.full(n, 0.3 - 0.2j)
    s = o.edwards_solve(w, n, L, Ns, kind)
    wf = o.edwards_field(w, kind).flat[0]
    assert abs(s.Q - np.exp(-wf)) <= 1e-14 * abs(np.exp(-wf))
    for k in (1, 5, Ns):
        assert np.max(np.abs(s.q[k] - np.exp(-wf * k / Ns))) < 1e-14
    assert np.max(np.abs(s.phi - 1.0)) < 1e-13


@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_edwards_equals_the_diblock_path_with_one_block(kind):
    """A homopolymer is a diblock with fA = 1 and no exchange field: the diblock path, which
    marches q-dagger separately, gives the same Q and phi_A = phi (pins q-dagger = q)."""
    n, L, Ns = (6, 4, 8), (3.0, 2.0, 4.0), 17
    rng = np.random.default_rng(50)
    w = rng.normal(0, 0.5, n)
    if kind == o.CL_COMPLEX:
        w = w + 1j * rng.normal(0, 0.3, n)
    e = o.edwards_solve(w, n, L, Ns, kind)
    d = o.solve(w, np.zeros(n, w.dtype), n, L, Ns, 1.0, kind)
    assert abs(e.Q - d.Q) <= 1e-13 * abs(d.Q)
    assert np.max(np.abs(e.phi - d.phiA)) < 1e-13 and np.max(np.abs(d.phiB)) == 0.0


@pytest.mark.parametrize("kind", [o.SCFT_REAL, o.CL_COMPLEX])
def test_edwards_force_is_the_gradient_of_H(kind):
    """dH/dW_j = C dV (phi_j - (B/C) W_j) for the discrete H of SCFT mode (5-point finite
    differences, 1e-8), and dH/domega_j = C dV ((B/C) omega_j + i phi_j) in CL mode."""
    n, L, Ns, B, C = (6, 4, 4), (3.0, 2.0, 2.0), 12, 2.0, 5.0
    rng = np.random.default_rng(51)
    w = rng.normal(0, 0.4, n)
    if kind == o.CL_COMPLEX:
        w = w + 1j * rng.normal(0, 0.2, n)
    s = o.edwards_solve(w, n, L, Ns, kind)
    dV = np.prod(L) / np.prod(n)
    if kind == o.SCFT_REAL:
        g = C * dV * (s.phi - (B / C) * w)
    else:
        g = C * dV * ((B / C) * w + 1j * s.phi)
    for idx in [(1, 2, 3), (4, 0, 1)]:
        def H(h, idx=idx):
            ww = w.copy()
            ww[idx] += h
            return o.edwards_hamiltonian(ww, o.edwards_solve(ww, n, L, Ns, kind).lnQ, B, C, n, L, kind)
        fd = fd5(H)
        assert abs(fd - g[idx]) <= 1e-8 * max(1.0, abs(g[idx])), (idx, fd, g[idx])


def test_edwards_debye_response_and_saddle():
    """W = W0 + eps cos(k x): the k-mode of phi is -eps g_D(k) (whole-chain Debye function)
    up to O(eps^2) and O(ds^2) (Richardson over Ns = 64, 128, 256); the homogeneous
    saddle W = C/B is a fixed point of the SCFT step."""
    eps = 1e-4
    n, L = (16, 2, 2), (5.0, 1.0, 1.0)
    x = np.arange(16) * 5.0 / 16
    k = 2 * np.pi / 5.0
    W = 0.3 + np.broadcast_to(eps * np.cos(k * x)[:, None, None], n).copy()
    amps = []
    for Ns in (64, 128, 256):
        s = o.edwards_solve(W, n, L, Ns, o.SCFT_REAL)
        amps.append(2 * np.mean(s.phi[:, 0, 0] * np.cos(k * x)))
    r1 = (4 * amps[1] - amps[0]) / 3
    r2 = (4 * amps[2] - amps[1]) / 3
    rr = (16 * r2 - r1) / 15
    ex = -eps * float(o.debye_chain(k * k))
    assert abs(rr - ex) <= 1e-6 * abs(ex), (rr, ex)
    B, C = 2.0, 5.0
    W0 = np.full((4, 4, 4), C / B)
    s = o.edwards_solve(W0, (4, 4, 4), (2.0, 2.0, 2.0), 10, o.SCFT_REAL)
    assert np.max(np.abs(o.edwards_scft_step(W0, s.phi, B, C, 0.5) - W0)) < 1e-13


# ------------------------------------------------------- reverse-mode adjoint (f3)
def _adj_setup(seed=5):
    n, L, Ns, fA = (6, 4, 4), (3.0, 2.0, 2.0), 12, 0.4
    rng = np.random.default_rng(seed)
    return n, L, Ns, fA, rng.normal(0, 0.3, n), rng.normal(0, 0.8, n), rng


def test_adjoint_gradient_of_a_linear_loss_matches_finite_differences():
    """L = sum_x (UA phiA + UB phiB) with random UA, UB: the adjoint gradients with respect
    to W+ and W- equal 5-point finite differences of L through the full solve (1e-9)."""
    n, L, Ns, fA, wp, wm, rng = _adj_setup()
    UA, UB = rng.normal(size=n), rng.normal(size=n)

    def loss(a, b):
        s = o.solve(a, b, n, L, Ns, fA, o.SCFT_REAL)
        return float(np.sum(UA * s.phiA + UB * s.phiB))
    gp, gm = o.adjoint_field_gradient(wp, wm, n, L, Ns, fA, UA, UB)
    for idx in [(1, 2, 3), (4, 0, 1), (0, 3, 2)]:
        for which, g in ((0, gp), (1, gm)):
            def f(h, idx=idx, which=which):
                a, b = wp.copy(), wm.copy()
                (a if which == 0 else b)[idx] += h
                return loss(a, b)
            fd = fd5(f, 1e-4)
            assert abs(fd - g[idx]) <= 1e-9 * max(1.0, abs(g[idx])), (idx, which, fd, g[idx])


def test_adjoint_gradient_of_a_quadratic_loss_matches_finite_differences():
    """L = (1/2) sum_x (phiA - t)^2, so dL/dphiA = phiA - t and dL/dphiB = 0."""
    n, L, Ns, fA, wp, wm, rng = _adj_setup(6)
    t = rng.uniform(0.2, 0.6, n)

    def loss(a, b):
        s = o.solve(a, b, n, L, Ns, fA, o.SCFT_REAL)
        return 0.5 * float(np.sum((s.phiA - t) ** 2))
    s0 = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    gp, gm = o.adjoint_field_gradient(wp, wm, n, L, Ns, fA, s0.phiA - t, np.zeros(n))
    for idx in [(2, 1, 0), (5, 3, 3)]:
        for which, g in ((0, gp), (1, gm)):
            def f(h, idx=idx, which=which):
                a, b = wp.copy(), wm.copy()
                (a if which == 0 else b)[idx] += h
                return loss(a, b)
            fd = fd5(f, 1e-4)
            assert abs(fd - g[idx]) <= 1e-9 * max(1.0, abs(g[idx])), (idx, which, fd, g[idx])


@pytest.mark.parametrize("GA,GB", [(1.0, 1.0), (1.0, 0.0), (0.0, 1.0)])
def test_adjoint_gradient_of_the_sum_rules_vanishes(GA, GB):
    """sum_x phiA = M fA_eff and sum_x phiB = M (1 - fA_eff) hold exactly for every field
    (trapezoid rule), so the adjoint gradient of these losses is zero to round-off: a
    dropped term or a wrong sign in the Q normalisation or in either adjoint march breaks
    the cancellation."""
    n, L, Ns, fA, wp, wm, rng = _adj_setup(7)
    gp, gm = o.adjoint_field_gradient(wp, wm, n, L, Ns, fA, np.full(n, GA), np.full(n, GB))
    assert np.max(np.abs(gp)) < 1e-13 and np.max(np.abs(gm)) < 1e-13
