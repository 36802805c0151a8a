"""Plain FP64 CPU oracle of the pseudo-spectral diblock propagator path.

TEST INFRASTRUCTURE ONLY.  Slow and obviously correct on purpose: it follows the
method of Delaney & Fredrickson, "Polymer Field-Theory Simulations on Graphics
Processing Units" (arXiv:1204.5434), step by step, in numpy float64/complex128, with
``numpy.fft`` as the only library primitive (``fft_workers`` swaps in ``scipy.fft`` on
several threads for the all-core CPU baseline; the arithmetic stays the same).  Nothing
here is blocked, fused or
reordered.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may call it; the CUDA library never does.

Conventions (the readings of the paper the whole project uses):

* grid ``n = (nx, ny, nz)``, box ``L = (Lx, Ly, Lz)`` in units of Rg, arrays are
  row-major ``[x][y][z]`` (z fastest).  ``M = nx*ny*nz``, ``V = Lx*Ly*Lz``,
  ``dV = V/M`` and a spatial integral is ``dV * sum``.
* contour ``s`` in ``[0, 1]`` (Eq. 5), ``ds = 1/Ns``; the A block holds the first
  ``NsA = floor(fA*Ns + 1/2)`` steps, so the effective A fraction is ``NsA/Ns``.
* wavenumbers ``k_a = 2*pi*m/L_a`` with ``m`` the signed FFT index; the diffusion
  factor of one contour step is ``exp(-k^2 ds)`` (the Laplacian of Eq. 5 in Rg units).
* forward DFT unnormalised with ``exp(-i k.x)``; the inverse carries ``1/M``.
* real SCFT mode ("scft") stores the Wick-rotated real fields ``W+ = i*omega+`` and
  ``W- = omega-``, so ``wA = W+ - W-`` and ``wB = W+ + W-``; complex Langevin mode
  ("cl") stores complex ``omega+`` and ``omega-`` with ``wA = i*omega+ - omega-`` and
  ``wB = i*omega+ + omega-`` (mapping below Eq. 3).
* ``q`` starts at the A end, ``q_0 = 1``; ``qd`` (the conjugate propagator) starts at
  the B end, ``qd_0 = 1``; they pair as ``q(s) qd(1-s)`` in the densities of Eq. 8.
* contour quadrature: the trapezoid rule on each block, split at ``NsA``.  With this
  rule the densities are the exact gradient of the discrete ``ln Q`` (pinned in the
  tests), which is why it is the reading taken where Eq. 8 leaves the rule open.

Every function cites the passage of the paper it follows.
"""
from __future__ import annotations

import math
from contextlib import contextmanager
from dataclasses import dataclass

import numpy as np

SCFT_REAL = "scft"
CL_COMPLEX = "cl"

__all__ = [
    "SCFT_REAL", "CL_COMPLEX", "Solution", "wavenumbers", "k_squared", "n_A_steps",
    "species_fields", "boltzmann_factor", "diffusion_factor", "split_step",
    "forward_march", "backward_march", "quadrature_weights", "solve",
    "slice_partition_functions", "field_term", "hamiltonian", "mean_field_forces",
    "scft_euler_step", "cl_noise_std", "cl_euler_maruyama_step", "cl_noise",
    "dlnQ_dL", "dH_dL", "dH_dfields", "dft_matrix", "dft3_bruteforce",
    "dense_propagator_matrix", "forward_march_dense", "continuum_Q", "debye_g",
    "variable_cell_step", "rqm4_step", "simpson_weights", "SPLIT2", "RQM4",
    "debye_chain", "scft_sis_step", "cl_sis_step", "fft_workers", "EdwardsSolution", "edwards_field", "edwards_solve",
    "edwards_hamiltonian", "edwards_scft_step", "edwards_cl_step", "adjoint_field_gradient",
]

class _Transforms:
    """The n-dimensional DFT pair every transform of the oracle goes through."""

    def __init__(self, fftn, ifftn):
        self.fftn = fftn
        self.ifftn = ifftn


_FFT = _Transforms(np.fft.fftn, np.fft.ifftn)


@contextmanager
def fft_workers(workers: int):
    """Inside the block, the oracle's transforms run through ``scipy.fft`` on ``workers``
    threads instead of ``numpy.fft`` (one thread): the same DFT definition, for timing the
    oracle on every core of a host.  Nothing else changes."""
    import scipy.fft as sf
    global _FFT
    saved = _FFT
    _FFT = _Transforms(lambda x: sf.fftn(x, workers=workers), lambda x: sf.ifftn(x, workers=workers))
    try:
        yield
    finally:
        _FFT = saved


SPLIT2 = "split2"   # 2nd-order operator splitting, the A(ds) block of Eq. 13
RQM4 = "rqm4"       # Richardson-extrapolated 4th-order scheme of Eq. 13


# ----------------------------------------------------------------------------
# grid and chain
# ----------------------------------------------------------------------------
def wavenumbers(n: int, L: float) -> np.ndarray:
    """Plane-wave numbers k = 2*pi*m/L of a periodic axis (pseudo-spectral basis,
    Sec. "Algorithms", Eq. 13).  m is the signed FFT index; the Nyquist mode only
    enters through k^2, so its sign is immaterial."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    return 2.0 * np.pi * m / L


def k_squared(n, L) -> np.ndarray:
    """|k|^2 on the full [nx][ny][nz] spectrum."""
    kx, ky, kz = (wavenumbers(int(n[a]), float(L[a])) for a in range(3))
    return kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2


def n_A_steps(Ns: int, fA: float) -> int:
    """Number of contour steps on the A block: nearest integer to fA*Ns (Eq. 8 splits
    the contour at s = fA; on a grid of Ns steps the split lands on a step boundary)."""
    return int(math.floor(fA * Ns + 0.5))


def species_fields(wp, wm, kind: str):
    """Fields felt by A and B segments (mapping stated below Eq. 3)."""
    if kind == SCFT_REAL:
        return wp - wm, wp + wm
    if kind == CL_COMPLEX:
        return 1j * wp - wm, 1j * wp + wm
    raise ValueError(kind)


def boltzmann_factor(w, ds: float):
    """Half-step Boltzmann factor exp(-w ds/2) of the operator splitting (Eq. 13)."""
    return np.exp(-w * ds / 2.0)


def diffusion_factor(n, L, ds: float) -> np.ndarray:
    """Diffusion factor exp(-k^2 ds), the Fourier-space form of exp(laplacian ds) (Eq. 13)."""
    return np.exp(-k_squared(n, L) * ds)


# ----------------------------------------------------------------------------
# modified diffusion equation (Eq. 5) by 2nd-order operator splitting
# ----------------------------------------------------------------------------
def split_step(q, Bn, D):
    """One contour step q -> B * F^-1[ D * F[ B * q ] ]: the A(ds) block of Eq. 13,
    i.e. exp(-w ds/2) exp(laplacian ds) exp(-w ds/2) applied to q."""
    y = _FFT.ifftn(D * _FFT.fftn(Bn * q))
    if np.isrealobj(q) and np.isrealobj(Bn):
        y = y.real
    return Bn * y


def rqm4_step(q, w, D_full, D_half, ds):
    """One step of Eq. 13: q -> -(1/3)[A(ds) - 4 A(ds/2) A(ds/2)] q, where
    A(h) = exp(-w h/2) exp(laplacian h) exp(-w h/2) (cancels the ds^2 error of A)."""
    full = split_step(q, boltzmann_factor(w, ds), D_full)
    Bh = boltzmann_factor(w, ds / 2.0)
    half = split_step(split_step(q, Bh, D_half), Bh, D_half)
    return (4.0 * half - full) / 3.0


def simpson_weights(n0: int, n1: int, size: int) -> np.ndarray:
    """Composite Simpson weights (in units of ds) on slices n0..n1 of an array of length
    `size`: Simpson 1-4-2-4-1 over an even number of intervals; with an odd number (>= 3)
    the last three intervals take Simpson's 3/8 rule; one interval takes the trapezoid
    rule; none gives no weight.  Exact for cubics, so the contour integrals of Eq. 8 stay
    4th order alongside the scheme of Eq. 13."""
    c = np.zeros(size)
    m = n1 - n0
    if m <= 0:
        return c
    if m == 1:
        c[n0] += 0.5
        c[n1] += 0.5
        return c
    even = m if m % 2 == 0 else m - 3
    for k in range(0, even, 2):
        c[n0 + k] += 1.0 / 3.0
        c[n0 + k + 1] += 4.0 / 3.0
        c[n0 + k + 2] += 1.0 / 3.0
    if m % 2 == 1:
        a = n0 + even
        for j, wgt in enumerate((3.0 / 8.0, 9.0 / 8.0, 9.0 / 8.0, 3.0 / 8.0)):
            c[a + j] += wgt
    return c


def forward_march(BA, BB, D, Ns: int, NsA: int, q0=None) -> np.ndarray:
    """Propagator q(x, s) from the A end (Eq. 5, q(x, 0) = 1): q_n = T_n q_{n-1} with
    the A-block factor for n <= NsA and the B-block factor after.  Returns q_0..q_Ns."""
    dtype = np.result_type(BA, BB, np.float64)
    if q0 is not None:
        dtype = np.result_type(dtype, q0)
    q = np.empty((Ns + 1,) + BA.shape, dtype)
    q[0] = 1.0 if q0 is None else q0
    for n in range(1, Ns + 1):
        q[n] = split_step(q[n - 1], BA if n <= NsA else BB, D)
    return q


def backward_march(BA, BB, D, Ns: int, NsA: int, q0=None) -> np.ndarray:
    """Conjugate propagator qd from the B end (qd = 1 at the free B end, Eq. 5):
    qd_m = T_{Ns+1-m} qd_{m-1}, so the B-block factors come first.  Returns qd_0..qd_Ns."""
    dtype = np.result_type(BA, BB, np.float64)
    if q0 is not None:
        dtype = np.result_type(dtype, q0)
    qd = np.empty((Ns + 1,) + BA.shape, dtype)
    qd[0] = 1.0 if q0 is None else q0
    for m in range(1, Ns + 1):
        n = Ns + 1 - m
        qd[m] = split_step(qd[m - 1], BA if n <= NsA else BB, D)
    return qd


def quadrature_weights(Ns: int, NsA: int):
    """Trapezoid weights c_n (n = 0..Ns) of the contour integrals of Eq. 8 on each block:
    1/2 at both ends of a block, 1 inside, 0 outside; a block of zero length has none."""
    cA = np.zeros(Ns + 1)
    cB = np.zeros(Ns + 1)
    if NsA > 0:
        cA[0:NsA + 1] = 1.0
        cA[0] = cA[NsA] = 0.5
    if NsA < Ns:
        cB[NsA:Ns + 1] = 1.0
        cB[NsA] = cB[Ns] = 0.5
    return cA, cB


@dataclass
class Solution:
    Q: complex
    lnQ: complex
    phiA: np.ndarray
    phiB: np.ndarray
    q: np.ndarray
    qd: np.ndarray
    NsA: int
    BA: np.ndarray
    BB: np.ndarray
    D: np.ndarray


def _rqm4_march(wA, wB, n, L, Ns, NsA, q0, backward):
    ds = 1.0 / Ns
    Df = diffusion_factor(n, L, ds)
    Dh = diffusion_factor(n, L, ds / 2.0)
    dtype = np.result_type(wA, wB, np.float64)
    if q0 is not None:
        dtype = np.result_type(dtype, q0)
    q = np.empty((Ns + 1,) + wA.shape, dtype)
    q[0] = 1.0 if q0 is None else q0
    for m in range(1, Ns + 1):
        k = (Ns + 1 - m) if backward else m
        w = wA if k <= NsA else wB
        q[m] = rqm4_step(q[m - 1], w, Df, Dh, ds)
    return q


def solve(wp, wm, n, L, Ns: int, fA: float, kind: str, q0=None, qd0=None, scheme: str = SPLIT2) -> Solution:
    """Propagators, partition function and segment densities for fixed fields.

    Q = (1/V) int dx q(x, 1) (Eq. 4) and phi_A,B = (1/Q) int ds q(x,s) qd(x,1-s) over
    each block (Eq. 8, phi = rho/rho0).  scheme SPLIT2: the 2nd-order step A(ds) and the
    trapezoid rule per block; scheme RQM4: the 4th-order step of Eq. 13 and the
    composite Simpson rule per block."""
    ds = 1.0 / Ns
    NsA = n_A_steps(Ns, fA)
    wA, wB = species_fields(wp, wm, kind)
    BA, BB = boltzmann_factor(wA, ds), boltzmann_factor(wB, ds)
    D = diffusion_factor(n, L, ds)
    if scheme == SPLIT2:
        q = forward_march(BA, BB, D, Ns, NsA, q0)
        qd = backward_march(BA, BB, D, Ns, NsA, qd0)
        cA, cB = quadrature_weights(Ns, NsA)
    elif scheme == RQM4:
        q = _rqm4_march(wA, wB, n, L, Ns, NsA, q0, backward=False)
        qd = _rqm4_march(wA, wB, n, L, Ns, NsA, qd0, backward=True)
        cA, cB = simpson_weights(0, NsA, Ns + 1), simpson_weights(NsA, Ns, Ns + 1)
    else:
        raise ValueError(scheme)
    Q = q[Ns].mean()
    accA = np.zeros(q.shape[1:], np.result_type(q, qd))
    accB = np.zeros_like(accA)
    for k in range(Ns + 1):
        prod = q[k] * qd[Ns - k]
        if cA[k]:
            accA = accA + cA[k] * prod
        if cB[k]:
            accB = accB + cB[k] * prod
    phiA = ds * accA / Q
    phiB = ds * accB / Q
    lnQ = np.log(Q) if np.iscomplexobj(Q) else math.log(Q)
    return Solution(Q=Q, lnQ=lnQ, phiA=phiA, phiB=phiB, q=q, qd=qd, NsA=NsA, BA=BA, BB=BB, D=D)


def slice_partition_functions(sol: Solution) -> np.ndarray:
    """Q evaluated at every cut n of the chain: (1/M) sum_x q_n qd_{Ns-n}."""
    Ns = sol.q.shape[0] - 1
    return np.array([(sol.q[k] * sol.qd[Ns - k]).mean() for k in range(Ns + 1)])


# ----------------------------------------------------------------------------
# Hamiltonian (Eq. 3), forces (Eq. 7) and field updates (Eq. 9)
# ----------------------------------------------------------------------------
def field_term(wp, wm, chiN: float, kind: str):
    """Local integrand of Eq. 3: omega-^2/chiN - i omega+ (i omega+ = W+ in SCFT mode)."""
    if kind == SCFT_REAL:
        return wm * wm / chiN - wp
    return wm * wm / chiN - 1j * wp


def hamiltonian(wp, wm, lnQ, chiN: float, C: float, n, L, kind: str):
    """H = C int dx [omega-^2/chiN - i omega+] - C V lnQ (Eq. 3)."""
    M = int(np.prod(n))
    V = float(np.prod(L))
    dV = V / M
    return C * dV * field_term(wp, wm, chiN, kind).sum() - C * V * lnQ


def mean_field_forces(wp, wm, phiA, phiB, chiN: float, kind: str):
    """Functional derivatives of H per unit C (Eq. 7, phi = rho/rho0).

    SCFT mode returns dH/dW+ = phiA+phiB-1 and dH/dW- = 2W-/chiN + phiB - phiA;
    CL mode returns dH/domega+ = i(phiA+phiB-1) and dH/domega- likewise."""
    fm = 2.0 * wm / chiN + phiB - phiA
    fp = phiA + phiB - 1.0
    if kind == CL_COMPLEX:
        fp = 1j * fp
    return fp, fm


def scft_euler_step(wp, wm, phiA, phiB, chiN: float, lam: float):
    """Explicit Euler relaxation of Eq. 9 without noise, Wick-rotated: ascent on the
    pressure field W+ and descent on the exchange field W-, with the force per C."""
    fp, fm = mean_field_forces(wp, wm, phiA, phiB, chiN, SCFT_REAL)
    return wp + lam * fp, wm - lam * fm


def cl_noise_std(dt: float, C: float, dV: float, lam: float = 1.0) -> float:
    """Standard deviation of the discretised real Gaussian noise: variance
    2 lam dt / dV (stated below Eq. 10), with the force taken per C, i.e. 2 lam dt/(C dV)."""
    return math.sqrt(2.0 * lam * dt / (C * dV))


def cl_euler_maruyama_step(wp, wm, phiA, phiB, chiN: float, dt: float, eta_p, eta_m, lam: float = 1.0):
    """One Euler-Maruyama step of the complex Langevin equation of motion (Eq. 9) with
    real noise eta (already scaled to its standard deviation), force per C."""
    fp, fm = mean_field_forces(wp, wm, phiA, phiB, chiN, CL_COMPLEX)
    return wp - lam * dt * fp + eta_p, wm - lam * dt * fm + eta_m


def debye_chain(x):
    """Debye function of the whole chain (ideal homopolymer of the full contour length),
    g_D(x) = 2 (e^{-x} + x - 1) / x^2 at x = k^2 Rg^2, with g_D(0) = 1.  Below x = 0.1,
    where the closed form cancels, the Taylor series 2 sum_{m>=2} (-x)^(m-2) / m! through
    x^9 (truncation below 1e-16)."""
    x = np.asarray(x, dtype=float)
    small = x < 0.1
    xs = np.where(small, 1.0, x)
    g = 2.0 * (np.exp(-xs) + xs - 1.0) / xs ** 2
    ser = np.zeros_like(x)
    for m in range(11, 1, -1):  # Horner on the coefficients 2 (-1)^(m-2) / m!
        ser = ser * x + 2.0 * (-1.0) ** (m - 2) / math.factorial(m)
    return np.where(small, ser, g)


def scft_sis_step(wp, wm, phiA, phiB, chiN: float, lam: float, n, L):
    """Semi-implicit SCFT relaxation (Eq. 11 without noise, Wick-rotated).  W+: the
    linear density response to W+, -g_D(k) W+, is taken at the new time, which gives the
    wavevector-dependent step W+^ += lam F+^ / (1 + lam g_D(k)).  W-: the explicit linear
    term 2 W-/chiN is taken fully implicitly, the density difference explicitly:
    W- <- (W- - lam (phiB - phiA)) / (1 + 2 lam/chiN)."""
    fp = phiA + phiB - 1.0
    gD = debye_chain(k_squared(n, L))
    wp_new = wp + _FFT.ifftn(_FFT.fftn(lam * fp) / (1.0 + lam * gD)).real
    wm_new = (wm - lam * (phiB - phiA)) / (1.0 + 2.0 * lam / chiN)
    return wp_new, wm_new


def cl_sis_step(wp, wm, phiA, phiB, chiN: float, dt: float, eta_p, eta_m, n, L):
    """Semi-implicit complex Langevin step (Eq. 11 with lam = 1): the linear part of the
    omega+ force, g_D(k) omega+, at the new time, so the force and the noise are divided
    by 1 + dt g_D(k) in reciprocal space; the 2 omega-/chiN term fully implicit:
    omega- <- (omega- - dt (phiB - phiA) + eta-) / (1 + 2 dt/chiN)."""
    fp = 1j * (phiA + phiB - 1.0)
    gD = debye_chain(k_squared(n, L))
    wp_new = wp + _FFT.ifftn(_FFT.fftn(-dt * fp + eta_p) / (1.0 + dt * gD))
    wm_new = (wm - dt * (phiB - phiA) + eta_m) / (1.0 + 2.0 * dt / chiN)
    return wp_new, wm_new


def cl_noise(seed: int, instance: int, step: int, M: int, std: float):
    """Noise arrays (eta+, eta-) of one CL step from the counter-based generator."""
    from .philox import philox_normals
    eta_p = std * philox_normals(seed, instance, step, 0, M)
    eta_m = std * philox_normals(seed, instance, step, 1, M)
    return eta_p, eta_m


# ----------------------------------------------------------------------------
# Edwards model of homopolymers in implicit solvent (Eq. 2): one field omega entering
# Q as i omega; the chain is reversible, so q-dagger = q and half of the march is needed
# ----------------------------------------------------------------------------
@dataclass
class EdwardsSolution:
    Q: complex
    lnQ: complex
    phi: np.ndarray
    q: np.ndarray


def edwards_field(w, kind: str):
    """Field felt by every segment: W = i omega is stored directly in SCFT mode (Wick
    rotation of the pressure-like field), i omega in CL mode."""
    return w if kind == SCFT_REAL else 1j * w


def edwards_solve(w, n, L, Ns: int, kind: str, q0=None) -> EdwardsSolution:
    """q from Eqs. 5 and 13 with one field for the whole chain, Q (Eq. 4), and the
    segment density phi = (1/Q) int_0^1 ds q(s) q(1-s) (q-dagger = q for a homopolymer;
    trapezoid rule over the whole contour)."""
    ds = 1.0 / Ns
    B = boltzmann_factor(edwards_field(w, kind), ds)
    D = diffusion_factor(n, L, ds)
    q = forward_march(B, B, D, Ns, Ns, q0)
    Q = q[Ns].mean()
    c = np.ones(Ns + 1)
    c[0] = c[Ns] = 0.5
    acc = np.zeros(q.shape[1:], q.dtype)
    for k in range(Ns + 1):
        acc = acc + c[k] * q[k] * q[Ns - k]
    phi = ds * acc / Q
    lnQ = np.log(Q) if np.iscomplexobj(Q) else math.log(Q)
    return EdwardsSolution(Q=Q, lnQ=lnQ, phi=phi, q=q)


def edwards_hamiltonian(w, lnQ, B: float, C: float, n, L, kind: str):
    """H = (B/2) int dx omega^2 - C V lnQ (Eq. 2); in SCFT mode omega^2 = -W^2."""
    M = int(np.prod(n))
    V = float(np.prod(L))
    w2 = -w * w if kind == SCFT_REAL else w * w
    return 0.5 * B * (V / M) * w2.sum() - C * V * lnQ


def edwards_scft_step(W, phi, B: float, C: float, lam: float):
    """Relaxation of the Wick-rotated field towards the saddle W = (C/B) phi, ascent on
    the pressure-like field with the force per C: W += lam (phi - (B/C) W)."""
    return W + lam * (phi - (B / C) * W)


def edwards_cl_step(w, phi, B: float, C: float, dt: float, eta):
    """Euler-Maruyama complex Langevin step with the force per C,
    dH/domega / C = (B/C) omega + i phi, and real noise eta of variance 2 dt/(C dV)."""
    return w - dt * ((B / C) * w + 1j * phi) + eta


# ----------------------------------------------------------------------------
# exact gradients of the discrete H: fields and box lengths (stress)
# ----------------------------------------------------------------------------
def dH_dfields(wp, wm, sol: Solution, chiN: float, C: float, n, L, kind: str):
    """Gradient of the discrete H with respect to the grid values of the two stored
    fields: dV * C * (Eq. 7 forces).  In SCFT mode these are d/dW+ and d/dW-."""
    M = int(np.prod(n))
    dV = float(np.prod(L)) / M
    fp, fm = mean_field_forces(wp, wm, sol.phiA, sol.phiB, chiN, kind)
    return C * dV * fp, C * dV * fm


def adjoint_field_gradient(wp, wm, n, L, Ns: int, fA: float, GA, GB):
    """Gradient of a loss L(phiA, phiB) with respect to the real SCFT fields W+ and W-,
    through the discrete march (2nd-order steps, trapezoid quadrature), given
    GA = dL/dphiA and GB = dL/dphiB on the grid.

    Derivation (step by step, the order used below): with T_n = B_n K B_n, K the
    diffusion operator (real symmetric for real fields) and g_n = (ds/Q)(cA_n GA + cB_n GB),
      L_acc = sum_n <g_n, q_n qd_{Ns-n}>: the sources a_n = g_n qd_{Ns-n} of the q march
      are propagated backwards by lambda_Ns = a_Ns, lambda_{n-1} = T_n lambda_n + a_{n-1},
      and each step contributes -(ds/2) [lambda_n q_n + B_n q_{n-1} K(B_n lambda_n)] to
      dL/dw of its block; likewise the qd march with sources b_m = g_{Ns-m} q_{Ns-m};
      the normalisation by Q adds gamma phi / M with gamma = sum_x (GA phiA + GB phiB)
      (d lnQ / dw = -phi / M); then dL/dW+ = dL/dwA + dL/dwB, dL/dW- = dL/dwB - dL/dwA."""
    sol = solve(wp, wm, n, L, Ns, fA, SCFT_REAL)
    ds = 1.0 / Ns
    NsA = sol.NsA
    M = int(np.prod(n))
    q, qd, Q = sol.q, sol.qd, sol.Q
    cA, cB = quadrature_weights(Ns, NsA)
    D = sol.D

    def K(v):
        return _FFT.ifftn(D * _FFT.fftn(v)).real

    def g(k):
        return (ds / Q) * (cA[k] * GA + cB[k] * GB)

    dwA = np.zeros(q.shape[1:])
    dwB = np.zeros(q.shape[1:])
    # adjoint of the forward march
    lam = g(Ns) * qd[0]
    for k in range(Ns, 0, -1):
        Bk = sol.BA if k <= NsA else sol.BB
        z = K(Bk * lam)
        term = -0.5 * ds * (lam * q[k] + Bk * q[k - 1] * z)
        if k <= NsA:
            dwA += term
        else:
            dwB += term
        lam = Bk * z + g(k - 1) * qd[Ns - k + 1]
    # adjoint of the conjugate march (step m uses the factor of split step Ns + 1 - m)
    mu = g(0) * q[0]
    for m in range(Ns, 0, -1):
        nb = Ns + 1 - m
        Bm = sol.BA if nb <= NsA else sol.BB
        z = K(Bm * mu)
        term = -0.5 * ds * (mu * qd[m] + Bm * qd[m - 1] * z)
        if nb <= NsA:
            dwA += term
        else:
            dwB += term
        mu = Bm * z + g(Ns - m + 1) * q[Ns - m + 1]
    gamma = float(np.sum(GA * sol.phiA + GB * sol.phiB))
    dwA += gamma * sol.phiA / M
    dwB += gamma * sol.phiB / M
    return dwA + dwB, dwB - dwA


def dlnQ_dL(sol: Solution, n, L):
    """d lnQ / dL_a with the fields held fixed on the grid.

    Only the diffusion factor depends on the box: dD/dL_a = D * 2 ds k_a^2 / L_a, so
    differentiating Q = (1/M) 1^T T_Ns ... T_1 1 slice by slice gives
    dQ/dL_a = (1/M) sum_n u_n . F^-1[(2 ds k_a^2/L_a) D F v_n] with v_n = B_n q_{n-1}
    and u_n = B_n qd_{Ns-n} (each split step is a symmetric operator).  The paper leaves
    stress out of scope; this is the derivative of its discrete Q (Eqs. 4, 13)."""
    Ns = sol.q.shape[0] - 1
    ds = 1.0 / Ns
    M = int(np.prod(n))
    out = np.zeros(3, dtype=np.result_type(sol.q, sol.qd, np.float64))
    ks = [wavenumbers(int(n[a]), float(L[a])) for a in range(3)]
    shapes = [(-1, 1, 1), (1, -1, 1), (1, 1, -1)]
    for a in range(3):
        g = (2.0 * ds * ks[a] ** 2 / float(L[a])).reshape(shapes[a]) * sol.D
        tot = 0.0
        for k in range(1, Ns + 1):
            Bn = sol.BA if k <= sol.NsA else sol.BB
            v = Bn * sol.q[k - 1]
            u = Bn * sol.qd[Ns - k]
            w = _FFT.ifftn(g * _FFT.fftn(v))
            if np.isrealobj(v):
                w = w.real
            tot = tot + (u * w).sum()
        out[a] = tot / (sol.Q * M)
    return out


def dH_dL(H, sol: Solution, C: float, n, L):
    """dH/dL_a = H/L_a - C V dlnQ/dL_a (fields fixed on the grid; from Eq. 3)."""
    V = float(np.prod(L))
    g = dlnQ_dL(sol, n, L)
    return np.array([H / float(L[a]) for a in range(3)]) - C * V * g


def variable_cell_step(L, sol: Solution, n, lam_L: float):
    """Cell relaxation on the intensive h = H/(C V): dh/dL_a = -dlnQ/dL_a, so
    L_a <- L_a - lam_L dh/dL_a."""
    g = np.real(dlnQ_dL(sol, n, L))
    return np.array([float(L[a]) + lam_L * g[a] for a in range(3)])


# ----------------------------------------------------------------------------
# brute force and continuum references (for pinning the oracle itself)
# ----------------------------------------------------------------------------
def dft_matrix(n: int) -> np.ndarray:
    """Unnormalised forward DFT matrix exp(-2 pi i j k / n), written out entry by entry."""
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


def dft3_bruteforce(x) -> np.ndarray:
    """O(M^2) 3D DFT: the dense Kronecker product of the three 1D DFT matrices."""
    nx, ny, nz = x.shape
    F = np.kron(dft_matrix(nx), np.kron(dft_matrix(ny), dft_matrix(nz)))
    return (F @ x.reshape(-1)).reshape(x.shape)


def dense_propagator_matrix(n, D) -> np.ndarray:
    """The diffusion operator F^-1 diag(D) F as an explicit M x M matrix."""
    F = np.kron(dft_matrix(int(n[0])), np.kron(dft_matrix(int(n[1])), dft_matrix(int(n[2]))))
    M = F.shape[0]
    return (F.conj().T / M) @ (D.reshape(-1)[:, None] * F)


def forward_march_dense(BA, BB, Dmat, Ns: int, NsA: int) -> np.ndarray:
    """Forward march with the diffusion factor applied as a dense matrix product."""
    shape = BA.shape
    q = np.ones(BA.size, dtype=np.result_type(BA, BB, Dmat))
    for k in range(1, Ns + 1):
        Bn = (BA if k <= NsA else BB).reshape(-1)
        q = Bn * (Dmat @ (Bn * q))
    return q.reshape(shape)


def continuum_Q(wA, wB, n, L, fA_eff: float) -> complex:
    """Exact-in-s partition function of Eqs. 4-5 on the spatial grid:
    Q* = (1/M) 1^T expm(fB (Lap - WB)) expm(fA (Lap - WA)) 1, with Lap the spectral
    Laplacian F^-1 diag(-k^2) F written as a dense matrix."""
    from scipy.linalg import expm
    F = np.kron(dft_matrix(int(n[0])), np.kron(dft_matrix(int(n[1])), dft_matrix(int(n[2]))))
    M = F.shape[0]
    lap = (F.conj().T / M) @ (-k_squared(n, L).reshape(-1)[:, None] * F)
    if np.isrealobj(wA) and np.isrealobj(wB):
        lap = lap.real
    one = np.ones(M)
    qa = expm(fA_eff * (lap - np.diag(wA.reshape(-1)))) @ one
    q1 = expm((1.0 - fA_eff) * (lap - np.diag(wB.reshape(-1)))) @ qa
    return q1.mean()


def debye_g(x: float, f: float):
    """Ideal diblock correlation functions (weak-inhomogeneity linear response, the
    Debye functions mentioned under Eq. 10) at x = k^2 Rg^2:
    g_AA = 2[f x + e^{-f x} - 1]/x^2, g_BB the same with 1-f,
    g_AB = (1 - e^{-f x})(1 - e^{-(1-f) x})/x^2."""
    gAA = 2.0 * (f * x + math.exp(-f * x) - 1.0) / x ** 2
    gBB = 2.0 * ((1 - f) * x + math.exp(-(1 - f) * x) - 1.0) / x ** 2
    gAB = (1.0 - math.exp(-f * x)) * (1.0 - math.exp(-(1 - f) * x)) / x ** 2
    return gAA, gBB, gAB
