"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle.

Tolerances (GPU vs oracle on the same seeded inputs):
  FP64 path      : relative 1e-12 on Q and H, 1e-10 max-abs on phi, 1e-12 relative
                   (to the slice maximum) on propagator slices and fields.
  FP32-mixed path: FP32 propagators and FFTs with FP64 quadrature/reductions; the
                   error is dominated by float rounding in ~2*Ns FFT round trips:
                   relative 2e-5 on Q, absolute 2e-5 on phi, and absolute 2e-5 on the
                   intensive h = H/(C V) (= field average - lnQ; H itself is a small
                   difference of two large terms, so its relative error is not a
                   property of the propagator).  Derived bound: unit roundoff 6e-8 x
                   log2(M) ~ 21 per transform, growing like a random walk over 2 Ns
                   <= 200 steps -> ~2e-5.  Measured errors are printed by the tests.
"""
import math

import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft
from paper_1204_5434_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64, FP32 = pft.PFT_FP64, pft.PFT_FP32_MIXED
SCFT, CL = pft.PFT_SCFT_REAL, pft.PFT_CL_COMPLEX
OKIND = {SCFT: o.SCFT_REAL, CL: o.CL_COMPLEX}
TOL = {FP64: dict(Q=1e-12, H=1e-12, phi=1e-10, q=1e-12), FP32: dict(Q=2e-5, h=2e-5, phi=2e-5, q=2e-5)}


def _check_H(H, Href, C, L, prec):
    """FP64: relative 1e-12 on H; FP32-mixed: absolute 2e-5 on h = H/(C V)."""
    if prec == FP64:
        return _rel(H, Href) <= TOL[FP64]["H"]
    return abs(H - Href) / (C * float(np.prod(L))) <= TOL[FP32]["h"]


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


def _rel(a, b):
    return abs(a - b) / abs(b)


# ------------------------------------------------------------------------ FFT
FFT_SHAPES = [(8, 12, 16), (48, 32, 24), (6, 4, 96), (128, 4, 8), (4, 256, 4), (192, 6, 4), (64, 64, 64), (12, 12, 12)]


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-13), (FP32, 3e-6)])
@pytest.mark.parametrize("shape", FFT_SHAPES)
def test_fft3d_matches_numpy(prec, tol, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    with pft.System(shape, (1, 1, 1), 4, 0.5, 10.0, 1.0, CL, prec) as s:
        y = s.fft3d(x)
        ref = np.fft.fftn(x)
        assert np.max(np.abs(y - ref)) <= tol * np.max(np.abs(ref))
        z = s.fft3d(x, inverse=True)
        ref = np.fft.ifftn(x) * x.size
        assert np.max(np.abs(z - ref)) <= tol * np.max(np.abs(ref))


def test_fft3d_matches_bruteforce_dft_8cubed():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(8, 8, 8)) + 1j * rng.normal(size=(8, 8, 8))
    with pft.System((8, 8, 8), (1, 1, 1), 4, 0.5, 10.0, 1.0, CL, FP64) as s:
        y = s.fft3d(x)
    ref = o.dft3_bruteforce(x)
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))


# ------------------------------------------------------------------ one solve
SOLVE_CASES = [
    ((16, 12, 8), (4.0, 3.0, 2.0), 20, 0.35),
    ((12, 12, 12), (3.0, 3.0, 3.0), 13, 0.5),     # ragged column and pencil tiles
    ((8, 6, 24), (2.0, 1.5, 6.0), 8, 0.25),
    ((48, 4, 6), (6.0, 1.0, 1.5), 10, 0.6),       # radix-3 lengths on x and z
    ((32, 32, 32), (4.0, 4.0, 4.0), 16, 0.5),
]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("kind", [SCFT, CL])
@pytest.mark.parametrize("case", SOLVE_CASES)
def test_solve_matches_oracle(case, kind, prec):
    n, L, Ns, fA = case
    chiN, C = 17.0, 3.0
    wp, wm = _fields(n, kind, 7 + Ns)
    ref = o.solve(wp, wm, n, L, Ns, fA, OKIND[kind])
    with pft.System(n, L, Ns, fA, chiN, C, kind, prec) as s:
        s.set_fields(wp, wm)
        s.solve()
        obs = s.observables()
        phiA, phiB = s.densities()
        t = TOL[prec]
        Q = obs["Q"] if kind == CL else obs["Q"].real
        H = obs["H"] if kind == CL else obs["H"].real
        Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, OKIND[kind])
        eQ, eH = _rel(Q, ref.Q), _rel(H, Href)
        ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
        print(f"\nsolve {n} Ns={Ns} kind={kind} prec={prec}: Q rel {eQ:.2e}  H rel {eH:.2e}  phi abs {ephi:.2e}")
        assert eQ <= t["Q"], (Q, ref.Q)
        assert _check_H(H, Href, C, L, prec), (H, Href)
        assert ephi <= t["phi"]
        assert abs(obs["fA_eff"] - ref.NsA / Ns) == 0
        NsA = ref.NsA
        for k in sorted({0, 1, NsA, Ns}):
            q = s.propagator(0, k)
            assert np.max(np.abs(q - ref.q[k])) <= t["q"] * np.max(np.abs(ref.q[k])), k
        qd = s.propagator(1, 0)
        assert np.max(np.abs(qd - ref.qd[Ns])) <= t["q"] * np.max(np.abs(ref.qd[Ns]))


@pytest.mark.parametrize("kind", [SCFT, CL])
@pytest.mark.parametrize("Ns,fA", [(1, 0.5), (6, 0.0), (6, 1.0), (7, 0.93)])
def test_solve_degenerate_chains(kind, Ns, fA):
    """Ns = 1 and pure A or pure B chains (a block of zero length has no quadrature)."""
    n, L = (8, 8, 8), (3.0, 3.0, 3.0)
    wp, wm = _fields(n, kind, 3)
    ref = o.solve(wp, wm, n, L, Ns, fA, OKIND[kind])
    with pft.System(n, L, Ns, fA, 12.0, 1.0, kind, FP64) as s:
        s.set_fields(wp, wm)
        s.solve()
        obs = s.observables()
        phiA, phiB = s.densities()
    Q = obs["Q"] if kind == CL else obs["Q"].real
    assert _rel(Q, ref.Q) <= 1e-12
    assert np.max(np.abs(phiA - ref.phiA)) <= 1e-10 and np.max(np.abs(phiB - ref.phiB)) <= 1e-10


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_uniform_fields_closed_form(prec):
    n, L, Ns, fA = (8, 12, 16), (2.0, 3.0, 4.0), 20, 0.35
    fa = o.n_A_steps(Ns, fA) / Ns
    with pft.System(n, L, Ns, fA, 15.0, 1.0, SCFT, prec) as s:
        s.set_fields(np.full(n, 0.7), np.full(n, -1.3))
        s.solve()
        obs = s.observables()
        phiA, _ = s.densities()
    Qx = math.exp(-(fa * 2.0 + (1 - fa) * (-0.6)))
    # FP32: each step multiplies the k=0 mode by float(1/M); with M = 1536 not a power
    # of two that rounding (<= 6e-8) repeats in all 2*Ns steps: 40 * 6e-8 = 2.4e-6.
    tol = 1e-13 if prec == FP64 else 2 * 20 * 2 * 6e-8
    assert _rel(obs["Q"].real, Qx) <= tol
    assert np.max(np.abs(phiA - fa)) <= (1e-13 if prec == FP64 else 1e-6)


def test_diffusion_alone_real_and_complex():
    """w = 0, q_0 a Laplacian eigenmode: q_Ns = exp(-k^2) q_0 (Eq. 5)."""
    n, L, Ns = (16, 8, 12), (4.0, 2.0, 3.0), 10
    x = [np.arange(n[a]) * L[a] / n[a] for a in range(3)]
    m = (1, -2, 1)
    k = [2 * np.pi * m[a] / L[a] for a in range(3)]
    ph = k[0] * x[0][:, None, None] + k[1] * x[1][None, :, None] + k[2] * x[2][None, None, :]
    k2 = sum(v * v for v in k)
    zero = np.zeros(n)
    with pft.System(n, L, Ns, 0.5, 10.0, 1.0, SCFT, FP64) as s:
        s.set_fields(zero, zero)
        pft.pft_debug_set_q0(s.h, np.ascontiguousarray(np.cos(ph)))
        s.solve()
        q = s.propagator(0, Ns)
    assert np.max(np.abs(q - math.exp(-k2) * np.cos(ph))) < 1e-13
    with pft.System(n, L, Ns, 0.5, 10.0, 1.0, CL, FP64) as s:
        s.set_fields(zero.astype(complex), zero.astype(complex))
        pft.pft_debug_set_q0(s.h, np.ascontiguousarray(np.exp(1j * ph)))
        s.solve()
        q = s.propagator(0, Ns)
    assert np.max(np.abs(q - math.exp(-k2) * np.exp(1j * ph))) < 1e-13


def test_graph_and_eager_paths_agree():
    n, L = (16, 16, 16), (4.0, 4.0, 4.0)
    wp, wm = _fields(n, SCFT, 11)
    res = []
    for g in (True, False):
        with pft.System(n, L, 24, 0.4, 15.0, 1.0, SCFT, FP64, use_graph=g) as s:
            s.set_fields(wp, wm)
            s.solve()
            s.solve()
            res.append((s.observables()["Q"], s.densities()[0]))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


# ---------------------------------------------------------------- field steps
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_scft_relaxation_matches_oracle(prec):
    n, L, Ns, fA, chiN, lam = (16, 12, 8), (4.0, 3.0, 2.0), 16, 0.4, 15.0, 0.1
    wp, wm = _fields(n, SCFT, 21)
    with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, prec) as s:
        s.set_fields(wp, wm)
        for it in range(4):
            s.solve()
            obs = s.observables()
            ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
            Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, 1.0, n, L, o.SCFT_REAL)
            assert _check_H(obs["H"].real, Href, 1.0, L, prec)
            s.field_step(lam)
            wp, wm = o.scft_euler_step(wp, wm, ref.phiA, ref.phiB, chiN, lam)
            gp, gm = s.get_fields()
            tol = 1e-12 if prec == FP64 else 1e-5
            assert np.max(np.abs(gp - wp)) <= tol and np.max(np.abs(gm - wm)) <= tol * 10


def test_cl_steps_with_supplied_noise_match_oracle():
    n, L, Ns, fA, chiN, C, dt = (16, 8, 12), (4.0, 2.0, 3.0), 12, 0.3, 20.0, 50.0, 0.01
    wp, wm = _fields(n, CL, 22, 0.05, 0.2)
    wm = wm + chiN * (2 * fA - 1) / 2
    dV = np.prod(L) / np.prod(n)
    std = o.cl_noise_std(dt, C, dV)
    rng = np.random.default_rng(5)
    with pft.System(n, L, Ns, fA, chiN, C, CL, FP64) as s:
        s.set_fields(wp, wm)
        for it in range(3):
            s.solve()
            ref = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
            obs = s.observables()
            Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, o.CL_COMPLEX)
            assert _rel(obs["H"], Href) <= 1e-12
            ep = std * rng.normal(size=n)
            em = std * rng.normal(size=n)
            s.field_step(dt, ep, em)
            wp, wm = o.cl_euler_maruyama_step(wp, wm, ref.phiA, ref.phiB, chiN, dt, ep, em)
            gp, gm = s.get_fields()
            assert np.max(np.abs(gp - wp)) <= 1e-10 and np.max(np.abs(gm - wm)) <= 1e-10


def test_cl_step_with_device_philox_matches_oracle_generator():
    n, L, Ns, fA, chiN, C, dt = (8, 8, 16), (2.0, 2.0, 4.0), 10, 0.3, 20.0, 50.0, 0.01
    wp, wm = _fields(n, CL, 23, 0.05, 0.2)
    seed, inst = 0x1234_5678_9ABC, 3
    dV = np.prod(L) / np.prod(n)
    std = o.cl_noise_std(dt, C, dV)
    with pft.System(n, L, Ns, fA, chiN, C, CL, FP64, seed=seed, instance=inst) as s:
        s.set_fields(wp, wm)
        for step in range(2):
            s.solve()
            ref = o.solve(wp, wm, n, L, Ns, fA, o.CL_COMPLEX)
            s.field_step(dt)
            ep, em = o.cl_noise(seed, inst, step, wp.size, std)
            wp, wm = o.cl_euler_maruyama_step(wp, wm, ref.phiA, ref.phiB, chiN, dt, ep.reshape(n), em.reshape(n))
            gp, gm = s.get_fields()
            assert np.max(np.abs(gp - wp)) <= 1e-10 and np.max(np.abs(gm - wm)) <= 1e-10


# ---------------------------------------------------------------- generator
def test_device_philox_bits_match_oracle():
    torch = pytest.importorskip("torch")
    count = 1 << 20
    ctr = (7, 0xDEADBEEF, 3, 0xFFFFFFFF)
    key = (0x243F6A88, 0x85A308D3)
    out = torch.empty(4 * count, dtype=torch.int32, device="cuda")
    pft.pft_philox_raw(ctr, key, count, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(count, 4)
    c = np.zeros((count, 4), dtype=np.uint64)
    c[:, 0] = (np.arange(count, dtype=np.uint64) + ctr[0]) & 0xFFFFFFFF
    c[:, 1], c[:, 2], c[:, 3] = ctr[1], ctr[2], ctr[3]
    ref = o.philox4x32_10(c, key)
    assert np.array_equal(got, ref)


def test_device_philox_normals_match_oracle():
    torch = pytest.importorskip("torch")
    M = 100003
    out = torch.empty(M, dtype=torch.float64, device="cuda")
    pft.pft_philox_normals(99, 2, 17, 1, M, out)
    torch.cuda.synchronize()
    ref = o.philox_normals(99, 2, 17, 1, M)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-13


# ---------------------------------------------------- the paper's workloads
def test_lamellar_scft_32cubed_50_steps():
    """32^3, L=4, Ns=64, fA=0.5, chiN=15: one solve then 50 Euler steps (lambda=0.1)."""
    w = wl.LAM32
    wp, wm = wl.fields(w)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, FP64) as s:
        s.set_fields(wp, wm)
        for it in range(w.steps):
            s.solve()
            ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
            s.field_step(w.lam)
            wp, wm = o.scft_euler_step(wp, wm, ref.phiA, ref.phiB, w.chiN, w.lam)
        s.solve()
        obs = s.observables()
        gp, gm = s.get_fields()
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    Href = o.hamiltonian(wp, wm, ref.lnQ, w.chiN, w.C, w.n, w.L, o.SCFT_REAL)
    assert np.max(np.abs(gm - wm)) <= 1e-9 and np.max(np.abs(gp - wp)) <= 1e-9
    assert _rel(obs["H"].real, Href) <= 1e-11


def test_lamellar_scft_32cubed_50_steps_fp32_error_table():
    """The same 50-step trajectory in FP32-mixed against the FP64 oracle trajectory: the
    error per quantity after 50 updates (printed; bounds from the one-solve tolerance 2e-5
    carried through 50 relaxation steps of lambda = 0.1, which contract the field error)."""
    w = wl.LAM32
    wp, wm = wl.fields(w)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, FP32) as s:
        s.set_fields(wp, wm)
        for it in range(w.steps):
            s.solve()
            ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
            s.field_step(w.lam)
            wp, wm = o.scft_euler_step(wp, wm, ref.phiA, ref.phiB, w.chiN, w.lam)
        s.solve()
        obs = s.observables()
        phiA, phiB = s.densities()
        gp, gm = s.get_fields()
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    Href = o.hamiltonian(wp, wm, ref.lnQ, w.chiN, w.C, w.n, w.L, o.SCFT_REAL)
    V = float(np.prod(w.L))
    err = {"Q rel": _rel(obs["Q"].real, ref.Q), "lnQ abs": abs(obs["lnQ"].real - ref.lnQ),
           "h abs": abs(obs["H"].real - Href) / (w.C * V),
           "phi abs": max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB))),
           "W+ abs": np.max(np.abs(gp - wp)), "W- abs": np.max(np.abs(gm - wm))}
    print("\nFP32-mixed after 50 SCFT steps: " + ", ".join(f"{k} {v:.2e}" for k, v in err.items()))
    assert err["Q rel"] <= 1e-4 and err["lnQ abs"] <= 1e-4 and err["h abs"] <= 1e-4
    assert err["phi abs"] <= 1e-4 and err["W+ abs"] <= 1e-4 and err["W- abs"] <= 1e-4


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_gyroid_128cubed_full_size(prec):
    """The 128^3 gyroid-seeded SCFT workload (Ns=100, fA=0.35, chiN=18) at full size:
    Q, H and phi sampled at 4096 random points against the oracle."""
    w = wl.GYR128
    wp, wm = wl.fields(w)
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    Href = o.hamiltonian(wp, wm, ref.lnQ, w.chiN, w.C, w.n, w.L, o.SCFT_REAL)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, prec) as s:
        s.set_fields(wp, wm)
        s.solve()
        obs = s.observables()
        phiA, phiB = s.densities()
    idx = np.random.default_rng(0).choice(phiA.size, 4096, replace=False)
    t = TOL[prec]
    eQ, eH = _rel(obs["Q"].real, ref.Q), _rel(obs["H"].real, Href)
    ephi = max(np.max(np.abs(phiA.ravel()[idx] - ref.phiA.ravel()[idx])),
               np.max(np.abs(phiB.ravel()[idx] - ref.phiB.ravel()[idx])))
    print(f"\n128^3 prec={prec}: Q rel {eQ:.2e} H rel {eH:.2e} phi abs {ephi:.2e}")
    assert eQ <= t["Q"] and _check_H(obs["H"].real, Href, w.C, w.L, prec) and ephi <= t["phi"]
    assert abs(phiA.mean() - ref.NsA / w.Ns) <= (1e-12 if prec == FP64 else 1e-6)


# ------------------------------------------------------------ resident march
def _gyroid_like(n, L, seed):
    x = [np.arange(n[a]) * L[a] / n[a] for a in range(3)]
    X = (2 * np.pi * x[0] / L[0])[:, None, None]
    Y = (2 * np.pi * x[1] / L[1])[None, :, None]
    Z = (2 * np.pi * x[2] / L[2])[None, None, :]
    G = np.sin(X) * np.cos(Y) + np.sin(Y) * np.cos(Z) + np.sin(Z) * np.cos(X)
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.1, n), 4.0 * G + rng.normal(0, 0.1, n)


@pytest.mark.parametrize("nn", [64, 96, 128])
def test_resident_march_matches_oracle_and_passes(nn):
    """The persistent resident march (FP32) against the oracle and the pass-kernel path."""
    n, L, Ns, fA, chiN = (nn, nn, nn), (8.0, 8.0, 8.0), 20, 0.35, 18.0
    wp, wm = _gyroid_like(n, L, nn)
    ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, 1.0, n, L, o.SCFT_REAL)
    out = {}
    for march in (pft.PFT_MARCH_RESIDENT, pft.PFT_MARCH_PASSES):
        with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, FP32, march=march) as s:
            assert pft.pft_get_march(s.h) == (2 if march == pft.PFT_MARCH_RESIDENT else 1)
            s.set_fields(wp, wm)
            s.solve()
            s.solve()
            obs = s.observables()
            phiA, phiB = s.densities()
            q = s.propagator(0, Ns)
            qd = s.propagator(1, 0)
        eQ = _rel(obs["Q"].real, ref.Q)
        ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
        print(f"\nresident={march} {nn}^3: Q rel {eQ:.2e} phi abs {ephi:.2e}")
        assert eQ <= TOL[FP32]["Q"] and ephi <= TOL[FP32]["phi"]
        assert _check_H(obs["H"].real, Href, 1.0, L, FP32)
        assert np.max(np.abs(q - ref.q[Ns])) <= TOL[FP32]["q"] * np.max(np.abs(ref.q[Ns]))
        assert np.max(np.abs(qd - ref.qd[Ns])) <= TOL[FP32]["q"] * np.max(np.abs(ref.qd[Ns]))
        out[march] = (phiA, obs["Q"].real)
    a, b = out[pft.PFT_MARCH_RESIDENT], out[pft.PFT_MARCH_PASSES]
    assert abs(a[1] - b[1]) <= 1e-5 * abs(b[1]) and np.max(np.abs(a[0] - b[0])) <= 1e-5


def test_resident_march_refuses_unsupported_configs():
    with pytest.raises(pft.PftError) as e:
        pft.System((32, 32, 32), (4, 4, 4), 10, 0.5, 15.0, 1.0, SCFT, FP32, march=pft.PFT_MARCH_RESIDENT)
    assert e.value.status == pft.PFT_ERR_UNSUPPORTED
    with pytest.raises(pft.PftError) as e:
        pft.System((64, 64, 64), (4, 4, 4), 10, 0.5, 15.0, 1.0, SCFT, FP64, march=pft.PFT_MARCH_RESIDENT)
    assert e.value.status == pft.PFT_ERR_UNSUPPORTED


def test_resident_barrier_timeout_is_reported_and_recoverable():
    """A barrier wait budget of one cycle makes the grid barriers give up: the march
    returns early, the host sees PFT_ERR_TIMEOUT, and the context still works."""
    n, L, Ns, fA = (64, 64, 64), (8.0, 8.0, 8.0), 8, 0.35
    wp, wm = _gyroid_like(n, L, 5)
    with pft.System(n, L, Ns, fA, 18.0, 1.0, SCFT, FP32, march=pft.PFT_MARCH_RESIDENT) as s:
        s.set_fields(wp, wm)
        pft.pft_debug_set_spin_limit(s.h, 1)
        s.solve()
        with pytest.raises(pft.PftError) as e:
            s.observables()
        assert e.value.status == pft.PFT_ERR_TIMEOUT
        pft.pft_debug_set_spin_limit(s.h, 4_000_000_000)
        s.solve()
        obs = s.observables()
    ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    assert _rel(obs["Q"].real, ref.Q) <= TOL[FP32]["Q"]


# ---------------------------------------------------------- persistent march
@pytest.mark.parametrize("nn,Ns", [(64, 20), (128, 20), (256, 4)])
def test_persistent_march_matches_oracle(nn, Ns):
    """The persistent multi-pass march (FP32, one cooperative launch per march) against
    the oracle and against the pass-kernel path."""
    n, L, fA, chiN = (nn, nn, nn), (8.0, 8.0, 8.0), 0.35, 18.0
    wp, wm = _gyroid_like(n, L, nn + 1)
    ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, 1.0, n, L, o.SCFT_REAL)
    out = {}
    for march in (pft.PFT_MARCH_PERSISTENT, pft.PFT_MARCH_PASSES):
        with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, FP32, march=march) as s:
            s.set_fields(wp, wm)
            s.solve()
            s.solve()
            obs = s.observables()
            phiA, phiB = s.densities()
            q = s.propagator(0, Ns)
            qd = s.propagator(1, 0)
        eQ = _rel(obs["Q"].real, ref.Q)
        ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
        print(f"\npersistent={march} {nn}^3: Q rel {eQ:.2e} phi abs {ephi:.2e}")
        assert eQ <= TOL[FP32]["Q"] and ephi <= TOL[FP32]["phi"]
        assert _check_H(obs["H"].real, Href, 1.0, L, FP32)
        assert np.max(np.abs(q - ref.q[Ns])) <= TOL[FP32]["q"] * np.max(np.abs(ref.q[Ns]))
        assert np.max(np.abs(qd - ref.qd[Ns])) <= TOL[FP32]["q"] * np.max(np.abs(ref.qd[Ns]))
        out[march] = (phiA, obs["Q"].real)
    a, b = out[pft.PFT_MARCH_PERSISTENT], out[pft.PFT_MARCH_PASSES]
    assert abs(a[1] - b[1]) <= 1e-5 * abs(b[1]) and np.max(np.abs(a[0] - b[0])) <= 1e-5


def test_persistent_barrier_timeout_is_reported_and_recoverable():
    n, L, Ns, fA = (64, 64, 64), (8.0, 8.0, 8.0), 8, 0.35
    wp, wm = _gyroid_like(n, L, 6)
    with pft.System(n, L, Ns, fA, 18.0, 1.0, SCFT, FP32, march=pft.PFT_MARCH_PERSISTENT) as s:
        s.set_fields(wp, wm)
        pft.pft_debug_set_spin_limit(s.h, 1)
        s.solve()
        with pytest.raises(pft.PftError) as e:
            s.observables()
        assert e.value.status == pft.PFT_ERR_TIMEOUT
        pft.pft_debug_set_spin_limit(s.h, 4_000_000_000)
        s.solve()
        obs = s.observables()
    ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    assert _rel(obs["Q"].real, ref.Q) <= TOL[FP32]["Q"]
