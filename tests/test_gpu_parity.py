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
@pytest.mark.parametrize("plan", [None, 4])
def test_lamellar_scft_32cubed_50_steps(plan):
    """32^3, L=4, Ns=64, fA=0.5, chiN=15: one solve then 50 Euler steps (lambda=0.1); the
    default FP64 plan and the double-float march (plan 4)."""
    w = wl.LAM32
    wp, wm = wl.fields(w)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, FP64) as s:
        if plan is not None:
            pft.pft_set_plan(s.h, plan, 1)
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
    """The 128^3 gyroid-seeded SCFT workload (Ns=100, fA=0.35, chiN=18) at full size, in
    the plan the bench times (FP32: the separable march, two chains) and, in FP32, also in
    the plane-kernel plan: Q and H, phiA and phiB over every one of the 2,097,152 points,
    and the propagator slices q_1, q_NsA, q_Ns and qd_1, qd_(Ns-NsA), qd_Ns element by
    element against the oracle (a fault confined to one kz column or one x-plane of a
    transform touches every slice after it).
    FP32 slices: the maximum over all 2,097,152 points of the error relative to the slice
    maximum, bounded by 1e-4 -- the per-point random-walk estimate of the derivation above
    (1.8e-5 after 2 Ns = 200 transforms of log2(M) = 21 stages) times the tail factor
    sqrt(2 ln M) = 5.4 of the largest of M such errors."""
    w = wl.GYR128
    wp, wm = wl.fields(w)
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    Href = o.hamiltonian(wp, wm, ref.lnQ, w.chiN, w.C, w.n, w.L, o.SCFT_REAL)
    NsA, Ns = ref.NsA, w.Ns
    t = TOL[prec]
    for plan in ((None,) if prec == FP64 else (None, (1, 1))):
        with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, prec) as s:
            if plan is not None:
                pft.pft_set_plan(s.h, *plan)
            elif prec == FP32:
                assert pft.pft_get_plan(s.h) == (2, 1)
            assert pft.pft_get_checkpoint(s.h) == 1
            s.set_fields(wp, wm)
            s.solve()
            obs = s.observables()
            phiA, phiB = s.densities()
            eq = 0.0
            for which, hist in ((0, ref.q), (2, ref.qd)):
                for k in sorted({1, NsA if which == 0 else Ns - NsA, Ns}):
                    g = s.propagator(which, k)
                    e = np.max(np.abs(g - hist[k])) / np.max(np.abs(hist[k]))
                    eq = max(eq, e)
                    assert e <= (t["q"] if prec == FP64 else 1e-4), (plan, which, k, e)
        eQ, eH = _rel(obs["Q"].real, ref.Q), _rel(obs["H"].real, Href)
        ephi = max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB)))
        print(f"\n128^3 prec={prec} plan={plan}: Q rel {eQ:.2e} H rel {eH:.2e} phi abs {ephi:.2e} (all points) "
              f"slices rel {eq:.2e}")
        assert eQ <= t["Q"] and _check_H(obs["H"].real, Href, w.C, w.L, prec) and ephi <= t["phi"]
        assert abs(phiA.mean() - ref.NsA / w.Ns) <= (1e-12 if prec == FP64 else 1e-6)


@pytest.mark.parametrize("n,Ns,fA", [((32, 32, 32), 40, 0.35), ((128, 128, 128), 100, 0.35)])
def test_fp32_quadrature_is_an_fp64_sum_of_the_fp32_products(n, Ns, fA):
    """FP32-mixed: the contour quadrature of Eq. 8 sums the FP32 products q_n qd_(Ns-n)
    in FP64 (compensated FP32 partial sums over chunks of slices, flushed into FP64 sums).
    Recomputed here from the GPU's own stored histories with a plain float64 sum of the
    same float32 products: the densities must agree to FP64 rounding, far below the FP32
    rounding of the products (6e-8)."""
    L = (8.0, 8.0, 8.0) if n[0] == 128 else (4.0, 4.0, 4.0)
    wp, wm = _fields(n, SCFT, 91)
    with pft.System(n, L, Ns, fA, 18.0, 1.0, SCFT, FP32) as s:
        s.set_fields(wp, wm)
        s.solve()
        phiA, phiB = s.densities()
        NsA = o.n_A_steps(Ns, fA)
        cA, cB = o.quadrature_weights(Ns, NsA)
        accA = np.zeros(n)
        accB = np.zeros(n)
        for k in range(Ns + 1):
            prod = (s.propagator(0, k).astype(np.float32) * s.propagator(2, Ns - k).astype(np.float32))
            prod = prod.astype(np.float64)
            accA += cA[k] * prod
            accB += cB[k] * prod
        Q = s.propagator(0, Ns).mean()
    ds = 1.0 / Ns
    eA = np.max(np.abs(phiA - ds * accA / Q))
    eB = np.max(np.abs(phiB - ds * accB / Q))
    print(f"\nFP32 quadrature {n} Ns={Ns} vs FP64 sum of the same products: {eA:.2e} {eB:.2e}")
    assert eA <= 1e-12 and eB <= 1e-12
