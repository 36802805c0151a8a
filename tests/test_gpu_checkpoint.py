"""GPU parity of the checkpointed q history: the forward march keeps every K-th slice
(and q_Ns), and the conjugate march recomputes each segment of K-1 slices from its
checkpoint before the steps that pair with it.  Results are the same arithmetic as with
the full history, so the tolerances are those of the solve (FP64: relative 1e-12 on Q
and H, 1e-10 absolute on phi; FP32-mixed: 2e-5)."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft
from paper_1204_5434_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64, FP32 = pft.PFT_FP64, pft.PFT_FP32_MIXED
SCFT, CL = pft.PFT_SCFT_REAL, pft.PFT_CL_COMPLEX
OKIND = {SCFT: o.SCFT_REAL, CL: o.CL_COMPLEX}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _fields(n, kind, seed):
    rng = np.random.default_rng(seed)
    wp = rng.normal(0, 0.3, n)
    wm = rng.normal(0, 1.0, n)
    if kind == CL:
        wp = wp + 1j * rng.normal(0, 0.3, n)
        wm = wm + 1j * rng.normal(0, 0.3, n)
    return wp, wm


def _rel(a, b):
    return abs(a - b) / abs(b)


# K divides Ns or not, segments shorter than K at the top, K = Ns (only q_0 kept)
@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("kind", [SCFT, CL])
@pytest.mark.parametrize("Ns,K", [(20, 2), (20, 3), (20, 5), (13, 4), (13, 13), (7, 6)])
def test_checkpointed_solve_matches_oracle(Ns, K, kind, prec):
    n, L, fA, chiN, C = (16, 12, 8), (4.0, 3.0, 2.0), 0.35, 17.0, 3.0
    wp, wm = _fields(n, kind, 60 + Ns + K)
    ref = o.solve(wp, wm, n, L, Ns, fA, OKIND[kind])
    Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, OKIND[kind])
    tol = 1e-12 if prec == FP64 else 2e-5
    with pft.System(n, L, Ns, fA, chiN, C, kind, prec, checkpoint=K) as s:
        assert pft.pft_get_checkpoint(s.h) == K
        s.set_fields(wp, wm)
        s.solve()
        obs = s.observables()
        phiA, phiB = s.densities()
        Q = obs["Q"] if kind == CL else obs["Q"].real
        H = obs["H"] if kind == CL else obs["H"].real
        assert _rel(Q, ref.Q) <= tol
        if prec == FP64:
            assert _rel(H, Href) <= 1e-12
        else:
            assert abs(H - Href) / (C * float(np.prod(L))) <= 2e-5
        assert max(np.max(np.abs(phiA - ref.phiA)), np.max(np.abs(phiB - ref.phiB))) <= (1e-10 if prec == FP64 else 2e-5)
        # kept slices: every K-th and q_Ns; the others are refused
        for k in range(0, Ns + 1):
            if k % K == 0 or k == Ns:
                q = s.propagator(0, k)
                assert np.max(np.abs(q - ref.q[k])) <= tol * np.max(np.abs(ref.q[k])), k
            else:
                with pytest.raises(pft.PftError) as ei:
                    s.propagator(0, k)
                assert ei.value.status == pft.PFT_ERR_UNSUPPORTED
        qd = s.propagator(1, 0)
        assert np.max(np.abs(qd - ref.qd[Ns])) <= tol * np.max(np.abs(ref.qd[Ns]))


def test_checkpointed_history_uses_less_memory():
    n, L, Ns = (32, 32, 32), (4.0, 4.0, 4.0), 100
    with pft.System(n, L, Ns, 0.5, 15.0, 1.0, SCFT, FP64, checkpoint=1) as s:
        full = pft.pft_memory_bytes(s.h)
    with pft.System(n, L, Ns, 0.5, 15.0, 1.0, SCFT, FP64, checkpoint=10) as s:
        ck = pft.pft_memory_bytes(s.h)
    slice_b = 8 * 32 ** 3
    # 101 slices against 11 checkpoints + q_Ns slot + 9 segment slots
    assert full - ck >= (101 - 21) * slice_b


def test_checkpointed_gradients_match_full_history_and_oracle():
    n, L, Ns, fA, chiN, C = (16, 12, 8), (4.0, 3.0, 2.0), 20, 0.35, 18.0, 2.0
    wp, wm = _fields(n, SCFT, 70)
    ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    gq = o.dlnQ_dL(ref, n, L)
    out = {}
    for K in (1, 4, 7):
        with pft.System(n, L, Ns, fA, chiN, C, SCFT, FP64, checkpoint=K) as s:
            s.set_fields(wp, wm)
            s.solve()
            out[K] = s.gradients()
    for K in (4, 7):
        a, b, dL, dq = out[K]
        a1, b1, dL1, dq1 = out[1]
        assert np.max(np.abs(a - a1)) <= 1e-13 * np.max(np.abs(a1))
        assert max(abs(dq[i] - dq1[i]) / abs(dq1[i]) for i in range(3)) <= 1e-12
        assert max(abs(dq[i] - gq[i]) / abs(gq[i]) for i in range(3)) <= 1e-9


def test_checkpointed_scft_relaxation_matches_oracle():
    n, L, Ns, fA, chiN, lam = (16, 12, 8), (4.0, 3.0, 2.0), 16, 0.4, 15.0, 0.1
    wp, wm = _fields(n, SCFT, 21)
    with pft.System(n, L, Ns, fA, chiN, 1.0, SCFT, FP64, checkpoint=5) as s:
        s.set_fields(wp, wm)
        for it in range(3):
            s.solve()
            obs = s.observables()
            ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
            Href = o.hamiltonian(wp, wm, ref.lnQ, chiN, 1.0, n, L, o.SCFT_REAL)
            assert _rel(obs["H"].real, Href) <= 1e-12
            s.field_step(lam)
            wp, wm = o.scft_euler_step(wp, wm, ref.phiA, ref.phiB, chiN, lam)
        gp, gm = s.get_fields()
    assert np.max(np.abs(gp - wp)) <= 1e-12 and np.max(np.abs(gm - wm)) <= 1e-11


def test_checkpoint_refuses_other_schemes():
    with pytest.raises(pft.PftError) as ei:
        pft.System((64, 64, 64), (8.0, 8.0, 8.0), 10, 0.5, 15.0, 1.0, SCFT, FP64, checkpoint=3,
                   scheme=pft.PFT_SCHEME_RQM4)
    assert ei.value.status == pft.PFT_ERR_UNSUPPORTED


@pytest.mark.parametrize("K", [10])
def test_checkpointed_gyroid_128cubed_fp32(K):
    """The 128^3 gyroid workload (Ns = 100) with q kept every 10th slice: Q, H and phi at
    4096 sampled points against the oracle (FP32-mixed tolerances)."""
    w = wl.GYR128
    wp, wm = wl.fields(w)
    ref = o.solve(wp, wm, w.n, w.L, w.Ns, w.fA, o.SCFT_REAL)
    Href = o.hamiltonian(wp, wm, ref.lnQ, w.chiN, w.C, w.n, w.L, o.SCFT_REAL)
    with pft.System(w.n, w.L, w.Ns, w.fA, w.chiN, w.C, SCFT, FP32, checkpoint=K) as s:
        s.set_fields(wp, wm)
        s.solve()
        obs = s.observables()
        phiA, phiB = s.densities()
    idx = np.random.default_rng(2).choice(phiA.size, 4096, replace=False)
    assert _rel(obs["Q"].real, ref.Q) <= 2e-5
    assert abs(obs["H"].real - Href) / (w.C * float(np.prod(w.L))) <= 2e-5
    assert max(np.max(np.abs(phiA.ravel()[idx] - ref.phiA.ravel()[idx])),
               np.max(np.abs(phiB.ravel()[idx] - ref.phiB.ravel()[idx]))) <= 2e-5
