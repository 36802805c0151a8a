"""The torch.autograd wrapper: H(W+, W-, L) through the C ABI, its gradients against the
oracle's exact discrete gradients and against finite differences of its own forward."""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _setup():
    n, L, Ns, fA, chiN, C = (16, 12, 8), (4.0, 3.0, 2.0), 20, 0.35, 18.0, 2.0
    rng = np.random.default_rng(31)
    return n, L, Ns, fA, chiN, C, rng.normal(0, 0.3, n), rng.normal(0, 1.0, n)


def test_autograd_gradients_match_the_oracle():
    torch = pytest.importorskip("torch")
    from paper_1204_5434_gb300.autograd import pft_hamiltonian
    n, L, Ns, fA, chiN, C, wp, wm = _setup()
    ref = o.solve(wp, wm, n, L, Ns, fA, o.SCFT_REAL)
    H = o.hamiltonian(wp, wm, ref.lnQ, chiN, C, n, L, o.SCFT_REAL)
    gp, gm = o.dH_dfields(wp, wm, ref, chiN, C, n, L, o.SCFT_REAL)
    gL = o.dH_dL(H, ref, C, n, L)
    with pft.System(n, L, Ns, fA, chiN, C, pft.PFT_SCFT_REAL, pft.PFT_FP64) as s:
        twp = torch.tensor(wp, device="cuda", requires_grad=True)
        twm = torch.tensor(wm, device="cuda", requires_grad=True)
        tL = torch.tensor(L, dtype=torch.float64, requires_grad=True)
        Ht = pft_hamiltonian(s, twp, twm, tL)
        Ht.backward()
    assert abs(Ht.item() - H) <= 1e-12 * abs(H)
    assert np.max(np.abs(twp.grad.cpu().numpy() - gp)) <= 1e-12 * np.max(np.abs(gp))
    assert np.max(np.abs(twm.grad.cpu().numpy() - gm)) <= 1e-12 * np.max(np.abs(gm))
    assert np.max(np.abs(tL.grad.numpy() - np.asarray(gL)) / np.abs(np.asarray(gL))) <= 1e-9


def test_autograd_box_gradient_matches_finite_differences_of_the_forward():
    torch = pytest.importorskip("torch")
    from paper_1204_5434_gb300.autograd import pft_hamiltonian
    n, L, Ns, fA, chiN, C, wp, wm = _setup()
    with pft.System(n, L, Ns, fA, chiN, C, pft.PFT_SCFT_REAL, pft.PFT_FP64) as s:
        twp = torch.tensor(wp, device="cuda")
        twm = torch.tensor(wm, device="cuda")
        tL = torch.tensor(L, dtype=torch.float64, requires_grad=True)
        pft_hamiltonian(s, twp, twm, tL).backward()
        g = tL.grad.numpy().copy()
        h = 1e-4
        for a in range(3):
            def H(d):
                LL = torch.tensor(L, dtype=torch.float64)
                LL[a] += d
                return pft_hamiltonian(s, twp, twm, LL).item()
            fd = (8 * (H(h) - H(-h)) - (H(2 * h) - H(-2 * h))) / (12 * h)
            assert abs(fd - g[a]) <= 1e-7 * max(1.0, abs(g[a])), (a, fd, g[a])


def test_autograd_refuses_complex_fields():
    pytest.importorskip("torch")
    from paper_1204_5434_gb300.autograd import pft_hamiltonian
    with pft.System((8, 8, 8), (2.0, 2.0, 2.0), 8, 0.5, 10.0, 1.0, pft.PFT_CL_COMPLEX, pft.PFT_FP64) as s:
        with pytest.raises(ValueError):
            pft_hamiltonian(s, None, None, None)
