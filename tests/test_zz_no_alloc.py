"""The allocation-free contour step (pft_contour_step_static) against the oracle's split
step and against the context path.

Some callers cannot call cudaMalloc -- for example code running while another
framework owns the device allocator, or a plug-in that may only use the buffers it is
handed -- so the library offers one step whose scratch is a static device array.  This
file checks, through the C ABI, that two calls in a row give q_{n+1} = B F^-1[D F[B q_n]]
(Eq. 13's A(ds) block) as the FP64 oracle computes it, and the same q_{n+1} as a context
solve (pft_debug_set_q0 + pft_solve + pft_get_propagator slice 1), both within the FP64
propagator tolerance of the other GPU tests (1e-12 relative to the slice maximum), and
that grids beyond the static limit are refused.  It is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle as o
from paper_1204_5434_gb300 import pft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1204_5434_gb300 import build
    build.build()


def _reference(n, L, Ns, w, q_in):
    # W+ = w and W- = 0 make wA = wB = w, so slice 1 of the forward history is one
    # split step of q_0 = q_in with B = exp(-w/(2 Ns)).
    with pft.System(n, L, Ns, 0.5, 10.0, 1.0, pft.PFT_SCFT_REAL, pft.PFT_FP64) as s:
        s.set_fields(w, np.zeros(n))
        pft.pft_debug_set_q0(s.h, np.ascontiguousarray(q_in))
        s.solve()
        return s.propagator(0, 1)


@pytest.mark.parametrize("n,L,Ns", [((16, 12, 8), (4.0, 3.0, 2.0), 20), ((64, 48, 64), (8.0, 6.0, 8.0), 100)])
def test_static_step_matches_context_step_twice(n, L, Ns):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(sum(n) + Ns)
    for call in range(2):
        w = rng.normal(0, 1.0, n)
        q_in = np.exp(rng.normal(0, 0.3, n))
        ref = _reference(n, L, Ns, w, q_in)
        dw = torch.from_numpy(w).cuda()
        dq = torch.from_numpy(q_in).cuda()
        out = torch.empty_like(dq)
        torch.cuda.synchronize()
        pft.pft_contour_step_static(n, L, Ns, dw, dq, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ds = 1.0 / Ns
        oref = o.split_step(q_in, o.boltzmann_factor(w, ds), o.diffusion_factor(n, L, ds))
        assert np.max(np.abs(got - oref)) <= 1e-12 * np.max(np.abs(oref)), call
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), call


def test_static_step_rejects_grids_beyond_the_limit():
    torch = pytest.importorskip("torch")
    n = (128, 64, 64)
    dw = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pft.PftError) as e:
        pft.pft_contour_step_static(n, (8.0, 4.0, 4.0), 10, dw, dw, dw)
    assert e.value.status == pft.PFT_ERR_ARG
    assert "static scratch" in pft.pft_last_error()
