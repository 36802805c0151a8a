"""H of a real SCFT diblock context as a differentiable torch function.

    H = pft_hamiltonian(system, wp, wm, L)

wp, wm: float64 CUDA tensors (the Wick-rotated fields W+ and W-, row-major [x][y][z]);
L: float64 tensor of the three box lengths (Rg).  The forward pass sets the box and the
fields, runs one solve and returns H (Eq. 3) as a 0-d float64 tensor on the fields'
device.  The backward pass returns the exact gradients of the discrete H computed by the
library (pft_gradients): dH/dW+ = C dV (phiA + phiB - 1), dH/dW- = C dV (2 W-/chiN +
phiB - phiA), and dH/dL_a at fixed grid values.  All arithmetic runs in the library's
kernels; this module only moves tensors across the C ABI.  The gradients are evaluated
in the forward pass when any input requires them (the context holds one solve at a time).
"""
from __future__ import annotations

import torch

from . import pft


class _Hamiltonian(torch.autograd.Function):
    @staticmethod
    def forward(ctx, wp, wm, L, system):
        h = system.h
        pft.pft_set_box(h, [float(v) for v in L.detach().cpu().tolist()])
        wp_c = wp.detach().contiguous()
        wm_c = wm.detach().contiguous()
        pft.pft_set_fields(h, wp_c, wm_c)
        pft.pft_solve(h)
        obs = pft.pft_get_observables(h)
        if any(ctx.needs_input_grad[:3]):
            gp = torch.empty_like(wp_c)
            gm = torch.empty_like(wm_c)
            dL, _ = pft.pft_gradients(h, gp, gm)
            pft.pft_synchronize(h)
            ctx.save_for_backward(gp, gm, torch.tensor(dL, dtype=torch.float64, device=L.device))
        return torch.tensor(obs["H"].real, dtype=torch.float64, device=wp.device)

    @staticmethod
    def backward(ctx, g):
        gp, gm, dL = ctx.saved_tensors
        gw = g.to(gp.device)
        return gw * gp, gw * gm, g.to(dL.device) * dL, None


def pft_hamiltonian(system, wp, wm, L):
    """Differentiable H(W+, W-, L) of `system` (a pft.System in real SCFT mode, SPLIT2)."""
    if system.kind != pft.PFT_SCFT_REAL:
        raise ValueError("the differentiable Hamiltonian needs real SCFT fields")
    return _Hamiltonian.apply(wp, wm, L, system)
