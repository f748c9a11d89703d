"""The pseudofermion action as a differentiable function of phi.

Forward: S(phi) = sum over the selected Hasenbusch terms of S_i (plus the
Gaussian term (1/2) phi^2/(delta U) when `gaussian` is set) at fixed
pseudofermions chi (Section 5.1), computed by libhmc's hmc_action.
Backward: dS/dphi from libhmc's hmc_force -- the adjoint of the operator's
phi dependence, Eqs. p_dot and f_chi_i -- scaled by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import _abi


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, hmc, masses, chis, opts=None, gaussian=False, term=-1):
        from . import SolverOpts
        opts = opts or SolverOpts()
        flags = _abi.HMC_FERMION | (_abi.HMC_GAUSSIAN if gaussian else 0)
        phi_c = phi.detach().contiguous()
        S, _ = hmc.action(phi_c, list(masses), list(chis), term=term, flags=flags, opts=opts)
        ctx.save_for_backward(phi_c)
        ctx.hmc, ctx.masses, ctx.chis, ctx.opts, ctx.flags, ctx.term = hmc, list(masses), list(chis), opts, flags, term
        return torch.tensor(S, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_S):
        (phi,) = ctx.saved_tensors
        g, _ = ctx.hmc.force(phi, ctx.masses, ctx.chis, term=ctx.term, flags=ctx.flags, opts=ctx.opts)
        return grad_S * g, None, None, None, None, None, None
