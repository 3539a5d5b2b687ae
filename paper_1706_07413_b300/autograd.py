"""torch.autograd interface to the discrete adjoint (adscl_grad) and the adjoint-driven refinement
of mode-sum initial data (arXiv:1706.07413, Sec. II: initial data Pi(x,0) = sum_k a_k e_k(x)
built from the AdS normal modes, and the mode-energy spectrum E_j that the paper monitors).

J(a) = sum_{j<spec_J} (E_j(T) - E_j(0))^2 per instance measures how far the spectrum drifts over
[0, T]; data with a small drift are close to quasi-periodic (non-collapsing) solutions.  One
adscl_grad call runs the forward pass (checkpoints every ckpt_every steps), the per-segment
recomputation and the backward sweep, so forward() computes dJ/da at once and backward() only
scales it by the incoming gradient.  Every step runs in the library's kernels; this module only
marshals tensors."""
from __future__ import annotations

import numpy as np
import torch

from . import adscl


def _grad_call(solver: adscl.Solver, a: torch.Tensor, T: float):
    """(J, dJ/da) as tensors on a's device; a: (B, K) float64."""
    a = a.detach().to(torch.float64).contiguous()
    B, K = a.shape
    J = torch.empty(B, dtype=torch.float64, device=a.device)
    g = torch.empty((B, K), dtype=torch.float64, device=a.device)
    if a.is_cuda:
        torch.cuda.current_stream(a.device).synchronize()   # a is ready for the solver's stream
        solver._check(solver.lib.adscl_grad(solver.ctx, a.data_ptr(), K, float(T), J.data_ptr(),
                                            g.data_ptr(), 1))
        if solver.stream:
            ext = torch.cuda.ExternalStream(solver.stream, device=a.device)
        else:
            ext = torch.cuda.default_stream(a.device)
        torch.cuda.current_stream(a.device).wait_stream(ext)
    else:
        solver._check(solver.lib.adscl_grad(solver.ctx, a.data_ptr(), K, float(T), J.data_ptr(),
                                            g.data_ptr(), 0))
    return J, g


class ModeDrift(torch.autograd.Function):
    """J = ModeDrift.apply(a, solver, T): per-instance spectral drift of the evolution from
    Pi(x,0) = sum_k a[b, k] e_k, Phi = 0, over [0, T]; differentiable in a (B x K, float64)."""

    @staticmethod
    def forward(ctx, a, solver, T):
        J, g = _grad_call(solver, a, T)
        ctx.save_for_backward(g)
        return J

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ.to(g.dtype)[:, None] * g, None, None


def mode_drift(solver: adscl.Solver, a: torch.Tensor, T: float) -> torch.Tensor:
    return ModeDrift.apply(a, solver, T)


def refine_modes(solver: adscl.Solver, a0, T: float, iters: int = 5, step: float = 0.02):
    """Adjoint-driven refinement of mode amplitudes towards small spectral drift: per instance,
    normalised gradient steps a <- a - step * |a| * g / |g| on J(a), halving the step for an
    instance whose J did not decrease (that step is undone).  Returns (a, J history (iters+1,
    B))."""
    a = torch.as_tensor(np.asarray(a0, dtype=np.float64)).clone()
    B = a.shape[0]
    lr = torch.full((B,), float(step), dtype=torch.float64)
    J, g = _grad_call(solver, a, T)
    hist = [J.clone()]
    for _ in range(iters):
        gn = g.norm(dim=1).clamp_min(1e-300)
        an = a.norm(dim=1)
        trial = a - (lr * an / gn)[:, None] * g
        Jt, gt = _grad_call(solver, trial, T)
        ok = Jt < J
        a = torch.where(ok[:, None], trial, a)
        J = torch.where(ok, Jt, J)
        g = torch.where(ok[:, None], gt, g)
        lr = torch.where(ok, lr, 0.5 * lr)
        hist.append(J.clone())
    return a, torch.stack(hist)
