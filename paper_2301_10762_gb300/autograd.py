"""torch.autograd wrappers of the Helmholtz solve, the restriction and the FWI misfit.

Every forward and backward step runs in libhelm's kernels through the C ABI (helm.py); these
classes only decide which calls to make.  Conventions: for a complex tensor z PyTorch passes
the gradient G with dL = Re sum conj(G) dz (twice the conjugate Wirtinger derivative), and for
the real model m the ordinary gradient.

    U = A(m)^{-1} B  (helm_solve, per frequency):
        grad_B = (A^H)^{-1} G                          (helm_adjoint_solve)
        grad_m = Re sum g U conj((A^H)^{-1} G)          (helm_field_grad; dU/dm_k = A^{-1}(g_k e_k U_k),
                                                        Proposition prop:elem of the paper)
    Y = R(P) U      (helm_restrict):   grad_U = R(P)^T G (helm_restrict_adjoint)
    phi(m)          (fwi_misfit_grad): grad_m = grad phi (Theorem th:grad), computed in the forward

With recompute=True the solve keeps only its factor and recomputes U from it in the backward
pass instead of storing the wavefields of every source and frequency.
"""
from __future__ import annotations

import numpy as np
import torch

from . import helm as hm


class HelmholtzProblem:
    """Grid, frequencies and acquisition of a family of Helmholtz problems A(m, w) u = b.

    solve(m, B) and restrict(U) are differentiable; misfit(m, data, alpha, mu) is the FWI
    objective phi of the paper with its adjoint-state gradient."""

    def __init__(self, nx, nz, lx, lz, omegas, acq: hm.Acq | None = None, prec=hm.HELM_MIXED, rtol=1e-10,
                 max_iter=8):
        self.nx, self.nz, self.lx, self.lz = int(nx), int(nz), float(lx), float(lz)
        self.omegas = np.atleast_1d(np.asarray(omegas, dtype=np.float64))
        self.acq = acq
        self.prec, self.rtol, self.max_iter = prec, float(rtol), int(max_iter)
        self.N = self.nx * self.nz
        self._geom = None   # an operator of this grid for the restriction (any m)

    def operator(self, m: torch.Tensor) -> hm.Op:
        return hm.helm_assemble(self.nx, self.nz, self.lx, self.lz, m.detach().contiguous(), self.omegas)

    def geometry_op(self) -> hm.Op:
        if self._geom is None:
            ones = torch.ones(self.N, dtype=torch.float64, device="cuda")
            self._geom = self.operator(ones)
        return self._geom

    def sources(self) -> torch.Tensor:
        return hm.helm_sources(self.geometry_op(), self._need_acq())

    def solve(self, m: torch.Tensor, B: torch.Tensor, recompute: bool = False) -> torch.Tensor:
        return HelmholtzSolve.apply(m, B, self, recompute)

    def restrict(self, U: torch.Tensor) -> torch.Tensor:
        return Restrict.apply(U, self)

    def misfit(self, m: torch.Tensor, data: torch.Tensor, alpha=0.0, mu=0.0) -> torch.Tensor:
        return FwiMisfit.apply(m, data, self, float(alpha), float(mu))

    def _need_acq(self) -> hm.Acq:
        if self.acq is None:
            raise ValueError("this operation needs an acquisition (sources, receivers)")
        return self.acq


class HelmholtzSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, B, prob: HelmholtzProblem, recompute: bool):
        op = prob.operator(m)
        f = hm.helm_factor(op, prob.prec)
        Bc = B.detach().contiguous()
        U, _ = hm.helm_solve(f, Bc, rtol=prob.rtol, max_iter=prob.max_iter)
        ctx.prob, ctx.op, ctx.f, ctx.recompute = prob, op, f, recompute
        ctx.save_for_backward(Bc if recompute else U)
        return U

    @staticmethod
    def backward(ctx, G):
        prob, op, f = ctx.prob, ctx.op, ctx.f
        (saved,) = ctx.saved_tensors
        Lam, _ = hm.helm_adjoint_solve(f, G.contiguous(), rtol=prob.rtol, max_iter=prob.max_iter)
        grad_m = grad_B = None
        if ctx.needs_input_grad[0]:
            U = hm.helm_solve(f, saved, rtol=prob.rtol, max_iter=prob.max_iter)[0] if ctx.recompute else saved
            grad_m = hm.helm_field_grad(op, U, Lam)
        if ctx.needs_input_grad[1]:
            grad_B = Lam
        return grad_m, grad_B, None, None


class Restrict(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, prob: HelmholtzProblem):
        ctx.prob = prob
        return hm.helm_restrict(prob.geometry_op(), prob._need_acq(), U.detach().contiguous())

    @staticmethod
    def backward(ctx, G):
        prob = ctx.prob
        return hm.helm_restrict_adjoint(prob.geometry_op(), prob._need_acq(), G.contiguous()), None


class FwiMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, data, prob: HelmholtzProblem, alpha: float, mu: float):
        op = prob.operator(m)
        f = hm.helm_factor(op, prob.prec)
        phi, grad, _, _ = hm.fwi_misfit_grad(f, prob._need_acq(), data.detach().contiguous(), alpha, mu, prob.rtol)
        ctx.save_for_backward(grad)
        return torch.tensor(phi, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, gphi):
        (grad,) = ctx.saved_tensors
        return grad * gphi, None, None, None, None
