"""Preconditioners for the Hessian system H rho = m' - m_FWI, and the study that compares them
(Section "Preconditioning the Hessian").

The upper-level gradient needs rho from H rho = m' - m_FWI (Eq. rho), solved by PCG without
forming H.  The paper proposes two preconditioners:
  P1 = H(m_FWI(P0, alpha0, m'), P0, alpha0): the full Hessian at chosen design parameters,
       formed column by column (one Hessian product per column) and applied through its
       Cholesky factor;
  P2 = Gamma(alpha0, mu) (Eq. P2): cheap, independent of the sensors, the model and the
       frequency; applied here by `helm_gamma_solve` (the DCT solver of the library's PCG).
Its study counts the PCG iterations to ||r_n|| / ||r_0|| <= 1e-6 with none, P1 (sensors P0 near
and far from the current ones) and P2, for several alpha, and reports the reduction as a
percentage of the unpreconditioned count.

`pcg` works on numpy arrays and on torch tensors (CPU or CUDA) alike; on the GPU every Hessian
product is `fwi_hessian_vec` and every P2 application `helm_gamma_solve`.
"""
from __future__ import annotations

import math

import numpy as np


def _copy(v):
    return v.clone() if hasattr(v, "clone") else np.array(v, copy=True)


def _dot(a, b):
    return float(a @ b)


def pcg(apply_H, b, apply_Minv=None, x0=None, rtol=1e-6, max_iter=1000):
    """Preconditioned conjugate gradients for H x = b (H symmetric positive definite).

    apply_Minv(r) applies the inverse of the preconditioner (None: no preconditioner).  x0: the
    initial guess (None: zero).  Stops when ||r_n||_2 / ||r_0||_2 <= rtol or after max_iter
    iterations.  Returns a dict: x, iters (iterations n, i.e. Hessian products after the one of
    the initial residual), relres, history (||r_k|| / ||r_0|| for k = 0..n), converged."""
    if x0 is None:
        x = b * 0.0
        r = _copy(b)
        products = 0
    else:
        x = _copy(x0)
        r = b - apply_H(x)
        products = 1
    r0 = math.sqrt(_dot(r, r))
    hist = [1.0]
    if r0 == 0.0:
        return {"x": x, "iters": 0, "relres": 0.0, "history": hist, "converged": True, "products": products}
    z = apply_Minv(r) if apply_Minv is not None else _copy(r)
    p = _copy(z)
    rz = _dot(r, z)
    n = 0
    rel = 1.0
    while rel > rtol and n < max_iter:
        Hp = apply_H(p)
        products += 1
        pHp = _dot(p, Hp)
        if not pHp > 0.0:
            raise ValueError(f"p.Hp = {pHp:.3e} <= 0 at iteration {n}: the matrix is not positive definite")
        a = rz / pHp
        x = x + a * p
        r = r - a * Hp
        n += 1
        rel = math.sqrt(_dot(r, r)) / r0
        hist.append(rel)
        if rel <= rtol:
            break
        z = apply_Minv(r) if apply_Minv is not None else _copy(r)
        rz_new = _dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return {"x": x, "iters": n, "relres": rel, "history": hist, "converged": rel <= rtol, "products": products}


def dense_from_products(apply_H, n, like=None):
    """The n x n matrix of a symmetric operator, one product per column (H e_k), symmetrised as
    (H + H^T) / 2 to remove the rounding asymmetry of the products.  like: a vector whose type
    and device the unit vectors take (numpy when None)."""
    if like is None:
        cols = [np.asarray(apply_H(np.eye(1, n, k)[0])) for k in range(n)]
        H = np.stack(cols, axis=1)
        return 0.5 * (H + H.T)
    import torch
    H = torch.empty((n, n), dtype=like.dtype, device=like.device)
    e = torch.zeros(n, dtype=like.dtype, device=like.device)
    for k in range(n):
        e.zero_()
        e[k] = 1.0
        H[:, k] = apply_H(e)
    return 0.5 * (H + H.T)


class CholeskyPreconditioner:
    """Applies P^{-1} for a dense symmetric positive definite P (e.g. P1, the Hessian at P0) by
    its Cholesky factor; numpy or torch (on the matrix's device)."""

    def __init__(self, P):
        self.torch = hasattr(P, "clone")
        if self.torch:
            import torch
            self.L = torch.linalg.cholesky(P)
        else:
            import scipy.linalg
            self.cf = scipy.linalg.cho_factor(np.asarray(P, dtype=np.float64))

    def __call__(self, r):
        if self.torch:
            import torch
            return torch.cholesky_solve(r.reshape(-1, 1), self.L).reshape(-1)
        import scipy.linalg
        return scipy.linalg.cho_solve(self.cf, r)


def gamma_preconditioner(nx, nz, alpha0, mu):
    """P2^{-1} = Gamma(alpha0, mu)^{-1} on the GPU (FP64 CUDA tensors)."""
    from . import helm as hm
    return lambda r: hm.helm_gamma_solve(nx, nz, alpha0, mu, r.contiguous())


def reduction_percent(n_plain, n_prec):
    """Reduction in iterations as a percentage of the unpreconditioned count, rounded to the
    nearest whole number (negative when the preconditioner needs more iterations)."""
    return int(round(100.0 * (n_plain - n_prec) / n_plain))


def study_row(apply_H, rhs, preconditioners, x0=None, rtol=1e-6, max_iter=1000):
    """PCG iteration counts for one Hessian system with each preconditioner.

    preconditioners: {name: apply_Minv or None}.  Returns {name: {"iters", "relres",
    "converged", "reduction"}}, where reduction is relative to the entry whose preconditioner is
    None (if there is one)."""
    out = {}
    for name, M in preconditioners.items():
        r = pcg(apply_H, rhs, M, x0=x0, rtol=rtol, max_iter=max_iter)
        out[name] = {"iters": r["iters"], "relres": r["relres"], "converged": r["converged"]}
    plain = [k for k, M in preconditioners.items() if M is None]
    if plain:
        n0 = out[plain[0]]["iters"]
        for v in out.values():
            v["reduction"] = reduction_percent(n0, v["iters"]) if n0 > 0 else 0
    return out


class GpuHessian:
    """The Hessian of phi at m (full, Lemmas thm:H1 and thm:H2) as an operator on FP64 CUDA
    vectors: the factor, wavefields and adjoint fields are computed once (fwi_misfit_grad) and
    every product is one fwi_hessian_vec call."""

    def __init__(self, problem, m, data, alpha, mu):
        import torch

        from . import helm as hm
        self.hm = hm
        self.acq = problem._need_acq()
        m = torch.as_tensor(m, dtype=torch.float64, device="cuda").contiguous()
        self.op = problem.operator(m)
        self.f = hm.helm_factor(self.op, problem.prec)
        self.alpha, self.mu, self.rtol = float(alpha), float(mu), problem.rtol
        self.phi, self.grad, self.U, self.Lam = hm.fwi_misfit_grad(self.f, self.acq, data.contiguous(), alpha, mu,
                                                                   problem.rtol, want_fields=True)
        self.N = problem.N
        self.products = 0

    def __call__(self, v):
        self.products += 1
        return self.hm.fwi_hessian_vec(self.f, self.acq, self.U, self.Lam, v.contiguous(), self.alpha, self.mu,
                                       self.rtol)

    def dense(self):
        return dense_from_products(self, self.N, like=self.grad)
