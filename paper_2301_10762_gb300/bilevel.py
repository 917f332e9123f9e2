"""Upper level of the bilevel learning of receiver positions and of the regularisation weight.

Bilevel frequency continuation (Algorithm allg:fcb1): the frequencies are arranged in groups of
increasing frequency, the bilevel problem is solved on each group in turn, and the design
parameters and the lower-level solutions of one group start the next.  On each group the
upper-level objective psi (Eq. SOobj averaged over the training models) is minimised by a bounded
L-BFGS (the L-BFGS-B of Byrd, Lu, Nocedal and Zhu, named in Section subsec:Quasi; SciPy's
implementation) with the stopping rules of the numerical experiments: projected gradient
infinity norm <= 1e-10, a stalled objective, or 50 iterations.  The receivers stay in their
borehole: x is fixed and the depths z are bounded.  As the paper recommends, alpha is kept fixed
and only optimised in the final frequency group (free_alpha="last"); "all" frees it from the
first group, "none" never.

`GpuBilevelProblem.evaluate` is the function the loop minimises.  For the current receiver depths
and alpha, and for every training model, it synthesises the data at the receivers, solves the
lower level (`lbfgs.fwi_lower_level`, warm-started from that model's previous solution, to
||grad phi|| <= 1e-10), and evaluates psi, dpsi/dz and dpsi/dalpha with `bilevel_hypergrad`.
Every Helmholtz solve is the GPU path; only the small design vectors and the lower-level
optimiser's N-vectors live on the host.
"""
from __future__ import annotations

import numpy as np


def frequency_continuation(evaluate, z0, alpha0, groups, z_bounds, alpha_bounds=(1e-10, None), free_alpha="last",
                           max_iter=50, pgtol=1e-10, ftol=1e-15, callback=None):
    """Algorithm allg:fcb1 with L-BFGS-B on each frequency group.

    evaluate(omegas, z, alpha) -> (psi, dpsi_dz [n_rec], dpsi_dalpha) on the group's frequencies.
    z0: initial receiver depths; z_bounds: (low, high) for every depth.
    Returns {"z", "alpha", "history"}; history has one entry per group with the psi at its start
    and at its end, the iterations, whether alpha was free and the stopping message."""
    from scipy.optimize import minimize

    z = np.array(z0, dtype=np.float64)
    alpha = float(alpha0)
    nz = z.size
    history = []
    for k, grp in enumerate(groups):
        omegas = np.atleast_1d(np.asarray(grp, dtype=np.float64))
        free = free_alpha == "all" or (free_alpha == "last" and k == len(groups) - 1)
        start = {}

        def fun(x, omegas=omegas, free=free):
            zz = x[:nz]
            a = float(x[nz]) if free else alpha
            psi, dz, da = evaluate(omegas, zz, a)
            if "psi" not in start:
                start["psi"] = float(psi)
            g = np.concatenate([np.asarray(dz, dtype=np.float64), [da]]) if free else np.asarray(dz, dtype=np.float64)
            return float(psi), g

        x0 = np.concatenate([z, [alpha]]) if free else z.copy()
        bounds = [tuple(z_bounds)] * nz + ([tuple(alpha_bounds)] if free else [])
        res = minimize(fun, x0, jac=True, method="L-BFGS-B", bounds=bounds,
                       options={"maxiter": int(max_iter), "gtol": float(pgtol), "ftol": float(ftol)})
        z = np.array(res.x[:nz])
        if free:
            alpha = float(res.x[nz])
        entry = {"omegas": omegas.tolist(), "psi_start": start.get("psi", float(res.fun)), "psi": float(res.fun),
                 "iters": int(res.nit), "alpha_free": free, "message": str(res.message)}
        history.append(entry)
        if callback is not None:
            callback(k, z, alpha, entry)
    return {"z": z, "alpha": alpha, "history": history}


class GpuBilevelProblem:
    """Training models on one grid, fixed sources, receivers in a vertical borehole x = rec_x.

    m_true: list of squared-slowness models m' (host arrays, N values); m0: the lower-level initial
    guess shared by all models; src_xz: [n_src][2]; alpha0, mu: P2 = Gamma(alpha0, mu) and the
    Tikhonov mu; prec: factor precision of every solve."""

    def __init__(self, nx, nz, lx, lz, m_true, m0, src_xz, rec_x, alpha0, mu, prec=None, refine_rtol=1e-10,
                 lower_gtol=1e-10, lower_max_iter=500, cg_rtol=1e-15, cg_max_iter=500):
        import torch

        from . import helm as hm
        self.hm, self.torch = hm, torch
        self.grid = (int(nx), int(nz), float(lx), float(lz))
        self.m_true = [torch.tensor(np.asarray(m, dtype=np.float64), device="cuda") for m in m_true]
        self.warm = [np.array(m0, dtype=np.float64) for _ in m_true]
        self.src_xz = np.asarray(src_xz, dtype=np.float64).reshape(-1, 2)
        self.rec_x = float(rec_x)
        self.alpha0, self.mu = float(alpha0), float(mu)
        self.prec = hm.HELM_MIXED if prec is None else prec
        self.refine_rtol, self.lower_gtol, self.lower_max_iter = refine_rtol, lower_gtol, lower_max_iter
        self.cg_rtol, self.cg_max_iter = cg_rtol, cg_max_iter
        self.evaluations = 0

    def acquisition(self, z):
        z = np.asarray(z, dtype=np.float64)
        rec = np.stack([np.full(z.size, self.rec_x), z], axis=1)
        return self.hm.Acq(self.src_xz, rec)

    def data(self, omegas, acq, m_true):
        """d = R(P) u(m') at the current receivers (the training data of model m')."""
        hm = self.hm
        op = hm.helm_assemble(*self.grid, m_true, omegas)
        f = hm.helm_factor(op, self.prec)
        U, _ = hm.helm_solve(f, hm.helm_sources(op, acq), rtol=self.refine_rtol, max_iter=40)
        return hm.helm_restrict(op, acq, U)

    def evaluate(self, omegas, z, alpha):
        """(psi, dpsi/dz, dpsi/dalpha) at receiver depths z and Tikhonov weight alpha."""
        from .autograd import HelmholtzProblem
        from .lbfgs import fwi_lower_level
        hm, torch = self.hm, self.torch
        acq = self.acquisition(z)
        m_fwi = []
        for k, mt in enumerate(self.m_true):
            prob = HelmholtzProblem(*self.grid, omegas, acq=acq, prec=self.prec, rtol=self.refine_rtol)
            res = fwi_lower_level(prob, self.data(omegas, acq, mt), alpha, self.mu, self.warm[k],
                                  gtol=self.lower_gtol, max_iter=self.lower_max_iter)
            if not res["converged"]:
                raise RuntimeError(f"lower level of model {k} stopped at ||grad phi|| = {res['gnorm']:.3e} "
                                   f"({res['message']})")
            self.warm[k] = res["x"]
            m_fwi.append(torch.tensor(res["x"], device="cuda"))
        out = hm.bilevel_hypergrad([self.grid] * len(self.m_true), m_fwi, self.m_true, acq, omegas, alpha,
                                   self.alpha0, self.mu, prec=self.prec, cg_rtol=self.cg_rtol,
                                   cg_max_iter=self.cg_max_iter, refine_rtol=self.refine_rtol)
        self.evaluations += 1
        return out["psi"], out["dpsi_dp"][:, 1].copy(), out["dpsi_dalpha"]
