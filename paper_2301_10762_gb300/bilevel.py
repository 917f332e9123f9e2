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


def mre(recon, truth):
    """Mean relative percentage error (Eq. relerr): the mean over the parameters j of
    |recon_j - truth_j| / |truth_j| * 100."""
    recon = np.asarray(recon, dtype=np.float64)
    truth = np.asarray(truth, dtype=np.float64)
    return float(np.mean(np.abs((recon - truth) / truth)) * 100.0)


def improvement_factor(psi_initial, psi_optimised):
    """IF = psi(alpha_0, P_0) / psi(alpha_opt, P_opt)."""
    return float(psi_initial) / float(psi_optimised)


def add_noise(data, draws, level=0.01):
    """Data with white noise at the given relative level (1 % is 40 dB SNR, the setting of the
    paper's tests).  draws: standard complex Gaussian samples of data's shape [n_omega, ...],
    drawn by the caller from a seeded generator; each frequency's noise is scaled to
    ||eta_w||_2 = level * ||d_w||_2.  Works on numpy arrays and torch tensors alike."""
    if tuple(draws.shape) != tuple(data.shape):
        raise ValueError(f"draws {tuple(draws.shape)} must have the data's shape {tuple(data.shape)}")
    out = data.clone() if hasattr(data, "clone") else np.array(data, copy=True)
    for q in range(data.shape[0]):
        dn = float((abs(data[q]) ** 2).sum()) ** 0.5
        en = float((abs(draws[q]) ** 2).sum()) ** 0.5
        if en == 0.0:
            raise ValueError("noise draws of a frequency are all zero")
        out[q] = data[q] + draws[q] * (level * dn / en)
    return out


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


def run_protocol(problem, z0, alpha0, groups, z_bounds, m_tests, m0, alpha_bounds=(1e-10, None),
                 free_alpha="last", max_iter=50, noise_draws=None, level=0.01, data_models=None):
    """The experiments' protocol: learn the design by bilevel frequency continuation on the
    training models, then report IF and MRE (Eq. relerr) on the training set and on test models.

    problem: an object with evaluate(omegas, z, alpha) -> (psi, dpsi/dz, dpsi/dalpha) over the
    training models, and test_metrics(omegas, z, alpha, m_tests, m0, noise_draws, level,
    data_models) -> (psi, [MRE per test model]) (e.g. GpuBilevelProblem).  Both IFs are taken
    on the final group's frequencies; the training psi at the initial design is evaluated last,
    so that the lower-level warm starts of the continuation are those of the algorithm.
    Returns a dict: z, alpha, history, train_psi (initial, learned), train_if, test_psi
    (initial, learned), test_if, test_mre (initial, learned; lists per test model)."""
    out = frequency_continuation(problem.evaluate, z0, alpha0, groups, z_bounds, alpha_bounds=alpha_bounds,
                                 free_alpha=free_alpha, max_iter=max_iter)
    last = np.atleast_1d(np.asarray(groups[-1], dtype=np.float64))
    psi_opt = problem.evaluate(last, out["z"], out["alpha"])[0]
    psi_init = problem.evaluate(last, np.asarray(z0, dtype=np.float64), alpha0)[0]
    kw = {"noise_draws": noise_draws, "level": level, "data_models": data_models}
    t_init, mre_init = problem.test_metrics(last, np.asarray(z0, dtype=np.float64), alpha0, m_tests, m0, **kw)
    t_opt, mre_opt = problem.test_metrics(last, out["z"], out["alpha"], m_tests, m0, **kw)
    return {"z": out["z"], "alpha": out["alpha"], "history": out["history"],
            "train_psi": (float(psi_init), float(psi_opt)), "train_if": improvement_factor(psi_init, psi_opt),
            "test_psi": (float(t_init), float(t_opt)), "test_if": improvement_factor(t_init, t_opt),
            "test_mre": (list(mre_init), list(mre_opt))}


def lower_level_set(models, prec=None, refine_rtol=1e-12, gtol=1e-10, max_iter=5000, memory=10):
    """m_FWI of the lower level (Section 4's L-BFGS to ||grad phi||_2 <= gtol) for a set of
    training models, e.g. the uneven-grid set of workloads.config_hypergrad: each entry has
    nx, nz, lx, lz, omegas, acq (workloads.Acquisition), m (the initial guess), m_true, alpha,
    mu.  The data d = R u(m') come from FP64 factors of A(m'); every phi / grad phi evaluation
    of the lower level is the library's (mixed by default, refined to refine_rtol, so that the
    gradient stays accurate well below gtol).  Returns one dict per model: x (m_FWI, host),
    gnorm, iters, evals, seconds, message."""
    import time

    import torch

    from . import helm as hm
    from .autograd import HelmholtzProblem
    from .lbfgs import fwi_lower_level
    prec = hm.HELM_MIXED if prec is None else prec
    out = []
    for w in models:
        acq = hm.Acq.from_workload(w.acq)
        op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, torch.tensor(w.m_true, device="cuda"), w.omegas)
        f = hm.helm_factor(op, hm.HELM_FP64)
        U, _ = hm.helm_solve(f, hm.helm_sources(op, acq), rtol=refine_rtol, max_iter=40)
        d = hm.helm_restrict(op, acq, U)
        f.close()
        op.close()
        prob = HelmholtzProblem(w.nx, w.nz, w.lx, w.lz, w.omegas, acq=acq, prec=prec, rtol=refine_rtol, max_iter=40)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fwi_lower_level(prob, d, w.alpha, w.mu, np.asarray(w.m, dtype=np.float64), gtol=gtol,
                              max_iter=max_iter, memory=memory)
        torch.cuda.synchronize()
        res["seconds"] = time.perf_counter() - t0
        out.append(res)
    return out


class GpuBilevelProblem:
    """Training models on one grid, fixed sources, receivers in a vertical borehole x = rec_x.

    m_true: list of squared-slowness models m' (host arrays, N values); m0: the lower-level initial
    guess shared by all models; src_xz: [n_src][2]; alpha0, mu: P2 = Gamma(alpha0, mu) and the
    Tikhonov mu; prec: factor precision of every solve.  cg_rtol: the PCG tolerance for rho; the
    paper's 1e-15 lies below what FP64 PCG reaches on an ill-conditioned Hessian (the library then
    reports non-convergence), so the default is 1e-13.  train_data_models: None (training data
    from m_true on the inversion grid), or per training model (nx_d, nz_d, m_d): the data computed
    from m_d on an nx_d x nz_d grid of the same domain, in the lower level and in the
    hypergradient alike (the Appendix generates u(m') on another grid than u(m))."""

    def __init__(self, nx, nz, lx, lz, m_true, m0, src_xz, rec_x, alpha0, mu, prec=None, refine_rtol=1e-10,
                 lower_gtol=1e-10, lower_max_iter=500, cg_rtol=1e-13, cg_max_iter=500, train_data_models=None):
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
        self.train_data = None
        if train_data_models is not None:
            if len(train_data_models) != len(m_true):
                raise ValueError("one data model per training model")
            self.train_data = [((int(a), int(b), float(lx), float(lz)),
                                torch.tensor(np.asarray(md, dtype=np.float64), device="cuda"))
                               for (a, b, md) in train_data_models]
        self.evaluations = 0

    def acquisition(self, z):
        z = np.asarray(z, dtype=np.float64)
        rec = np.stack([np.full(z.size, self.rec_x), z], axis=1)
        return self.hm.Acq(self.src_xz, rec)

    def data(self, omegas, acq, m_true, grid=None):
        """d = R(P) u(m') at the current receivers (the training data of model m'), on the
        inversion grid or on another grid (nx, nz) of the same domain, on which m_true is then
        given (data from a finer grid avoid the inverse crime)."""
        hm = self.hm
        g = self.grid if grid is None else (int(grid[0]), int(grid[1]), self.grid[2], self.grid[3])
        op = hm.helm_assemble(*g, m_true, omegas)
        f = hm.helm_factor(op, self.prec)
        U, _ = hm.helm_solve(f, hm.helm_sources(op, acq), rtol=self.refine_rtol, max_iter=40)
        return hm.helm_restrict(op, acq, U)

    def reconstruct(self, omegas, z, alpha, m_true, m0, noise_draws=None, level=0.01, data_model=None):
        """m_FWI for one model from data at receiver depths z (with noise at the given level if
        noise_draws, [n_omega, n_src, n_rec] complex, are given), by the lower level from m0.
        data_model: None (data from m_true on the inversion grid) or (nx, nz, m) to generate the
        data from m on another nx x nz grid of the same domain."""
        from .autograd import HelmholtzProblem
        from .lbfgs import fwi_lower_level
        torch = self.torch
        omegas = np.atleast_1d(np.asarray(omegas, dtype=np.float64))
        acq = self.acquisition(z)
        if data_model is None:
            mt = torch.as_tensor(np.asarray(m_true, dtype=np.float64), device="cuda")
            d = self.data(omegas, acq, mt)
        else:
            md = torch.as_tensor(np.asarray(data_model[2], dtype=np.float64), device="cuda")
            d = self.data(omegas, acq, md, grid=data_model[:2])
        if noise_draws is not None:
            d = add_noise(d, torch.as_tensor(np.asarray(noise_draws), dtype=torch.complex128, device="cuda"), level)
        prob = HelmholtzProblem(*self.grid, omegas, acq=acq, prec=self.prec, rtol=self.refine_rtol)
        res = fwi_lower_level(prob, d, alpha, self.mu, np.asarray(m0, dtype=np.float64), gtol=self.lower_gtol,
                              max_iter=self.lower_max_iter)
        return res["x"], res

    def test_metrics(self, omegas, z, alpha, m_tests, m0, noise_draws=None, level=0.01, data_models=None):
        """psi (Eq. SOobj averaged over the test models) and the MRE of the reconstructed
        wavespeed c = m^(-1/2) against the ground truth, per test model.  data_models: None or
        one (nx, nz, m) per test model (data from another grid, see reconstruct)."""
        psi, mres = 0.0, []
        for k, mt in enumerate(m_tests):
            draws = None if noise_draws is None else noise_draws[k]
            dm = None if data_models is None else data_models[k]
            m_fwi, _ = self.reconstruct(omegas, z, alpha, mt, m0, draws, level, data_model=dm)
            mt = np.asarray(mt, dtype=np.float64)
            psi += 0.5 * float(np.sum((mt - m_fwi) ** 2)) / len(m_tests)
            mres.append(mre(1.0 / np.sqrt(m_fwi), 1.0 / np.sqrt(mt)))
        return psi, mres

    def evaluate(self, omegas, z, alpha):
        """(psi, dpsi/dz, dpsi/dalpha) at receiver depths z and Tikhonov weight alpha."""
        from .autograd import HelmholtzProblem
        from .lbfgs import fwi_lower_level
        hm, torch = self.hm, self.torch
        acq = self.acquisition(z)
        m_fwi = []
        for k, mt in enumerate(self.m_true):
            prob = HelmholtzProblem(*self.grid, omegas, acq=acq, prec=self.prec, rtol=self.refine_rtol)
            if self.train_data is None:
                d = self.data(omegas, acq, mt)
            else:
                dg, md = self.train_data[k]
                d = self.data(omegas, acq, md, grid=dg[:2])
            res = fwi_lower_level(prob, d, alpha, self.mu, self.warm[k],
                                  gtol=self.lower_gtol, max_iter=self.lower_max_iter)
            if not res["converged"]:
                raise RuntimeError(f"lower level of model {k} stopped at ||grad phi|| = {res['gnorm']:.3e} "
                                   f"({res['message']})")
            self.warm[k] = res["x"]
            m_fwi.append(torch.tensor(res["x"], device="cuda"))
        dgs = None if self.train_data is None else [dg for dg, _ in self.train_data]
        mds = None if self.train_data is None else [md for _, md in self.train_data]
        out = hm.bilevel_hypergrad([self.grid] * len(self.m_true), m_fwi, self.m_true, acq, omegas, alpha,
                                   self.alpha0, self.mu, prec=self.prec, cg_rtol=self.cg_rtol,
                                   cg_max_iter=self.cg_max_iter, refine_rtol=self.refine_rtol,
                                   data_grids=dgs, m_data=mds)
        self.evaluations += 1
        return out["psi"], out["dpsi_dp"][:, 1].copy(), out["dpsi_dalpha"]
