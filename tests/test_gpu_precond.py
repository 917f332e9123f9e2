"""GPU checks of the preconditioners of the Hessian system (Section "Preconditioning the
Hessian"): helm_gamma_solve (P2 = Gamma(alpha0, mu), Eq. P2) against the oracle's Gamma solved
directly, and the preconditioner study on the GPU Hessian against the same study on the oracle's
Hessian."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import dense as D
from oracle import helmholtz as H

hm = pytest.importorskip("paper_2301_10762_gb300.helm")
PC = pytest.importorskip("paper_2301_10762_gb300.precond")

pytestmark = pytest.mark.gpu


# cond(Gamma) = (8 alpha0 (n - 1)^2 + mu) / mu stays below 1e6, so that the sparse LU reference
# is itself accurate to about 1e-10
@pytest.mark.parametrize("shape,alpha0,mu", [((8, 7), 1e-3, 1e-6), ((64, 48), 2e-3, 1e-4), ((33, 95), 1e-3, 1e-2)])
def test_gamma_solve_matches_oracle(shape, alpha0, mu):
    import scipy.sparse.linalg as spla
    nx, nz = shape
    N = nx * nz
    R = np.random.default_rng(nx * nz).standard_normal((3, N))
    G = H.gamma(nx, nz, alpha0, mu).tocsc()
    ref = np.stack([spla.spsolve(G, R[c]) for c in range(3)])
    Rd = torch.tensor(R, device="cuda")
    Z = hm.helm_gamma_solve(nx, nz, alpha0, mu, Rd)
    err = np.linalg.norm(Z.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-9
    # one column, and in place
    z1 = hm.helm_gamma_solve(nx, nz, alpha0, mu, Rd[1].clone())
    assert np.linalg.norm(z1.cpu().numpy() - ref[1]) <= 1e-9 * np.linalg.norm(ref[1])
    hm.helm_gamma_solve(nx, nz, alpha0, mu, Rd, Z=Rd)
    assert np.linalg.norm(Rd.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)


def test_gamma_solve_rejects_bad_arguments():
    R = torch.zeros(20, dtype=torch.float64, device="cuda")
    for args in ((5, 4, 1e-3, 0.0), (5, 4, -1.0, 1e-6), (1, 20, 1e-3, 1e-6)):
        with pytest.raises(hm.HelmError):
            hm.helm_gamma_solve(*args, R)


def test_preconditioner_study_on_gpu_hessian_matches_oracle():
    from paper_2301_10762_gb300.autograd import HelmholtzProblem
    w = W.tiny_case(12, 11, seed=21, n_omega=2, n_src=3, n_rec=6)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    zs = np.linspace(0.2, 0.8, 6) * w.lz
    sensors = {"P": np.stack([np.full(6, 0.7 * w.lx), zs], 1),
               "near": np.stack([np.full(6, 0.72 * w.lx), zs + 0.03], 1)}
    alpha, mu = 1e-4, 1e-6
    src = w.acq.src_xz
    ops, m_fwis, datas = {}, {}, {}
    for k, rec in sensors.items():
        data, _ = H.synthetic_data(g, w.m_true, w.omegas, src, rec)
        m_fwi, gn = D.lower_level_newton(g, w.m, w.omegas, src, rec, data, alpha, mu)
        assert gn < 1e-10
        _, _, fields = H.fwi_objective_gradient(g, m_fwi, w.omegas, src, rec, data, alpha, mu, return_fields=True)
        ops[k] = (lambda v, m=m_fwi, f=fields: H.hessian_vec(g, m, w.omegas, f, v, alpha, mu))
        m_fwis[k], datas[k] = m_fwi, data
    # oracle study
    P1o = PC.CholeskyPreconditioner(PC.dense_from_products(ops["near"], g.N))
    P2o = PC.CholeskyPreconditioner(H.gamma(g.nx, g.nz, alpha, mu).toarray())
    rhs = w.m_true - m_fwis["P"]
    ref = PC.study_row(ops["P"], rhs, {"none": None, "P1near": P1o, "P2": P2o}, x0=np.ones(g.N), rtol=1e-6)
    # the same study on the GPU: Hessian products by fwi_hessian_vec, P2 by helm_gamma_solve
    gpu = {}
    for k, rec in sensors.items():
        prob = HelmholtzProblem(w.nx, w.nz, w.lx, w.lz, w.omegas, acq=hm.Acq(src, rec), prec=hm.HELM_FP64)
        gpu[k] = PC.GpuHessian(prob, m_fwis[k], torch.tensor(datas[k], device="cuda"), alpha, mu)
    Hd = gpu["near"].dense()
    Ho = PC.dense_from_products(ops["near"], g.N)
    assert np.abs(Hd.cpu().numpy() - Ho).max() <= 1e-8 * np.abs(Ho).max()
    P1g = PC.CholeskyPreconditioner(Hd)
    P2g = PC.gamma_preconditioner(g.nx, g.nz, alpha, mu)
    got = PC.study_row(gpu["P"], torch.tensor(rhs, device="cuda"), {"none": None, "P1near": P1g, "P2": P2g},
                       x0=torch.ones(g.N, dtype=torch.float64, device="cuda"), rtol=1e-6)
    for k in ref:
        assert got[k]["converged"]
        assert abs(got[k]["iters"] - ref[k]["iters"]) <= 1, (k, got[k], ref[k])


def test_bilevel_evaluate_matches_oracle_evaluator():
    """GpuBilevelProblem.evaluate (data at the receivers, GPU L-BFGS lower level to
    ||grad phi|| <= 1e-10, bilevel_hypergrad) against the same composition on the oracle (dense
    Newton lower level, Algorithm alg:box hypergradient), averaged over two training models.
    The lower-level solutions differ by up to ||grad phi|| / mu, hence the 1e-4 tolerance."""
    from paper_2301_10762_gb300.bilevel import GpuBilevelProblem
    w0 = W.tiny_case(7, 6, seed=11, n_omega=3, n_src=4, n_rec=6)
    w1 = W.tiny_case(7, 6, seed=12, n_omega=3, n_src=4, n_rec=6)
    g = H.Grid(w0.nx, w0.nz, w0.lx, w0.lz)
    alpha, alpha0, mu = 1e-4, 1e-4, 1e-4
    rec_x = 0.55 * w0.lx
    z = np.linspace(0.15, 0.75, 6) * w0.lz
    omegas = np.array([2.0, 3.0])
    src = w0.acq.src_xz
    rec = np.stack([np.full(6, rec_x), z], axis=1)
    psi_o, dz_o, da_o = 0.0, np.zeros(6), 0.0
    for mt in (w0.m_true, w1.m_true):
        data, _ = H.synthetic_data(g, mt, omegas, src, rec)
        m_fwi, gn = D.lower_level_newton(g, w0.m, omegas, src, rec, data, alpha, mu)
        assert gn < 1e-10
        hg = H.hypergradient(g, m_fwi, mt, omegas, src, rec, alpha, alpha0, mu, cg_rtol=1e-14)
        psi_o += hg["psi"] / 2
        dz_o += hg["dpsi_dp"][:, 1] / 2
        da_o += hg["dpsi_dalpha"] / 2
    prob = GpuBilevelProblem(w0.nx, w0.nz, w0.lx, w0.lz, [w0.m_true, w1.m_true], w0.m, src, rec_x, alpha0, mu,
                             prec=hm.HELM_FP64, lower_max_iter=2000)
    psi, dz, da = prob.evaluate(omegas, z, alpha)
    assert abs(psi - psi_o) <= 1e-4 * abs(psi_o)
    assert np.abs(dz - dz_o).max() <= 1e-4 * np.abs(dz_o).max()
    assert abs(da - da_o) <= 1e-4 * abs(da_o)
    assert prob.evaluations == 1
