"""GPU parity of the FWI misfit/gradient and the bilevel hypergradient against the CPU
oracle, through the C ABI (Algorithms alg:box1 and alg:box)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import helmholtz as H

hm = pytest.importorskip("paper_2301_10762_gb300.helm")

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
@pytest.mark.parametrize("shape", [(24, 20), (50, 47)])
def test_fwi_misfit_grad_matches_oracle(prec, tol, shape):
    w = W.tiny_case(*shape, n_omega=2, n_src=5, n_rec=11, seed=21)
    w.alpha, w.mu = 1e-3, 1e-6
    rw = np.linspace(0.5, 1.5, 11)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz)
    phi_o, grad_o, fields = H.fwi_objective_gradient(g, w.m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data,
                                                     w.alpha, w.mu, rec_w=rw, return_fields=True)
    op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, torch.tensor(w.m, device="cuda"), w.omegas)
    f = hm.helm_factor(op, prec)
    acq = hm.Acq(w.acq.src_xz, w.acq.rec_xz, rec_w=rw)
    phi, grad, U, Lam = hm.fwi_misfit_grad(f, acq, torch.tensor(data, device="cuda"), w.alpha, w.mu,
                                           rtol=1e-12, want_fields=True)
    assert abs(phi - phi_o) <= tol * abs(phi_o)
    assert relerr(grad.cpu().numpy(), grad_o) <= tol
    assert relerr(U.cpu().numpy(), fields["U"]) <= tol
    assert relerr(Lam.cpu().numpy(), fields["Lam"]) <= tol


def test_fwi_gradient_is_deterministic():
    w = W.tiny_case(40, 33, n_omega=2, n_src=4, n_rec=7, seed=22)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz)
    op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, torch.tensor(w.m, device="cuda"), w.omegas)
    f = hm.helm_factor(op, 0)
    acq = hm.Acq.from_workload(w.acq)
    d = torch.tensor(data, device="cuda")
    p1, g1, _, _ = hm.fwi_misfit_grad(f, acq, d, 1e-3, 1e-6)
    p2, g2, _, _ = hm.fwi_misfit_grad(f, acq, d, 1e-3, 1e-6)
    assert p1 == p2 and torch.equal(g1, g2)


def _two_models(mu, seed=3):
    rng = np.random.default_rng(seed)
    shapes = [(26, 22), (30, 30)]
    om = np.array([4.0, 7.5])
    src = np.array([[0.0, 0.2], [0.0, 0.5], [0.0, 0.8]])
    rec = np.array([[0.9, 0.25], [0.93, 0.55], [0.88, 0.71], [0.95, 0.4]])
    rw = np.array([1.0, 0.9, 1.1, 1.2])
    models = []
    for (nx, nz) in shapes:
        mtrue = W.layered_velocity(nx, nz, int(rng.integers(1000)))
        mfwi = W.gaussian_smooth(mtrue.reshape(nx, nz), 2.0).reshape(-1)
        models.append((nx, nz, mfwi, mtrue))
    return models, om, src, rec, rw


def _hyper_both(models, om, src, rec, rw, alpha, alpha0, mu, prec, oracle_kw, gpu_kw):
    ref = {"psi": 0.0, "dpsi_dalpha": 0.0, "dpsi_dp": 0.0, "dpsi_dw": 0.0}
    grids, mf, mt = [], [], []
    for (nx, nz, mfwi, mtrue) in models:
        o = H.hypergradient(H.Grid(nx, nz), mfwi, mtrue, om, src, rec, alpha, alpha0, mu, rec_w=rw, **oracle_kw)
        for k in ref:
            ref[k] = ref[k] + o[k] / len(models)
        grids.append((nx, nz, 1.0, 1.0))
        mf.append(torch.tensor(mfwi, device="cuda"))
        mt.append(torch.tensor(mtrue, device="cuda"))
    out = hm.bilevel_hypergrad(grids, mf, mt, hm.Acq(src, rec, rec_w=rw), om, alpha, alpha0, mu, prec=prec,
                               refine_rtol=1e-13, **gpu_kw)
    return out, ref


def _assert_hyper(out, ref, tol):
    assert abs(out["psi"] - ref["psi"]) <= 1e-12 * abs(ref["psi"])
    assert abs(out["dpsi_dalpha"] - ref["dpsi_dalpha"]) <= tol * abs(ref["dpsi_dalpha"])
    assert relerr(out["dpsi_dp"], ref["dpsi_dp"]) <= tol
    assert relerr(out["dpsi_dw"], ref["dpsi_dw"]) <= tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
@pytest.mark.parametrize("mu", [1e-4, 1e-6])
def test_hypergradient_converged_pcg_matches_oracle(prec, tol, mu):
    """Two training models on different grids, PCG run to ||r|| <= 1e-13 ||r_0|| on both sides:
    rho is then the solution of H rho = m' - m_fwi, which is well posed (a 1e-14 relative
    change of m_fwi moves the oracle's hypergradient by about 1e-13), unlike a short
    fixed-iteration PCG on an indefinite H (see the reading on PCG sensitivity)."""
    models, om, src, rec, rw = _two_models(mu)
    out, ref = _hyper_both(models, om, src, rec, rw, 1e-3, 2e-3, mu, prec, dict(cg_rtol=1e-13, cg_maxiter=500),
                           dict(cg_rtol=1e-13, cg_max_iter=500))
    assert out["cg_relres"] <= 1e-13
    _assert_hyper(out, ref, tol)


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
def test_hypergradient_with_data_from_a_finer_grid_matches_oracle(prec, tol):
    """Training data computed on a finer grid of the same domain (2n - 1 nodes per direction,
    the model carried there by bilinear interpolation), as the Appendix does against the
    inverse crime: the data and their receiver derivatives come from that grid's wavefields,
    and the hypergradient is compared with the oracle's data-grid branch (converged PCG)."""
    models, om, src, rec, rw = _two_models(1e-4)
    alpha, alpha0, mu = 1e-3, 2e-3, 1e-4
    ref = {"psi": 0.0, "dpsi_dalpha": 0.0, "dpsi_dp": 0.0, "dpsi_dw": 0.0}
    grids, dgrids, mf, mt, md = [], [], [], [], []
    for (nx, nz, mfwi, mtrue) in models:
        fx, fz = 2 * nx - 1, 2 * nz - 1
        mdata = W.resample_bilinear(mtrue, nx, nz, fx, fz)
        o = H.hypergradient(H.Grid(nx, nz), mfwi, mtrue, om, src, rec, alpha, alpha0, mu, rec_w=rw, cg_rtol=1e-13,
                            data_grid=H.Grid(fx, fz), m_true_data=mdata)
        for k in ref:
            ref[k] = ref[k] + o[k] / len(models)
        grids.append((nx, nz, 1.0, 1.0))
        dgrids.append((fx, fz, 1.0, 1.0))
        mf.append(torch.tensor(mfwi, device="cuda"))
        mt.append(torch.tensor(mtrue, device="cuda"))
        md.append(torch.tensor(mdata, device="cuda"))
    out = hm.bilevel_hypergrad(grids, mf, mt, hm.Acq(src, rec, rec_w=rw), om, alpha, alpha0, mu, prec=prec,
                               refine_rtol=1e-13, cg_rtol=1e-13, cg_max_iter=500, data_grids=dgrids, m_data=md)
    assert out["cg_relres"] <= 1e-13
    _assert_hyper(out, ref, tol)
    same = hm.bilevel_hypergrad(grids, mf, mt, hm.Acq(src, rec, rec_w=rw), om, alpha, alpha0, mu, prec=prec,
                                refine_rtol=1e-13, cg_rtol=1e-13, cg_max_iter=500)
    assert relerr(out["dpsi_dp"], same["dpsi_dp"]) > 1e-4   # the finer data do change the result


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
def test_hypergradient_fixed_iterations_matches_oracle(prec, tol):
    """Six PCG iterations on both sides at mu = 1e-6, where the fixed-iteration result is well
    conditioned (its sensitivity to a 1e-14 input change is about 1e-12); also the solve
    count of Theorem thm:cost."""
    models, om, src, rec, rw = _two_models(1e-6)
    out, ref = _hyper_both(models, om, src, rec, rw, 1e-3, 2e-3, 1e-6, prec, dict(cg_fixed_iters=6),
                           dict(cg_fixed_iters=6))
    _assert_hyper(out, ref, tol)
    assert out["cg_matvecs"] == 7
    n_data = len(om) * len(src)
    assert out["data_solves"] == len(models) * n_data
    assert out["solves"] == len(models) * (2 + 2 * 7 + 1) * n_data


@pytest.mark.parametrize("gn", [False, True])
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
def test_hessian_vec_matches_oracle(gn, prec, tol):
    w = W.tiny_case(30, 26, n_omega=2, n_src=4, n_rec=9, seed=31)
    w.alpha, w.mu = 1e-3, 1e-5
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz)
    _, _, fields = H.fwi_objective_gradient(g, w.m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu,
                                            return_fields=True)
    mt = np.random.default_rng(5).standard_normal(g.N)
    ref = H.hessian_vec(g, w.m, w.omegas, fields, mt, w.alpha, w.mu, gauss_newton=gn)
    op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, torch.tensor(w.m, device="cuda"), w.omegas)
    f = hm.helm_factor(op, prec)
    acq = hm.Acq.from_workload(w.acq)
    _, _, U, Lam = hm.fwi_misfit_grad(f, acq, torch.tensor(data, device="cuda"), w.alpha, w.mu, rtol=1e-12,
                                      want_fields=True)
    hv = hm.fwi_hessian_vec(f, acq, U, None if gn else Lam, torch.tensor(mt, device="cuda"), w.alpha, w.mu,
                            rtol=1e-12, gauss_newton=gn)
    assert relerr(hv.cpu().numpy(), ref) <= tol


def test_hypergradient_concurrent_models_match_sequential():
    """Training models processed 1, 2 or 4 at a time (own streams and host threads) give the
    same hypergradient: every model writes its own partial results, summed in model order."""
    rng = np.random.default_rng(8)
    shapes = [(26, 22), (30, 30), (22, 28), (26, 22)]
    om = np.array([4.0, 7.5])
    src = np.array([[0.0, 0.2], [0.0, 0.5], [0.0, 0.8]])
    rec = np.array([[0.9, 0.25], [0.93, 0.55], [0.88, 0.71], [0.95, 0.4]])
    acq = hm.Acq(src, rec, rec_w=np.array([1.0, 0.9, 1.1, 1.2]))
    grids, mf, mt = [], [], []
    for (nx, nz) in shapes:
        mtrue = W.layered_velocity(nx, nz, int(rng.integers(1000)))
        grids.append((nx, nz, 1.0, 1.0))
        mf.append(torch.tensor(W.gaussian_smooth(mtrue.reshape(nx, nz), 2.0).reshape(-1), device="cuda"))
        mt.append(torch.tensor(mtrue, device="cuda"))
    outs = [hm.bilevel_hypergrad(grids, mf, mt, acq, om, 1e-3, 2e-3, 1e-2, prec=hm.HELM_MIXED, cg_fixed_iters=3,
                                 refine_rtol=1e-11, concurrent_models=k) for k in (1, 2, 4)]
    for o in outs[1:]:
        assert o["psi"] == outs[0]["psi"]
        assert o["dpsi_dalpha"] == outs[0]["dpsi_dalpha"]
        assert np.array_equal(o["dpsi_dp"], outs[0]["dpsi_dp"])
        assert np.array_equal(o["dpsi_dw"], outs[0]["dpsi_dw"])
        assert o["solves"] == outs[0]["solves"]
