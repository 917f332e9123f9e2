"""torch.autograd through the C ABI (paper_2301_10762_gb300/autograd.py): the solve, the
restriction and the FWI misfit, against the oracle's adjoint-state gradient (Theorem th:grad)
and against finite differences."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import helmholtz as H

hm = pytest.importorskip("paper_2301_10762_gb300.helm")
from paper_2301_10762_gb300.autograd import HelmholtzProblem  # noqa: E402

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _setup(prec, shape=(24, 20), n_omega=2, n_src=3, n_rec=7, seed=31):
    w = W.tiny_case(*shape, n_omega=n_omega, n_src=n_src, n_rec=n_rec, seed=seed)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz)
    prob = HelmholtzProblem(w.nx, w.nz, w.lx, w.lz, w.omegas, hm.Acq.from_workload(w.acq), prec=prec, rtol=1e-12)
    return w, g, torch.tensor(data, device="cuda"), data, prob


def _loss(prob, m, B, d, recompute=False):
    U = prob.solve(m, B, recompute)
    eps = d - prob.restrict(U)
    return 0.5 * (eps.abs() ** 2).sum()


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
@pytest.mark.parametrize("shape", [(24, 20), (40, 33)])
def test_autograd_misfit_gradient_matches_oracle(prec, tol, shape):
    w, g, d, data, prob = _setup(prec, shape)
    phi_o, grad_o = H.fwi_objective_gradient(g, w.m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, 0.0, 0.0)
    m = torch.tensor(w.m, device="cuda", requires_grad=True)
    L = _loss(prob, m, prob.sources(), d)
    L.backward()
    assert abs(L.item() - phi_o) <= tol * abs(phi_o)
    assert relerr(m.grad.cpu().numpy(), grad_o) <= tol


def test_autograd_model_gradient_finite_differences():
    w, g, d, data, prob = _setup(hm.HELM_FP64)
    m0 = torch.tensor(w.m, device="cuda")
    B = prob.sources()
    m = m0.clone().requires_grad_(True)
    _loss(prob, m, B, d).backward()
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = torch.tensor(rng.standard_normal(m0.numel()), device="cuda")
        h = 1e-6 * (m0.norm() / v.norm()).item()
        with torch.no_grad():
            fd = (_loss(prob, m0 + h * v, B, d) - _loss(prob, m0 - h * v, B, d)).item() / (2 * h)
        assert abs(fd - float(m.grad @ v)) <= 1e-6 * abs(fd)


def test_autograd_source_gradient_finite_differences():
    w, g, d, data, prob = _setup(hm.HELM_FP64)
    m0 = torch.tensor(w.m, device="cuda")
    B0 = prob.sources()
    B = B0.clone().requires_grad_(True)
    _loss(prob, m0, B, d).backward()
    rng = np.random.default_rng(6)
    V = torch.tensor(rng.standard_normal(B0.shape) + 1j * rng.standard_normal(B0.shape), device="cuda")
    h = 1e-6
    with torch.no_grad():
        fd = (_loss(prob, m0, B0 + h * V, d) - _loss(prob, m0, B0 - h * V, d)).item() / (2 * h)
    an = float(torch.real(torch.sum(torch.conj(B.grad) * V)))
    assert abs(fd - an) <= 1e-6 * abs(fd)


def test_autograd_recomputed_wavefields_give_the_same_gradient():
    w, g, d, data, prob = _setup(hm.HELM_MIXED)
    B = prob.sources()
    grads = []
    for recompute in (False, True):
        m = torch.tensor(w.m, device="cuda", requires_grad=True)
        _loss(prob, m, B, d, recompute).backward()
        grads.append(m.grad)
    assert torch.equal(grads[0], grads[1])


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
def test_autograd_fwi_misfit_matches_oracle(prec, tol):
    w, g, d, data, prob = _setup(prec)
    alpha, mu = 1e-3, 1e-6
    phi_o, grad_o = H.fwi_objective_gradient(g, w.m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, alpha, mu)
    m = torch.tensor(w.m, device="cuda", requires_grad=True)
    phi = prob.misfit(m, d, alpha, mu)
    (2.0 * phi).backward()
    assert abs(phi.item() - phi_o) <= tol * abs(phi_o)
    assert relerr(m.grad.cpu().numpy() / 2.0, grad_o) <= tol
