"""GPU parity of the solve path (assemble, line factor, sweeps, refinement, sources,
restriction) against the CPU oracle, through the C ABI.

Tolerances: relative error per right-hand-side column, max over columns and
frequencies, <= 1e-9 for the FP64 path and <= 1e-8 for the mixed path after
refinement (the wavefield targets of the method's GPU path)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import helmholtz as H

hm = pytest.importorskip("paper_2301_10762_gb300.helm")

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9
TOL_MIXED = 1e-8


def colerr(X, ref):
    return float(np.max(np.linalg.norm(X - ref, axis=-1) / np.linalg.norm(ref, axis=-1)))


def oracle_solve(g, m, omegas, B, adjoint=False):
    out = np.empty_like(B)
    for q, om in enumerate(omegas):
        f = H.Factor(H.helmholtz_matrix(g, m, om))
        out[q] = f.adjoint_solve(B[q]) if adjoint else f.solve(B[q])
    return out


# grids chosen to cover: a single ragged 16-block (nz < 16), several blocks with a
# ragged tail, the cluster sizes 1, 2, 4, 8 and rectangular domains
CASES = [
    (12, 10, 1.0, 0.8, 2, 3),
    (40, 37, 1.3, 1.0, 3, 20),
    (33, 64, 1.0, 1.0, 1, 17),
    (64, 64, 1.0, 1.0, 2, 8),
    (20, 150, 0.5, 1.0, 2, 5),
]


def _setup(nx, nz, lx, lz, n_om, nrhs, seed=0):
    rng = np.random.default_rng(seed)
    c = 1.0 + 0.5 * rng.uniform(0, 1, (nx, nz))
    c = W.gaussian_smooth(c, 1.5)
    m = (1.0 / c ** 2).reshape(-1)
    om = np.sort(rng.uniform(5.0, 20.0, n_om))
    B = rng.standard_normal((n_om, nrhs, nx * nz)) + 1j * rng.standard_normal((n_om, nrhs, nx * nz))
    return m, om, B


@pytest.mark.parametrize("nx,nz,lx,lz,n_om,nrhs", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_solve_and_adjoint_match_oracle(nx, nz, lx, lz, n_om, nrhs, prec):
    m, om, B = _setup(nx, nz, lx, lz, n_om, nrhs)
    g = H.Grid(nx, nz, lx, lz)
    op = hm.helm_assemble(nx, nz, lx, lz, torch.tensor(m, device="cuda"), om)
    f = hm.helm_factor(op, prec)
    Bd = torch.tensor(B, device="cuda")
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    X, info = hm.helm_solve(f, Bd, rtol=1e-12, max_iter=10)
    assert colerr(X.cpu().numpy(), oracle_solve(g, m, om, B)) <= tol
    Y, info = hm.helm_adjoint_solve(f, Bd, rtol=1e-12, max_iter=10)
    assert colerr(Y.cpu().numpy(), oracle_solve(g, m, om, B, adjoint=True)) <= tol
    if prec == 1:
        assert info["max_relres"] <= 1e-12 and info["iters"] >= 2


@pytest.mark.parametrize("product", ["fma", "mma"])
@pytest.mark.parametrize("nx,nz,nrhs", [(24, 128, 11), (30, 64, 3), (24, 128, 1)])
def test_sweep_products_match_oracle(monkeypatch, product, nx, nz, nrhs):
    # 16 rows per CTA (n_z = 64: one K block per warp, n_z = 128: two): the FP32-FMA and the
    # tensor-pipe product of the complex-FP32 sweep, forced either way, with a ragged last
    # chunk of right-hand sides (11 = 8 + 3)
    monkeypatch.setenv("HELM_SWEEP_MMA", "0" if product == "fma" else "1")
    m, om, B = _setup(nx, nz, 1.0, 1.0, 2, nrhs, seed=3)
    g = H.Grid(nx, nz, 1.0, 1.0)
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    f = hm.helm_factor(op, 1)
    Bd = torch.tensor(B, device="cuda")
    X, info = hm.helm_solve(f, Bd, rtol=1e-12, max_iter=10)
    assert colerr(X.cpu().numpy(), oracle_solve(g, m, om, B)) <= TOL_MIXED
    assert info["max_relres"] <= 1e-12
    Y, _ = hm.helm_adjoint_solve(f, Bd, rtol=1e-12, max_iter=10)
    assert colerr(Y.cpu().numpy(), oracle_solve(g, m, om, B, adjoint=True)) <= TOL_MIXED


@pytest.mark.parametrize("tol", ["0", None])
def test_flagged_pivot_blocks_inverted_in_fp64(monkeypatch, tol):
    # tolerance 0 flags every pivot block that the complex-FP32 factor inverts by Gauss-Jordan
    # (first line of each team, ragged last block): those are redone in FP64 and the solve still
    # matches the oracle; the default tolerance flags none on this smooth medium
    if tol is not None:
        monkeypatch.setenv("HELM_FACTOR_FLAG_TOL", tol)
    nx, nz, lx, lz, n_om, nrhs = 40, 37, 1.3, 1.0, 3, 6
    m, om, B = _setup(nx, nz, lx, lz, n_om, nrhs, seed=4)
    g = H.Grid(nx, nz, lx, lz)
    op = hm.helm_assemble(nx, nz, lx, lz, torch.tensor(m, device="cuda"), om)
    f = hm.helm_factor(op, hm.HELM_MIXED)
    if tol is not None:
        assert f.fp64_blocks > 0
    else:
        assert f.fp64_blocks == 0
    X, info = hm.helm_solve(f, torch.tensor(B, device="cuda"), rtol=1e-12, max_iter=10)
    assert colerr(X.cpu().numpy(), oracle_solve(g, m, om, B)) <= TOL_MIXED
    assert hm.helm_factor(op, hm.HELM_FP64).fp64_blocks == 0


def test_plain_forward_config_64():
    """The plain forward workload: 64 x 64, omega = 10, Gaussian inclusion, 8 top-row
    sources; both precisions against the oracle."""
    w = W.config_plain()
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, torch.tensor(w.m, device="cuda"), w.omegas)
    acq = hm.Acq.from_workload(w.acq)
    B = hm.helm_sources(op, acq)
    E = H.source_vectors(g, w.acq.src_xz)
    assert np.array_equal(B.cpu().numpy()[0], E)
    ref = oracle_solve(g, w.m, w.omegas, E[None])
    for prec, tol in ((0, TOL_FP64), (1, TOL_MIXED)):
        f = hm.helm_factor(op, prec)
        X, _ = hm.helm_solve(f, B, rtol=1e-10)
        assert colerr(X.cpu().numpy(), ref) <= tol


def test_sources_off_grid_and_restriction_match_oracle():
    w = W.tiny_case(30, 26, n_src=4, n_rec=9, seed=5)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    src = np.array([[0.13, 0.0], [0.5, 0.31], [w.lx, w.lz], [0.0, 0.77]])
    rec = np.concatenate([w.acq.rec_xz, [[0.0, 0.0], [w.lx, 0.4], [0.5, w.lz]]])
    acq = hm.Acq(src, rec, src_amp=np.array([1.0, 2.0, -0.5, 0.25]))
    op = hm.helm_assemble(w.nx, w.nz, w.lx, w.lz, torch.tensor(w.m, device="cuda"), w.omegas)
    B = hm.helm_sources(op, acq).cpu().numpy()
    E = H.source_vectors(g, src, np.array([1.0, 2.0, -0.5, 0.25]))
    assert np.allclose(B[0], E, atol=1e-15) and np.allclose(B[1], E, atol=1e-15)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((len(w.omegas), 3, g.N)) + 1j * rng.standard_normal((len(w.omegas), 3, g.N))
    Y = hm.helm_restrict(op, acq, torch.tensor(X, device="cuda")).cpu().numpy()
    R, _, _ = H.restriction(g, rec)
    ref = np.einsum("rn,wcn->wcr", R.toarray(), X)
    assert np.max(np.abs(Y - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_invalid_arguments_are_rejected():
    m = torch.ones(16, dtype=torch.float64, device="cuda")
    with pytest.raises(hm.HelmError):
        hm.helm_assemble(3, 4, 1.0, 1.0, m[:12], [1.0])
    op = hm.helm_assemble(4, 4, 1.0, 1.0, m, [1.0])
    with pytest.raises(hm.HelmError):
        hm.helm_sources(op, hm.Acq([[2.0, 0.0]], [[0.5, 0.5]]))


def test_fp64_solve_is_deterministic():
    m, om, B = _setup(48, 40, 1.0, 1.0, 2, 12, seed=3)
    op = hm.helm_assemble(48, 40, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    f = hm.helm_factor(op, 0)
    Bd = torch.tensor(B, device="cuda")
    X1, _ = hm.helm_solve(f, Bd)
    X2, _ = hm.helm_solve(f, Bd)
    assert torch.equal(X1, X2)


@pytest.mark.parametrize("lumping,name", [(hm.HELM_LUMP_UP, "up"), (hm.HELM_LUMP_DOWN, "down")])
@pytest.mark.parametrize("prec,method", [(0, 0), (1, 1), (1, 2)])
def test_triangle_lumping_matches_oracle(lumping, name, prec, method):
    """The mass lumped on the triangles of either orientation (corner weights hx hz / 3 and
    hx hz / 6 instead of the trapezoid's hx hz / 4): solves and the FWI gradient against the
    oracle with the same lumping, and the corner weights do change the wavefield."""
    nx, nz, lx, lz, n_om, nrhs = 40, 48, 1.3, 1.0, 2, 6
    m, om, B = _setup(nx, nz, lx, lz, n_om, nrhs, seed=4)
    g = H.Grid(nx, nz, lx, lz, lumping=name)
    md = torch.tensor(m, device="cuda")
    op = hm.helm_assemble(nx, nz, lx, lz, md, om, lumping=lumping)
    f = hm.helm_factor(op, prec, method=method)
    Bd = torch.tensor(B, device="cuda")
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    X, _ = hm.helm_solve(f, Bd, rtol=1e-12, max_iter=10)
    ref = oracle_solve(g, m, om, B)
    assert colerr(X.cpu().numpy(), ref) <= tol
    assert colerr(oracle_solve(H.Grid(nx, nz, lx, lz), m, om, B), ref) > 1e-6   # the tensor weights differ
    # the gradient's g_k carries the same weights
    src = np.array([[0.0, 0.3], [0.0, 0.7]])
    rec = np.array([[1.2, 0.2], [1.1, 0.5], [1.25, 0.85], [1.0, 0.6]])
    mt = m * 1.05
    data, _ = H.synthetic_data(g, mt, om, src, rec)
    phi_o, grad_o = H.fwi_objective_gradient(g, m, om, src, rec, data, 1e-3, 1e-4)
    phi, grad, _, _ = hm.fwi_misfit_grad(f, hm.Acq(src, rec), torch.tensor(data, device="cuda"), 1e-3, 1e-4, 1e-12)
    assert abs(phi - phi_o) <= tol * abs(phi_o)
    assert np.linalg.norm(grad.cpu().numpy() - grad_o) <= tol * np.linalg.norm(grad_o)
