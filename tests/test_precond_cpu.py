"""CPU checks of the preconditioner study (paper_2301_10762_gb300/precond.py; Section
"Preconditioning the Hessian", preconditioners P1 and P2 of Eq. P2).

Pins: PCG reaches the solution of a dense SPD system; with an operator of three distinct
eigenvalues it converges in at most three iterations (the Krylov space is exhausted); with the
exact inverse as preconditioner in one; the torch path takes the numpy path's iteration count.  The
Hessian formed column by column from the oracle's adjoint-state products equals the oracle's dense
Hessian built from explicit second derivatives of the wavefield.  On a 12 x 11 stand-in for the
paper's preconditioning experiment, with the oracle's Hessian, the pattern the paper reports
appears: P1 with sensors near the current ones cuts the iterations most; P1 with far sensors
helps little at small alpha and more as alpha grows; P2 helps at every alpha, increasingly so."""
import numpy as np
import pytest

from paper_2301_10762_gb300 import precond as PC


def _spd(n, eigs, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * np.asarray(eigs)) @ Q.T


def test_pcg_solves_spd_system():
    rng = np.random.default_rng(0)
    A = _spd(40, np.geomspace(1e-2, 1e2, 40), 1)
    b = rng.standard_normal(40)
    r = PC.pcg(lambda v: A @ v, b, rtol=1e-12, max_iter=500)
    assert r["converged"] and r["relres"] <= 1e-12
    assert np.allclose(r["x"], np.linalg.solve(A, b), rtol=1e-9, atol=1e-9)
    assert r["history"][0] == 1.0 and len(r["history"]) == r["iters"] + 1


def test_pcg_three_distinct_eigenvalues_three_iterations():
    eigs = np.repeat([1.0, 4.0, 9.0], [10, 7, 13])
    A = _spd(30, eigs, 2)
    b = np.random.default_rng(3).standard_normal(30)
    r = PC.pcg(lambda v: A @ v, b, rtol=1e-10, max_iter=50)
    assert r["converged"] and r["iters"] <= 3


def test_pcg_exact_preconditioner_one_iteration_and_initial_guess():
    A = _spd(25, np.geomspace(1e-3, 1e3, 25), 4)
    b = np.random.default_rng(5).standard_normal(25)
    M = PC.CholeskyPreconditioner(A)
    r = PC.pcg(lambda v: A @ v, b, M, x0=np.ones(25), rtol=1e-8)
    assert r["iters"] == 1 and r["products"] == 2   # the initial residual costs one product
    assert np.allclose(r["x"], np.linalg.solve(A, b), rtol=1e-8)
    # the exact solution as initial guess: no iteration
    r = PC.pcg(lambda v: A @ v, A @ np.ones(25), x0=np.ones(25))
    assert r["iters"] == 0


def test_pcg_not_positive_definite_raises():
    A = np.diag([1.0, -1.0])
    with pytest.raises(ValueError):
        PC.pcg(lambda v: A @ v, np.array([1.0, 1.0]), rtol=1e-12)


def test_pcg_torch_path_matches_numpy():
    torch = pytest.importorskip("torch")
    A = _spd(30, np.geomspace(1e-2, 1e2, 30), 6)
    D = np.diag(1.0 / np.diag(A))
    b = np.random.default_rng(7).standard_normal(30)
    rn = PC.pcg(lambda v: A @ v, b, lambda r: D @ r, x0=np.ones(30), rtol=1e-10)
    At, Dt = torch.tensor(A), torch.tensor(D)
    rt = PC.pcg(lambda v: At @ v, torch.tensor(b), lambda r: Dt @ r, x0=torch.ones(30, dtype=torch.float64),
                rtol=1e-10)
    assert rn["iters"] == rt["iters"]
    # matrix products round differently in numpy and torch: both iterates are within
    # cond(A) * rtol = 1e-6 of the solution
    assert np.linalg.norm(rt["x"].numpy() - rn["x"]) <= 1e-6 * np.linalg.norm(rn["x"])
    Pt = PC.CholeskyPreconditioner(At)
    assert np.allclose(Pt(torch.tensor(b)).numpy(), np.linalg.solve(A, b), rtol=1e-10)


def test_reduction_percent():
    assert PC.reduction_percent(60, 16) == 73
    assert PC.reduction_percent(60, 108) == -80
    assert PC.reduction_percent(44, 13) == 70


def _setup(nx=12, nz=11):
    from oracle import helmholtz as H
    from workloads import tiny_case
    w = tiny_case(nx, nz, seed=21, n_omega=2, n_src=3, n_rec=6)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    zs = np.linspace(0.2, 0.8, 6) * w.lz
    sensors = {
        "P": np.stack([np.full(6, 0.7 * w.lx), zs], 1),
        "near": np.stack([np.full(6, 0.72 * w.lx), zs + 0.03], 1),
        "far": np.stack([np.full(6, 0.15 * w.lx), np.linspace(0.05, 0.3, 6) * w.lz], 1),
    }
    return w, g, sensors


def _oracle_hessian(w, g, rec, alpha, mu):
    from oracle import dense as D
    from oracle import helmholtz as H
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, rec)
    m_fwi, gn = D.lower_level_newton(g, w.m, w.omegas, w.acq.src_xz, rec, data, alpha, mu)
    assert gn < 1e-10
    _, _, fields = H.fwi_objective_gradient(g, m_fwi, w.omegas, w.acq.src_xz, rec, data, alpha, mu,
                                            return_fields=True)
    return (lambda v: H.hessian_vec(g, m_fwi, w.omegas, fields, v, alpha, mu)), m_fwi, data


def test_dense_from_products_equals_oracle_dense_hessian():
    from oracle import dense as D
    w, g, sensors = _setup(7, 6)
    alpha, mu = 1e-3, 1e-6
    Hop, m_fwi, data = _oracle_hessian(w, g, sensors["P"], alpha, mu)
    Hp = PC.dense_from_products(Hop, g.N)
    Hd = D.dense_hessian(g, m_fwi, w.omegas, w.acq.src_xz, sensors["P"], data, alpha, mu)
    assert np.abs(Hp - Hd).max() <= 1e-9 * np.abs(Hd).max()
    assert np.array_equal(Hp, Hp.T)


def test_preconditioner_study_pattern():
    """P1 near: >= 70 % fewer iterations at every alpha.  P1 far: much weaker than P1 near at the
    smallest alpha, better at the largest.  P2: fewer iterations at every alpha, the reduction
    growing with alpha to >= 60 % from alpha = 1e-4 on."""
    from oracle import helmholtz as H
    w, g, sensors = _setup()
    mu = 1e-6
    rows = {}
    for alpha in (1e-6, 1e-4, 1e-2):
        Hop, m_fwi, _ = _oracle_hessian(w, g, sensors["P"], alpha, mu)
        P1n = PC.CholeskyPreconditioner(PC.dense_from_products(_oracle_hessian(w, g, sensors["near"], alpha, mu)[0], g.N))
        P1f = PC.CholeskyPreconditioner(PC.dense_from_products(_oracle_hessian(w, g, sensors["far"], alpha, mu)[0], g.N))
        P2 = PC.CholeskyPreconditioner(H.gamma(g.nx, g.nz, alpha, mu).toarray())
        row = PC.study_row(Hop, w.m_true - m_fwi, {"none": None, "P1near": P1n, "P1far": P1f, "P2": P2},
                           x0=np.ones(g.N), rtol=1e-6)
        assert all(v["converged"] for v in row.values())
        rows[alpha] = {k: v["reduction"] for k, v in row.items()}
    a = sorted(rows)
    for al in a:
        assert rows[al]["P1near"] >= 70
        assert rows[al]["P2"] > 0
    assert rows[a[0]]["P1far"] <= rows[a[0]]["P1near"] - 40
    assert rows[a[-1]]["P1far"] > rows[a[0]]["P1far"] + 40
    assert rows[a[0]]["P2"] < rows[a[1]]["P2"] < rows[a[2]]["P2"]
    assert rows[a[1]]["P2"] >= 60 and rows[a[2]]["P2"] >= 60
