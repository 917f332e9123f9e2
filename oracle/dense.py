"""Brute-force dense counterparts of the oracle, for tiny grids only.

TEST INFRASTRUCTURE (see oracle/helmholtz.py).  These routines take a different
route to the same quantities, so that the sparse oracle can be pinned against them:
  * Gaussian elimination with partial pivoting written out by hand (no LAPACK);
  * the Hessian of phi formed entry by entry from explicit first and second
    derivatives of the wavefield (Eqs. (h1), (h2), (oneMgrad2a), (Jac_exp));
  * the lower-level minimiser by Newton's method with that dense Hessian, so that
    the hypergradient can be checked against finite differences of psi.
"""
from __future__ import annotations

import numpy as np

from . import helmholtz as H


def gauss_solve(A, B):
    """Solve A X = B (A dense n x n, B n x k) by Gaussian elimination with row partial
    pivoting and back substitution, written out in plain numpy row operations."""
    A = np.array(A, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128).reshape(A.shape[0], -1)
    n = A.shape[0]
    for c in range(n):
        p = c + int(np.argmax(np.abs(A[c:, c])))
        if A[p, c] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        if p != c:
            A[[c, p]] = A[[p, c]]
            X[[c, p]] = X[[p, c]]
        f = A[c + 1:, c] / A[c, c]
        A[c + 1:, c:] -= np.outer(f, A[c, c:])
        X[c + 1:] -= np.outer(f, X[c])
    for c in range(n - 1, -1, -1):
        X[c] = (X[c] - A[c, c + 1:] @ X[c + 1:]) / A[c, c]
    return X


def jacobian(grid, m, omega, Ainv, u):
    """J[:, k] = du/dm_k = A^{-1} (g_k u_k e_k) (Eq. (oneMgrad2a)); Ainv dense."""
    g = H.g_vec(grid, m, omega)
    return Ainv * (g * u)[None, :]


def dense_hessian(grid, m, omegas, src_xz, rec_xz, data, alpha, mu, rec_w=None):
    """Dense H = H1 + H2 + Gamma from Eqs. (h1), (h2), with d2u/dm_j dm_k from
    Eq. (Jac_exp):  A d2u = g_j (du/dm_k)_j e_j + g_k (du/dm_j)_k e_k + delta_jk g'_k u_k e_k."""
    R, _, _ = H.restriction(grid, rec_xz)
    R = R.toarray()
    w2 = np.ones(R.shape[0]) if rec_w is None else np.asarray(rec_w) ** 2
    E = H.source_vectors(grid, src_xz)
    N = grid.N
    Hm = np.zeros((N, N))
    for q, om in enumerate(omegas):
        A = H.helmholtz_matrix(grid, m, om).toarray()
        Ainv = gauss_solve(A, np.eye(N))
        g = H.g_vec(grid, m, om)
        gp = H.g_prime_vec(grid, m, om)
        for s in range(E.shape[0]):
            u = Ainv @ E[s]
            J = jacobian(grid, m, om, Ainv, u)                 # [N, N]
            RJ = R @ J                                         # [n_rec, N]
            eps = data[q, s] - R @ u
            # H1_jk = Re <R J_j, W^2 R J_k>
            Hm += np.real(RJ.T @ (w2[:, None] * np.conj(RJ)))
            # H2_jk = -Re <R d2u/dm_j dm_k, W^2 eps>; d2u = Ainv[:, j] g_j J[j, k] + Ainv[:, k] g_k J[k, j] + ...
            c = R.T @ (w2 * np.conj(eps))                      # so <R x, W^2 eps> = x^T c
            a = Ainv.T @ c                                     # a_j = (Ainv[:, j])^T c
            T = (a * g)[:, None] * J                           # T[j, k] = a_j g_j J[j, k]
            H2 = -np.real(T + T.T)
            H2 -= np.diag(np.real(a * gp * u))
            Hm += H2
    return Hm + H.gamma(grid.nx, grid.nz, alpha, mu).toarray()


def lower_level_newton(grid, m0, omegas, src_xz, rec_xz, data, alpha, mu, rec_w=None,
                       tol=1e-13, maxit=30):
    """m_FWI: minimise phi by Newton's method with the dense Hessian (tiny grids only).
    Stops when ||grad phi|| <= tol * max(1, ||grad phi(m0)||)."""
    m = np.array(m0, dtype=np.float64)
    g0 = None
    for _ in range(maxit):
        _, g = H.fwi_objective_gradient(grid, m, omegas, src_xz, rec_xz, data, alpha, mu, rec_w=rec_w)
        gn = np.linalg.norm(g)
        if g0 is None:
            g0 = max(1.0, gn)
        if gn <= tol * g0:
            return m, gn
        Hd = dense_hessian(grid, m, omegas, src_xz, rec_xz, data, alpha, mu, rec_w=rec_w)
        step = np.linalg.solve(Hd, g)
        t = 1.0
        while np.any(m - t * step <= 0):
            t *= 0.5
        m = m - t * step
    _, g = H.fwi_objective_gradient(grid, m, omegas, src_xz, rec_xz, data, alpha, mu, rec_w=rec_w)
    return m, np.linalg.norm(g)
