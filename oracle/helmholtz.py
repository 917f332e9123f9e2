"""Plain FP64 CPU oracle for the discrete Helmholtz / FWI / hypergradient computations
of Downing, Gazzola, Graham, Spence, "Optimising seismic imaging design parameters
via bilevel learning" (arXiv:2301.10762).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference leg may import this module.  The CUDA library never does,
and this module shares no code with it: assembly here goes element by element
over triangles, solves use a general sparse LU of the assembled matrix (and of
its explicitly formed conjugate transpose for adjoints), and every derivative
is written in the paper's order.

Every function cites the section / equation of the paper it follows.  Readings of
passages the paper leaves open are marked "Reading:".

Conventions: grid nx x nz nodes on [0, lx] x [0, lz], z = 0 the top row,
node (i, j) at (i*hx, j*hz), canonical index k = i*nz + j (z fastest, the
Kronecker order of the regulariser, Eq. (ThisGamma)).  Complex vectors are
numpy complex128.  Right-hand-side blocks are [n_rhs, N] (one row per RHS).
"""
from __future__ import annotations

import math
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SOLVE_COUNTER = {"solves": 0}


def reset_solve_counter():
    SOLVE_COUNTER["solves"] = 0


def spacing(nx, nz, lx, lz):
    return lx / (nx - 1), lz / (nz - 1)


def node_xz(nx, nz, lx, lz):
    """[N, 2] coordinates of the nodes in canonical order."""
    hx, hz = spacing(nx, nz, lx, lz)
    i, j = np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij")
    return np.stack([i.reshape(-1) * hx, j.reshape(-1) * hz], axis=1)


# ------------------------------------------------------------------ discrete operator

def stiffness(nx, nz, lx, lz, diagonal="up"):
    """S_ij = integral of grad(phi_i) . grad(phi_j) for P1 hat functions on the uniform
    rectangular grid with every cell cut into two triangles (Appendix 'Numerical
    forward model', S in A = S - w^2 M - i w B).  Assembled element by element from
    the barycentric-coordinate gradients of each triangle.  `diagonal` picks which
    diagonal cuts the cells ("up": (i,j)-(i+1,j+1), "down": (i+1,j)-(i,j+1))."""
    hx, hz = spacing(nx, nz, lx, lz)
    I, J = np.meshgrid(np.arange(nx - 1), np.arange(nz - 1), indexing="ij")
    I = I.reshape(-1)
    J = J.reshape(-1)
    k00 = I * nz + J
    k10 = (I + 1) * nz + J
    k01 = I * nz + J + 1
    k11 = (I + 1) * nz + J + 1
    if diagonal == "up":
        tris = [(k00, k10, k11), (k00, k11, k01)]
    else:
        tris = [(k00, k10, k01), (k10, k11, k01)]
    xz = node_xz(nx, nz, lx, lz)
    rows, cols, vals = [], [], []
    for tri in tris:
        P = np.stack([xz[t] for t in tri], axis=1)           # [ncell, 3, 2]
        # barycentric coordinates lam_a = c0 + c1 x + c2 z solve V c = e_a, V = [1 x z]
        V = np.concatenate([np.ones(P.shape[:2] + (1,)), P], axis=2)   # [ncell, 3, 3]
        C = np.linalg.inv(V)                                  # columns = coefficients of lam_a
        grads = C[:, 1:, :]                                   # [ncell, 2, 3]
        area = 0.5 * np.abs(np.linalg.det(V))
        K = area[:, None, None] * np.einsum("cda,cdb->cab", grads, grads)
        for a in range(3):
            for b in range(3):
                rows.append(tri[a])
                cols.append(tri[b])
                vals.append(K[:, a, b])
    N = nx * nz
    S = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    S = S.tocsr()
    S.sum_duplicates()
    S.data[np.abs(S.data) < 1e-14 * max(hx / hz, hz / hx)] = 0.0   # hypotenuse couplings are exact zeros
    S.eliminate_zeros()
    return S


def lumped_mass(nx, nz, lx, lz, lumping="tensor"):
    """d_k of M(m) = diag(d_k m_k) (Appendix 'Numerical forward model', nodal quadrature).
    lumping "tensor" (the default reading): the orientation-free tensor trapezoid weights
    d = hx hz qx(i) qz(j), q = 1/2 at end nodes and 1 otherwise (interior hx hz, edges
    hx hz / 2, corners hx hz / 4).  "up" / "down": the vertex quadrature of the P1 mass on the
    triangles themselves, cut along the diagonal (i,j)-(i+1,j+1) ("up") or (i+1,j)-(i,j+1)
    ("down"): every triangle gives a third of its area to each of its vertices (the four grid
    corners then depend on the orientation)."""
    hx, hz = spacing(nx, nz, lx, lz)
    if lumping == "tensor":
        qx = np.ones(nx)
        qx[[0, -1]] = 0.5
        qz = np.ones(nz)
        qz[[0, -1]] = 0.5
        return (hx * hz * np.outer(qx, qz)).reshape(-1)
    if lumping not in ("up", "down"):
        raise ValueError(f"lumping {lumping!r}")
    d = np.zeros(nx * nz)
    xz = node_xz(nx, nz, lx, lz)
    for i in range(nx - 1):
        for j in range(nz - 1):
            k00, k10, k01, k11 = i * nz + j, (i + 1) * nz + j, i * nz + j + 1, (i + 1) * nz + j + 1
            tris = [(k00, k10, k11), (k00, k11, k01)] if lumping == "up" else [(k00, k10, k01), (k10, k11, k01)]
            for t in tris:
                (x0, z0), (x1, z1), (x2, z2) = xz[t[0]], xz[t[1]], xz[t[2]]
                area = 0.5 * abs((x1 - x0) * (z2 - z0) - (x2 - x0) * (z1 - z0))
                for k in t:
                    d[k] += area / 3.0
    return d


def boundary_mass(nx, nz, lx, lz):
    """b_k of B(m) = diag(b_k sqrt(m_k)): nodal (trapezoid) quadrature of the boundary
    integral, i.e. every boundary edge gives half its length to each of its two end
    nodes (Appendix 'Numerical forward model'; b vanishes at interior nodes)."""
    hx, hz = spacing(nx, nz, lx, lz)
    b = np.zeros(nx * nz)
    for i in range(nx - 1):                      # top (j = 0) and bottom (j = nz-1) edges
        for j in (0, nz - 1):
            b[i * nz + j] += 0.5 * hx
            b[(i + 1) * nz + j] += 0.5 * hx
    for j in range(nz - 1):                      # left (i = 0) and right (i = nx-1) edges
        for i in (0, nx - 1):
            b[i * nz + j] += 0.5 * hz
            b[i * nz + j + 1] += 0.5 * hz
    return b


class Grid:
    """Grid plus the m-independent pieces of the operator."""

    def __init__(self, nx, nz, lx=1.0, lz=1.0, diagonal="up", lumping="tensor"):
        if nx < 4 or nz < 4:
            raise ValueError("the sliding-cubic restriction needs at least 4 nodes per direction")
        self.nx, self.nz, self.lx, self.lz = int(nx), int(nz), float(lx), float(lz)
        self.hx, self.hz = spacing(nx, nz, lx, lz)
        self.N = self.nx * self.nz
        self.S = stiffness(nx, nz, lx, lz, diagonal)
        self.d = lumped_mass(nx, nz, lx, lz, lumping)
        self.b = boundary_mass(nx, nz, lx, lz)


def helmholtz_matrix(grid: Grid, m, omega):
    """A(m, w) = S - w^2 diag(d m) - i w diag(b sqrt(m)) (Appendix 'Numerical forward
    model', Eq. (matrices) with nodal quadrature)."""
    m = np.asarray(m, dtype=np.float64)
    diag = -(omega ** 2) * grid.d * m - 1j * omega * grid.b * np.sqrt(m)
    return (grid.S.astype(np.complex128) + sp.diags(diag)).tocsc()


def g_vec(grid: Grid, m, omega):
    """Discrete G_{m,w} of Proposition (prop:elem): -dA/dm_k = g_k e_k e_k^T with
    g_k = w^2 d_k + i w b_k / (2 sqrt(m_k))."""
    return omega ** 2 * grid.d + 1j * omega * grid.b / (2.0 * np.sqrt(m))


def g_prime_vec(grid: Grid, m, omega):
    """d g_k / d m_k = -i w b_k / (4 m_k^{3/2}) (second-derivative term of Eq. (Jac_exp))."""
    return -1j * omega * grid.b / (4.0 * m ** 1.5)


class Factor:
    """Sparse LU of A and, separately, of its explicitly formed conjugate transpose."""

    def __init__(self, A):
        self.A = A
        self._lu = spla.splu(A.tocsc())
        self._luH = None

    def solve(self, B):
        """Rows of B are right-hand sides; returns rows of A^{-1} B."""
        B = np.atleast_2d(B)
        SOLVE_COUNTER["solves"] += B.shape[0]
        return self._lu.solve(np.ascontiguousarray(B.T)).T

    def adjoint_solve(self, B):
        """Rows of (A^H)^{-1} B, A^H = conj(A)^T formed explicitly (Eq. (adjoint),
        A^* = S - w^2 M + i w B of the Appendix)."""
        if self._luH is None:
            self._luH = spla.splu(self.A.conj().T.tocsc())
        B = np.atleast_2d(B)
        SOLVE_COUNTER["solves"] += B.shape[0]
        return self._luH.solve(np.ascontiguousarray(B.T)).T


# ------------------------------------------------------------------- sources / sensors

def source_vectors(grid: Grid, src_xz, src_amp=None):
    """Rows e_s (Appendix, 'Computing the wavefield'): value 1 at a grid-point source.
    Reading for off-grid sources: the bilinear weights of the four surrounding nodes
    (these reduce to e_s on a node)."""
    src_xz = np.atleast_2d(src_xz)
    E = np.zeros((src_xz.shape[0], grid.N), dtype=np.complex128)
    for q, (x, z) in enumerate(src_xz):
        tx, tz = x / grid.hx, z / grid.hz
        i0 = min(max(int(math.floor(tx)), 0), grid.nx - 2)
        j0 = min(max(int(math.floor(tz)), 0), grid.nz - 2)
        fx, fz = tx - i0, tz - j0
        amp = 1.0 if src_amp is None else src_amp[q]
        for di, wx in ((0, 1 - fx), (1, fx)):
            for dj, wz in ((0, 1 - fz), (1, fz)):
                E[q, (i0 + di) * grid.nz + (j0 + dj)] += amp * wx * wz
    return E


def lagrange_cubic(s):
    """Lagrange basis on the nodes 0, 1, 2, 3 at local coordinate s, and its derivative
    (the cubic interpolant through the four nearest nodes, Section 'Numerical
    restriction operator')."""
    L = np.empty(4)
    dL = np.empty(4)
    for a in range(4):
        others = [b for b in range(4) if b != a]
        den = np.prod([a - b for b in others])
        L[a] = np.prod([s - b for b in others]) / den
        dsum = 0.0
        for c in others:
            dsum += np.prod([s - b for b in others if b != c])
        dL[a] = dsum / den
    return L, dL


def cubic_window(t, n):
    """First node of the sliding 4-node window for the scaled position t = p/h
    (Figs. fig:Cub1 / fig:Cub2: p in [x1, x2] uses x0..x3, p in [x2, x3] uses x1..x4).
    Reading: the window is clamped inside the grid (one-sided cubic near the ends)
    and an exact node position uses the window of floor(t)."""
    i0 = int(math.floor(t)) - 1
    return min(max(i0, 0), n - 4)


def restriction(grid: Grid, rec_xz):
    """R(P) (N_r x N), dR/dx and dR/dz: bicubic sliding interpolation, tensor product of
    the 1D sliding cubic in x and in z (Section 'Numerical restriction operator')."""
    rec_xz = np.atleast_2d(rec_xz)
    nr = rec_xz.shape[0]
    R = sp.lil_matrix((nr, grid.N))
    Rx = sp.lil_matrix((nr, grid.N))
    Rz = sp.lil_matrix((nr, grid.N))
    for r, (x, z) in enumerate(rec_xz):
        tx, tz = x / grid.hx, z / grid.hz
        i0 = cubic_window(tx, grid.nx)
        j0 = cubic_window(tz, grid.nz)
        Lx, dLx = lagrange_cubic(tx - i0)
        Lz, dLz = lagrange_cubic(tz - j0)
        for a in range(4):
            for b in range(4):
                k = (i0 + a) * grid.nz + (j0 + b)
                R[r, k] += Lx[a] * Lz[b]
                Rx[r, k] += dLx[a] / grid.hx * Lz[b]
                Rz[r, k] += Lx[a] * dLz[b] / grid.hz
    return R.tocsr(), Rx.tocsr(), Rz.tocsr()


# ------------------------------------------------------------------------ regulariser

def difference_matrix(n):
    """D_n = (n-1) * bidiag(1, -1), (n-1) x n (Section 2, Regularisation)."""
    return (n - 1) * (sp.eye(n - 1, n) - sp.eye(n - 1, n, k=1))


def regulariser(nx, nz):
    """R = D_x^T D_x + D_z^T D_z, D_x = D_nx (x) I_nz, D_z = I_nx (x) D_nz (Eq. (ThisGamma)).
    Reading: the (n - 1) scaling is taken literally, whatever the physical size."""
    Dx = sp.kron(difference_matrix(nx), sp.eye(nz))
    Dz = sp.kron(sp.eye(nx), difference_matrix(nz))
    return (Dx.T @ Dx + Dz.T @ Dz).tocsr()


def gamma(nx, nz, alpha, mu):
    """Gamma(alpha, mu) = alpha R + mu I (Eq. (Gamma))."""
    return (alpha * regulariser(nx, nz) + mu * sp.eye(nx * nz)).tocsr()


# ---------------------------------------------------------------- lower-level problem

def wavefields(grid: Grid, m, omegas, src_xz, src_amp=None):
    """u(m, w, s) = A(m, w)^{-1} e_s for every w and s (Eq. (defu) discretised).
    Returns (factors per w, U [n_omega, n_src, N])."""
    E = source_vectors(grid, src_xz, src_amp)
    facs, U = [], []
    for w in omegas:
        f = Factor(helmholtz_matrix(grid, m, w))
        facs.append(f)
        U.append(f.solve(E))
    return facs, np.array(U)


def fwi_objective_gradient(grid: Grid, m, omegas, src_xz, rec_xz, data, alpha, mu,
                           rec_w=None, src_amp=None, return_fields=False):
    """phi and grad phi by the adjoint-state method (Algorithm alg:box1, Theorem th:grad,
    Eqs. (newphi), (I4), (lambda) and the discrete gradient formula that follows it).

    data: [n_omega, n_src, n_rec] complex, d = R u(m').  eps = d - R u (Eq. (resd)).
    phi = 1/2 sum |W eps|^2 + 1/2 m^T Gamma m, W = diag(rec_w) (rec_w = 1 is the paper).
    lambda solves A^H lambda = R^T (W^2 eps); grad_k = -Re sum g_k u_k conj(lambda_k) + (Gamma m)_k.
    """
    m = np.asarray(m, dtype=np.float64)
    R, _, _ = restriction(grid, rec_xz)
    w2 = np.ones(R.shape[0]) if rec_w is None else np.asarray(rec_w) ** 2
    G = gamma(grid.nx, grid.nz, alpha, mu)
    facs, U = wavefields(grid, m, omegas, src_xz, src_amp)
    phi = 0.0
    grad = np.zeros(grid.N)
    Lam = []
    for q, w in enumerate(omegas):
        eps = data[q] - (R @ U[q].T).T                    # [n_src, n_rec]
        phi += 0.5 * np.sum(w2 * np.abs(eps) ** 2)
        lam = facs[q].adjoint_solve((R.T @ (w2[:, None] * eps.T)).T)
        Lam.append(lam)
        gk = g_vec(grid, m, w)
        grad += -np.real(np.sum(gk[None, :] * U[q] * np.conj(lam), axis=0))
    Gm = G @ m
    phi += 0.5 * m @ Gm
    grad += Gm
    if return_fields:
        return phi, grad, {"U": U, "Lam": np.array(Lam), "facs": facs, "R": R, "w2": w2}
    return phi, grad


def synthetic_data(grid: Grid, m_true, omegas, src_xz, rec_xz, src_amp=None):
    """d(m', w, s) = R(P) u(m', w, s) (Section 2.3, data from a training model)."""
    R, _, _ = restriction(grid, rec_xz)
    _, Ut = wavefields(grid, m_true, omegas, src_xz, src_amp)
    return np.einsum("rn,wsn->wsr", R.toarray(), Ut), Ut


def hessian_vec(grid: Grid, m, omegas, fields, mt, alpha, mu, gauss_newton=False):
    """H m~ = (H1 + H2 + Gamma) m~ by the adjoint-state formulas of Lemmas thm:H1 and
    thm:H2 and Discussion disc:Hess, per (s, w):
        v = A^{-1} (g u m~)                       (Eq. (defv))
        z = A^{-H} (R^T W^2 R v - m~ conj(g) lambda)
        (H m~) += Re[g u conj(z)] - Re[g v conj(lambda)] - Re[g' u conj(lambda)] m~.
    Reading: the adjoint of G in the second term of Eq. (I6) (G^* lambda = conj(g)
    lambda), as in the proof of Lemma thm:H2, not G lambda as in its statement.
    With gauss_newton=True only H1 (z without the lambda term, no H2 terms)."""
    U, Lam, facs, R, w2 = fields["U"], fields["Lam"], fields["facs"], fields["R"], fields["w2"]
    out = np.zeros(grid.N)
    for q, w in enumerate(omegas):
        gk = g_vec(grid, m, w)
        gp = g_prime_vec(grid, m, w)
        V = facs[q].solve(gk[None, :] * U[q] * mt[None, :])
        rhs = (R.T @ (w2[:, None] * (R @ V.T))).T
        if not gauss_newton:
            rhs = rhs - mt[None, :] * np.conj(gk)[None, :] * Lam[q]
        Z = facs[q].adjoint_solve(rhs)
        out += np.real(np.sum(gk[None, :] * U[q] * np.conj(Z), axis=0))
        if not gauss_newton:
            out -= np.real(np.sum(gk[None, :] * V * np.conj(Lam[q]), axis=0))
            out -= np.real(np.sum(gp[None, :] * U[q] * np.conj(Lam[q]), axis=0)) * mt
    return out + gamma(grid.nx, grid.nz, alpha, mu) @ mt


def pcg(apply_H, rhs, apply_Minv, x0, rtol, maxiter):
    """Preconditioned conjugate gradients for H rho = rhs (Section 'Preconditioning the
    Hessian'); stops when ||r_n|| / ||r_0|| <= rtol.  Returns (x, n_matvec, relres).
    The initial residual costs one product with H (x0 = 1 in the paper, Section 4)."""
    x = np.array(x0, dtype=np.float64)
    r = rhs - apply_H(x)
    nmv = 1
    r0 = np.linalg.norm(r)
    z = apply_Minv(r)
    p = z.copy()
    rz = r @ z
    rel = 1.0 if r0 > 0 else 0.0
    for _ in range(maxiter):
        if r0 == 0 or np.linalg.norm(r) <= rtol * r0:
            break
        Hp = apply_H(p)
        nmv += 1
        a = rz / (p @ Hp)
        x = x + a * p
        r = r - a * Hp
        z = apply_Minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    rel = np.linalg.norm(r) / r0 if r0 > 0 else 0.0
    return x, nmv, rel


def hypergradient(grid: Grid, m_fwi, m_true, omegas, src_xz, rec_xz, alpha, alpha0, mu,
                  rec_w=None, src_amp=None, cg_rtol=1e-13, cg_maxiter=500, cg_fixed_iters=None,
                  x0=None, data_grid=None, m_true_data=None):
    """Upper-level derivatives for one training model (Algorithm alg:box, Theorems
    sogradt1 and sogradta), evaluated at the given m_fwi:
        rho solves H rho = m' - m_fwi by PCG with P2 = Gamma(alpha0, mu) (Eq. (P2)),
            initial guess the all-ones vector (Section 4);
        tau = A^{-1} (g u rho) (Eq. (tau_def));
        dpsi/dp_{j,l} = sum_{s,w} w_j^2 Re[conj((dR_l tau)_j) (R(u - u'))_j
                                            + conj((R tau)_j) (dR_l (u - u'))_j];
        dpsi/dalpha = m_fwi^T R rho (Eq. (sograda));
        dpsi/dw_j = -sum 2 w_j Re[conj((R tau)_j) (R(u' - u))_j] (receiver weights; not
            in the paper, reduces to it for w = 1);
        psi = 1/2 ||m' - m_fwi||^2 (Eq. (SOobj) for one model).
    Reading of Eq. (gradALT1): the conjugated form that the proof of Theorem sogradt1
    yields with the paper's inner product (f, delta_r) = f(r).
    data_grid, m_true_data: the training data u' computed on another grid of the same domain
    (Appendix, data generation: u(m) and u(m') on different grids against the inverse crime),
    with m' given on it; the data and their receiver derivatives are then that grid's:
    R(u - u') reads R u - R_d u'_d and dR_l(u - u') reads dR_l u - dR_{d,l} u'_d.  m_true
    stays the model on this grid (psi and the right-hand side of the rho system).
    Returns a dict (the 1/N_m' average over models is left to the caller)."""
    m_fwi = np.asarray(m_fwi, dtype=np.float64)
    R, Rx, Rz = restriction(grid, rec_xz)
    w = np.ones(R.shape[0]) if rec_w is None else np.asarray(rec_w, dtype=np.float64)
    if data_grid is None:
        data, Ut = synthetic_data(grid, m_true, omegas, src_xz, rec_xz, src_amp)
    else:   # receiver values d and dR_l u' of the data grid's wavefields
        Rd, Rdx, Rdz = restriction(data_grid, rec_xz)
        data, Ud = synthetic_data(data_grid, m_true_data, omegas, src_xz, rec_xz, src_amp)
        dRd = [np.einsum("rn,wsn->wsr", Rl.toarray(), Ud) for Rl in (Rdx, Rdz)]
    phi, grad, fields = fwi_objective_gradient(grid, m_fwi, omegas, src_xz, rec_xz, data, alpha, mu,
                                               rec_w=w, src_amp=src_amp, return_fields=True)
    U = fields["U"]
    P2 = gamma(grid.nx, grid.nz, alpha0, mu)
    P2lu = spla.splu(P2.tocsc())
    rhs = np.asarray(m_true, dtype=np.float64) - m_fwi
    x0 = np.ones(grid.N) if x0 is None else x0
    Hop = lambda v: hessian_vec(grid, m_fwi, omegas, fields, v, alpha, mu)
    if cg_fixed_iters is not None:
        rho, nmv, rel = pcg(Hop, rhs, P2lu.solve, x0, 0.0, cg_fixed_iters)
    else:
        rho, nmv, rel = pcg(Hop, rhs, P2lu.solve, x0, cg_rtol, cg_maxiter)
    dp = np.zeros((R.shape[0], 2))
    dw = np.zeros(R.shape[0])
    for q, om in enumerate(omegas):
        gk = g_vec(grid, m_fwi, om)
        T = fields["facs"][q].solve(gk[None, :] * U[q] * rho[None, :])
        Rt = (R @ T.T).T                         # [n_src, n_rec]
        if data_grid is None:
            du = U[q] - Ut[q]                    # u - u'
            Rdu = (R @ du.T).T
        else:
            Rdu = (R @ U[q].T).T - data[q]
        for l, Rl in enumerate((Rx, Rz)):
            Rlt = (Rl @ T.T).T
            Rldu = (Rl @ du.T).T if data_grid is None else (Rl @ U[q].T).T - dRd[l][q]
            dp[:, l] += (w ** 2) * np.sum(np.real(np.conj(Rlt) * Rdu + np.conj(Rt) * Rldu), axis=0)
        dw += -2.0 * w * np.sum(np.real(np.conj(Rt) * (-Rdu)), axis=0)
    return {
        "psi": 0.5 * np.sum(rhs ** 2),
        "dpsi_dalpha": m_fwi @ (regulariser(grid.nx, grid.nz) @ rho),
        "dpsi_dp": dp,
        "dpsi_dw": dw,
        "rho": rho,
        "cg_matvecs": nmv,
        "cg_relres": rel,
        "phi": phi,
        "grad": grad,
    }
