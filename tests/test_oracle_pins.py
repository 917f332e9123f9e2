"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(five-point / ghost-point finite-difference rows, the discrete plane wave and its
dispersion relation, Lagrange-cubic weights), brute force (hand-written dense
Gaussian elimination, a Hessian formed entry by entry from explicit derivatives,
a Newton-solved lower level), invariants (symmetry, reciprocity, adjoint
identities, partition of unity) and finite differences.  A few tests plant a
plausible mistake in the oracle and check that a pin catches it.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import helmholtz as H
from oracle import dense as D
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------- operator pins

def fd_ghost_point_matrix(nx, nz, lx, lz, m, omega):
    """Five-point FD rows of -(Lap + w^2 m) u = f with the first-order absorbing condition
    du/dn - i sqrt(m) w u = 0 imposed by centred ghost points, each row scaled by the
    area hx*hz*(1/2 on an x-boundary)*(1/2 on a z-boundary).  Written from the PDE of
    Definition def:solnop, independently of the finite-element assembly."""
    hx, hz = lx / (nx - 1), lz / (nz - 1)
    N = nx * nz
    A = np.zeros((N, N), dtype=complex)
    for i in range(nx):
        for j in range(nz):
            k = i * nz + j
            s = hx * hz * (0.5 if i in (0, nx - 1) else 1.0) * (0.5 if j in (0, nz - 1) else 1.0)
            sq = math.sqrt(m[k])
            row = {}

            def add(kk, v):
                row[kk] = row.get(kk, 0) + v
            # x direction: (2u - u_w - u_e)/hx^2; a missing neighbour is a ghost point,
            # u_ghost = u_inner + 2 h i w sqrt(m) u (outward derivative = i w sqrt(m) u)
            for (n1, n2, h, ok_lo, ok_hi, step) in ((i, nx, hx, i > 0, i < nx - 1, nz), (j, nz, hz, j > 0, j < nz - 1, 1)):
                add(k, 2.0 / h ** 2)
                lo = k - step if ok_lo else None
                hi = k + step if ok_hi else None
                if lo is None:
                    add(hi, -1.0 / h ** 2)
                    add(hi, -1.0 / h ** 2)
                    add(k, -2.0 * h * 1j * omega * sq / h ** 2)
                elif hi is None:
                    add(lo, -1.0 / h ** 2)
                    add(lo, -1.0 / h ** 2)
                    add(k, -2.0 * h * 1j * omega * sq / h ** 2)
                else:
                    add(lo, -1.0 / h ** 2)
                    add(hi, -1.0 / h ** 2)
            add(k, -omega ** 2 * m[k])
            for kk, v in row.items():
                A[k, kk] += s * v
    return A


@pytest.mark.parametrize("nx,nz,lx,lz", [(6, 5, 1.0, 1.0), (7, 9, 2.0, 0.7)])
def test_operator_equals_ghost_point_fd(nx, nz, lx, lz):
    rng = np.random.default_rng(1)
    m = rng.uniform(0.3, 1.2, nx * nz)
    g = H.Grid(nx, nz, lx, lz)
    A = H.helmholtz_matrix(g, m, 7.3).toarray()
    F = fd_ghost_point_matrix(nx, nz, lx, lz, m, 7.3)
    assert np.max(np.abs(A - F)) <= 1e-12 * np.max(np.abs(F))


def test_stiffness_orientation_free_and_row_sums():
    S1 = H.stiffness(7, 6, 1.3, 0.8, "up").toarray()
    S2 = H.stiffness(7, 6, 1.3, 0.8, "down").toarray()
    assert np.allclose(S1, S2, atol=1e-13)
    assert np.allclose(S1.sum(axis=1), 0, atol=1e-13)
    assert np.allclose(S1, S1.T)
    # five nonzeros per interior row: no hypotenuse couplings for right triangles
    k = 3 * 6 + 2
    assert np.count_nonzero(np.abs(S1[k]) > 1e-14) == 5


@pytest.mark.parametrize("lumping", ["up", "down"])
def test_triangle_lumping_closed_forms(lumping):
    """Mass lumped on the triangles themselves (the orientation reading): the row sums of the
    consistent P1 mass matrix (each triangle: area/12 (1 + delta_ab), a textbook closed form)
    equal the lumped weights; interior and edge nodes keep the tensor trapezoid's weights, the
    four corners get hx hz / 3 where the cutting diagonal ends and hx hz / 6 elsewhere; the
    weights sum to the domain's area."""
    nx, nz, lx, lz = 7, 6, 1.3, 0.8
    hx, hz = lx / (nx - 1), lz / (nz - 1)
    d = H.lumped_mass(nx, nz, lx, lz, lumping)
    t = H.lumped_mass(nx, nz, lx, lz, "tensor")
    M = np.zeros((nx * nz, nx * nz))
    for i in range(nx - 1):
        for j in range(nz - 1):
            k00, k10, k01, k11 = i * nz + j, (i + 1) * nz + j, i * nz + j + 1, (i + 1) * nz + j + 1
            tris = [(k00, k10, k11), (k00, k11, k01)] if lumping == "up" else [(k00, k10, k01), (k10, k11, k01)]
            for tri in tris:
                for a in tri:
                    for b in tri:
                        M[a, b] += (hx * hz / 2) / 12 * (2.0 if a == b else 1.0)
    assert np.allclose(M.sum(axis=1), d, rtol=1e-13, atol=0)
    corners = {(0, 0): 0, (nx - 1, 0): 1, (0, nz - 1): 2, (nx - 1, nz - 1): 3}
    on_diag = {0, 3} if lumping == "up" else {1, 2}
    for (i, j), c in corners.items():
        assert np.isclose(d[i * nz + j], hx * hz / (3.0 if c in on_diag else 6.0), rtol=1e-14)
    mask = np.ones(nx * nz, bool)
    mask[[i * nz + j for (i, j) in corners]] = False
    assert np.allclose(d[mask], t[mask], rtol=1e-14, atol=0)
    assert np.isclose(d.sum(), lx * lz, rtol=1e-14)
    # the two orientations are mirror images in x
    other = H.lumped_mass(nx, nz, lx, lz, "down" if lumping == "up" else "up")
    assert np.allclose(d.reshape(nx, nz)[::-1], other.reshape(nx, nz), rtol=1e-14, atol=0)


def test_quadrature_weights_sum_to_area_and_perimeter():
    g = H.Grid(9, 6, 2.0, 0.75)
    assert np.isclose(g.d.sum(), 2.0 * 0.75)
    assert np.isclose(g.b.sum(), 2 * (2.0 + 0.75))
    inner = np.zeros((9, 6), bool)
    inner[1:-1, 1:-1] = True
    assert np.all(g.b.reshape(9, 6)[inner] == 0)
    assert np.isclose(g.d.reshape(9, 6)[0, 0], g.hx * g.hz / 4)


def _plane_wave(nx, nz, lx, lz, m0, omega, kx):
    hx, hz = lx / (nx - 1), lz / (nz - 1)
    # discrete dispersion relation (hz/hx)(2 - 2cos kx hx) + (hx/hz)(2 - 2cos kz hz) = w^2 m hx hz
    c = 1 - (omega ** 2 * m0 * hx * hz - (hz / hx) * (2 - 2 * np.cos(kx * hx))) / (2 * hx / hz)
    kz = np.arccos(c) / hz
    X = np.repeat(np.arange(nx) * hx, nz)
    Z = np.tile(np.arange(nz) * hz, nx)
    return np.exp(1j * (kx * X + kz * Z))


def test_discrete_plane_wave_annihilated_in_interior():
    nx, nz, lx, lz, m0, om = 20, 17, 1.0, 0.8, 0.9, 12.0
    g = H.Grid(nx, nz, lx, lz)
    A = H.helmholtz_matrix(g, np.full(g.N, m0), om)
    u = _plane_wave(nx, nz, lx, lz, m0, om, kx=5.0)
    r = (A @ u).reshape(nx, nz)
    assert np.max(np.abs(r[1:-1, 1:-1])) < 1e-12
    assert np.max(np.abs(r[0, :])) > 1e-3      # boundary rows are not annihilated


def test_manufactured_plane_wave_solution():
    nx, nz, m0, om = 24, 21, 1.1, 15.0
    g = H.Grid(nx, nz)
    A = H.helmholtz_matrix(g, np.full(g.N, m0), om)
    u = _plane_wave(nx, nz, 1.0, 1.0, m0, om, kx=7.0)
    x = H.Factor(A).solve((A @ u)[None, :])[0]
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-10


# --------------------------------------------------------------------- solve pins

def test_sparse_lu_matches_handwritten_gauss():
    w = W.tiny_case(9, 8, seed=3)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    A = H.helmholtz_matrix(g, w.m, 6.0)
    rng = np.random.default_rng(0)
    B = rng.standard_normal((3, g.N)) + 1j * rng.standard_normal((3, g.N))
    f = H.Factor(A)
    X = f.solve(B)
    Xd = D.gauss_solve(A.toarray(), B.T).T
    assert np.max(np.abs(X - Xd)) <= 1e-12 * np.max(np.abs(Xd))
    Y = f.adjoint_solve(B)
    Yd = D.gauss_solve(A.toarray().conj().T, B.T).T
    assert np.max(np.abs(Y - Yd)) <= 1e-12 * np.max(np.abs(Yd))


def test_symmetry_reciprocity_and_adjoint_identity():
    w = W.tiny_case(10, 9, seed=4)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    A = H.helmholtz_matrix(g, w.m, 5.0)
    assert abs(A - A.T).max() == 0
    f = H.Factor(A)
    # node-source reciprocity u_s(r) = u_r(s)
    s, r = 2 * g.nz + 0, 7 * g.nz + 5
    es = np.zeros(g.N); es[s] = 1
    er = np.zeros(g.N); er[r] = 1
    us, ur = f.solve(es)[0], f.solve(er)[0]
    assert abs(us[r] - ur[s]) <= 1e-13 * abs(us[r])
    # restricted reciprocity R_a A^{-1} R_b^T = (R_b A^{-1} R_a^T)^T
    Ra, _, _ = H.restriction(g, [[0.31, 0.22], [0.55, 0.6]])
    Rb, _, _ = H.restriction(g, [[0.73, 0.41], [0.2, 0.7], [0.5, 0.5]])
    Mab = Ra @ f.solve(Rb.toarray()).T
    Mba = Rb @ f.solve(Ra.toarray()).T
    assert np.max(np.abs(Mab - Mba.T)) <= 1e-12 * np.max(np.abs(Mab))
    # <A^{-1} b, c> = <b, A^{-H} c>
    rng = np.random.default_rng(5)
    b = rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)
    c = rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)
    lhs = np.vdot(c, f.solve(b)[0])
    rhs = np.vdot(f.adjoint_solve(c)[0], b)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# --------------------------------------------------------------- restriction pins

def test_cubic_weights_golden_values():
    gold = json.load(open(os.path.join(GOLDEN, "cubic_weights.json")))
    for case in gold["cases"]:
        L, dL = H.lagrange_cubic(case["s"])
        assert np.allclose(L, [eval(v) for v in case["L"]], atol=1e-15)
        assert np.allclose(dL, [eval(v) for v in case["dL"]], atol=1e-14)


def test_cubic_weights_closed_form():
    for s in np.linspace(-0.3, 3.3, 37):
        L, _ = H.lagrange_cubic(s)
        ref = [-(s - 1) * (s - 2) * (s - 3) / 6, s * (s - 2) * (s - 3) / 2,
               -s * (s - 1) * (s - 3) / 2, s * (s - 1) * (s - 2) / 6]
        assert np.allclose(L, ref, atol=1e-14)


def test_sliding_window_rule_of_the_figures():
    # p in [x1, x2] -> x0..x3 ; p in [x2, x3] -> x1..x4 ; clamped at the ends
    assert H.cubic_window(1.4, 10) == 0
    assert H.cubic_window(2.6, 10) == 1
    assert H.cubic_window(0.2, 10) == 0
    assert H.cubic_window(8.7, 10) == 6
    assert H.cubic_window(9.0, 10) == 6


def test_restriction_exact_on_bicubic_polynomials():
    g = H.Grid(11, 9, 1.2, 0.9)
    xz = H.node_xz(g.nx, g.nz, g.lx, g.lz)
    p = lambda x, z: x ** 3 - 2 * x * z ** 2 + 0.5 * z ** 3 + x ** 2 * z ** 3 - 1.0
    px = lambda x, z: 3 * x ** 2 - 2 * z ** 2 + 2 * x * z ** 3
    pz = lambda x, z: -4 * x * z + 1.5 * z ** 2 + 3 * x ** 2 * z ** 2
    rec = np.array([[0.03, 0.05], [0.61, 0.33], [1.19, 0.88], [0.5, 0.0], [0.37, 0.9]])
    R, Rx, Rz = H.restriction(g, rec)
    vals = p(xz[:, 0], xz[:, 1])
    assert np.allclose(R @ vals, p(rec[:, 0], rec[:, 1]), atol=1e-12)
    assert np.allclose(Rx @ vals, px(rec[:, 0], rec[:, 1]), atol=1e-10)
    assert np.allclose(Rz @ vals, pz(rec[:, 0], rec[:, 1]), atol=1e-10)
    assert np.allclose(np.asarray(R.sum(axis=1)).ravel(), 1.0)
    assert np.allclose(np.asarray(Rx.sum(axis=1)).ravel(), 0.0, atol=1e-10)


def test_restriction_continuous_across_nodes():
    g = H.Grid(10, 10)
    u = np.random.default_rng(2).standard_normal(g.N)
    x_node = 3 * g.hx
    a, _, _ = H.restriction(g, [[x_node - 1e-12, 0.43]])
    b, _, _ = H.restriction(g, [[x_node + 1e-12, 0.43]])
    assert abs((a @ u)[0] - (b @ u)[0]) < 1e-9


def test_regulariser_stencil_and_spectrum():
    nx, nz = 6, 5
    Rg = H.regulariser(nx, nz).toarray()
    assert np.allclose(Rg, Rg.T)
    assert np.allclose(Rg @ np.ones(nx * nz), 0)
    # eigenvalues (nx-1)^2 (2 - 2 cos(pi a / nx)) + (nz-1)^2 (2 - 2 cos(pi b / nz))
    lam = np.sort(np.add.outer((nx - 1) ** 2 * (2 - 2 * np.cos(np.pi * np.arange(nx) / nx)),
                               (nz - 1) ** 2 * (2 - 2 * np.cos(np.pi * np.arange(nz) / nz))).ravel())
    assert np.allclose(np.sort(np.linalg.eigvalsh(Rg)), lam, atol=1e-9)
    # interior stencil
    k = 2 * nz + 2
    assert np.isclose(Rg[k, k], 2 * (nx - 1) ** 2 + 2 * (nz - 1) ** 2)
    assert np.isclose(Rg[k, k + nz], -(nx - 1) ** 2)
    assert np.isclose(Rg[k, k + 1], -(nz - 1) ** 2)


def test_source_vector_on_node_is_unit_vector():
    g = H.Grid(8, 7)
    E = H.source_vectors(g, [[3 * g.hx, 0.0], [2 * g.hx, 4 * g.hz]])
    assert E[0, 3 * 7 + 0] == 1 and np.count_nonzero(E[0]) == 1
    assert E[1, 2 * 7 + 4] == 1 and np.count_nonzero(E[1]) == 1


def test_off_grid_source_weights_reproduce_bilinear_functions():
    """Reading for off-grid sources: the bilinear (hat-function) weights of the containing cell.
    They reproduce every bilinear function f = a + b x + c z + d x z exactly (E f = f(p)), are
    non-negative with 4 nonzeros, sum to the amplitude, and put weight 1 on the node at the
    far corner (x = lx, z = lz).  Swapping the weights of a cell (a plausible slip) fails."""
    g = H.Grid(9, 7, 1.3, 0.8)
    X = np.repeat(np.arange(g.nx) * g.hx, g.nz)
    Z = np.tile(np.arange(g.nz) * g.hz, g.nx)
    rng = np.random.default_rng(3)
    pts = np.stack([rng.uniform(0, g.lx, 20), rng.uniform(0, g.lz, 20)], axis=1)
    E = H.source_vectors(g, pts, np.full(20, 2.5))
    for a, b, c, d in ((1.0, 0, 0, 0), (0, 1.0, 0, 0), (0, 0, 1.0, 0), (0.3, -1.2, 0.7, 2.0)):
        f = a + b * X + c * Z + d * X * Z
        assert np.allclose(np.real(E @ f), 2.5 * (a + b * pts[:, 0] + c * pts[:, 1] + d * pts[:, 0] * pts[:, 1]),
                           rtol=1e-13, atol=1e-13)
    assert np.all(np.real(E) >= 0) and np.all(np.count_nonzero(E, axis=1) <= 4)
    assert np.allclose(E.sum(axis=1), 2.5, rtol=1e-14)
    corner = H.source_vectors(g, [[g.lx, g.lz]])
    assert corner[0, g.N - 1] == 1 and np.count_nonzero(corner) == 1
    # planted slip: swapping the two x-weights of every cell breaks the linear reproduction
    Es = np.zeros_like(E)
    for q, (x, z) in enumerate(pts):
        i0 = min(int(x / g.hx), g.nx - 2)
        j0 = min(int(z / g.hz), g.nz - 2)
        fx, fz = x / g.hx - i0, z / g.hz - j0
        for di, wx in ((0, fx), (1, 1 - fx)):
            for dj, wz in ((0, 1 - fz), (1, fz)):
                Es[q, (i0 + di) * g.nz + j0 + dj] += wx * wz
    assert not np.allclose(np.real(Es @ X), pts[:, 0], atol=1e-6)


def test_receiver_data_converge_at_second_order():
    """Data of a smooth model on refined grids (same physical sources, receivers and model
    function) approach the data of a fine reference grid at second order in h, the order of the
    P1 elements with nodal quadrature.  Halving h divides the error by about 4 (the error of
    the 193 x 193 reference is 4-5x below that of the finest grid checked).  This also shows
    that data from another grid (inverse-crime avoidance) fit through the same restriction."""
    c = lambda X, Z: 1.0 + 0.3 * np.exp(-((X - 0.5) ** 2 + (Z - 0.55) ** 2) / 0.04)   # noqa: E731
    src = np.array([[0.25, 0.0], [0.75, 0.0]])
    rec = np.stack([np.full(7, 0.9), np.linspace(0.1, 0.9, 7)], axis=1)
    om = [4.0, 8.0]

    def data(n):
        g = H.Grid(n, n, 1.0, 1.0)
        return H.synthetic_data(g, W.sample_on_grid(lambda X, Z: 1.0 / c(X, Z) ** 2, n, n), om, src, rec)[0]

    ref = data(193)
    err = [np.linalg.norm(data(n) - ref) / np.linalg.norm(ref) for n in (13, 25, 49)]
    for coarse, fine in zip(err, err[1:]):
        assert 3.5 <= coarse / fine <= 4.6


# ------------------------------------------------------------------ derivative pins

def _tiny_fwi(seed=0, nx=8, nz=7):
    w = W.tiny_case(nx, nz, seed=seed)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz)
    return w, g, data


def test_gradient_matches_central_differences():
    w, g, data = _tiny_fwi()
    f = lambda m: H.fwi_objective_gradient(g, m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu)
    phi, grad = f(w.m)
    rng = np.random.default_rng(11)
    for _ in range(5):
        dm = rng.standard_normal(g.N) * w.m
        dm /= np.linalg.norm(dm)
        h = 1e-5 * np.linalg.norm(w.m)
        fd = (f(w.m + h * dm)[0] - f(w.m - h * dm)[0]) / (2 * h)
        assert abs(fd - grad @ dm) <= 1e-6 * max(abs(fd), np.linalg.norm(grad) * 1e-3)


def test_gradient_taylor_remainder_is_second_order():
    w, g, data = _tiny_fwi(seed=1)
    f = lambda m: H.fwi_objective_gradient(g, m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu)
    phi, grad = f(w.m)
    dm = np.random.default_rng(3).standard_normal(g.N) * w.m * 0.05
    r = [abs(f(w.m + t * dm)[0] - phi - t * grad @ dm) for t in (1e-1, 5e-2, 2.5e-2)]
    assert 3.0 < r[0] / r[1] < 5.0 and 3.0 < r[1] / r[2] < 5.0


def test_weighted_gradient_matches_differences():
    w, g, data = _tiny_fwi(seed=2)
    rw = np.array([0.7, 1.3, 1.1])
    f = lambda m: H.fwi_objective_gradient(g, m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu, rec_w=rw)
    _, grad = f(w.m)
    dm = np.random.default_rng(4).standard_normal(g.N) * w.m
    dm /= np.linalg.norm(dm)
    h = 1e-5
    fd = (f(w.m + h * dm)[0] - f(w.m - h * dm)[0]) / (2 * h)
    assert abs(fd - grad @ dm) <= 1e-6 * abs(fd)


def test_data_model_has_zero_misfit():
    w, g, data = _tiny_fwi(seed=3)
    phi, grad = H.fwi_objective_gradient(g, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu)
    G = H.gamma(g.nx, g.nz, w.alpha, w.mu)
    assert np.isclose(phi, 0.5 * w.m_true @ (G @ w.m_true), rtol=1e-12)
    assert np.allclose(grad, G @ w.m_true, rtol=1e-9, atol=1e-12)


def test_hessian_vec_matches_dense_hessian_and_differences():
    w, g, data = _tiny_fwi(seed=5, nx=7, nz=6)
    args = (g, w.m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu)
    _, grad, fields = H.fwi_objective_gradient(*args, return_fields=True)
    Hd = D.dense_hessian(*args)
    assert np.max(np.abs(Hd - Hd.T)) <= 1e-10 * np.max(np.abs(Hd))
    rng = np.random.default_rng(6)
    mt = rng.standard_normal(g.N)
    Hv = H.hessian_vec(g, w.m, w.omegas, fields, mt, w.alpha, w.mu)
    assert np.linalg.norm(Hv - Hd @ mt) <= 1e-9 * np.linalg.norm(Hd @ mt)
    h = 1e-6
    gp = H.fwi_objective_gradient(g, w.m + h * mt, *args[2:])[1]
    gm = H.fwi_objective_gradient(g, w.m - h * mt, *args[2:])[1]
    fd = (gp - gm) / (2 * h)
    assert np.linalg.norm(fd - Hv) <= 1e-6 * np.linalg.norm(Hv)
    a, b = rng.standard_normal(g.N), rng.standard_normal(g.N)
    Ha = H.hessian_vec(g, w.m, w.omegas, fields, a, w.alpha, w.mu)
    Hb = H.hessian_vec(g, w.m, w.omegas, fields, b, w.alpha, w.mu)
    assert abs(b @ Ha - a @ Hb) <= 1e-10 * abs(b @ Ha)


def test_gauss_newton_part_is_positive_semidefinite():
    w, g, data = _tiny_fwi(seed=6, nx=6, nz=6)
    _, _, fields = H.fwi_objective_gradient(g, w.m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, 0.0, 0.0,
                                            return_fields=True)
    H1 = np.stack([H.hessian_vec(g, w.m, w.omegas, fields, e, 0.0, 0.0, gauss_newton=True)
                   for e in np.eye(g.N)], axis=1)
    assert np.allclose(H1, H1.T, atol=1e-10 * np.abs(H1).max())
    assert np.linalg.eigvalsh(0.5 * (H1 + H1.T)).min() >= -1e-10 * np.abs(H1).max()


def test_statement_form_G_instead_of_Gstar_is_caught():
    """Lemma thm:H2's statement has G lambda where its proof has G^* lambda; the pin
    (finite differences of the gradient) must reject the statement's form, computed
    here inline with conj(g) replaced by g in the right-hand side of z."""
    w, g, data = _tiny_fwi(seed=5, nx=7, nz=6)
    args = (g, w.m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu)
    _, _, fields = H.fwi_objective_gradient(*args, return_fields=True)
    mt = np.random.default_rng(6).standard_normal(g.N)
    h = 1e-6
    fd = (H.fwi_objective_gradient(g, w.m + h * mt, *args[2:])[1]
          - H.fwi_objective_gradient(g, w.m - h * mt, *args[2:])[1]) / (2 * h)
    bad = H.gamma(g.nx, g.nz, w.alpha, w.mu) @ mt
    for q, om in enumerate(w.omegas):
        gk, gp = H.g_vec(g, w.m, om), H.g_prime_vec(g, w.m, om)
        U, Lam, f, R = fields["U"][q], fields["Lam"][q], fields["facs"][q], fields["R"]
        V = f.solve(gk * U * mt)
        Z = f.adjoint_solve((R.T @ (R @ V.T)).T - mt * gk * Lam)
        bad += np.real(np.sum(gk * U * np.conj(Z) - gk * V * np.conj(Lam) - gp * U * np.conj(Lam) * mt, axis=0))
    good = H.hessian_vec(g, w.m, w.omegas, fields, mt, w.alpha, w.mu)
    assert np.linalg.norm(fd - good) <= 1e-6 * np.linalg.norm(fd)
    assert np.linalg.norm(fd - bad) > 1e-4 * np.linalg.norm(fd)


def test_planted_mistake_dropped_boundary_term_is_caught(monkeypatch):
    w, g, data = _tiny_fwi(seed=0)
    f = lambda m: H.fwi_objective_gradient(g, m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu)
    good = H.g_vec
    monkeypatch.setattr(H, "g_vec", lambda grid, m, om: om ** 2 * grid.d + 0j)
    _, grad = f(w.m)
    monkeypatch.setattr(H, "g_vec", good)
    dm = np.zeros(g.N)
    dm[0] = 1.0                     # a corner node: boundary term matters
    h = 1e-6
    fd = (f(w.m + h * dm)[0] - f(w.m - h * dm)[0]) / (2 * h)
    assert abs(fd - grad @ dm) > 1e-4 * abs(fd)


# -------------------------------------------------------------- hypergradient pins

def _hyper_setup(seed=7, nx=7, nz=6):
    # an over-determined tiny problem (4 sources, 12 receivers, 3 frequencies) so that
    # the lower level has a well-conditioned minimiser near m' for the Newton solve
    w = W.tiny_case(nx, nz, seed=seed, n_omega=3, n_src=4, n_rec=12)
    w.alpha, w.mu = 1e-4, 1e-4
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    return w, g


def _psi(w, g, alpha, rec_xz, rec_w=None):
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, rec_xz)
    m_fwi, gn = D.lower_level_newton(g, w.m_true, w.omegas, w.acq.src_xz, rec_xz, data, alpha, w.mu, rec_w=rec_w)
    assert gn < 1e-10
    return 0.5 * np.sum((w.m_true - m_fwi) ** 2), m_fwi


def test_hypergradient_implicit_function_check():
    """dpsi/dalpha and dpsi/dp from Algorithm alg:box against central differences of psi,
    re-solving the lower level (Newton, dense Hessian) at every perturbed design."""
    w, g = _hyper_setup()
    rec = w.acq.rec_xz.copy()
    rw = np.linspace(0.8, 1.2, 12)
    psi0, m_fwi = _psi(w, g, w.alpha, rec, rw)
    hg = H.hypergradient(g, m_fwi, w.m_true, w.omegas, w.acq.src_xz, rec, w.alpha, w.alpha, w.mu,
                         rec_w=rw, cg_rtol=1e-14)
    assert np.isclose(hg["psi"], psi0, rtol=1e-12)
    da = 1e-3 * w.alpha
    fd_a = (_psi(w, g, w.alpha + da, rec, rw)[0] - _psi(w, g, w.alpha - da, rec, rw)[0]) / (2 * da)
    assert abs(fd_a - hg["dpsi_dalpha"]) <= 1e-5 * abs(fd_a)
    for j, l in ((0, 0), (1, 1), (2, 0)):
        dp = 1e-5
        rp, rm = rec.copy(), rec.copy()
        rp[j, l] += dp
        rm[j, l] -= dp
        fd_p = (_psi(w, g, w.alpha, rp, rw)[0] - _psi(w, g, w.alpha, rm, rw)[0]) / (2 * dp)
        assert abs(fd_p - hg["dpsi_dp"][j, l]) <= 1e-5 * max(abs(fd_p), 1e-3 * np.abs(hg["dpsi_dp"]).max())
    j = 1
    dw = 1e-5
    wp, wm = rw.copy(), rw.copy()
    wp[j] += dw
    wm[j] -= dw
    fd_w = (_psi(w, g, w.alpha, rec, wp)[0] - _psi(w, g, w.alpha, rec, wm)[0]) / (2 * dw)
    assert abs(fd_w - hg["dpsi_dw"][j]) <= 1e-5 * abs(fd_w)


def _fine_setup(nx=7, nz=6, fx=13, fz=11, seed=7):
    """The tiny over-determined problem with a smooth m' known everywhere, so that it can be
    sampled on the inversion grid and on a finer data grid of the same domain."""
    w = W.tiny_case(nx, nz, seed=seed, n_omega=3, n_src=4, n_rec=12)
    w.alpha, w.mu = 1e-4, 1e-4
    fn = lambda X, Z: 1.0 / (1.2 + 0.8 * Z + 0.3 * np.sin(3.0 * X) * Z) ** 2
    g, gd = H.Grid(nx, nz, w.lx, w.lz), H.Grid(fx, fz, w.lx, w.lz)
    m = W.sample_on_grid(fn, nx, nz, w.lx, w.lz)
    md = W.sample_on_grid(fn, fx, fz, w.lx, w.lz)
    return w, g, gd, m, md


def _psi_fine(w, g, gd, m, md, alpha, rec_xz):
    data, _ = H.synthetic_data(gd, md, w.omegas, w.acq.src_xz, rec_xz)
    m_fwi, gn = D.lower_level_newton(g, m, w.omegas, w.acq.src_xz, rec_xz, data, alpha, w.mu)
    assert gn < 1e-10
    return 0.5 * np.sum((m - m_fwi) ** 2), m_fwi


def test_hypergradient_with_data_from_a_finer_grid_implicit_function_check():
    """Training data computed on a finer grid (u(m') on 13 x 11 nodes, the inversion on 7 x 6):
    dpsi/dalpha and dpsi/dp against central differences of psi, the lower level re-solved
    with the finer grid's data at every perturbed design.  The data no longer fit exactly at
    m_FWI, so the Hessian's second-order part and the data-grid receiver derivatives both
    enter."""
    w, g, gd, m, md = _fine_setup()
    rec = w.acq.rec_xz.copy()
    psi0, m_fwi = _psi_fine(w, g, gd, m, md, w.alpha, rec)
    hg = H.hypergradient(g, m_fwi, m, w.omegas, w.acq.src_xz, rec, w.alpha, w.alpha, w.mu, cg_rtol=1e-14,
                         data_grid=gd, m_true_data=md)
    assert np.isclose(hg["psi"], psi0, rtol=1e-12)
    da = 1e-3 * w.alpha
    fd_a = (_psi_fine(w, g, gd, m, md, w.alpha + da, rec)[0] - _psi_fine(w, g, gd, m, md, w.alpha - da, rec)[0]) / (2 * da)
    assert abs(fd_a - hg["dpsi_dalpha"]) <= 1e-5 * abs(fd_a)
    for j, l in ((0, 0), (1, 1), (2, 0)):
        dp = 1e-5
        rp, rm = rec.copy(), rec.copy()
        rp[j, l] += dp
        rm[j, l] -= dp
        fd_p = (_psi_fine(w, g, gd, m, md, w.alpha, rp)[0] - _psi_fine(w, g, gd, m, md, w.alpha, rm)[0]) / (2 * dp)
        assert abs(fd_p - hg["dpsi_dp"][j, l]) <= 1e-5 * max(abs(fd_p), 1e-3 * np.abs(hg["dpsi_dp"]).max())
    # the same-grid data through the data-grid branch reproduce the default branch
    ref = H.hypergradient(g, m_fwi, m, w.omegas, w.acq.src_xz, rec, w.alpha, w.alpha, w.mu, cg_rtol=1e-14)
    same = H.hypergradient(g, m_fwi, m, w.omegas, w.acq.src_xz, rec, w.alpha, w.alpha, w.mu, cg_rtol=1e-14,
                           data_grid=g, m_true_data=m)
    assert np.allclose(same["dpsi_dp"], ref["dpsi_dp"], rtol=1e-10, atol=1e-12 * np.abs(ref["dpsi_dp"]).max())
    assert np.isclose(same["dpsi_dalpha"], ref["dpsi_dalpha"], rtol=1e-12)
    # and the finer data are not the same-grid data: the terms differ
    assert not np.allclose(hg["dpsi_dp"], ref["dpsi_dp"], rtol=1e-3)


def test_unconjugated_gradALT1_fails_the_pin():
    """Eq. (gradALT1) as printed (no conjugates) disagrees with the differences of psi."""
    w, g = _hyper_setup(seed=8)
    rec = w.acq.rec_xz.copy()
    psi0, m_fwi = _psi(w, g, w.alpha, rec)
    hg = H.hypergradient(g, m_fwi, w.m_true, w.omegas, w.acq.src_xz, rec, w.alpha, w.alpha, w.mu, cg_rtol=1e-14)
    # recompute the printed form tau * d(u - u') + d(tau) * (u - u') without conjugates
    data, Ut = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, rec)
    _, _, fields = H.fwi_objective_gradient(g, m_fwi, w.omegas, w.acq.src_xz, rec, data, w.alpha, w.mu,
                                            return_fields=True)
    R, Rx, _ = H.restriction(g, rec)
    printed = 0.0
    for q, om in enumerate(w.omegas):
        T = fields["facs"][q].solve(H.g_vec(g, m_fwi, om)[None, :] * fields["U"][q] * hg["rho"][None, :])
        du = fields["U"][q] - Ut[q]
        printed += np.sum(np.real((R @ T.T)[0] * (Rx @ du.T)[0] + (Rx @ T.T)[0] * (R @ du.T)[0]))
    dp = 1e-5
    rp, rm = rec.copy(), rec.copy()
    rp[0, 0] += dp
    rm[0, 0] -= dp
    fd = (_psi(w, g, w.alpha, rp)[0] - _psi(w, g, w.alpha, rm)[0]) / (2 * dp)
    assert abs(fd - hg["dpsi_dp"][0, 0]) <= 1e-5 * abs(fd)
    assert abs(fd - printed) > 1e-3 * abs(fd)


def test_dpsi_dalpha_algebraic_identity_at_any_m():
    w, g = _hyper_setup(seed=9)
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz)
    m = w.m * 1.02
    hg = H.hypergradient(g, m, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz, w.alpha, w.alpha, w.mu,
                         cg_rtol=1e-14)
    Hd = D.dense_hessian(g, m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, w.alpha, w.mu)
    rho = np.linalg.solve(Hd, w.m_true - m)
    assert np.allclose(hg["rho"], rho, rtol=1e-8, atol=1e-10 * np.abs(rho).max())
    ref = (H.regulariser(g.nx, g.nz) @ m) @ rho
    assert abs(hg["dpsi_dalpha"] - ref) <= 1e-8 * abs(ref)


def test_solve_count_matches_cost_theorem():
    """Theorem thm:cost / Discussion disc:Hess: per (s, w) one hypergradient pass costs
    u and lambda (lower level), 2 per Hessian product, and 1 for tau; the data fields
    u(m') are counted separately."""
    w, g = _hyper_setup(seed=10)
    H.reset_solve_counter()
    n_cg = 4
    hg = H.hypergradient(g, w.m, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz, w.alpha, w.alpha, w.mu,
                         cg_fixed_iters=n_cg)
    n_data = w.acq.n_src * len(w.omegas)
    n_matvec = hg["cg_matvecs"]
    assert n_matvec == n_cg + 1            # initial residual of x0 = 1 plus one per iteration
    assert H.SOLVE_COUNTER["solves"] == n_data + (2 + 2 * n_matvec + 1) * n_data
