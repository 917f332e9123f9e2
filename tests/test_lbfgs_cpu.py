"""CPU checks of the lower-level optimiser (paper_2301_10762_gb300/lbfgs.py): L-BFGS with a
strong Wolfe line search (Section subsec:Quasi; Nocedal & Wright, Algorithms 3.5/3.6, 9.1, 9.2).

Pins: the two-loop recursion equals the dense BFGS inverse-Hessian update applied pair by pair;
every accepted step satisfies both strong Wolfe inequalities, or, where f is flat to rounding,
the approximate Wolfe conditions; the minimisers of a quadratic and of
Rosenbrock's function are reached to ||g|| <= 1e-10, also where f carries rounding noise far
above the decrease of a step (the zoom then brackets by the slope); a domain where the objective is not finite
is backed out of; on a tiny FWI problem (the oracle's phi and grad phi) the minimiser agrees with
SciPy's L-BFGS-B."""
import math

import numpy as np
import pytest

from paper_2301_10762_gb300 import lbfgs as L


def test_two_loop_equals_dense_bfgs_update():
    rng = np.random.default_rng(0)
    n = 7
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    pairs = []
    for _ in range(4):
        s = rng.standard_normal(n)
        y = A @ s
        pairs.append((s, y, 1.0 / (s @ y)))
    gamma = (pairs[-1][0] @ pairs[-1][1]) / (pairs[-1][1] @ pairs[-1][1])
    H = gamma * np.eye(n)
    for s, y, rho in pairs:   # oldest first
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    g = rng.standard_normal(n)
    assert np.allclose(L.two_loop(g, pairs, gamma), H @ g, rtol=1e-12, atol=1e-12)
    # the secant condition of the newest pair: H y = s
    assert np.allclose(L.two_loop(pairs[-1][1], pairs, gamma), pairs[-1][0], rtol=1e-10, atol=1e-12)


def rosenbrock(x):
    f = np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1.0 - x[:-1]) ** 2)
    g = np.zeros_like(x)
    g[:-1] = -400.0 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2.0 * (1.0 - x[:-1])
    g[1:] += 200.0 * (x[1:] - x[:-1] ** 2)
    return f, g


@pytest.mark.parametrize("n", [2, 10])
def test_rosenbrock_minimum_and_wolfe_steps(n):
    c1, c2 = 1e-4, 0.9
    steps = []
    prev = {}

    def fun(x):
        return rosenbrock(x)

    x0 = np.full(n, -1.2)
    x0[1::2] = 1.0

    def cb(k, x, f, g, a):
        steps.append((k, x.copy(), f, g.copy(), a))

    out = L.lbfgs(fun, x0, gtol=1e-10, max_iter=500, c1=c1, c2=c2, callback=cb)
    assert out["converged"] and out["gnorm"] <= 1e-10
    assert np.allclose(out["x"], 1.0, atol=1e-8)
    # strong Wolfe at every accepted step: replay the directions
    x, (f, g) = x0, rosenbrock(x0)
    n_strong = 0
    for k, xn, fn, gn, a in steps:
        p = (xn - x) / a
        dg0, dg = g @ p, gn @ p
        strong = fn <= f + c1 * a * dg0 and abs(dg) <= -c2 * dg0
        approx = fn <= f + 1e-12 * abs(f) and c2 * dg0 <= dg <= (2 * c1 - 1) * dg0
        assert strong or approx, k
        n_strong += strong
        x, f, g = xn, fn, gn
    assert n_strong >= len(steps) - 5   # the approximate conditions only near the minimiser


def test_quadratic_minimiser():
    rng = np.random.default_rng(1)
    n = 30
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T / n + np.eye(n)
    b = rng.standard_normal(n)
    out = L.lbfgs(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b), np.zeros(n), gtol=1e-12, max_iter=300)
    assert out["converged"]
    assert np.linalg.norm(out["x"] - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(np.linalg.solve(A, b))


def test_converges_where_f_is_flat_to_rounding():
    # a quadratic with f carrying deterministic noise of 1e-14 |f| (an objective that is only
    # accurate to rounding, as the FWI misfit is) and an exact gradient: near the minimiser
    # the decrease per step falls far below the noise, so comparisons of f say nothing and the
    # line search has to bracket the step by the slope; ||g|| <= 1e-10 is still reached
    import hashlib
    rng = np.random.default_rng(4)
    n = 12
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T / n + 0.5 * np.eye(n)
    b = rng.standard_normal(n)
    f_min = 1e-2

    def fun(x):
        h = int.from_bytes(hashlib.sha256(np.ascontiguousarray(x).tobytes()).digest()[:8], "little")
        noise = 1e-14 * f_min * (h / 2.0 ** 64 - 0.5)
        return f_min + 0.5 * x @ A @ x - b @ x + noise, A @ x - b

    x_star = np.linalg.solve(A, b)
    out = L.lbfgs(fun, x_star + 1e-3 * rng.standard_normal(n), gtol=1e-10, max_iter=500)
    assert out["converged"], out["message"]
    assert np.linalg.norm(out["x"] - x_star) <= 1e-9


def test_line_search_brackets_by_slope_where_f_is_flat():
    # one dimension, the situation of an L-BFGS step near an FWI minimiser (slope -2.1e-17 at
    # f = 1e-2): the unit step overshoots the minimum of f(a) = f0 + dg0 a + k a^2 / 2 (at
    # a = 3/8, depth 4e-18), and the computed f carries rounding noise of 1e-16, far above that
    # depth but far below eps |f|, so comparisons of f point anywhere.  For 200 noise patterns
    # the search returns a step, and it satisfies the approximate Wolfe conditions (comparing
    # values of f inside the zoom lost the minimum for 30 of them).
    import hashlib
    f_base, dg0, c1, c2 = 1.02e-2, -2.1e-17, 1e-4, 0.9
    kappa = -dg0 / 0.375
    for salt in range(200):
        def fun(x):
            a = float(x[0])
            h = int.from_bytes(hashlib.sha256(np.float64(a).tobytes() + bytes([salt])).digest()[:8], "little")
            noise = 1e-16 * (h / 2.0 ** 64 - 0.5)
            return f_base + dg0 * a + 0.5 * kappa * a * a + noise, np.array([dg0 + kappa * a])

        f0, g0 = fun(np.zeros(1))
        a, f, g, _ = L.wolfe_line_search(fun, np.zeros(1), f0, g0, np.ones(1), alpha0=1.0, c1=c1, c2=c2)
        assert a is not None, salt
        dg = float(g[0])
        strong = f <= f0 + c1 * a * dg0 and abs(dg) <= -c2 * dg0
        approx = f <= f0 + 1e-12 * abs(f0) and c2 * dg0 <= dg <= (2 * c1 - 1) * dg0
        assert strong or approx, salt


def test_steps_out_of_the_domain_are_shortened():
    # f(x) = sum(x - log x) on x > 0 (minimum at 1), infinite elsewhere; the first full steps
    # from far away leave the domain
    def fun(x):
        if np.any(x <= 0):
            return math.inf, np.full_like(x, math.nan)
        return float(np.sum(x - np.log(x))), 1.0 - 1.0 / x

    out = L.lbfgs(fun, np.array([40.0, 0.05, 7.0]), gtol=1e-10, max_iter=200)
    assert out["converged"] and np.allclose(out["x"], 1.0, atol=1e-9)


def test_tiny_fwi_matches_scipy_lbfgsb():
    scipy_opt = pytest.importorskip("scipy.optimize")
    import workloads as W
    from oracle import helmholtz as H
    w = W.tiny_case(nx=9, nz=8, n_omega=2, n_src=2, n_rec=4, seed=3)
    g = H.Grid(w.nx, w.nz, w.lx, w.lz)
    data, _ = H.synthetic_data(g, w.m_true, w.omegas, w.acq.src_xz, w.acq.rec_xz)
    alpha, mu = 1e-3, 1e-6

    def fun(m):
        if np.any(m <= 0):
            return math.inf, np.full_like(m, math.nan)
        return H.fwi_objective_gradient(g, m, w.omegas, w.acq.src_xz, w.acq.rec_xz, data, alpha, mu)

    out = L.lbfgs(fun, w.m, gtol=1e-10, max_iter=400)
    assert out["converged"], out["message"]
    ref = scipy_opt.minimize(fun, w.m, jac=True, method="L-BFGS-B",
                             options={"gtol": 1e-12, "ftol": 1e-16, "maxiter": 2000, "maxcor": 10})
    assert np.linalg.norm(out["x"] - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    assert out["f"] <= ref.fun * (1 + 1e-9) + 1e-15
