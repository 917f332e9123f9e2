"""L-BFGS with a strong Wolfe line search, and the lower-level FWI solve built on it.

The paper minimises the FWI objective phi(m) (Eq. newphi, with the adjoint-state gradient of
Theorem th:grad) by L-BFGS with a Wolfe line search (Section subsec:Quasi: the two-loop recursion
and the limited-memory BFGS iteration, Algorithms 9.1 and 9.2 of Nocedal & Wright), stopping when
||grad phi||_2 <= 1e-10 (the tolerance of its numerical experiments).

The optimiser here is host logic: the iterate, the search directions and the curvature pairs are
numpy vectors.  In `fwi_lower_level` every evaluation of phi and grad phi is the GPU path
(helm_assemble, helm_factor, fwi_misfit_grad), and only the N-vector gradient comes back.

Line search: strong Wolfe conditions
    f(x + a p) <= f(x) + c1 a g.p,    |g(x + a p).p| <= c2 |g.p|,
found by bracketing and zoom (Nocedal & Wright, Algorithms 3.5 and 3.6) with safeguarded cubic
interpolation.  Close to a minimiser the decrease of f per step falls to the rounding level of f
itself (an FP64 objective cannot resolve ||g|| = 1e-10 through f), so a step is also accepted on
the approximate Wolfe conditions of Hager & Zhang (2005):
    f(x + a p) <= f(x) + eps |f(x)|   and   c2 g.p <= g(x + a p).p <= (2 c1 - 1) g.p,
which test the slope instead; where f is flat in that sense the zoom also keeps the step
bracketed by the sign of the slope rather than by comparing values of f (their interval update).  A trial point where the objective is not finite (a model with
m <= 0, where sqrt(m) is undefined) is treated as a step that is too long.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np


def two_loop(g, pairs, gamma):
    """H g for the L-BFGS inverse-Hessian approximation (two-loop recursion, Algorithm 9.1):
    H0 = gamma I updated by the curvature pairs (s, y, rho = 1 / y.s), oldest first."""
    q = np.array(g, dtype=np.float64, copy=True)
    alphas = []
    for s, y, rho in reversed(pairs):
        a = rho * (s @ q)
        alphas.append(a)
        q -= a * y
    r = gamma * q
    for (s, y, rho), a in zip(pairs, reversed(alphas)):
        b = rho * (y @ r)
        r += (a - b) * s
    return r


def _cubic_min(a, fa, da, b, fb, db):
    """Minimiser of the cubic interpolating f and f' at a and b (None if it does not exist)."""
    if not (math.isfinite(fa) and math.isfinite(fb) and math.isfinite(da) and math.isfinite(db)) or a == b:
        return None
    d1 = da + db - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - da * db
    if disc < 0.0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = db - da + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (db + d2 - d1) / den


def wolfe_line_search(fun, x, f0, g0, p, alpha0=1.0, c1=1e-4, c2=0.9, max_evals=40, alpha_max=1e10,
                      eps_f=1e-12):
    """Step a along p satisfying the strong Wolfe conditions, or the approximate Wolfe
    conditions where f is flat to eps_f |f|.  fun(x) -> (f, g).
    Returns (a, f, g, evaluations); a is None if no such step was found."""
    dg0 = float(g0 @ p)
    if not dg0 < 0.0:
        return None, f0, g0, 0
    n_ev = 0
    flat = eps_f * abs(float(f0))

    def accept(a, f, dg):
        if not math.isfinite(f):
            return False
        if f <= f0 + c1 * a * dg0 and abs(dg) <= -c2 * dg0:
            return True   # strong Wolfe
        return f <= f0 + flat and c2 * dg0 <= dg <= (2.0 * c1 - 1.0) * dg0   # approximate Wolfe

    def phi(a):
        nonlocal n_ev
        n_ev += 1
        f, g = fun(x + a * p)
        f = float(f)
        dg = float(g @ p) if math.isfinite(f) else math.nan
        return f, g, dg

    def zoom(lo, f_lo, dg_lo, g_lo, hi, f_hi, dg_hi):
        while n_ev < max_evals:
            w = hi - lo
            a = _cubic_min(lo, f_lo, dg_lo, hi, f_hi, dg_hi)
            left, right = min(lo, hi), max(lo, hi)
            if a is None or not (left + 0.1 * abs(w) <= a <= right - 0.1 * abs(w)):
                a = 0.5 * (lo + hi)   # safeguard: bisection
            f, g, dg = phi(a)
            if accept(a, f, dg):
                return a, f, g
            if math.isfinite(f) and f <= f0 + flat:
                # f is flat to rounding here, so its comparisons carry no information: keep the
                # minimiser bracketed by the sign of the slope (Hager & Zhang's interval update)
                if dg * (hi - lo) >= 0.0:
                    hi, f_hi, dg_hi = a, f, dg
                else:
                    lo, f_lo, dg_lo, g_lo = a, f, dg, g
                continue
            if not math.isfinite(f) or f > f0 + c1 * a * dg0 or f >= f_lo:
                hi, f_hi, dg_hi = a, f, dg
            else:
                if abs(dg) <= -c2 * dg0:
                    return a, f, g
                if dg * (hi - lo) >= 0.0:
                    hi, f_hi, dg_hi = lo, f_lo, dg_lo
                lo, f_lo, dg_lo, g_lo = a, f, dg, g
        return None, f_lo, g_lo

    a_prev, f_prev, dg_prev, g_prev = 0.0, float(f0), dg0, g0
    a = float(alpha0)
    first = True
    while n_ev < max_evals:
        f, g, dg = phi(a)
        if accept(a, f, dg):
            return a, f, g, n_ev
        if not math.isfinite(f) or f > f0 + c1 * a * dg0 or (not first and f >= f_prev):
            r = zoom(a_prev, f_prev, dg_prev, g_prev, a, f, dg)
            return r[0], r[1], r[2], n_ev
        if dg >= 0.0:
            r = zoom(a, f, dg, g, a_prev, f_prev, dg_prev)
            return r[0], r[1], r[2], n_ev
        a_prev, f_prev, dg_prev, g_prev = a, f, dg, g
        a = min(2.0 * a, alpha_max)
        first = False
    return None, f0, g0, n_ev


def lbfgs(fun, x0, m=10, gtol=1e-10, max_iter=1000, c1=1e-4, c2=0.9, callback=None):
    """Minimise fun (x -> (f, grad)) from x0 by L-BFGS (Algorithm 9.2) with strong Wolfe steps.

    Stops when ||grad||_2 <= gtol, after max_iter iterations, or when the line search finds no
    step.  Curvature pairs with y.s <= 0 are not stored.  callback(k, x, f, g, step) is called
    after every accepted step.  Returns a dict: x, f, g, gnorm, iters, evals, converged, message."""
    x = np.array(x0, dtype=np.float64, copy=True)
    f, g = fun(x)
    f = float(f)
    g = np.asarray(g, dtype=np.float64)
    evals = 1
    pairs = deque(maxlen=int(m))
    gamma = 1.0
    k = 0
    message = "max_iter"
    while True:
        gn = float(np.linalg.norm(g))
        if gn <= gtol:
            message = "gtol"
            break
        if k >= max_iter:
            break
        if pairs:
            p = -two_loop(g, list(pairs), gamma)
            a0 = 1.0
        else:   # first step: steepest descent of unit length
            p = -g
            a0 = 1.0 / gn
        a, f_new, g_new, n_ev = wolfe_line_search(fun, x, f, g, p, alpha0=a0, c1=c1, c2=c2)
        evals += n_ev
        if a is None:
            message = "line search failed"
            break
        g_new = np.asarray(g_new, dtype=np.float64)
        s = a * p
        y = g_new - g
        sy = float(s @ y)
        if sy > 1e-300:
            pairs.append((s, y, 1.0 / sy))
            gamma = sy / float(y @ y)   # H0 = gamma I (Eq. 9.6)
        x = x + s
        f, g = float(f_new), g_new
        k += 1
        if callback is not None:
            callback(k, x, f, g, a)
    return {"x": x, "f": f, "g": g, "gnorm": float(np.linalg.norm(g)), "iters": k, "evals": evals,
            "converged": message == "gtol", "message": message}


def fwi_lower_level(problem, data, alpha, mu, m0, gtol=1e-10, max_iter=500, memory=10, callback=None):
    """m_FWI = argmin phi(m) for one training model (the lower-level problem), by L-BFGS.

    problem: autograd.HelmholtzProblem (grid, frequencies, acquisition, precision, refinement
    tolerance); data: [n_omega, n_src, n_rec] complex128 CUDA tensor; m0: initial squared
    slowness (host array or tensor, N values).  Each evaluation assembles and factors A(m, w) and
    calls fwi_misfit_grad on the GPU."""
    import torch

    from . import helm as hm

    acq = problem._need_acq()
    data = data.detach().contiguous()

    def fun(mv):
        mv = np.asarray(mv, dtype=np.float64)
        if not np.all(mv > 0.0):   # outside the model space (sqrt(m)): a step that is too long
            return math.inf, np.full(mv.shape, math.nan)
        m = torch.as_tensor(mv, dtype=torch.float64, device="cuda")
        try:
            op = problem.operator(m)
            f = hm.helm_factor(op, problem.prec)
            phi, grad, _, _ = hm.fwi_misfit_grad(f, acq, data, alpha, mu, problem.rtol)
        except hm.HelmError as err:
            if err.status not in (4, 5):   # only a failed solve or a singular line makes the step too long
                raise
            return math.inf, np.full(mv.shape, math.nan)
        return phi, grad.cpu().numpy()

    x0 = m0.detach().cpu().numpy() if hasattr(m0, "detach") else np.asarray(m0, dtype=np.float64)
    return lbfgs(fun, x0, m=memory, gtol=gtol, max_iter=max_iter, callback=callback)
