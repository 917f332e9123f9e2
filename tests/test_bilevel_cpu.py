"""CPU checks of the upper-level loop (paper_2301_10762_gb300/bilevel.py): bilevel frequency
continuation (Algorithm allg:fcb1) with L-BFGS-B on each frequency group.

Pins: on a separable quadratic whose minimiser moves with the frequency group, each group ends at
the closed-form box-constrained minimiser (the unconstrained one clipped to the bounds), alpha
stays at its initial value until the final group ("last"), moves in every group ("all") or never
("none"), and every evaluation stays inside the bounds.  On a tiny bilevel problem evaluated by
the oracle (dense Newton lower level, Algorithm alg:box hypergradient averaged over two training
models), the loop lowers psi in every group, keeps the receivers in the borehole, starts each
group from the previous group's design and ends with an improvement factor above 1.  The metrics
of the experiments: MRE (Eq. relerr) and IF on closed-form cases, and the 1 % test-time noise is
40 dB SNR per frequency."""
import numpy as np
import pytest

from paper_2301_10762_gb300 import bilevel as B


def _quadratic(calls, targets, a_star, scale_a=3.0):
    def evaluate(omegas, z, alpha):
        c = targets[float(omegas[0])]
        calls.append((float(omegas[0]), np.array(z), float(alpha)))
        psi = 0.5 * np.sum((z - c) ** 2) + 0.5 * scale_a * (alpha - a_star) ** 2
        return psi, z - c, scale_a * (alpha - a_star)
    return evaluate


def test_groups_end_at_box_constrained_minimiser_alpha_last():
    targets = {1.0: np.array([0.2, 0.5, 1.4, -0.3]), 2.0: np.array([0.7, 0.1, 0.95, 0.4])}
    lo, hi = 0.0, 1.0
    calls = []
    out = B.frequency_continuation(_quadratic(calls, targets, 0.03), [0.5, 0.5, 0.5, 0.5], 0.01,
                                   [[1.0], [2.0]], (lo, hi), alpha_bounds=(1e-6, None), max_iter=50)
    assert len(out["history"]) == 2
    for om, z, a in calls:
        assert np.all(z >= lo) and np.all(z <= hi)
        if om == 1.0:
            assert a == 0.01   # alpha fixed outside the final group
    assert out["history"][0]["alpha_free"] is False and out["history"][1]["alpha_free"] is True
    assert np.allclose(out["z"], np.clip(targets[2.0], lo, hi), atol=1e-8)
    assert abs(out["alpha"] - 0.03) <= 1e-8
    # group 1 ended at its own clipped minimiser: the first call of group 2 starts there
    first2 = next(z for om, z, a in calls if om == 2.0)
    assert np.allclose(first2, np.clip(targets[1.0], lo, hi), atol=1e-8)
    for h in out["history"]:
        assert h["psi"] <= h["psi_start"]


@pytest.mark.parametrize("mode", ["all", "none"])
def test_free_alpha_modes(mode):
    targets = {1.0: np.array([0.3, 0.6]), 2.0: np.array([0.4, 0.5])}
    calls = []
    out = B.frequency_continuation(_quadratic(calls, targets, 0.05), [0.5, 0.5], 0.01, [[1.0], [2.0]],
                                   (0.0, 1.0), free_alpha=mode)
    alphas_g1 = {a for om, z, a in calls if om == 1.0}
    if mode == "none":
        assert alphas_g1 == {0.01} and out["alpha"] == 0.01
        assert all(not h["alpha_free"] for h in out["history"])
    else:
        assert len(alphas_g1) > 1 and abs(out["alpha"] - 0.05) <= 1e-8
        assert all(h["alpha_free"] for h in out["history"])


def test_alpha_lower_bound_holds():
    targets = {1.0: np.array([0.5])}
    calls = []
    out = B.frequency_continuation(_quadratic(calls, targets, -1.0), [0.5], 0.01, [[1.0]], (0.0, 1.0),
                                   alpha_bounds=(1e-4, None))
    assert all(a >= 1e-4 for _, _, a in calls)
    assert abs(out["alpha"] - 1e-4) <= 1e-12


def _oracle_evaluate(models, g, src_xz, rec_x, alpha0, mu, counter):
    """psi, dpsi/dz, dpsi/dalpha averaged over the training models (Eq. SOobj with 1/N_m'),
    each lower level solved by Newton with the dense Hessian from the model's previous m_FWI."""
    from oracle import dense as D
    from oracle import helmholtz as H
    warm = [np.array(m0) for m0, _ in models]

    def evaluate(omegas, z, alpha):
        counter[0] += 1
        rec = np.stack([np.full(len(z), rec_x), z], axis=1)
        psi, dz, da = 0.0, np.zeros(len(z)), 0.0
        for k, (_, mt) in enumerate(models):
            data, _ = H.synthetic_data(g, mt, omegas, src_xz, rec)
            m_fwi, gn = D.lower_level_newton(g, warm[k], omegas, src_xz, rec, data, alpha, mu)
            assert gn < 1e-10
            warm[k] = m_fwi
            hg = H.hypergradient(g, m_fwi, mt, omegas, src_xz, rec, alpha, alpha0, mu, cg_rtol=1e-14)
            psi += hg["psi"] / len(models)
            dz += hg["dpsi_dp"][:, 1] / len(models)
            da += hg["dpsi_dalpha"] / len(models)
        return psi, dz, da
    return evaluate


def test_oracle_bilevel_continuation_lowers_psi():
    from oracle import helmholtz as H
    from workloads import tiny_case
    w0 = tiny_case(7, 6, seed=11, n_omega=3, n_src=4, n_rec=6)
    w1 = tiny_case(7, 6, seed=12, n_omega=3, n_src=4, n_rec=6)
    g = H.Grid(w0.nx, w0.nz, w0.lx, w0.lz)
    models = [(w0.m, w0.m_true), (w1.m, w1.m_true)]
    src = w0.acq.src_xz
    rec_x = 0.55 * w0.lx
    z0 = np.linspace(0.15, 0.75, 6) * w0.lz
    bounds = (0.05 * w0.lz, 0.85 * w0.lz)
    counter = [0]
    evaluate = _oracle_evaluate(models, g, src, rec_x, 1e-4, 1e-4, counter)
    groups = [[2.0, 3.0], [4.0, 5.0]]
    seen = []

    def cb(k, z, alpha, entry):
        seen.append((k, z.copy(), alpha))

    out = B.frequency_continuation(evaluate, z0, 1e-4, groups, bounds, alpha_bounds=(1e-8, 1.0),
                                   max_iter=6, callback=cb)
    assert [k for k, _, _ in seen] == [0, 1]
    assert np.all(out["z"] >= bounds[0]) and np.all(out["z"] <= bounds[1])
    for h in out["history"]:
        assert h["psi"] < h["psi_start"]
        assert 1 <= h["iters"] <= 6
    assert seen[0][2] == 1e-4                # alpha fixed in the first group
    assert counter[0] <= 2 * 6 * 3           # a handful of evaluations per iteration
    # the second group starts where the first ended: re-evaluating the first group's design on
    # the second group's frequencies gives that group's starting psi
    psi_g2, _, _ = evaluate(np.array(groups[1]), seen[0][1], seen[0][2])
    assert np.isclose(psi_g2, out["history"][1]["psi_start"], rtol=1e-9)
    # improvement factor on the final group's frequencies: the learned design beats the initial one
    psi_init, _, _ = evaluate(np.array(groups[-1]), z0, 1e-4)
    assert B.improvement_factor(psi_init, out["history"][-1]["psi"]) > 1.0


def test_mre_and_improvement_factor_closed_forms():
    # errors of 10 %, 5 % and 0 %: mean 5 %
    assert np.isclose(B.mre([1.1, 1.9, 3.0], [1.0, 2.0, 3.0]), 5.0, rtol=1e-12)
    assert B.mre([-2.0], [-1.0]) == 100.0          # relative to |truth|
    assert B.improvement_factor(3.0, 1.5) == 2.0


@pytest.mark.parametrize("backend", ["numpy", "torch"])
def test_noise_is_40db_per_frequency(backend):
    rng = np.random.default_rng(3)
    scale = np.array([1.0, 1e-3, 1e4])[:, None, None]        # very different amplitudes per frequency
    d = (rng.standard_normal((3, 4, 5)) + 1j * rng.standard_normal((3, 4, 5))) * scale
    eta = rng.standard_normal((3, 4, 5)) + 1j * rng.standard_normal((3, 4, 5))
    if backend == "torch":
        torch = pytest.importorskip("torch")
        dn = B.add_noise(torch.tensor(d), torch.tensor(eta)).numpy()
    else:
        dn = B.add_noise(d, eta)
    for q in range(3):
        snr = 10 * np.log10(np.sum(np.abs(d[q]) ** 2) / np.sum(np.abs(dn[q] - d[q]) ** 2))
        assert abs(snr - 40.0) <= 1e-9
        # the noise is the draws, rescaled: same direction
        r = (dn[q] - d[q]) / eta[q]
        assert np.allclose(r, r.flat[0], rtol=1e-12)
    assert np.array_equal(B.add_noise(d, eta, level=0.0), d)
    with pytest.raises(ValueError):
        B.add_noise(d, eta[:2])
    with pytest.raises(ValueError):
        B.add_noise(d, np.zeros_like(eta))


class _OracleProblem:
    """The interface of GpuBilevelProblem (evaluate, test_metrics) on the oracle: data from the
    training models at the current receivers, the lower level by Newton with the dense Hessian
    (warm-started per model), the hypergradient of Algorithm alg:box averaged over the models."""

    def __init__(self, g, train, m0, src, rec_x, alpha0, mu):
        self.g, self.train, self.m0, self.src, self.rec_x = g, train, m0, src, rec_x
        self.alpha0, self.mu = alpha0, mu
        self.warm = [m0.copy() for _ in train]
        self.calls = []

    def _rec(self, z):
        return np.stack([np.full(len(z), self.rec_x), z], axis=1)

    def evaluate(self, om, z, alpha):
        from oracle import dense as D
        from oracle import helmholtz as H
        self.calls.append((float(om[-1]), float(alpha)))
        rec = self._rec(z)
        psi, dz, da = 0.0, np.zeros(len(z)), 0.0
        for k, mt in enumerate(self.train):
            data, _ = H.synthetic_data(self.g, mt, om, self.src, rec)
            m_fwi, gn = D.lower_level_newton(self.g, self.warm[k], om, self.src, rec, data, alpha, self.mu)
            assert gn < 1e-10
            self.warm[k] = m_fwi
            hg = H.hypergradient(self.g, m_fwi, mt, om, self.src, rec, alpha, self.alpha0, self.mu, cg_rtol=1e-13)
            psi += hg["psi"] / len(self.train)
            dz += hg["dpsi_dp"][:, 1] / len(self.train)
            da += hg["dpsi_dalpha"] / len(self.train)
        return psi, dz, da

    def test_metrics(self, om, z, alpha, m_tests, m0, noise_draws=None, level=0.01, data_models=None):
        from oracle import dense as D
        from oracle import helmholtz as H
        rec = self._rec(z)
        psi, mres = 0.0, []
        for k, mt in enumerate(m_tests):
            data, _ = H.synthetic_data(self.g, mt, om, self.src, rec)
            if noise_draws is not None:
                data = B.add_noise(data, noise_draws[k], level)
            m_fwi, _ = D.lower_level_newton(self.g, m0, om, self.src, rec, data, alpha, self.mu)
            psi += 0.5 * np.sum((mt - m_fwi) ** 2) / len(m_tests)
            mres.append(B.mre(1 / np.sqrt(m_fwi), 1 / np.sqrt(mt)))
        return psi, mres


def test_oracle_miniature_of_the_experiment_protocol():
    """The paper's protocol in miniature, through bilevel.run_protocol with the oracle as the
    problem (the GPU run passes a GpuBilevelProblem instead).
    - Setup: 8 x 8 grid, two layered training models, crosswell (3 sources at x = 0.05,
      4 receivers in a borehole at x = 0.9, depths bounded to [0.05, 0.95]).
    - Lower level: from a vertically varying start model.
    - Frequency groups: overlapping, [(2), (2, 4), (4, 8)]; alpha freed in the last group only.
    - Test: a held-out layered model, data with 1 % noise (40 dB).
    The learned design beats the initial one on the training set and on the held-out model, in
    psi (IF > 1) and in the wavespeed MRE."""
    from oracle import helmholtz as H
    import workloads as W
    n = 8
    g = H.Grid(n, n, 1.0, 1.0)
    train = [W.layered_velocity(n, n, 100 + k) for k in range(2)]
    test = W.layered_velocity(n, n, 200)
    m0 = W.sample_on_grid(lambda X, Z: 1.0 / (1.5 + 3.0 * Z) ** 2, n, n)
    h = 1.0 / (n - 1)
    src = np.stack([np.full(3, round(0.05 / h) * h), np.round(np.array([0.2, 0.5, 0.8]) / h) * h], axis=1)
    z0, alpha0 = np.linspace(0.3, 0.7, 4), 1e-2
    prob = _OracleProblem(g, train, m0, src, 0.9, alpha0, 1e-4)
    rng = np.random.default_rng(7)
    draws = [rng.standard_normal((2, 3, 4)) + 1j * rng.standard_normal((2, 3, 4))]
    # alpha >= 1e-5 keeps every lower-level problem well posed for the Newton solve (at 1e-6 a
    # trial point's Newton iteration stalled); the optimum lies inside, at about 2.7e-5
    res = B.run_protocol(prob, z0, alpha0, [[2.0], [2.0, 4.0], [4.0, 8.0]], (0.05, 0.95), [test], m0,
                         alpha_bounds=(1e-5, 1.0), max_iter=15, noise_draws=draws)
    assert all(a == alpha0 for top, a in prob.calls if top < 8.0)     # alpha fixed before the last group
    assert res["alpha"] != alpha0
    assert np.all((res["z"] >= 0.05) & (res["z"] <= 0.95))
    assert res["train_if"] > 5.0
    assert res["test_if"] > 2.0
    assert res["test_mre"][1][0] < 0.5 * res["test_mre"][0][0]
