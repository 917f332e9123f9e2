"""The experiments' protocol end to end on the GPU (Algorithm allg:fcb1 with the lower level of
Section 4): bilevel.run_protocol with a GpuBilevelProblem -- every phi / grad phi evaluation of
the L-BFGS lower level, every data synthesis and every hypergradient runs in the library's
kernels.  The same miniature as the oracle-driven CPU test: an 8 x 8 grid, two layered training
models, crosswell (3 sources at x = 0.05, 4 receivers in a borehole at x = 0.9, depths bounded to
[0.05, 0.95]), overlapping frequency groups [(2), (2, 4), (4, 8)] with alpha freed in the last,
a held-out layered test model with 1 % noise.  FP64 factors, so that the lower level reaches
||grad phi|| <= 1e-10."""
import numpy as np
import pytest

import workloads as W

hm = pytest.importorskip("paper_2301_10762_gb300.helm")
B = pytest.importorskip("paper_2301_10762_gb300.bilevel")

pytestmark = pytest.mark.gpu


def test_protocol_miniature_on_the_gpu():
    n = 8
    train = [W.layered_velocity(n, n, 100 + k) for k in range(2)]
    test = W.layered_velocity(n, n, 200)
    m0 = W.sample_on_grid(lambda X, Z: 1.0 / (1.5 + 3.0 * Z) ** 2, n, n)
    h = 1.0 / (n - 1)
    src = np.stack([np.full(3, round(0.05 / h) * h), np.round(np.array([0.2, 0.5, 0.8]) / h) * h], axis=1)
    z0, alpha0 = np.linspace(0.3, 0.7, 4), 1e-2
    prob = B.GpuBilevelProblem(n, n, 1.0, 1.0, train, m0, src, 0.9, alpha0, 1e-4, prec=hm.HELM_FP64,
                               refine_rtol=1e-12, lower_gtol=1e-10, lower_max_iter=2000)
    rng = np.random.default_rng(7)
    draws = [rng.standard_normal((2, 3, 4)) + 1j * rng.standard_normal((2, 3, 4))]
    res = B.run_protocol(prob, z0, alpha0, [[2.0], [2.0, 4.0], [4.0, 8.0]], (0.05, 0.95), [test], m0,
                         alpha_bounds=(1e-5, 1.0), max_iter=15, noise_draws=draws)
    assert res["alpha"] != alpha0
    assert np.all((res["z"] >= 0.05) & (res["z"] <= 0.95))
    assert res["train_if"] > 2.0
    assert res["test_if"] > 1.0
    assert res["test_mre"][1][0] < res["test_mre"][0][0]
    assert prob.evaluations > 3


def test_evaluate_with_training_data_from_a_finer_grid():
    """One upper-level evaluation with the training data computed on a finer grid (23 x 23
    nodes for the 12 x 12 inversion grid, the layered models sampled there): the lower level
    runs on the finer data to ||grad phi|| <= 1e-10 on the GPU, and the hypergradient at the
    m_FWI it found matches the oracle's data-grid branch (FP64 path: 1e-9)."""
    from oracle import helmholtz as H
    n, nf = 12, 23   # (on 8 x 8 the finer data drive the lower level to the boundary m = 0)
    seeds = (100, 101)
    train = [W.layered_velocity(n, n, s) for s in seeds]
    fine = [W.layered_velocity(nf, nf, s) for s in seeds]
    m0 = W.sample_on_grid(lambda X, Z: 1.0 / (1.5 + 3.0 * Z) ** 2, n, n)
    h = 1.0 / (n - 1)
    src = np.stack([np.full(3, round(0.05 / h) * h), np.round(np.array([0.2, 0.5, 0.8]) / h) * h], axis=1)
    z, alpha, alpha0, mu = np.linspace(0.3, 0.7, 4), 1e-2, 1e-2, 1e-4
    om = [2.0, 4.0]
    prob = B.GpuBilevelProblem(n, n, 1.0, 1.0, train, m0, src, 0.9, alpha0, mu, prec=hm.HELM_FP64,
                               refine_rtol=1e-12, lower_gtol=1e-10, lower_max_iter=2000,
                               train_data_models=[(nf, nf, m) for m in fine])
    psi, dz, da = prob.evaluate(om, z, alpha)
    rec = np.stack([np.full(z.size, 0.9), z], axis=1)
    ref = {"psi": 0.0, "dpsi_dalpha": 0.0, "dpsi_dp": 0.0}
    for k in range(2):
        o = H.hypergradient(H.Grid(n, n), prob.warm[k], train[k], np.array(om), src, rec, alpha, alpha0, mu,
                            cg_rtol=1e-13, data_grid=H.Grid(nf, nf), m_true_data=fine[k])
        for key in ref:
            ref[key] = ref[key] + o[key] / 2
    assert abs(psi - ref["psi"]) <= 1e-12 * abs(ref["psi"])
    assert abs(da - ref["dpsi_dalpha"]) <= 1e-9 * abs(ref["dpsi_dalpha"])
    assert np.linalg.norm(dz - ref["dpsi_dp"][:, 1]) <= 1e-9 * np.linalg.norm(ref["dpsi_dp"][:, 1])
