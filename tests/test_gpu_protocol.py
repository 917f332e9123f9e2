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
