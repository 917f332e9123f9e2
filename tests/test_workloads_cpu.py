"""The seeded workload generators follow their stated recipes.

Every input of the tests and the benchmark comes from workloads/; these checks pin what the
recipes promise: determinism per seed, the canonical node order (z fastest), the documented
source and receiver positions, value ranges, the Gaussian covariance of the random fields, speeds
that increase with depth in the layered models, and the structure of the batched hypergradient
and solve-server loads."""
import numpy as np
import pytest

import workloads as W


def test_node_order_is_z_fastest():
    nx, nz, lx, lz = 9, 6, 2.0, 1.0
    m = W.gaussian_inclusion_velocity(nx, nz, lx, lz, centre=(0.7, 0.4), radius=0.3)
    hx, hz = lx / (nx - 1), lz / (nz - 1)
    for i, j in ((0, 0), (3, 1), (8, 5), (2, 4)):
        x, z = i * hx, j * hz
        c = 1.0 + 0.2 * np.exp(-((x - 0.7) ** 2 + (z - 0.4) ** 2) / 0.3 ** 2)
        assert m[i * nz + j] == pytest.approx(1.0 / c ** 2, rel=1e-14)


def test_generators_are_deterministic_per_seed():
    a = W.gaussian_random_field(40, 30, 0.1, 7)
    assert np.array_equal(a, W.gaussian_random_field(40, 30, 0.1, 7))
    assert not np.array_equal(a, W.gaussian_random_field(40, 30, 0.1, 8))
    assert np.array_equal(W.layered_velocity(32, 32, 3), W.layered_velocity(32, 32, 3))
    assert np.array_equal(W.random_rhs(50, 3, 1, 2), W.random_rhs(50, 3, 1, 2))
    w1, w2 = W.tiny_case(seed=4), W.tiny_case(seed=4)
    assert np.array_equal(w1.m_true, w2.m_true) and np.array_equal(w1.acq.rec_xz, w2.acq.rec_xz)


def test_plain_forward_geometry():
    w = W.config_plain()
    h = 1.0 / 63
    idx = np.round(w.acq.src_xz[:, 0] / h).astype(int)
    assert idx.tolist() == [4, 12, 20, 28, 35, 43, 51, 59]
    assert np.allclose(w.acq.src_xz[:, 0], idx * h, rtol=0, atol=1e-15) and np.all(w.acq.src_xz[:, 1] == 0)
    assert np.allclose(w.acq.rec_xz[:, 0], (np.arange(16) + 0.5) / 16) and np.all(w.acq.rec_xz[:, 1] == 0)
    c = 1.0 / np.sqrt(w.m)
    assert c.min() >= 1.0 and 1.19 < c.max() <= 1.2
    assert w.omegas.tolist() == [10.0]


def test_gaussian_random_field_moments_and_covariance():
    """Zero mean, max |g| = 1, and the correlation length of the covariance exp(-r^2 / (2 l^2)):
    l is recovered from the sample correlation at short lags, rho(r) = exp(-r^2 / (2 l^2)),
    where removing the sample mean barely biases it (a filter with the wrong exponent, e.g.
    covariance exp(-r^2 / (4 l^2)), would give sqrt(2) l)."""
    n, ell = 128, 0.05
    h = 1.0 / (n - 1)
    est = []
    for seed in range(12):
        g = W.gaussian_random_field(n, n, ell, seed)
        assert abs(g.mean()) < 1e-12 and np.abs(g).max() == pytest.approx(1.0, abs=1e-15)
        c0 = np.mean(g * g)
        for lag in (2, 3):
            for rho in (np.mean(g[:-lag] * g[lag:]) / c0, np.mean(g[:, :-lag] * g[:, lag:]) / c0):
                est.append(lag * h / np.sqrt(-2.0 * np.log(rho)))
    assert np.mean(est) == pytest.approx(ell, rel=0.08)


@pytest.mark.parametrize("seed", [0, 4001, 4017])
def test_layered_velocity_range_and_depth_trend(seed):
    n = 96
    c = (1.0 / np.sqrt(W.layered_velocity(n, n, seed))).reshape(n, n)
    assert c.min() >= 1.5 * 0.85 - 1e-12 and c.max() <= 4.5 * 1.15 + 1e-12
    profile = c.mean(axis=0)                    # horizontal average at each depth
    assert profile[:5].mean() < 1.8 and profile[-5:].mean() > 3.9
    assert np.corrcoef(np.arange(n), profile)[0, 1] > 0.9


def test_fwi_step_and_mixed_ranges():
    w = W.config_fwi_step(64)
    c = 1.0 / np.sqrt(w.m_true)
    assert 0.7 - 1e-12 <= c.min() and c.max() <= 1.3 + 1e-12
    assert np.max(np.abs(c - 1.0)) == pytest.approx(0.3, rel=1e-12)   # max |g| = 1
    assert np.all(w.m == 1.0) and w.omegas.tolist() == [5.0, 10.0, 15.0]
    assert (w.acq.n_src, w.acq.n_rec, w.alpha, w.mu) == (16, 32, 1e-3, 1e-6)
    wm = W.config_mixed(64)
    cm = 1.0 / np.sqrt(wm.m)
    assert cm.min() == pytest.approx(1.0, abs=1e-12) and cm.max() == pytest.approx(3.0, abs=1e-12)
    assert wm.omegas.tolist() == [5.0 * k for k in range(1, 9)] and wm.acq.n_src == 64


def test_hypergrad_set_structure():
    models = W.config_hypergrad(n_models=7)
    assert [w.nx for w in models] == [96, 128, 160, 192, 224, 256, 96]
    n_src = models[0].acq.n_src
    assert 16 <= n_src <= 64
    rec = models[0].acq.rec_xz
    for w in models:
        h = 1.0 / (w.nx - 1)
        assert w.acq.n_src == n_src and np.array_equal(w.acq.rec_xz, rec)
        assert np.allclose(w.acq.src_xz[:, 0], round(0.05 / h) * h)
        assert np.allclose(w.acq.src_xz[:, 1] / h, np.round(w.acq.src_xz[:, 1] / h), atol=1e-9)   # on nodes
        assert w.omegas.tolist() == [3.0, 9.0, 18.0, 36.0]
        m_fwi = W.gaussian_smooth(w.m_true.reshape(w.nx, w.nz), 4.0).reshape(-1)
        assert np.array_equal(w.m, m_fwi)
    assert np.all(rec[:, 0] == 0.95) and np.all((rec[:, 1] >= 0.05) & (rec[:, 1] <= 0.95))


def test_server_load():
    cfg = W.config_server(sizes=(32, 48), n_models=3, n_freq=5)
    for ms, oms in zip(cfg["m"], cfg["omegas"]):
        for m, om in zip(ms, oms):
            c = 1.0 / np.sqrt(m)
            assert c.min() == pytest.approx(1.5, abs=1e-12) and c.max() == pytest.approx(4.5, abs=1e-12)
            assert np.all(np.diff(om) >= 0) and om.min() >= 5.0 and om.max() <= 60.0
    reqs = W.server_requests(cfg, 400, seed=1)
    assert {r[0] for r in reqs} == {0, 1} and {r[3] for r in reqs} == {0, 1}
    assert all(1 <= r[4] <= 128 for r in reqs)
    assert all(r[2] in cfg["omegas"][r[0]][r[1]] for r in reqs)
    t = W.poisson_arrivals(20000, 50.0, seed=2)
    assert np.all(np.diff(t) > 0) and np.mean(np.diff(t)) == pytest.approx(1 / 50.0, rel=0.03)


def test_tiny_case_geometry():
    w = W.tiny_case(8, 7, n_src=3, n_rec=4, seed=9)
    hx = w.lx / (w.nx - 1)
    i = np.round(w.acq.src_xz[:, 0] / hx)
    assert np.all((i >= 1) & (i <= w.nx - 2)) and len(set(i)) == 3 and np.all(w.acq.src_xz[:, 1] == 0)
    assert np.all((w.acq.rec_xz[:, 0] > 0) & (w.acq.rec_xz[:, 0] < w.lx))
    assert np.all((w.acq.rec_xz[:, 1] > 0) & (w.acq.rec_xz[:, 1] < w.lz))
    assert np.all(w.m > 0.25 - 1e-12) and np.all(w.m <= 1.0)


def test_resample_bilinear_exact_on_bilinear_fields_and_shared_nodes():
    fn = lambda X, Z: 1.0 + 2.0 * X - 3.0 * Z + 0.5 * X * Z   # noqa: E731
    f = W.sample_on_grid(fn, 7, 5, 1.4, 0.8)
    g = W.resample_bilinear(f, 7, 5, 13, 9)
    assert np.allclose(g, W.sample_on_grid(fn, 13, 9, 1.4, 0.8), rtol=0, atol=1e-14)
    # the 13 x 9 grid contains every node of the 7 x 5 grid: going back copies them
    assert np.array_equal(W.resample_bilinear(g, 13, 9, 7, 5), f)
    assert np.array_equal(W.resample_bilinear(f, 7, 5, 7, 5), f)
    # a non-bilinear field is reproduced at shared nodes and bounded by its neighbours elsewhere
    h = W.sample_on_grid(lambda X, Z: np.sin(3 * X) * np.cos(2 * Z), 7, 5)
    hr = W.resample_bilinear(h, 7, 5, 13, 9).reshape(13, 9)
    assert np.array_equal(hr[::2, ::2].reshape(-1), h)
    assert hr.min() >= h.min() - 1e-15 and hr.max() <= h.max() + 1e-15
