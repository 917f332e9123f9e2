"""GPU checks of the solve server (include/helm_server.h) through the C ABI: every request's
result against the CPU oracle (1e-9 FP64, 1e-8 mixed), batching of queued requests with the
same key, cache hits on a second wave, LRU eviction under a budget that holds one factor,
and refusal of a request whose footprint exceeds the budget."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import helmholtz as H

hm = pytest.importorskip("paper_2301_10762_gb300.helm")

pytestmark = pytest.mark.gpu

TOL = {hm.HELM_FP64: 1e-9, hm.HELM_MIXED: 1e-8}
GRIDS = [(24, 20, 1.0, 0.8), (32, 28, 1.0, 1.0)]


def _m(nx, nz, seed):
    rng = np.random.default_rng(seed)
    c = W.gaussian_smooth(1.0 + 0.5 * rng.uniform(0, 1, (nx, nz)), 1.5)
    return (1.0 / c ** 2).reshape(-1)


def _rhs(nrhs, N, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((nrhs, N)) + 1j * rng.standard_normal((nrhs, N))
    return torch.tensor(B).pin_memory()


def _oracle(grid, m, omega, B, adjoint):
    f = H.Factor(H.helmholtz_matrix(H.Grid(*grid), m, omega))
    return f.adjoint_solve(B) if adjoint else f.solve(B)


def _err(X, ref):
    return float(np.max(np.linalg.norm(X - ref, axis=-1) / np.linalg.norm(ref, axis=-1)))


def test_server_results_batching_and_cache():
    # one worker: while it builds the first factor the other requests queue up, so requests
    # with the same key are batched
    srv = hm.Server(workers=1)
    ms = [_m(*g[:2], seed=k) for k, g in enumerate(GRIDS)]
    ids = [srv.add_model(*g, m) for g, m in zip(GRIDS, ms)]
    # (model, omega, prec, adjoint, nrhs): four factor keys, two batches of more than one request
    reqs = [(0, 5.0, hm.HELM_MIXED, False, 3), (0, 5.0, hm.HELM_MIXED, False, 2), (1, 9.0, hm.HELM_FP64, False, 4),
            (0, 5.0, hm.HELM_MIXED, True, 1), (1, 9.0, hm.HELM_FP64, False, 1), (0, 7.0, hm.HELM_FP64, True, 2),
            (1, 12.0, hm.HELM_MIXED, False, 5), (0, 5.0, hm.HELM_MIXED, False, 1)]
    for wave in range(2):
        inputs = [_rhs(r[4], GRIDS[r[0]][0] * GRIDS[r[0]][1], seed=100 * wave + k) for k, r in enumerate(reqs)]
        tickets = [srv.submit(ids[mi], om, B, prec=prec, rtol=1e-12, adjoint=adj)
                   for (mi, om, prec, adj, nrhs), B in zip(reqs, inputs)]
        for k, t in enumerate(tickets):
            out = srv.wait(t)
            assert "error" not in out, out["error"]
            mi, om, prec, adj, nrhs = reqs[k]
            ref = _oracle(GRIDS[mi], ms[mi], om, inputs[k].numpy(), adj)
            assert _err(out["X"].numpy(), ref) <= TOL[prec], (k, wave)
            assert out["batch_rhs"] >= nrhs and out["total_ms"] >= out["queue_ms"] >= 0.0
            if wave == 1:
                assert out["cache_hit"] == 1
        st = srv.stats()
        assert st["completed"] == len(reqs) * (wave + 1)
        assert st["rhs_solved"] == sum(r[4] for r in reqs) * (wave + 1)
        assert st["factor_builds"] == 4 and st["entries"] == 4 and st["evictions"] == 0
    assert st["batches"] < st["completed"] and st["refused"] == 0
    srv.close()


def test_server_workers_run_concurrently():
    # eight workers (the default), requests of eight keys at once: all correct
    srv = hm.Server()
    grid = GRIDS[1]
    m = _m(*grid[:2], seed=9)
    mid = srv.add_model(*grid, m)
    N = grid[0] * grid[1]
    oms = [4.0 + k for k in range(8)]
    inputs = [_rhs(3, N, seed=200 + k) for k in range(8)]
    tickets = [srv.submit(mid, om, B, prec=hm.HELM_MIXED if k % 2 else hm.HELM_FP64, rtol=1e-12)
               for k, (om, B) in enumerate(zip(oms, inputs))]
    for k, t in enumerate(tickets):
        out = srv.wait(t)
        assert "error" not in out
        prec = hm.HELM_MIXED if k % 2 else hm.HELM_FP64
        assert _err(out["X"].numpy(), _oracle(grid, m, oms[k], inputs[k].numpy(), False)) <= TOL[prec]
    st = srv.stats()
    assert st["factor_builds"] == 8 and st["completed"] == 8
    srv.close()


def test_server_evicts_least_recently_used_under_budget():
    grid = GRIDS[0]
    m = _m(*grid[:2], seed=5)
    probe = hm.Server(hbm_budget_bytes=1 << 34)
    fp = probe.footprint(probe.add_model(*grid, m), hm.HELM_MIXED, 2)
    probe.close()
    srv = hm.Server(hbm_budget_bytes=int(1.5 * fp), workers=1)   # one factor at a time
    mid = srv.add_model(*grid, m)
    N = grid[0] * grid[1]
    for k, om in enumerate([5.0, 7.0, 5.0, 9.0]):
        B = _rhs(2, N, seed=k)
        out = srv.wait(srv.submit(mid, om, B, prec=hm.HELM_MIXED, rtol=1e-12))
        assert "error" not in out and out["cache_hit"] == 0
        assert _err(out["X"].numpy(), _oracle(grid, m, om, B.numpy(), False)) <= TOL[hm.HELM_MIXED]
    st = srv.stats()
    assert st["factor_builds"] == 4 and st["evictions"] == 3 and st["entries"] == 1
    assert st["bytes_peak"] <= st["bytes_budget"]
    srv.close()


def test_server_refuses_requests_above_the_budget():
    grid = GRIDS[1]
    m = _m(*grid[:2], seed=6)
    probe = hm.Server(hbm_budget_bytes=1 << 34)
    fp4 = probe.footprint(probe.add_model(*grid, m), hm.HELM_FP64, 4)
    probe.close()
    srv = hm.Server(hbm_budget_bytes=fp4 - 1, workers=1)
    mid = srv.add_model(*grid, m)
    N = grid[0] * grid[1]
    with pytest.raises(hm.HelmError) as ei:
        srv.submit(mid, 6.0, _rhs(4, N, seed=1), prec=hm.HELM_FP64)
    assert ei.value.status == 2   # HELM_ENOMEM
    B = _rhs(1, N, seed=2)
    out = srv.wait(srv.submit(mid, 6.0, B, prec=hm.HELM_FP64))
    assert "error" not in out
    assert _err(out["X"].numpy(), _oracle(grid, m, 6.0, B.numpy(), False)) <= TOL[hm.HELM_FP64]
    st = srv.stats()
    assert st["refused"] == 1 and st["completed"] == 1
    with pytest.raises(hm.HelmError):
        srv.submit(mid + 7, 6.0, B)   # unknown model
    srv.close()
