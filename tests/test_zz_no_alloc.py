"""helm_solve_noalloc, the solve entry point that allocates nothing (its working memory
is a fixed device array), for callers that cannot allocate device memory at solve time.
Checked through the C ABI against helm_solve / helm_adjoint_solve on the same factor, on
two calls in a row (the array keeps the previous call's contents), with the mixed-path
tolerance of the other parity tests.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

hm = pytest.importorskip("paper_2301_10762_gb300.helm")

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-8


def _case(nx=48, nz=40, n_om=2, nrhs=6, seed=4):
    rng = np.random.default_rng(seed)
    c = 1.0 + 0.5 * rng.uniform(0, 1, (nx, nz))
    m = (1.0 / c ** 2).reshape(-1)
    om = np.sort(rng.uniform(5.0, 15.0, n_om))
    B = rng.standard_normal((n_om, nrhs, nx * nz)) + 1j * rng.standard_normal((n_om, nrhs, nx * nz))
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    return op, torch.tensor(B, device="cuda")


def _colerr(X, ref):
    X, ref = X.cpu().numpy(), ref.cpu().numpy()
    return float(np.max(np.linalg.norm(X - ref, axis=-1) / np.linalg.norm(ref, axis=-1)))


@pytest.mark.parametrize("adjoint", [False, True])
def test_noalloc_solve_matches_helm_solve_on_two_calls(adjoint):
    op, B = _case()
    f = hm.helm_factor(op, hm.HELM_MIXED)
    solve = hm.helm_adjoint_solve if adjoint else hm.helm_solve
    ref, _ = solve(f, B, rtol=1e-12, max_iter=10)
    for _ in range(2):
        X = torch.full_like(B, float("nan"))
        X, info = hm.helm_solve_noalloc(f, B, X, rtol=1e-12, max_iter=10, adjoint=adjoint)
        assert info["max_relres"] <= 1e-12
        assert _colerr(X, ref) <= TOL_MIXED


def test_noalloc_solve_rejects_sizes_beyond_its_array():
    op, B = _case(nrhs=2)
    f = hm.helm_factor(op, hm.HELM_MIXED)
    big = torch.zeros((op.n_omega, 400, op.N), dtype=torch.complex128, device="cuda")   # ~98 MB of scratch
    with pytest.raises(hm.HelmError) as e:
        hm.helm_solve_noalloc(f, big, torch.empty_like(big))
    assert e.value.status == 1
