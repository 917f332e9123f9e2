"""helm_solve_noalloc, the solve entry point that allocates nothing.

Some callers cannot allocate device memory at solve time: a serving process that carved up
the device memory once at start-up, a host framework whose caching allocator already owns
the free memory, or a loop that cannot take the device-wide synchronisation of cudaMalloc /
cudaFree.  For them the solve's working memory is a fixed array in device global memory.

Checked through the C ABI against helm_solve / helm_adjoint_solve on the same factor, on two
calls in a row (the array keeps the previous call's contents), on both factor precisions, at
the tolerances of the other parity tests; once directly against the CPU oracle; and by the
default memory pool's used-bytes counter, which a call on a fresh factor leaves unchanged
(while helm_solve on a fresh factor raises it).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import helmholtz as H

hm = pytest.importorskip("paper_2301_10762_gb300.helm")

pytestmark = pytest.mark.gpu

TOL = {hm.HELM_FP64: 1e-9, hm.HELM_MIXED: 1e-8}


def _case(nx=48, nz=40, n_om=2, nrhs=6, seed=4):
    rng = np.random.default_rng(seed)
    c = 1.0 + 0.5 * rng.uniform(0, 1, (nx, nz))
    m = (1.0 / c ** 2).reshape(-1)
    om = np.sort(rng.uniform(5.0, 15.0, n_om))
    B = rng.standard_normal((n_om, nrhs, nx * nz)) + 1j * rng.standard_normal((n_om, nrhs, nx * nz))
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    return op, torch.tensor(B, device="cuda"), m, om, B


def _colerr(X, ref):
    X = X.cpu().numpy() if torch.is_tensor(X) else X
    ref = ref.cpu().numpy() if torch.is_tensor(ref) else ref
    return float(np.max(np.linalg.norm(X - ref, axis=-1) / np.linalg.norm(ref, axis=-1)))


def _pool_used_bytes():
    """cudaMemPoolAttrUsedMemCurrent of the current device's default memory pool (the pool the
    library's stream-ordered allocations come from), through the CUDA runtime the library
    links."""
    rt = C.CDLL("libcudart.so.13")
    dev = C.c_int()
    assert rt.cudaGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    used = C.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 0x7, C.byref(used)) == 0   # cudaMemPoolAttrUsedMemCurrent
    return used.value


@pytest.mark.parametrize("prec", [hm.HELM_FP64, hm.HELM_MIXED])
@pytest.mark.parametrize("adjoint", [False, True])
def test_noalloc_solve_matches_helm_solve_on_two_calls(prec, adjoint):
    op, B, _, _, _ = _case()
    f = hm.helm_factor(op, prec)
    solve = hm.helm_adjoint_solve if adjoint else hm.helm_solve
    ref, _ = solve(f, B, rtol=1e-12, max_iter=10)
    for _ in range(2):
        X = torch.full_like(B, float("nan"))
        X, info = hm.helm_solve_noalloc(f, B, X, rtol=1e-12, max_iter=10, adjoint=adjoint)
        if prec == hm.HELM_MIXED:
            assert info["max_relres"] <= 1e-12
        else:
            assert 0.0 <= info["max_relres"] <= 1e-12
        assert _colerr(X, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [hm.HELM_FP64, hm.HELM_MIXED])
def test_noalloc_solve_matches_oracle(prec):
    op, B, m, om, Bh = _case(nx=30, nz=26, nrhs=3, seed=6)
    f = hm.helm_factor(op, prec)
    X = torch.empty_like(B)
    X, _ = hm.helm_solve_noalloc(f, B, X, rtol=1e-12, max_iter=10)
    g = H.Grid(30, 26)
    for q, w in enumerate(om):
        ref = H.Factor(H.helmholtz_matrix(g, m, w)).solve(Bh[q])
        assert _colerr(X[q], ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [hm.HELM_FP64, hm.HELM_MIXED])
def test_noalloc_solve_allocates_nothing_on_a_fresh_factor(prec):
    import gc
    op, B, _, _, _ = _case(nrhs=5, seed=7)
    X = torch.empty_like(B)
    f = hm.helm_factor(op, prec)             # fresh: no solve has reserved working memory yet
    gc.collect()                             # handles of earlier tests are freed before, not during
    gc.disable()
    try:
        torch.cuda.synchronize()
        used0 = _pool_used_bytes()
        hm.helm_solve_noalloc(f, B, X, rtol=1e-12, max_iter=10)
        hm.helm_solve_noalloc(f, B, X, rtol=1e-12, max_iter=10, adjoint=True)
        torch.cuda.synchronize()
        used1 = _pool_used_bytes()
        # the counter does see the working memory that helm_solve reserves on its first call
        hm.helm_solve(f, B, X, rtol=1e-12, max_iter=10)
        torch.cuda.synchronize()
        used2 = _pool_used_bytes()
    finally:
        gc.enable()
    assert used1 == used0
    assert used2 > used0


def test_noalloc_solve_rejects_sizes_beyond_its_array():
    op, B, _, _, _ = _case(nrhs=2)
    f = hm.helm_factor(op, hm.HELM_MIXED)
    big = torch.zeros((op.n_omega, 400, op.N), dtype=torch.complex128, device="cuda")   # ~98 MB of scratch
    with pytest.raises(hm.HelmError) as e:
        hm.helm_solve_noalloc(f, big, torch.empty_like(big))
    assert e.value.status == 1
