"""The tensor-core building blocks and the block-cyclic-reduction (BCR) factor.

helm_zgemm_batched (tcgen05, 3xTF32) against a complex128 product of the same FP32 inputs;
helm_zinv_batched against numpy's inverse of complex symmetric matrices, in shared memory
(n <= 128) and by the recursive 2 x 2 block inverse (n > 128); and the BCR factor of the
mixed path against the CPU oracle's sparse LU, element by element per column, at the mixed
tolerance 1e-8, on square, rectangular and ragged grids (nx not a power of two, odd nx)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import helmholtz as H

hm = pytest.importorskip("paper_2301_10762_gb300.helm")

pytestmark = pytest.mark.gpu


def _c64(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.mark.parametrize("M,N,K", [(128, 64, 128), (256, 256, 256), (96, 16, 160), (200, 40, 50), (130, 130, 34),
                                   (64, 24, 200)])
def test_zgemm_matches_complex128_product(M, N, K):
    rng = np.random.default_rng(M + N + K)
    b = 3
    A, Bt, C0 = _c64(rng, b, M, K), _c64(rng, b, N, K), _c64(rng, b, M, N)
    ref = C0.astype(np.complex128) - np.einsum("tmk,tnk->tmn", A.astype(np.complex128), Bt.astype(np.complex128))
    C = hm.helm_zgemm_batched(torch.tensor(A, device="cuda"), torch.tensor(Bt, device="cuda"),
                              torch.tensor(C0, device="cuda"), sign=-1.0)
    out = C.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    # 3xTF32 with FP32 accumulation: about FP32 accuracy (a single TF32 product is ~1e-3 off)
    assert err <= 1e-5, err
    C2 = hm.helm_zgemm_batched(torch.tensor(A, device="cuda"), torch.tensor(Bt, device="cuda"))
    ref2 = np.einsum("tmk,tnk->tmn", A.astype(np.complex128), Bt.astype(np.complex128))
    assert np.linalg.norm(C2.cpu().numpy() - ref2) / np.linalg.norm(ref2) <= 1e-5


@pytest.mark.parametrize("n", [32, 64, 100, 128, 160, 256])
def test_zinv_matches_numpy_inverse(n):
    rng = np.random.default_rng(n)
    b = 4
    M = _c64(rng, b, n, n)
    M = ((M + np.transpose(M, (0, 2, 1))) / 2 + 3.0 * np.sqrt(n) * np.eye(n)).astype(np.complex64)   # symmetric
    X = hm.helm_zinv_batched(torch.tensor(M, device="cuda")).cpu().numpy().astype(np.complex128)
    ref = np.linalg.inv(M.astype(np.complex128))
    err = np.linalg.norm(X - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err


@pytest.mark.parametrize("n", [128, 256])
def test_zinv_needs_pivoting(n):
    """Complex symmetric blocks with a small shift (zero and tiny diagonal entries, so the
    Gauss-Jordan pivots are chosen off the diagonal), against numpy's inverse; the bound scales
    with the condition number."""
    rng = np.random.default_rng(n + 7)
    b = 3
    M = _c64(rng, b, n, n)
    M = ((M + np.transpose(M, (0, 2, 1))) / 2 + 0.5 * np.sqrt(n) * np.eye(n)).astype(np.complex64)
    M[:, np.arange(0, n, 5), np.arange(0, n, 5)] = 0.0
    M64 = M.astype(np.complex128)
    X = hm.helm_zinv_batched(torch.tensor(M, device="cuda")).cpu().numpy().astype(np.complex128)
    for i in range(b):
        ref = np.linalg.inv(M64[i])
        err = np.linalg.norm(X[i] - ref) / np.linalg.norm(ref)
        assert err <= 2e-6 * np.linalg.cond(M64[i]), (i, err, np.linalg.cond(M64[i]))


def _oracle_cols(nx, nz, m, om, B):
    g = H.Grid(nx, nz)
    return [H.Factor(H.helmholtz_matrix(g, m, w)).solve(B[q]) for q, w in enumerate(om)]


@pytest.mark.parametrize("nx,nz,nrhs", [(48, 40, 3), (64, 64, 8), (37, 32, 5), (33, 50, 2), (128, 128, 16),
                                          (20, 200, 2)])
def test_bcr_solve_matches_oracle(nx, nz, nrhs):
    rng = np.random.default_rng(nx * nz)
    c = 1.0 + 0.5 * W.gaussian_smooth(rng.uniform(0, 1, (nx, nz)), 2.0)
    m = (1.0 / c ** 2).reshape(-1)
    om = np.array([4.0, 9.5, 17.0])
    B = rng.standard_normal((3, nrhs, nx * nz)) + 1j * rng.standard_normal((3, nrhs, nx * nz))
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    f = hm.helm_factor(op, hm.HELM_MIXED, method=hm.HELM_FACTOR_BCR)
    Bd = torch.tensor(B, device="cuda")
    X, info = hm.helm_solve(f, Bd, rtol=1e-12, max_iter=20)
    Y, _ = hm.helm_adjoint_solve(f, Bd, rtol=1e-12, max_iter=20)
    assert info["max_relres"] <= 1e-12
    g = H.Grid(nx, nz)
    Xc, Yc = X.cpu().numpy(), Y.cpu().numpy()
    for q, w in enumerate(om):
        fo = H.Factor(H.helmholtz_matrix(g, m, w))
        rx, ry = fo.solve(B[q]), fo.adjoint_solve(B[q])
        ex = np.max(np.linalg.norm(Xc[q] - rx, axis=1) / np.linalg.norm(rx, axis=1))
        ey = np.max(np.linalg.norm(Yc[q] - ry, axis=1) / np.linalg.norm(ry, axis=1))
        assert ex <= 1e-8 and ey <= 1e-8, (q, ex, ey)


def test_bcr_and_line_factors_agree_and_the_automatic_choice():
    """Both methods solve the same system to the refinement tolerance; the automatic choice is
    the line recurrence on short lines and BCR from nz = 192 on (mixed), the line factor for
    FP64, and BCR is refused for FP64."""
    nx, nz = 40, 36
    rng = np.random.default_rng(5)
    m = (1.0 / (1.0 + 0.4 * rng.uniform(0, 1, (nx, nz))) ** 2).reshape(-1)
    om = np.array([7.0])
    B = torch.tensor(rng.standard_normal((1, 4, nx * nz)) + 0j, device="cuda")
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    X = {}
    for meth in (hm.HELM_FACTOR_LINE, hm.HELM_FACTOR_BCR):
        f = hm.helm_factor(op, hm.HELM_MIXED, method=meth)
        assert f.method == meth
        X[meth], _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=20)
    ref = X[hm.HELM_FACTOR_LINE]
    err = torch.linalg.vector_norm(X[hm.HELM_FACTOR_BCR] - ref, dim=-1) / torch.linalg.vector_norm(ref, dim=-1)
    assert float(err.max()) <= 1e-10
    assert hm.helm_factor(op, hm.HELM_MIXED).method == hm.HELM_FACTOR_LINE
    assert hm.helm_factor(op, hm.HELM_FP64).method == hm.HELM_FACTOR_LINE
    with pytest.raises(hm.HelmError):
        hm.helm_factor(op, hm.HELM_FP64, method=hm.HELM_FACTOR_BCR)   # no FP64 tensor path
    m2 = np.full(20 * 192, 0.5)
    op2 = hm.helm_assemble(20, 192, 1.0, 1.0, torch.tensor(m2, device="cuda"), om)
    assert hm.helm_factor(op2, hm.HELM_MIXED).method == hm.HELM_FACTOR_BCR
