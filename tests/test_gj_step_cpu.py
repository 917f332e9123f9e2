"""The algebra of one block Gauss-Jordan step as the batched inversion performs it, in numpy.

For pivot columns K = k0 .. k0 + 15 with P = W[K, K]^{-1}, the step is a single product
    W <- W' + A' R',  W' = W with the rows and columns K zeroed,
    A'[r, :] = -W[r, K] off the pivot rows, the identity rows on them,
    R' = P W[K, :] off the pivot columns, P on them,
which the GPU kernel accumulates into the block held in tensor memory.  Eight such steps over a
128 x 128 block must give its inverse; each step must equal the textbook in-place Gauss-Jordan
update (pivot rows scaled by P, the other rows eliminated, the pivot columns replaced)."""
import numpy as np
import pytest


def _one_product_step(W, k0, kb=16):
    K = slice(k0, k0 + kb)
    P = np.linalg.inv(W[K, K])
    R = P @ W[K, :]
    R[:, K] = P
    A = -W[:, K].copy()
    A[K, :] = np.eye(kb)
    Wp = W.copy()
    Wp[K, :] = 0
    Wp[:, K] = 0
    return Wp + A @ R


def _textbook_step(W, k0, kb=16):
    n = W.shape[0]
    K = np.arange(k0, k0 + kb)
    rest = np.setdiff1d(np.arange(n), K)
    P = np.linalg.inv(W[np.ix_(K, K)])
    out = np.empty_like(W)
    rows_k = P @ W[K, :]                                        # pivot rows scaled
    out[K, :] = rows_k
    out[np.ix_(rest, np.arange(n))] = W[rest, :] - W[np.ix_(rest, K)] @ rows_k   # eliminated
    out[np.ix_(K, K)] = P                                       # pivot columns replaced
    out[np.ix_(rest, K)] = -W[np.ix_(rest, K)] @ P
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_one_product_steps_invert_the_block(seed):
    rng = np.random.default_rng(seed)
    n = 128
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    M = (M + M.T) / 2 + 3.0 * np.sqrt(n) * np.eye(n)           # complex symmetric
    W = M.astype(np.complex128)
    for k0 in range(0, n, 16):
        step = _one_product_step(W, k0)
        assert np.allclose(step, _textbook_step(W, k0), rtol=1e-12, atol=1e-12)
        W = step
    ref = np.linalg.inv(M)
    assert np.linalg.norm(W - ref) <= 1e-12 * np.linalg.norm(ref) * np.linalg.cond(M)


def test_a_dropped_term_is_caught():
    # the pivot rows left in W' (not zeroed): the result is no longer the inverse
    rng = np.random.default_rng(5)
    n = 32
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4.0 * np.eye(n)
    W = M.copy()
    for k0 in range(0, n, 16):
        K = slice(k0, k0 + 16)
        P = np.linalg.inv(W[K, K])
        R = P @ W[K, :]
        R[:, K] = P
        A = -W[:, K].copy()
        A[K, :] = np.eye(16)
        Wp = W.copy()
        Wp[:, K] = 0   # rows K not zeroed
        W = Wp + A @ R
    assert not np.allclose(W, np.linalg.inv(M), rtol=1e-6, atol=1e-9)
