"""The algebra of the level-0 block inverse of the block-cyclic-reduction factor, in numpy.

A complex symmetric tridiagonal block D = [[D11, D21^T], [D21, D22]] (the line block of A: its
diagonal and the line's vertical couplings) has an off-diagonal block D21 = c e_0 e_{n1-1}^T
with a single entry, so its 2 x 2 block inverse needs two half-size inverses and rank-one
updates only (x = X11[:, n1 - 1], X11 = D11^{-1}):
    S = D22 - c^2 X11[n1-1, n1-1] e_0 e_0^T,  X22 = S^{-1},
    X12 = -c x X22[0, :],  X21 = X12^T,  X11 <- X11 + c^2 X22[0, 0] x x^T.
The GPU kernels compute exactly these steps; here they are checked against numpy's inverse on
random and Helmholtz-like blocks, for even and uneven halves."""
import numpy as np
import pytest


def _tridiag(rng, n, helmholtz):
    if helmholtz:   # 4 - k^2 h^2 - i omega h b sqrt(m) on the diagonal, -1 couplings (indefinite)
        d = 4.0 - rng.uniform(0.5, 3.5, n) - 1j * rng.uniform(0.0, 0.2, n)
        c = -1.0 + 0.0j
    else:
        d = rng.standard_normal(n) + 1j * rng.standard_normal(n) + 3.0
        c = complex(rng.standard_normal(), rng.standard_normal())
    D = np.diag(d).astype(np.complex128)
    i = np.arange(n - 1)
    D[i, i + 1] = c
    D[i + 1, i] = c
    return D, c


def _rank_one_inverse(D, n1, c):
    n = D.shape[0]
    X11 = np.linalg.inv(D[:n1, :n1])
    x = X11[:, n1 - 1].copy()
    S = D[n1:, n1:].copy()
    S[0, 0] -= c * c * X11[n1 - 1, n1 - 1]
    X22 = np.linalg.inv(S)
    X = np.empty((n, n), dtype=np.complex128)
    X[n1:, n1:] = X22
    X[:n1, n1:] = -c * np.outer(x, X22[0, :])
    X[n1:, :n1] = X[:n1, n1:].T
    X[:n1, :n1] = X11 + c * c * X22[0, 0] * np.outer(x, x)
    return X


@pytest.mark.parametrize("n,n1", [(256, 128), (200, 128), (130, 128), (16, 8)])
@pytest.mark.parametrize("helmholtz", [False, True])
def test_rank_one_block_inverse_matches_numpy(n, n1, helmholtz):
    rng = np.random.default_rng(n + n1 + helmholtz)
    D, c = _tridiag(rng, n, helmholtz)
    ref = np.linalg.inv(D)
    X = _rank_one_inverse(D, n1, c)
    assert np.linalg.norm(X - ref) <= 1e-10 * np.linalg.norm(ref) * np.linalg.cond(D)
    # a planted slip (the corner correction with the wrong sign) is caught
    S_bad = D[n1:, n1:].copy()
    S_bad[0, 0] += c * c * np.linalg.inv(D[:n1, :n1])[n1 - 1, n1 - 1]
    assert not np.allclose(np.linalg.inv(S_bad), ref[n1:, n1:], rtol=1e-6, atol=0)
