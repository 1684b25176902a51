"""The structure of the GPU's SR solve (Sec. 2.1: (O O^T / B + lambda) x = c),
checked on CPU in FP64 against a dense solve: the matrix padded to whole
64 x 64 blocks with the identity, a blocked right-looking Cholesky in which
each step stores X_k = L_kk^-T (the panel solve applied to the identity)
and leaves the diagonal block of A untouched, and the two triangular solves
as block reductions plus products with X_k^T and X_k.  A mistake in the
padding, the block order or the use of X_k fails the comparison."""
import numpy as np
import pytest

import oracle
from paper_2106_13308_gb300 import inputs

NB = 64


def _factor_and_solve(A_lower, B, rhs):
    T = (B + NB - 1) // NB
    N = T * NB
    A = np.eye(N)
    A[:B, :B] = np.tril(A_lower)
    X = np.zeros((T, NB, NB))
    for k in range(T):
        s = slice(k * NB, (k + 1) * NB)
        Lkk = np.linalg.cholesky(np.tril(A[s, s]) + np.tril(A[s, s], -1).T)
        X[k] = np.linalg.inv(Lkk).T                   # the panel solve on the identity
        for i in range(k + 1, T):                      # panels in place: A_ik L_kk^-T
            r = slice(i * NB, (i + 1) * NB)
            A[r, s] = A[r, s] @ X[k]
        for i in range(k + 1, T):                      # trailing lower triangle
            for j in range(k + 1, i + 1):
                r, c = slice(i * NB, (i + 1) * NB), slice(j * NB, (j + 1) * NB)
                A[r, c] -= A[r, s] @ A[c, s].T
    y = np.zeros(N)
    y[:B] = rhs
    for k in range(T):                                 # L y = rhs
        s = slice(k * NB, (k + 1) * NB)
        y[s] = X[k].T @ (y[s] - A[s, :k * NB] @ y[:k * NB])
    for k in range(T - 1, -1, -1):                     # L^T x = y
        s = slice(k * NB, (k + 1) * NB)
        y[s] = X[k] @ (y[s] - A[(k + 1) * NB:, s].T @ y[(k + 1) * NB:])
    assert np.all(y[B:] == 0.0)
    return y[:B]


@pytest.mark.parametrize("B", [1, 64, 150, 200])
def test_blocked_solve_equals_a_dense_solve(B):
    n, h, lam = 10, 8, 1e-2
    theta = inputs.lively_params(n, h, 3)
    P = oracle.theta_to_made(theta, n, h)
    S = inputs.spins(B, n, 4)
    G = oracle.sr_gram(P, S, oracle.SIGMOID)
    A = G / B + lam * np.eye(B)
    c = np.random.default_rng(5).standard_normal(B)
    x = _factor_and_solve(A, B, c)
    assert np.allclose(x, np.linalg.solve(A, c), rtol=1e-9, atol=1e-12)
