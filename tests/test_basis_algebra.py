"""The expansion behind the stored-basis assembly of the shifted solutions
(Algorithm 1's shifted updates), checked in FP64 on random blocks: running the
recurrences
    X^(s) += P^(s) alpha_k,   P^(s) = Q_k + P^(s) M2_k      (k = 1 .. L, P^(s)_0 = Q_0)
gives the same X^(s) and P^(s) as the sums over the stored blocks
    X^(s) = sum_{i < L} Q_i C_i,   C_{L-1} = alpha_L,  C_i = alpha_{i+1} + M2_{i+1} C_{i+1},
    P^(s)_K = sum_{i <= K} Q_i D_i, D_K = 1,         D_i = M2_{i+1} D_{i+1},
and the real embedding used for the GEMM reproduces the complex products."""
import numpy as np


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _recurrence(Q, alpha, M2, L):
    P = Q[0].copy()
    X = np.zeros_like(P)
    for k in range(1, L + 1):
        X = X + P @ alpha[k]
        P = Q[k] + P @ M2[k]
    return X, P


def _backward_X(Q, alpha, M2, L):
    C = alpha[L].copy()
    X = Q[L - 1] @ C
    for i in range(L - 2, -1, -1):
        C = alpha[i + 1] + M2[i + 1] @ C
        X = X + Q[i] @ C
    return X


def _backward_P(Q, M2, K):
    n = Q[0].shape[1]
    D = np.eye(n, dtype=complex)
    P = Q[K] @ D
    for i in range(K - 1, -1, -1):
        D = M2[i + 1] @ D
        P = P + Q[i] @ D
    return P


def test_backward_recursions_equal_the_recurrences():
    rng = np.random.default_rng(5)
    rows, n, L = 40, 4, 23
    Q = [_crandn(rng, rows, n) for _ in range(L + 1)]
    # contracting coefficients keep the products bounded, as in a converging solve
    alpha = [None] + [0.3 * _crandn(rng, n, n) for _ in range(L)]
    M2 = [None] + [0.25 * _crandn(rng, n, n) for _ in range(L)]
    X, P = _recurrence(Q, alpha, M2, L)
    assert np.allclose(_backward_X(Q, alpha, M2, L), X, rtol=0, atol=1e-12 * np.abs(X).max())
    assert np.allclose(_backward_P(Q, M2, L), P, rtol=0, atol=1e-12 * np.abs(P).max())
    # a shift that stopped updating at L' < L: its X uses blocks below L' only
    Lp = 11
    Xp, _ = _recurrence(Q, alpha, M2, Lp)
    assert np.allclose(_backward_X(Q, alpha, M2, Lp), Xp, rtol=0, atol=1e-12 * np.abs(Xp).max())


def test_real_embedding_reproduces_complex_products():
    """Row (x_0re, x_0im, x_1re, ...) times B with B[2q][2j] = Re C, B[2q][2j+1] = Im C,
    B[2q+1][2j] = -Im C, B[2q+1][2j+1] = Re C gives (y_0re, y_0im, ...) = x C."""
    rng = np.random.default_rng(6)
    n, m, rows = 5, 7, 9
    C = _crandn(rng, n, m)
    Xc = _crandn(rng, rows, n)
    B = np.zeros((2 * n, 2 * m))
    B[0::2, 0::2] = C.real
    B[0::2, 1::2] = C.imag
    B[1::2, 0::2] = -C.imag
    B[1::2, 1::2] = C.real
    Xr = np.stack([Xc.real, Xc.imag], axis=-1).reshape(rows, 2 * n)
    Yr = Xr @ B
    Y = Yr[:, 0::2] + 1j * Yr[:, 1::2]
    assert np.allclose(Y, Xc @ C, rtol=0, atol=1e-13)
