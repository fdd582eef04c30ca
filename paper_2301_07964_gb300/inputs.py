"""Seeded synthetic pencils.

This module is shared by the GPU tests, the benchmark and the oracle checks.  It draws random
numbers and arranges them into the shapes of the paper's workloads; it contains none of the
reduction's arithmetic.

The paper measures on random pencils whose B is QR-factorised first (Section
"Experiments") and on synthetic saddle-point pencils.  The generators below produce:

* ``random_pencil``          A, B iid N(0, 1)                             (dense input)
* ``ill_conditioned_pencil`` A iid N(0, 1), B = U diag(10^(-e i/(n-1))) V^T, U, V Haar
* ``random_rht_pencil``      an r-Hessenberg-triangular pencil: A iid N(0, 1) on and above
                             the r-th subdiagonal, zero below; B = the R factor of an iid
                             N(0, 1) matrix (the distribution stage 0 hands to stage 1)
* ``ill_conditioned_rht_pencil``  the r-HT pencil of the same family: A iid N(0, 1) on and
                             above the r-th subdiagonal, B = the R factor of
                             U diag(10^(-e i/(n-1))) V^T (condition number 10^e)
* ``saddle_point_pencil``    (A, B) = ([[X, Y], [Y^T, 0]], diag(I_m, 0)) with X = G G^T / m + I
                             symmetric positive definite, Y iid N(0, 1) and m = n - n // 8, so
                             that a quarter of the eigenvalues (2 (n - m)) are infinite
* ``batch_sizes``            pencil sizes n_i ~ U{32..512} with r_i = min(8, n_i // 8)

All arrays are float64 in Fortran (column-major) order.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_pencil(n: int, seed: int):
    """Dense pencil with A, B iid N(0, 1)."""
    g = _rng(seed)
    A = np.asfortranarray(g.standard_normal((n, n)))
    B = np.asfortranarray(g.standard_normal((n, n)))
    return A, B


def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the columns of Q
    multiplied by sign(diag(R)) (Mezzadri's recipe)."""
    X = g.standard_normal((n, n))
    Qm, R = np.linalg.qr(X)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Qm * d[None, :]


def ill_conditioned_pencil(n: int, seed: int, decades: float = 8.0):
    """A iid N(0, 1); B = U diag(logspace(0, -decades, n)) V^T with Haar U, V."""
    g = _rng(seed)
    A = np.asfortranarray(g.standard_normal((n, n)))
    U = haar_orthogonal(n, g)
    V = haar_orthogonal(n, g)
    s = 10.0 ** (-decades * np.arange(n) / max(n - 1, 1))
    B = np.asfortranarray((U * s[None, :]) @ V.T)
    return A, B


def random_rht_pencil(n: int, r: int, seed: int):
    """r-Hessenberg-triangular pencil: A(i, j) = 0 for i > j + r, B upper triangular."""
    g = _rng(seed)
    A = g.standard_normal((n, n))
    A = np.asfortranarray(np.triu(A, -r))
    X = g.standard_normal((n, n))
    B = np.linalg.qr(X, mode="r")
    B = np.asfortranarray(np.triu(B))
    return A, B


def ill_conditioned_rht_pencil(n: int, r: int, seed: int, decades: float = 8.0):
    """r-HT pencil with an ill-conditioned triangular B: A(i, j) iid N(0, 1) for i <= j + r
    (zero below), B = R of the QR factorisation of U diag(logspace(0, -decades, n)) V^T."""
    g = _rng(seed)
    A = np.asfortranarray(np.triu(g.standard_normal((n, n)), -r))
    U = haar_orthogonal(n, g)
    V = haar_orthogonal(n, g)
    s = 10.0 ** (-decades * np.arange(n) / max(n - 1, 1))
    B = np.linalg.qr((U * s[None, :]) @ V.T, mode="r")
    return A, np.asfortranarray(np.triu(B))


def saddle_point_pencil(n: int, seed: int):
    """Saddle-point pencil of the paper's experiment: A = [[X, Y], [Y^T, 0]] with X symmetric
    positive definite (X = G G^T / m + I) and Y iid N(0, 1); B = diag(I_m, 0) with
    m = n - n // 8, so that 2 (n - m) = n / 4 eigenvalues are infinite."""
    g = _rng(seed)
    m = n - n // 8
    G = g.standard_normal((m, m))
    X = G @ G.T / m + np.eye(m)
    Y = g.standard_normal((m, n - m))
    A = np.zeros((n, n))
    A[:m, :m] = X
    A[:m, m:] = Y
    A[m:, :m] = Y.T
    B = np.zeros((n, n))
    B[np.arange(m), np.arange(m)] = 1.0
    return np.asfortranarray(A), np.asfortranarray(B)


def batch_sizes(count: int, seed: int, lo: int = 32, hi: int = 512):
    """Sizes of a batch of pencils: n_i uniform in [lo, hi], r_i = min(8, n_i // 8)."""
    g = _rng(seed)
    n = g.integers(lo, hi + 1, size=count)
    r = np.minimum(8, n // 8)
    return n.astype(np.int64), r.astype(np.int64)
