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


def batch_sizes(count: int, seed: int, lo: int = 32, hi: int = 512):
    """Sizes of a batch of pencils: n_i uniform in [lo, hi], r_i = min(8, n_i // 8)."""
    g = _rng(seed)
    n = g.integers(lo, hi + 1, size=count)
    r = np.minimum(8, n // 8)
    return n.astype(np.int64), r.astype(np.int64)
