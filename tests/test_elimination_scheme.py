"""The arithmetic of the chase's direction for the opposite reflector (reading R9), modelled
on the CPU bit for bit and checked against what the method requires.

The opposite reflector Z^ of a chase step needs only z with W z parallel to e_1, W the B block
after the left reflector (the first column of the RQ's accumulated right factor, Section
"Blocked stage one").  The GPU finds z by column elimination with partial pivoting, last row
first:
- the pivot p of a row is its active column of largest |x_c|, compared on the high 32 bits of
  the IEEE-754 encoding;
- with 2^e the power of two of x_p, a = x_p 2^-e and b_c = x_c 2^-e (b_c = 0 where the
  exponent arithmetic would leave the normal range); column c becomes a col_c - b_c col_p for
  every active c != p, each entry one rounded product and one fused multiply-add;
- the accumulated column operations M start at the identity, and z is the column no step
  retired.

The tests pin:
- the residual the reflector zeroes, max_i>0 |(W z)_i|, against max|W| max|z| on blocks like
  the chase's, graded and rank-deficient ones, and against the RQ direction;
- exact structure: a block that is already upper triangular gives z = e_1 with exact zeros;
- the sparse form of M used on the GPU (only the retired pivots' rows, with every active
  column's diagonal the same running product D) equals the dense M bit for bit.
"""
import struct
from fractions import Fraction

import numpy as np
import pytest


def _hi(x):
    return struct.unpack('<Q', struct.pack('<d', x))[0] >> 32


def _lo(x):
    return struct.unpack('<Q', struct.pack('<d', x))[0] & 0xffffffff


def _mk(h, l):
    return struct.unpack('<d', struct.pack('<Q', ((h & 0xffffffff) << 32) | (l & 0xffffffff)))[0]


def fma(a, b, c):
    """a b + c rounded once (exact in Fraction, then to the nearest double)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def elim_step(x, act):
    """Pivot, a and the multipliers b of one row x (16 entries) on the active columns."""
    keys = [(_hi(x[c]) & 0x7fffffff) if (act >> c) & 1 else 0 for c in range(16)]
    kmax = max(keys)
    if kmax == 0:
        return -1, 1.0, [0.0] * 16
    p = keys.index(kmax)
    hp = _hi(x[p])
    ebp = (hp >> 20) & 0x7ff
    a = _mk((hp & 0x800fffff) | 0x3ff00000, _lo(x[p]))
    b = [0.0] * 16
    for c in range(16):
        hx = _hi(x[c])
        ebx = (hx >> 20) & 0x7ff
        ebn = ebx - ebp + 1023
        if (act >> c) & 1 and c != p and ebx != 0 and ebn >= 1:
            b[c] = _mk((hx & 0x800fffff) | (ebn << 20), _lo(x[c]))
    return p, a, b


def direction(W0, sparse=False):
    """z for the m x m block W0, with the dense M or the sparse form (retired rows + D)."""
    m = W0.shape[0]
    W = np.zeros((16, 16))
    W[:m, :m] = W0
    M = np.eye(16)
    act = (1 << m) - 1
    retired = []
    D = 1.0
    for rho in range(m - 1, 0, -1):
        p, a, b = elim_step(list(W[rho]), act)
        if p < 0:
            continue
        cols = [c for c in range(16) if (act >> c) & 1 and c != p]
        for i in range(rho):
            vp = W[i, p]
            for c in cols:
                W[i, c] = fma(-b[c], vp, a * W[i, c])
        if sparse:
            rows = retired + [p]
            for r in rows:
                vp = D if r == p else M[r, p]
                for c in cols:
                    M[r, c] = fma(-b[c], vp, a * M[r, c])
        else:
            for r in range(16):
                vp = M[r, p]
                for c in cols:
                    M[r, c] = fma(-b[c], vp, a * M[r, c])
        retired.append(p)
        D = D * a
        act &= ~(1 << p)
    cs = (act & -act).bit_length() - 1
    if sparse:
        return np.array([D if r == cs else M[r, cs] for r in range(m)])
    return M[:m, cs].copy()


def residual(W0, z):
    r = W0 @ z
    return float(np.max(np.abs(r[1:])) / (np.max(np.abs(W0)) * np.max(np.abs(z))))


def rq_direction(W0):
    """The RQ's direction (numpy): the first column of Q^T in W0 = R Q."""
    q, _ = np.linalg.qr(W0[::-1, ::-1].T)
    return q[::-1, ::-1][:, 0]


def _block(kind, rng, m=16):
    if kind == "chase":          # triangular with a large diagonal, as the R factor of a Gaussian
        T = np.triu(rng.standard_normal((m, m)), 1) + np.diag(np.sqrt(rng.chisquare(4000 - np.arange(m))))
    elif kind == "graded":       # triangular factor of U diag(logspace(0, -12)) V^T
        U = np.linalg.qr(rng.standard_normal((m, m)))[0]
        V = np.linalg.qr(rng.standard_normal((m, m)))[0]
        T = np.linalg.qr(U @ np.diag(np.logspace(0, -12, m)) @ V.T)[1]
    else:                        # rank-deficient: two rows of the triangle vanish
        T = np.triu(rng.standard_normal((m, m)))
        T[4, 4:] = 0.0
        T[11, 11:] = 0.0
    x = rng.standard_normal(m)
    u = x.copy()
    u[0] += np.copysign(np.linalg.norm(x), x[0])
    return T - np.outer(u, (2.0 / (u @ u)) * (u @ T))   # after the left reflector


@pytest.mark.parametrize("kind", ["chase", "graded", "rank-deficient"])
def test_residual_within_the_kernel_bound(kind):
    rng = np.random.default_rng({"chase": 1, "graded": 2, "rank-deficient": 3}[kind])
    worst = 0.0
    for _ in range(6):
        W0 = _block(kind, rng)
        z = direction(W0)
        res = residual(W0, z)
        worst = max(worst, res)
        assert res <= 2.0 ** -44, res          # the kernel's acceptance test
        zr = rq_direction(W0)
        assert res <= 8.0 * max(residual(W0, zr), 2.0 ** -53)
    assert worst < 2.0 ** -49


def test_triangular_block_gives_e1_exactly():
    rng = np.random.default_rng(4)
    for m in (2, 5, 16):
        W0 = np.triu(rng.standard_normal((m, m)))
        z = direction(W0)
        assert z[0] != 0.0 and np.all(z[1:] == 0.0)


def test_sparse_column_operations_equal_dense_bitwise():
    rng = np.random.default_rng(6)
    for kind in ("chase", "rank-deficient"):
        W0 = _block(kind, rng)
        assert np.array_equal(direction(W0), direction(W0, sparse=True))
    for m in (2, 3, 7):
        W0 = rng.standard_normal((m, m))
        assert np.array_equal(direction(W0), direction(W0, sparse=True))


def test_direction_matches_the_unique_solution():
    # for a nonsingular block z is unique up to scale: compare with W^{-1} e_1
    rng = np.random.default_rng(7)
    W0 = _block("chase", rng)
    z = direction(W0)
    y = np.linalg.solve(W0, np.eye(16)[:, 0])
    cosang = abs(z @ y) / (np.linalg.norm(z) * np.linalg.norm(y))
    assert cosang > 1.0 - 1e-12
