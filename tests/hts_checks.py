"""Checks shared by the oracle pins and the GPU parity tests.

Nothing here calls the oracle or the GPU library: these are independent textbook routines
(a Givens-rotation Moler-Stewart HT reduction) and residual / invariant computations that
use only numpy.
"""
from __future__ import annotations

import numpy as np


def _sgn(x):
    return 1.0 if x >= 0 else -1.0


def givens_ht(A, B):
    """Textbook one-stage HT reduction with Givens rotations (Moler & Stewart) of a pencil
    whose B is upper triangular.  Returns (H, T, Q, Z) with A = Q H Z^T, B = Q T Z^T.
    Rotations act on rows/columns 2..n only, so Q e_1 = e_1 and Z e_1 = e_1."""
    A = np.array(A, dtype=np.float64)
    B = np.array(B, dtype=np.float64)
    n = A.shape[0]
    Q = np.eye(n)
    Z = np.eye(n)
    for j in range(n - 2):
        for i in range(n - 1, j + 1, -1):
            a, b = A[i - 1, j], A[i, j]
            rr = np.hypot(a, b)
            if rr != 0.0:
                c, s = a / rr, b / rr
                G = np.array([[c, s], [-s, c]])
                A[i - 1:i + 1, :] = G @ A[i - 1:i + 1, :]
                B[i - 1:i + 1, :] = G @ B[i - 1:i + 1, :]
                Q[:, i - 1:i + 1] = Q[:, i - 1:i + 1] @ G.T
            A[i, j] = 0.0
            # B(i, i-1) is now filled; rotate columns i-1, i to remove it
            a, b = B[i, i - 1], B[i, i]
            rr = np.hypot(a, b)
            if rr != 0.0:
                c, s = b / rr, a / rr
                G2 = np.array([[c, s], [-s, c]])
                B[:, i - 1:i + 1] = B[:, i - 1:i + 1] @ G2
                A[:, i - 1:i + 1] = A[:, i - 1:i + 1] @ G2
                Z[:, i - 1:i + 1] = Z[:, i - 1:i + 1] @ G2
            B[i, i - 1] = 0.0
    return A, B, Q, Z


def canonical(H, T, Q, Z, B_in=None):
    """Remove the diagonal sign freedom of an HT decomposition: choose D_Q, D_Z = diag(+-1)
    with d_q1 = +1, T_ii >= 0 and H_{i+1,i} >= 0, then (if B_in is given) flip Q and Z
    together so that Q(:,1) . B_in(:,1) >= 0.  Returns (D_Q H D_Z, D_Q T D_Z, Q D_Q, Z D_Z)."""
    H = np.array(H, dtype=np.float64)
    T = np.array(T, dtype=np.float64)
    n = H.shape[0]
    dq = np.ones(n)
    dz = np.ones(n)
    for i in range(n):
        dz[i] = _sgn(dq[i] * T[i, i])
        if i + 1 < n:
            dq[i + 1] = _sgn(H[i + 1, i] * dz[i])
    Hc = dq[:, None] * H * dz[None, :]
    Tc = dq[:, None] * T * dz[None, :]
    Qc = None if Q is None else np.array(Q, dtype=np.float64) * dq[None, :]
    Zc = None if Z is None else np.array(Z, dtype=np.float64) * dz[None, :]
    if B_in is not None and Qc is not None and Zc is not None:
        if float(Qc[:, 0] @ np.asarray(B_in, dtype=np.float64)[:, 0]) < 0:
            Qc, Zc = -Qc, -Zc
    return Hc, Tc, Qc, Zc


def last_nonzero_rows(M):
    """1-based index of the last row holding a nonzero in each column (0 if none)."""
    M = np.asarray(M)
    out = []
    for c in range(M.shape[1]):
        nz = np.nonzero(M[:, c] != 0)[0]
        out.append(int(nz[-1]) + 1 if nz.size else 0)
    return out


def below_band(M, band):
    """Largest |M_ij| with i > j + band (band = 1: Hessenberg, 0: triangular)."""
    M = np.asarray(M, dtype=np.float64)
    L = np.tril(M, -band - 1)
    return float(np.abs(L).max()) if L.size else 0.0


def rel_residual(Q, H, Z, A):
    """||Q H Z^T - A||_F / ||A||_F."""
    Q, H, Z, A = (np.asarray(x, dtype=np.float64) for x in (Q, H, Z, A))
    return float(np.linalg.norm(Q @ H @ Z.T - A) / np.linalg.norm(A))


def orth_error(Q):
    """||Q^T Q - I||_F / sqrt(n)."""
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[0]
    return float(np.linalg.norm(Q.T @ Q - np.eye(n)) / np.sqrt(n))


def det_identity_error(A, B, H, T, Q, Z, lams):
    """Max over lambda of the mismatch between det(A - lam B) and det(Q) det(Z) det(H - lam T),
    compared through slogdet: returns (max relative log|det| mismatch, all signs equal)."""
    worst = 0.0
    signs_ok = True
    sq, lq = np.linalg.slogdet(Q)
    sz, lz = np.linalg.slogdet(Z)
    for lam in lams:
        s1, l1 = np.linalg.slogdet(A - lam * B)
        s2, l2 = np.linalg.slogdet(H - lam * T)
        s2 = s2 * sq * sz
        l2 = l2 + lq + lz
        worst = max(worst, abs(l1 - l2) / max(1.0, abs(l1)))
        signs_ok &= bool(s1 == s2)
    return worst, signs_ok


def rht_pencil_checks(A_in, B_in, H, T, Q, Z):
    """Dictionary of the invariants every HT decomposition must satisfy."""
    return {
        "H_below_hessenberg": below_band(H, 1),
        "T_below_diag": below_band(T, 0),
        "bwd_A": rel_residual(Q, H, Z, A_in),
        "bwd_B": rel_residual(Q, T, Z, B_in),
        "orth_Q": orth_error(Q),
        "orth_Z": orth_error(Z),
    }
