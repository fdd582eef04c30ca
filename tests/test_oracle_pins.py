"""Pins for the CPU oracle: each test ties the oracle to something other than itself --
values and patterns the paper prints, closed forms, an independent textbook reduction,
library eigenvalue routines, invariants that any HT decomposition must satisfy, and a
higher-precision run of the same algorithm.  ``test_planted_mistakes_are_caught`` plants
plausible mistakes in copies of the oracle and checks that this battery catches each one.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from hts_checks import (below_band, canonical, det_identity_error, givens_ht,
                        last_nonzero_rows, orth_error, rel_residual, rht_pencil_checks)
from paper_2301_07964_gb300.inputs import random_pencil, random_rht_pencil

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "stage2_fig_n10_r3.txt")
ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle")


def _golden_profiles():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows.append((parts[0], int(parts[1]), parts[2], [int(x) for x in parts[3:]]))
    return rows


# ---------------------------------------------------------------------------------------
# the battery (each check returns a list of failure strings; empty = pass)
# ---------------------------------------------------------------------------------------

def check_larfg(oracle):
    """Closed forms of the Householder reflector in the dlarfg convention."""
    fails = []
    for prec in ("d", "ld"):
        cases = [  # x, beta, tau, v
            ([3.0, 4.0], -5.0, 1.6, [1.0, 0.5]),
            ([-3.0, 4.0], 5.0, 1.6, [1.0, -0.5]),
            ([0.0, 2.0], -2.0, 1.0, [1.0, 1.0]),
            ([-3.0, 0.0], -3.0, 0.0, [1.0, 0.0]),
            ([2.0, 0.0, 0.0], 2.0, 0.0, [1.0, 0.0, 0.0]),
            ([1.0, 2.0, 2.0], -3.0, 4.0 / 3.0, [1.0, 0.5, 0.5]),
        ]
        for x, beta, tau, v in cases:
            b, vv, t = oracle.larfg(x, precision=prec)
            if not (abs(float(b) - beta) < 1e-15 and abs(float(t) - tau) < 1e-15
                    and np.allclose(np.asarray(vv, dtype=float), v, atol=1e-15, rtol=0)):
                fails.append("larfg(%s, %s) = (%r, %r, %r)" % (x, prec, b, t, vv))
    # random vector: H x = beta e1 and H orthogonal
    x = np.random.default_rng(5).standard_normal(9)
    b, v, t = oracle.larfg(x)
    H = np.eye(9) - t * np.outer(v, v)
    y = H @ x
    if abs(y[0] - b) > 1e-14 or np.abs(y[1:]).max() > 1e-14 or np.abs(H.T @ H - np.eye(9)).max() > 1e-14:
        fails.append("larfg random vector")
    return fails


def check_figure(oracle):
    """Sparsity profiles of Alg. 2 at n = 10, r = 3 after each half step of the first
    sweep, against the paper's illustration of the unblocked algorithm."""
    fails = []
    A, B = random_rht_pencil(10, 3, 11)
    for state, hs, mat, prof in _golden_profiles():
        H, T, _, _ = oracle.stage2(A, B, 3, max_half_steps=hs)
        got = last_nonzero_rows(H if mat == "A" else T)
        if got != prof:
            fails.append("%s %s: %s != %s" % (state, mat, got, prof))
    return fails


def check_vs_givens(oracle):
    """Stage 2 alone and the full reduction against the textbook Givens reduction: the HT
    form is unique up to signs once Q e1 is fixed, so canonical forms must agree."""
    fails = []
    for n, r, seed in ((5, 2, 1), (8, 3, 2), (10, 3, 3), (11, 2, 4)):
        A, B = random_rht_pencil(n, r, seed)
        H, T, Q, Z = oracle.stage2(A, B, r)
        G = givens_ht(A, B)
        c1, c2 = canonical(H, T, Q, Z), canonical(*G)
        err = max(np.abs(a - b).max() for a, b in zip(c1, c2))
        if err > 1e-13:
            fails.append("stage2 vs Givens n=%d r=%d: %.2e" % (n, r, err))
        if not (np.array_equal(Q[:, 0], np.eye(n)[:, 0]) and np.array_equal(Z[:, 0], np.eye(n)[:, 0])):
            fails.append("stage2 Q e1 / Z e1 not exactly e1 (n=%d)" % n)
    for n, r, seed in ((6, 2, 5), (9, 2, 6), (10, 3, 7)):
        A, B = random_pencil(n, seed)
        H, T, Q, Z = oracle.reduce(A, B, r, p=3)
        Q0, R0 = np.linalg.qr(B)
        G = givens_ht(Q0.T @ A, R0)
        Hg, Tg, Qg, Zg = G
        c1 = canonical(H, T, Q, Z, B_in=B)
        c2 = canonical(Hg, Tg, Q0 @ Qg, Zg, B_in=B)
        err = max(np.abs(a - b).max() for a, b in zip(c1, c2))
        if err > 1e-12:
            fails.append("reduce vs QR+Givens n=%d: %.2e" % (n, err))
    return fails


def check_invariants(oracle):
    """Structure, backward error, orthogonality and det(A - lam B) on larger pencils."""
    fails = []
    lam = np.random.default_rng(99).standard_normal(3)
    for n, r in ((37, 4), (64, 8), (50, 3)):
        A, B = random_rht_pencil(n, r, n + r)
        H, T, Q, Z = oracle.stage2(A, B, r)
        c = rht_pencil_checks(A, B, H, T, Q, Z)
        tol = 1e-14 * n
        if c["H_below_hessenberg"] != 0 or c["T_below_diag"] != 0:
            fails.append("stage2 structure n=%d r=%d" % (n, r))
        for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
            if not c[key] < tol:
                fails.append("stage2 %s=%.2e n=%d r=%d" % (key, c[key], n, r))
        d, signs = det_identity_error(A, B, H, T, Q, Z, lam)
        if d > 1e-10 or not signs:
            fails.append("det identity n=%d: %.2e %s" % (n, d, signs))
    for n, r, p in ((40, 4, 3), (57, 5, 4), (64, 8, 8)):
        A, B = random_pencil(n, n * 7 + r)
        A1, B1, Q0 = oracle.stage0(A, B)
        if below_band(B1, 0) != 0 or rel_residual(Q0, B1, np.eye(n), B) > 1e-14 * n:
            fails.append("stage0 n=%d" % n)
        A2, B2, Q1, Z1 = oracle.stage1(A1, B1, r, p, Q=Q0)
        if below_band(A2, r) != 0 or below_band(B2, 0) != 0:
            fails.append("stage1 structure n=%d r=%d p=%d: %.2e %.2e" % (n, r, p, below_band(A2, r), below_band(B2, 0)))
        if rel_residual(Q1, A2, Z1, A) > 1e-14 * n or rel_residual(Q1, B2, Z1, B) > 1e-14 * n:
            fails.append("stage1 backward error n=%d" % n)
        if orth_error(Q1) > 1e-14 * n or orth_error(Z1) > 1e-14 * n:
            fails.append("stage1 orthogonality n=%d" % n)
        if not np.array_equal(Z1[:, 0], np.eye(n)[:, 0]):
            fails.append("stage1 Z e1 != e1 n=%d" % n)
        H, T, Q, Z = oracle.stage2(A2, B2, r, Q=Q1, Z=Z1)
        c = rht_pencil_checks(A, B, H, T, Q, Z)
        if c["H_below_hessenberg"] != 0 or c["T_below_diag"] != 0 or max(
                c[k] for k in ("bwd_A", "bwd_B", "orth_Q", "orth_Z")) > 1e-14 * n:
            fails.append("full reduction n=%d: %s" % (n, c))
    return fails


def check_hand_n3(oracle):
    """n = 3, r = 2, B = I, A(2:3, 1) = (3, 4): one left reflector with beta = -5 and an
    orthogonal B block, so H(2, 1) = -5 and T = diag(1, +-1, +-1) exactly up to rounding."""
    A = np.array([[1.0, 2.0, 3.0], [3.0, 5.0, 7.0], [4.0, 11.0, 13.0]], order="F")
    B = np.eye(3, order="F")
    H, T, Q, Z = oracle.stage2(A, B, 2)
    fails = []
    if abs(H[1, 0] + 5.0) > 1e-15 or H[2, 0] != 0.0:
        fails.append("n=3 H(2:3,1) = %r" % H[1:, 0])
    if abs(T[0, 0] - 1.0) > 1e-15 or np.abs(np.abs(np.diag(T)) - 1.0).max() > 1e-15 \
            or np.abs(np.triu(T, 1)).max() > 1e-15 or T[1, 0] != 0 or T[2, 0] != 0 or T[2, 1] != 0:
        fails.append("n=3 T = %r" % T)
    if rel_residual(Q, H, Z, A) > 1e-15 * 10:
        fails.append("n=3 residual")
    return fails


def check_r1_noop(oracle):
    """r = 1: the input is already HT; every reflector has length 1 and the stage is a no-op."""
    A, B = random_rht_pencil(12, 1, 3)
    H, T, Q, Z = oracle.stage2(A, B, 1)
    ok = (np.array_equal(H, A) and np.array_equal(T, B) and np.array_equal(Q, np.eye(12))
          and np.array_equal(Z, np.eye(12)))
    return [] if ok else ["r=1 not a no-op"]


def check_eigenvalues(oracle):
    """Generalised eigenvalues of (H, T) against scipy's QZ on the input pencil."""
    fails = []
    for n, r, seed in ((8, 3, 21), (12, 4, 22)):
        A, B = random_rht_pencil(n, r, seed)
        H, T, _, _ = oracle.stage2(A, B, r)
        e1 = scipy.linalg.eigvals(A, B)
        e2 = scipy.linalg.eigvals(H, T)
        cost = np.abs(e1[:, None] - e2[None, :])
        ri, ci = scipy.optimize.linear_sum_assignment(cost)
        if cost[ri, ci].max() > 1e-9 * max(1.0, np.abs(e1).max()):
            fails.append("eigenvalues n=%d" % n)
    return fails


def check_long_double(oracle):
    """FP64 oracle against the same algorithm in long double: the FP64 run must sit within
    FP64 rounding of the higher-precision one."""
    fails = []
    n, r = 48, 4
    A, B = random_rht_pencil(n, r, 31)
    Hd, Td, Qd, Zd = oracle.stage2(A, B, r)
    Hl, Tl, Ql, Zl = oracle.stage2(A, B, r, precision="ld")
    c1 = canonical(Hd, Td, Qd, Zd)
    c2 = canonical(*(np.asarray(x, dtype=np.float64) for x in (Hl, Tl, Ql, Zl)))
    err = max(np.abs(a - b).max() for a, b in zip(c1, c2))
    if err > 1e-12:
        fails.append("long double mismatch %.2e" % err)
    return fails


BATTERY = [check_larfg, check_figure, check_vs_givens, check_invariants, check_hand_n3,
           check_r1_noop, check_eigenvalues, check_long_double]


def run_battery(oracle):
    fails = []
    for chk in BATTERY:
        try:
            fails += chk(oracle)
        except Exception as e:  # a crash in a mutant counts as caught
            fails.append("%s raised %r" % (chk.__name__, e))
    return fails


# ---------------------------------------------------------------------------------------
# tests
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("chk", BATTERY, ids=[c.__name__ for c in BATTERY])
def test_oracle_pin(oracle_mod, chk):
    assert chk(oracle_mod) == []


def test_long_double_is_wider(oracle_mod):
    assert oracle_mod.ldbl_mant_dig() > 53


# Plausible mistakes: (description, exact text in hts_oracle_body.inc, replacement)
MUTANTS = [
    ("reflector sign convention", "REAL beta = (a >= 0 ? -1 : 1) * FN(pyth)(a, xnorm);",
     "REAL beta = (a >= 0 ? 1 : -1) * FN(pyth)(a, xnorm);"),
    ("tau sign", "REAL tau = (beta - a) / beta;", "REAL tau = (a - beta) / beta;"),
    ("dropped term in left dot", "for (int i = 0; i < m; ++i) s += v[i] * AT(M, ld, r0 + i, c);",
     "for (int i = 0; i < m - 1; ++i) s += v[i] * AT(M, ld, r0 + i, c);"),
    ("wrong sign in right update", "for (int x = xa; x <= xb; ++x) AT(M, ld, x, c0 + i) -= s[x - xa] * v[i];",
     "for (int x = xa; x <= xb; ++x) AT(M, ld, x, c0 + i) += s[x - xa] * v[i];"),
    ("norm scale dropped", "return scale * SQRT(ssq);", "return SQRT(ssq);"),
    ("i3 off by one block", "int i3 = (j + (k + 2) * r < n) ? j + (k + 2) * r : n;",
     "int i3 = (j + (k + 1) * r < n) ? j + (k + 1) * r : n;"),
    ("pivot column index", "int jb = j + ((k - 1) * r + 1 > 0 ? (k - 1) * r + 1 : 0);",
     "int jb = j + ((k - 1) * r + 1 > 0 ? (k - 1) * r + 1 : 1);"),
    ("transposed RQ factor", "for (int c = 1; c <= m; ++c) x[c - 1] = AT(G, m, c, 1);",
     "for (int c = 1; c <= m; ++c) x[c - 1] = AT(G, m, 1, c);"),
    ("Q update dropped in stage 2", "if (Q) FN(apply_right)(m, v, tau, Q, ldq, 1, n, i1);", ""),
    ("RQ stops one row early", "for (int s = m; s >= 2; --s) {", "for (int s = m; s >= 3; --s) {"),
    ("stage-1 block stride", "int i1 = j + nb + k * (p - 1) * nb;", "int i1 = j + nb + k * p * nb;"),
    ("stage-1 B rows", "FN(apply_right)(len, v, tau, B, ldb, 1, i2, i1 + t - 1);",
     "FN(apply_right)(len, v, tau, B, ldb, 1, i2 - 1, i1 + t - 1);"),
    ("stage-0 A not updated", "FN(apply_left)(m, v, tau, A, lda, j, 1, n);", ""),
]


def test_planted_mistakes_are_caught(oracle_mod, tmp_path):
    body = open(os.path.join(ORACLE_DIR, "hts_oracle_body.inc")).read()
    shutil.copy(os.path.join(ORACLE_DIR, "hts_oracle.c"), tmp_path / "hts_oracle.c")
    missed = []
    for i, (desc, old, new) in enumerate(MUTANTS):
        assert body.count(old) == 1, "mutation site not unique: " + desc
        (tmp_path / "hts_oracle_body.inc").write_text(body.replace(old, new))
        so = str(tmp_path / ("mutant%d.so" % i))
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               str(tmp_path / "hts_oracle.c"), "-o", so, "-lm"])
        with oracle_mod.using_library(so):
            fails = run_battery(oracle_mod)
        if not fails:
            missed.append(desc)
    assert missed == [], "planted mistakes not caught: %s" % missed
