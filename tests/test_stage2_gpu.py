"""GPU parity of stage 2 (r-HT -> HT) through the C ABI against the CPU oracle (Alg. 2).

The HT decomposition is unique up to diagonal signs once Q e1 is fixed (both the GPU's
blocked schedule and the oracle's unblocked one leave row/column 1 alone), so H, T, Q, Z are
compared element by element after sign normalisation, within 1e-12 * n relative.  Each case
also checks exact structural zeros, backward errors, orthogonality and the fixed first
columns.  Full-size pencils (n = 4096 and 8192, r = 16) are checked through properties that
hold at any size, with residual products formed by cuBLAS DGEMM (independent of both
implementations).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hts_checks import canonical, rht_pencil_checks  # noqa: E402
from paper_2301_07964_gb300 import binding as b  # noqa: E402
from paper_2301_07964_gb300.inputs import random_rht_pencil  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def red():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_07964_gb300 import build
    build.build()
    from paper_2301_07964_gb300.device import Reducer
    r = Reducer(0)
    yield r
    r.close()


def _gpu_stage2(red, A, B, r, q, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, flags=0, Q0=None, Z0=None,
                stream=None):
    from paper_2301_07964_gb300.device import colmajor_empty, to_device, to_host
    n = A.shape[0]
    dA, dB = to_device(A), to_device(B)
    dQ = to_device(Q0) if Q0 is not None else colmajor_empty(n)
    dZ = to_device(Z0) if Z0 is not None else colmajor_empty(n)
    red.stage2(dA, dB, r, dQ if compq else None, dZ if compz else None, compq=compq, compz=compz, q=q,
               flags=flags, stream=stream)
    st, info = red.sync_status(stream)
    assert st == b.HTS_OK, (b.status_string(st), info)
    return tuple(to_host(x) for x in (dA, dB, dQ, dZ))


def _compare(oracle, A, B, r, H, T, Q, Z, tol_scale=1e-12):
    n = A.shape[0]
    Ho, To, Qo, Zo = oracle.stage2(A, B, r)
    g = canonical(H, T, Q, Z)
    o = canonical(Ho, To, Qo, Zo)
    scale = max(1.0, float(np.abs(A).max()), float(np.abs(B).max()))
    return max(float(np.abs(x - y).max()) for x, y in zip(g, o)) / scale, tol_scale * n


CASES = [  # n, r, q
    (5, 2, 1), (10, 3, 2), (10, 3, 3), (33, 8, 8), (64, 2, 2), (64, 3, 1), (64, 3, 2), (64, 3, 3),
    (97, 4, 3), (100, 8, 8), (129, 8, 5), (150, 5, 5), (256, 8, 1), (256, 8, 8), (255, 16, 7),
    (256, 16, 16), (300, 32, 32), (301, 32, 13), (200, 31, 9),
]


@pytest.mark.parametrize("n,r,q", CASES)
def test_stage2_matches_oracle(red, oracle_mod, n, r, q):
    A, B = random_rht_pencil(n, r, 1000 * n + 10 * r + q)
    H, T, Q, Z = _gpu_stage2(red, A, B, r, q)
    c = rht_pencil_checks(A, B, H, T, Q, Z)
    assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c
    for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
        assert c[key] < 1e-14 * max(n, 10), c
    e1 = np.eye(n)[:, 0]
    assert np.array_equal(Q[:, 0], e1) and np.array_equal(Z[:, 0], e1)
    assert np.array_equal(Q[0, :], e1) and np.array_equal(Z[0, :], e1)
    err, tol = _compare(oracle_mod, A, B, r, H, T, Q, Z)
    assert err <= tol, "max |GPU - oracle| = %.3e > %.3e" % (err, tol)


@pytest.mark.parametrize("n,r,q", [(33, 8, 8), (129, 8, 5), (255, 16, 7), (256, 16, 16)])
def test_rq_fallback_matches_oracle(red, oracle_mod, n, r, q):
    """The r <= 16 chase finds each opposite reflector's direction by pivoted elimination and
    falls back to the RQ of the B block when the residual check fails; HTS_FLAG_TEST_DIRECT_RQ
    takes the fallback in every step, which must meet the same bar."""
    A, B = random_rht_pencil(n, r, 3000 * n + 10 * r + q)
    H, T, Q, Z = _gpu_stage2(red, A, B, r, q, flags=b.HTS_FLAG_TEST_DIRECT_RQ)
    c = rht_pencil_checks(A, B, H, T, Q, Z)
    assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c
    for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
        assert c[key] < 1e-14 * max(n, 10), c
    err, tol = _compare(oracle_mod, A, B, r, H, T, Q, Z)
    assert err <= tol, "max |GPU - oracle| = %.3e > %.3e" % (err, tol)
    # both paths find the same reduction (the direction is unique up to scale)
    H2, T2, Q2, Z2 = _gpu_stage2(red, A, B, r, q)
    g, g2 = canonical(H, T, Q, Z), canonical(H2, T2, Q2, Z2)
    scale = max(1.0, float(np.abs(A).max()), float(np.abs(B).max()))
    assert max(float(np.abs(x - y).max()) for x, y in zip(g, g2)) / scale <= 1e-12 * n


@pytest.mark.parametrize("n,r,q", [(128, 8, 4), (200, 16, 16)])
def test_structure_exact_without_final_cleanup(red, n, r, q):
    """The chase annihilates every entry exactly where it reduces it, so the structural
    zeros are exact even without the final zeroing pass."""
    A, B = random_rht_pencil(n, r, 77 + n)
    H, T, Q, Z = _gpu_stage2(red, A, B, r, q, flags=b.HTS_FLAG_NO_CLEAN)
    c = rht_pencil_checks(A, B, H, T, Q, Z)
    assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c


def test_comp_modes(red, oracle_mod):
    n, r, q = 80, 6, 4
    A, B = random_rht_pencil(n, r, 5)
    rng = np.random.default_rng(6)
    Q0 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Z0 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    # UPDATE multiplies into the given factors
    H, T, Q, Z = _gpu_stage2(red, A, B, r, q, compq=b.HTS_COMP_UPDATE, compz=b.HTS_COMP_UPDATE, Q0=Q0, Z0=Z0)
    A_in, B_in = Q0 @ A @ Z0.T, Q0 @ B @ Z0.T
    c = rht_pencil_checks(A_in, B_in, H, T, Q, Z)
    assert max(c["bwd_A"], c["bwd_B"], c["orth_Q"], c["orth_Z"]) < 1e-13, c
    # NONE leaves the buffers alone and gives the same H, T
    H2, T2, Qn, Zn = _gpu_stage2(red, A, B, r, q, compq=b.HTS_COMP_NONE, compz=b.HTS_COMP_NONE, Q0=Q0, Z0=Z0)
    assert np.array_equal(Qn, Q0) and np.array_equal(Zn, Z0)
    H3, T3, _, _ = _gpu_stage2(red, A, B, r, q)
    assert np.array_equal(H2, H3) and np.array_equal(T2, T3)
    assert np.array_equal(H, H3) and np.array_equal(T, T3)


def test_r1_and_tiny_are_noops(red):
    A, B = random_rht_pencil(40, 1, 3)
    H, T, Q, Z = _gpu_stage2(red, A, B, 1, 1)
    assert np.array_equal(H, A) and np.array_equal(T, B)
    assert np.array_equal(Q, np.eye(40)) and np.array_equal(Z, np.eye(40))
    for n in (1, 2):
        A, B = random_rht_pencil(n, 1, n)
        H, T, Q, Z = _gpu_stage2(red, A, B, 1, 1)
        assert np.array_equal(H, A) and np.array_equal(Q, np.eye(n))


def test_n3_hand_case(red):
    """n = 3, B = I, A(2:3, 1) = (3, 4): H(2, 1) = -5, T = diag(1, +-1, +-1)."""
    A = np.array([[1.0, 2.0, 3.0], [3.0, 5.0, 7.0], [4.0, 11.0, 13.0]], order="F")
    H, T, Q, Z = _gpu_stage2(red, A, np.eye(3, order="F"), 2, 1)
    assert abs(H[1, 0] + 5.0) < 1e-15 and H[2, 0] == 0.0
    assert abs(T[0, 0] - 1.0) < 1e-15 and np.abs(np.abs(np.diag(T)) - 1).max() < 1e-15
    assert np.abs(np.triu(T, 1)).max() < 1e-15


def test_bad_arguments(red):
    from paper_2301_07964_gb300.device import colmajor_empty
    n = 32
    A, B = colmajor_empty(n), colmajor_empty(n)
    work = red.workspace(n, 4)
    f = b.hts_reduce_stage2
    assert f(red.ctx, n, 4, A, n - 1, B, n, 0, None, 1, 0, None, 1, 0, None, work, work.numel()) == b.HTS_ERR_ARG
    assert f(red.ctx, n, 4, A, n, B, n, 0, None, 1, 0, None, 1, 0, None, None, 0) == b.HTS_ERR_WORKSPACE
    assert f(red.ctx, n, 4, A, n, B, n, 0, None, 1, 0, None, 1, 0, None, work, 8) == b.HTS_ERR_WORKSPACE
    assert f(red.ctx, n, 4, A, n, B, n, 0, None, 1, 0, None, 1, 0, b.hts_params(q=5), work,
             work.numel()) == b.HTS_ERR_ARG
    assert f(red.ctx, n, 4, A, n, B, n, 1, None, 1, 0, None, 1, 0, None, work, work.numel()) == b.HTS_ERR_ARG
    assert f(red.ctx, n, 40, A, n, B, n, 0, None, 1, 0, None, 1, 0, None, work, work.numel()) == b.HTS_ERR_UNSUPPORTED


def test_bounded_wait_reports_timeout_and_context_survives(red):
    """Fault injection on the host side of the protocol: the first sweep never publishes
    its progress, the next block's bounded wait ends after ~2 s with HTS_ERR_TIMEOUT, and the
    context stays usable for a correct call afterwards."""
    from paper_2301_07964_gb300.device import to_device
    n, r = 64, 4
    A, B = random_rht_pencil(n, r, 9)
    dA, dB = to_device(A), to_device(B)
    red.stage2(dA, dB, r, q=4, flags=b.HTS_FLAG_TEST_STALL)
    st, info = red.sync_status()
    assert st == b.HTS_ERR_TIMEOUT
    # group 0; the first sweep's helper block and every later sweep wait on the stalled block
    # (directly or through their predecessor) and run out at about the same time, so the
    # first one recorded may be any of sweeps 1 .. q
    assert info[1] == 0 and 1 <= info[3] <= 4
    H, T, Q, Z = _gpu_stage2(red, A, B, r, 4)
    c = rht_pencil_checks(A, B, H, T, Q, Z)
    assert c["T_below_diag"] == 0.0 and c["bwd_A"] < 1e-13


def test_side_stream(red, oracle_mod):
    n, r, q = 120, 8, 8
    A, B = random_rht_pencil(n, r, 4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        H, T, Q, Z = _gpu_stage2(red, A, B, r, q, stream=s)
    err, tol = _compare(oracle_mod, A, B, r, H, T, Q, Z)
    assert err <= tol


def _device_properties(A, B, dH, dT, dQ, dZ):
    """Invariants at full size with the residual products on the GPU (cuBLAS DGEMM)."""
    n = A.shape[0]
    dA0 = torch.from_numpy(A).cuda()
    dB0 = torch.from_numpy(B).cuda()
    H, T, Q, Z = dH, dT, dQ, dZ
    out = {}
    out["H_below_hessenberg"] = float(torch.tril(H, -2).abs().max())
    out["T_below_diag"] = float(torch.tril(T, -1).abs().max())
    out["bwd_A"] = float(torch.linalg.norm(Q @ H @ Z.T - dA0) / torch.linalg.norm(dA0))
    out["bwd_B"] = float(torch.linalg.norm(Q @ T @ Z.T - dB0) / torch.linalg.norm(dB0))
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    out["orth_Q"] = float(torch.linalg.norm(Q.T @ Q - I) / n ** 0.5)
    out["orth_Z"] = float(torch.linalg.norm(Z.T @ Z - I) / n ** 0.5)
    out["Qe1"] = bool(torch.equal(Q[:, 0], I[:, 0]))
    out["Ze1"] = bool(torch.equal(Z[:, 0], I[:, 0]))
    return out


@pytest.mark.parametrize("n,r,q,seed", [(4096, 16, 16, 2), (8192, 16, 16, 4)])
def test_full_size_properties(red, n, r, q, seed):
    from paper_2301_07964_gb300.device import colmajor_empty, to_device
    A, B = random_rht_pencil(n, r, seed)
    dA, dB = to_device(A), to_device(B)
    dQ, dZ = colmajor_empty(n), colmajor_empty(n)
    red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=q)
    st, info = red.sync_status()
    assert st == b.HTS_OK, info
    p = _device_properties(A, B, dA, dB, dQ, dZ)
    assert p["H_below_hessenberg"] == 0.0 and p["T_below_diag"] == 0.0, p
    assert p["Qe1"] and p["Ze1"], p
    for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
        assert p[key] < 1e-12 * n, p


@pytest.mark.parametrize("n,r,q,mode", [(300, 16, 16, b.HTS_GEMM_FP64), (300, 16, 16, b.HTS_GEMM_EMU_BF16),
                                        (301, 32, 13, b.HTS_GEMM_FP64), (129, 8, 5, b.HTS_GEMM_FP64),
                                        (700, 16, 16, b.HTS_GEMM_EMU_BF16), (517, 16, 9, b.HTS_GEMM_EMU_BF16),
                                        (97, 4, 3, b.HTS_GEMM_FP64)])
def test_lookahead_and_serial_schedules_match_oracle(red, oracle_mod, n, r, q, mode):
    """The default schedule runs group g's delayed updates beside group g+1's chase (each chase
    step waits for the update tiles it touches); HTS_FLAG_SERIAL_UPDATES runs them after the
    chase.  Both must give the oracle's reduction, and agree with each other."""
    from paper_2301_07964_gb300.device import colmajor_empty, to_device, to_host
    A, B = random_rht_pencil(n, r, 5000 * n + 10 * r + q)
    res = []
    for flags in (0, b.HTS_FLAG_SERIAL_UPDATES):
        dA, dB = to_device(A), to_device(B)
        dQ, dZ = colmajor_empty(n), colmajor_empty(n)
        red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=q, flags=flags, mode=mode)
        st, info = red.sync_status()
        assert st == b.HTS_OK, (b.status_string(st), info)
        H, T, Q, Z = (to_host(x) for x in (dA, dB, dQ, dZ))
        c = rht_pencil_checks(A, B, H, T, Q, Z)
        assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c
        for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
            assert c[key] < 1e-14 * max(n, 10), c
        err, tol = _compare(oracle_mod, A, B, r, H, T, Q, Z)
        assert err <= tol, (flags, err, tol)
        res.append(canonical(H, T, Q, Z))
    scale = max(1.0, float(np.abs(A).max()), float(np.abs(B).max()))
    assert max(float(np.abs(x - y).max()) for x, y in zip(*res)) / scale <= 1e-12 * n
