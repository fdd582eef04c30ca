"""GPU stage 0 (QR of B), stage 1 (Alg. 1) and the full reduction through the C ABI.

Stage 1 runs the same algorithm as the oracle (the same p and n_b, the same reflector
conventions), so its r-HT output is compared with the oracle's element by element, besides
the invariants (exact r-HT structure, backward error, orthogonality, Z e1 = e1).  The full
reduction's HT form is unique up to signs once Q e1 = +-B(:,1)/||B(:,1)|| is fixed, so it is
compared with the oracle's in canonical signs (tolerance 1e-12 n, relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hts_checks import below_band, canonical, orth_error, rel_residual, rht_pencil_checks  # noqa: E402
from paper_2301_07964_gb300 import binding as b  # noqa: E402
from paper_2301_07964_gb300.inputs import ill_conditioned_pencil, random_pencil  # noqa: E402

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


def _dev(*Ms):
    from paper_2301_07964_gb300.device import to_device
    return [to_device(M) for M in Ms]


def _host(*ts):
    from paper_2301_07964_gb300.device import to_host
    return [to_host(t) for t in ts]


@pytest.mark.parametrize("n,r,p", [(40, 4, 3), (57, 5, 4), (100, 8, 8), (129, 16, 8), (200, 32, 4), (33, 2, 2)])
def test_stage1_matches_oracle(red, oracle_mod, n, r, p):
    from paper_2301_07964_gb300.device import colmajor_empty
    A, B0 = random_pencil(n, 100 * n + r)
    B = np.asfortranarray(np.triu(np.linalg.qr(B0)[1]))
    dA, dB = _dev(A, B)
    dQ, dZ = colmajor_empty(n), colmajor_empty(n)
    red.stage1(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, p=p)
    st, info = red.sync_status()
    assert st == b.HTS_OK, info
    A1, B1, Q1, Z1 = _host(dA, dB, dQ, dZ)
    assert below_band(A1, r) == 0.0 and below_band(B1, 0) == 0.0
    assert rel_residual(Q1, A1, Z1, A) < 1e-14 * n and rel_residual(Q1, B1, Z1, B) < 1e-14 * n
    assert orth_error(Q1) < 1e-14 * n and orth_error(Z1) < 1e-14 * n
    e1 = np.eye(n)[:, 0]
    assert np.array_equal(Z1[:, 0], e1) and np.array_equal(Q1[:, 0], e1)
    Ao, Bo, Qo, Zo = oracle_mod.stage1(A, B, r, p)
    scale = max(np.abs(A).max(), np.abs(B).max())
    err = max(np.abs(x - y).max() for x, y in zip((A1, B1, Q1, Z1), (Ao, Bo, Qo, Zo))) / scale
    assert err < 1e-12 * n, err


@pytest.mark.parametrize("n,r", [(10, 3), (64, 4), (256, 8), (300, 16), (257, 32)])
def test_reduce_matches_oracle(red, oracle_mod, n, r):
    """Full reduction of a dense pencil (config 1 is n = 256, r = 8)."""
    from paper_2301_07964_gb300.device import colmajor_empty
    A, B = random_pencil(n, n + 7 * r)
    dA, dB = _dev(A, B)
    dQ, dZ = colmajor_empty(n), colmajor_empty(n)
    red.reduce(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT)
    st, info = red.sync_status()
    assert st == b.HTS_OK, info
    H, T, Q, Z = _host(dA, dB, dQ, dZ)
    c = rht_pencil_checks(A, B, H, T, Q, Z)
    assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c
    for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
        assert c[key] < 1e-14 * n, c
    assert np.array_equal(Z[:, 0], np.eye(n)[:, 0])
    q1 = B[:, 0] / np.linalg.norm(B[:, 0])
    assert min(np.abs(Q[:, 0] - q1).max(), np.abs(Q[:, 0] + q1).max()) < 1e-13
    Ho, To, Qo, Zo = oracle_mod.reduce(A, B, r)
    g = canonical(H, T, Q, Z, B_in=B)
    o = canonical(Ho, To, Qo, Zo, B_in=B)
    scale = max(np.abs(A).max(), np.abs(B).max())
    err = max(float(np.abs(x - y).max()) for x, y in zip(g, o)) / scale
    assert err <= 1e-12 * n, err


def test_reduce_tiny_and_r1(red):
    from paper_2301_07964_gb300.device import colmajor_empty
    for n, r in ((1, 1), (2, 1), (3, 1), (5, 1), (6, 5)):
        A, B = random_pencil(n, 3 * n + r)
        dA, dB = _dev(A, B)
        dQ, dZ = colmajor_empty(n), colmajor_empty(n)
        red.reduce(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT)
        st, info = red.sync_status()
        assert st == b.HTS_OK, (n, r, info)
        H, T, Q, Z = _host(dA, dB, dQ, dZ)
        c = rht_pencil_checks(A, B, H, T, Q, Z)
        assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, (n, r, c)
        assert max(c["bwd_A"], c["bwd_B"], c["orth_Q"], c["orth_Z"]) < 1e-14 * max(n, 10), (n, r, c)


def test_reduce_ill_conditioned_b(red):
    """Config 3's pencil family at a reduced size: B = U diag(logspace(0,-8)) V^T."""
    from paper_2301_07964_gb300.device import colmajor_empty
    n, r = 512, 32
    A, B = ill_conditioned_pencil(n, 3)
    dA, dB = _dev(A, B)
    dQ, dZ = colmajor_empty(n), colmajor_empty(n)
    red.reduce(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT)
    st, info = red.sync_status()
    assert st == b.HTS_OK, info
    H, T, Q, Z = _host(dA, dB, dQ, dZ)
    c = rht_pencil_checks(A, B, H, T, Q, Z)
    assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c
    for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
        assert c[key] < 1e-14 * n, c


def test_stage1_argument_errors(red):
    from paper_2301_07964_gb300.device import colmajor_empty
    n = 64
    A, B = colmajor_empty(n), colmajor_empty(n)
    work = red.workspace(n, 16, b.hts_params(p=8))
    f = b.hts_reduce_stage1
    assert f(red.ctx, n, n, A, n, B, n, 0, None, 1, 0, None, 1, 0, None, work, work.numel()) == b.HTS_ERR_ARG
    assert f(red.ctx, n, 16, A, n, B, n, 0, None, 1, 0, None, 1, 0, b.hts_params(p=16), work,
             work.numel()) == b.HTS_ERR_UNSUPPORTED
    assert f(red.ctx, n, 16, A, n, B, n, 0, None, 1, 0, None, 1, 0, None, work, 64) == b.HTS_ERR_WORKSPACE
    assert f(red.ctx, n, 16, A, n, B, n, 0, None, 1, 0, None, 1, b.HTS_GEMM_EMU_BF16, None, work,
             work.numel()) == b.HTS_ERR_UNSUPPORTED
