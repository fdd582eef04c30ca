"""GPU parity of stage 2 with the emulated-FP64 delayed updates (HTS_GEMM_EMU_BF16).

The chase is the same native-FP64 code as in HTS_GEMM_FP64 mode; the delayed updates form
each block's reflector product U_k and apply it on the BF16 tensor cores with 8 base-256
digits per operand.  The result must meet the same bar as the native mode: element-wise
agreement with the CPU oracle (Alg. 2, unblocked, FP64) after sign normalisation within
1e-12 * n, exact structural zeros, and backward errors / orthogonality within 1e-14 * n.
Pencils are n x n r-HT pencils with r = 16 (the only r this mode implements) at sizes that
span several 64-line tiles, ragged tails and both full and partial sweep groups.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hts_checks import canonical, rht_pencil_checks  # noqa: E402
from paper_2301_07964_gb300 import binding as b  # noqa: E402
from paper_2301_07964_gb300.inputs import random_pencil, random_rht_pencil  # noqa: E402

pytestmark = pytest.mark.gpu

EMU = b.HTS_GEMM_EMU_BF16


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


def _run(red, A, B, r, q, mode, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, Q0=None, Z0=None):
    from paper_2301_07964_gb300.device import colmajor_empty, to_device, to_host
    n = A.shape[0]
    dA, dB = to_device(A), to_device(B)
    dQ = to_device(Q0) if Q0 is not None else colmajor_empty(n)
    dZ = to_device(Z0) if Z0 is not None else colmajor_empty(n)
    red.stage2(dA, dB, r, dQ if compq else None, dZ if compz else None, compq=compq, compz=compz, q=q, mode=mode)
    st, info = red.sync_status()
    assert st == b.HTS_OK, (b.status_string(st), info)
    return tuple(to_host(x) for x in (dA, dB, dQ, dZ))


CASES = [  # n, q (r = 16)
    (20, 16), (40, 16), (64, 16), (100, 8), (129, 16), (200, 16), (255, 7), (300, 16), (513, 16), (700, 11),
]


@pytest.mark.parametrize("n,q", CASES)
def test_emu_stage2_matches_oracle(red, oracle_mod, n, q):
    r = 16
    A, B = random_rht_pencil(n, r, 31 * n + q)
    H, T, Q, Z = _run(red, A, B, r, q, EMU)
    c = rht_pencil_checks(A, B, H, T, Q, Z)
    assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c
    for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
        assert c[key] < 1e-14 * max(n, 10), c
    e1 = np.eye(n)[:, 0]
    assert np.array_equal(Q[:, 0], e1) and np.array_equal(Z[:, 0], e1)
    Ho, To, Qo, Zo = oracle_mod.stage2(A, B, r)
    g = canonical(H, T, Q, Z)
    o = canonical(Ho, To, Qo, Zo)
    scale = max(1.0, float(np.abs(A).max()), float(np.abs(B).max()))
    err = max(float(np.abs(x - y).max()) for x, y in zip(g, o)) / scale
    assert err <= 1e-12 * n, "max |GPU(emu) - oracle| = %.3e" % err


def test_emu_and_native_agree(red):
    """Both update modes compute the same reduction; at n = 1024 they agree to rounding."""
    n, r, q = 1024, 16, 16
    A, B = random_rht_pencil(n, r, 11)
    e = canonical(*_run(red, A, B, r, q, EMU))
    f = canonical(*_run(red, A, B, r, q, b.HTS_GEMM_FP64))
    scale = max(float(np.abs(A).max()), float(np.abs(B).max()))
    err = max(float(np.abs(x - y).max()) for x, y in zip(e, f)) / scale
    assert err <= 1e-12 * n, err


def test_emu_comp_update_and_scaled_rows(red):
    """COMP_UPDATE multiplies into given factors; rows of very different magnitude (the
    per-row scales of the emulation) keep their relative accuracy."""
    n, r, q = 160, 16, 16
    A, B = random_rht_pencil(n, r, 21)
    d = 2.0 ** np.arange(-40, 40, 80 / n)[:n]
    A = np.asfortranarray(d[:, None] * A)   # row scaling keeps the r-HT structure
    B = np.asfortranarray(d[:, None] * B)
    rng = np.random.default_rng(22)
    Q0 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Z0 = np.linalg.qr(rng.standard_normal((n, n)))[0]
    H, T, Q, Z = _run(red, A, B, r, q, EMU, compq=b.HTS_COMP_UPDATE, compz=b.HTS_COMP_UPDATE, Q0=Q0, Z0=Z0)
    c = rht_pencil_checks(Q0 @ A @ Z0.T, Q0 @ B @ Z0.T, H, T, Q, Z)
    assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c
    assert max(c["orth_Q"], c["orth_Z"]) < 1e-13, c
    Hn, Tn, Qn, Zn = _run(red, A, B, r, q, b.HTS_GEMM_FP64, compq=b.HTS_COMP_UPDATE, compz=b.HTS_COMP_UPDATE,
                          Q0=Q0, Z0=Z0)
    cn = rht_pencil_checks(Q0 @ A @ Z0.T, Q0 @ B @ Z0.T, Hn, Tn, Qn, Zn)
    for key in ("bwd_A", "bwd_B"):
        assert c[key] < 4 * cn[key] + 1e-15, (c, cn)


def test_emu_full_reduction(red, oracle_mod):
    from paper_2301_07964_gb300.device import colmajor_empty, to_device, to_host
    n, r = 300, 16
    A, B = random_pencil(n, 4242)
    dA, dB = to_device(A), to_device(B)
    dQ, dZ = colmajor_empty(n), colmajor_empty(n)
    red.reduce(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, mode=EMU)
    st, info = red.sync_status()
    assert st == b.HTS_OK, info
    H, T, Q, Z = (to_host(x) for x in (dA, dB, dQ, dZ))
    c = rht_pencil_checks(A, B, H, T, Q, Z)
    assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, c
    for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
        assert c[key] < 1e-14 * n, c
    Ho, To, Qo, Zo = oracle_mod.reduce(A, B, r)
    g = canonical(H, T, Q, Z, B_in=B)
    o = canonical(Ho, To, Qo, Zo, B_in=B)
    scale = max(np.abs(A).max(), np.abs(B).max())
    assert max(float(np.abs(x - y).max()) for x, y in zip(g, o)) / scale <= 1e-12 * n


def test_emu_argument_errors(red):
    from paper_2301_07964_gb300.device import colmajor_empty
    n = 64
    A, B = colmajor_empty(n), colmajor_empty(n)
    f = b.hts_reduce_stage2
    work = red.workspace(n, 8)
    # r != 16 is not implemented in this mode
    assert f(red.ctx, n, 8, A, n, B, n, 0, None, 1, 0, None, 1, EMU, None, work, work.numel()) == \
        b.HTS_ERR_UNSUPPORTED
    work = red.workspace(n, 16)
    assert f(red.ctx, n, 16, A, n, B, n, 0, None, 1, 0, None, 1, EMU, b.hts_params(emu_slices=7), work,
             work.numel()) == b.HTS_ERR_UNSUPPORTED
    # the digit planes are part of the workspace size; one KiB short is refused (at n = 1024 the
    # stage-2 layout with its planes is the largest part of the reported size, which also covers
    # stage 1 and the cuBLAS workspace of its block-reflector products)
    n2 = 1024
    A2, B2 = colmajor_empty(n2), colmajor_empty(n2)
    need = b.hts_workspace_size(n2, 16)
    work2 = torch.empty(need, dtype=torch.uint8, device="cuda")
    assert f(red.ctx, n2, 16, A2, n2, B2, n2, 0, None, 1, 0, None, 1, EMU, None, work2, need - 1024) == \
        b.HTS_ERR_WORKSPACE


@pytest.mark.parametrize("n,seed", [(4096, 2), (8192, 4)])
def test_emu_full_size_properties(red, n, seed):
    """Full size (config 2's n = 4096 and the metric's n = 8192 at r = 16): invariants with
    the residual products on the GPU (cuBLAS DGEMM), and backward errors no worse than the
    native mode's on the same pencil (the precision comparison of config 4)."""
    from paper_2301_07964_gb300.device import colmajor_empty, to_device
    r, q = 16, 16
    A, B = random_rht_pencil(n, r, seed)
    dA0, dB0 = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    res = {}
    for mode in (EMU, b.HTS_GEMM_FP64):
        dA, dB = to_device(A), to_device(B)
        dQ, dZ = colmajor_empty(n), colmajor_empty(n)
        red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=q, mode=mode)
        st, info = red.sync_status()
        assert st == b.HTS_OK, info
        p = {"H": float(torch.tril(dA, -2).abs().max()), "T": float(torch.tril(dB, -1).abs().max()),
             "bwd_A": float(torch.linalg.norm(dQ @ dA @ dZ.T - dA0) / torch.linalg.norm(dA0)),
             "bwd_B": float(torch.linalg.norm(dQ @ dB @ dZ.T - dB0) / torch.linalg.norm(dB0)),
             "orth_Q": float(torch.linalg.norm(dQ.T @ dQ - I) / n ** 0.5),
             "orth_Z": float(torch.linalg.norm(dZ.T @ dZ - I) / n ** 0.5)}
        res[mode] = p
        del dA, dB, dQ, dZ
    e, f = res[EMU], res[b.HTS_GEMM_FP64]
    assert e["H"] == 0.0 and e["T"] == 0.0, e
    for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
        assert e[key] < 1e-12 * n, e
        assert e[key] <= 1.5 * f[key], (key, e, f)


@pytest.mark.parametrize("n,q", [(40, 16), (129, 16), (300, 16), (513, 9), (700, 16)])
def test_tensor_core_and_warp_kernels_match_oracle(red, oracle_mod, n, q):
    """The emulated updates run either on the tcgen05 kernel (64-line tiles, TMEM accumulators,
    U planes by TMA; the default) or on the mma.sync kernel (32-line tiles): both must give the
    oracle's reduction within 1e-12 n, and agree with each other."""
    from paper_2301_07964_gb300.device import colmajor_empty, to_device, to_host
    r = 16
    A, B = random_rht_pencil(n, r, 71 * n + q)
    scale = max(1.0, float(np.abs(A).max()), float(np.abs(B).max()))
    Ho, To, Qo, Zo = oracle_mod.stage2(A, B, r)
    o = canonical(Ho, To, Qo, Zo)
    res = []
    for tile_m in (64, 32):
        dA, dB = to_device(A), to_device(B)
        dQ, dZ = colmajor_empty(n), colmajor_empty(n)
        red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=q, mode=EMU, tile_m=tile_m)
        st, info = red.sync_status()
        assert st == b.HTS_OK, (tile_m, b.status_string(st), info)
        H, T, Q, Z = (to_host(x) for x in (dA, dB, dQ, dZ))
        c = rht_pencil_checks(A, B, H, T, Q, Z)
        assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, (tile_m, c)
        for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
            assert c[key] < 1e-14 * max(n, 10), (tile_m, c)
        g = canonical(H, T, Q, Z)
        err = max(float(np.abs(x - y).max()) for x, y in zip(g, o)) / scale
        assert err <= 1e-12 * n, (tile_m, err)
        res.append(g)
    assert max(float(np.abs(x - y).max()) for x, y in zip(*res)) / scale <= 1e-12 * n
