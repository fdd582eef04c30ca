"""hts_reduce_batched: many independent pencils of different sizes in one launch.

Each pencil's result is checked against the oracle's full reduction in canonical signs, plus
the invariants.  The full batch configuration (4096 pencils, n uniform in [32, 512],
r = min(8, n // 8)) is checked by invariants on every pencil and by oracle parity on a
sample.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hts_checks import canonical, rht_pencil_checks  # noqa: E402
from paper_2301_07964_gb300 import binding as b  # noqa: E402
from paper_2301_07964_gb300.inputs import batch_sizes, random_pencil  # noqa: E402

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


def _run_batch(red, pencils, rs, params=None):
    from paper_2301_07964_gb300.device import colmajor_empty, to_device
    ns = [A.shape[0] for A, _ in pencils]
    dA = [to_device(A) for A, _ in pencils]
    dB = [to_device(B) for _, B in pencils]
    dQ = [colmajor_empty(n) for n in ns]
    dZ = [colmajor_empty(n) for n in ns]
    nbytes = b.hts_workspace_size_batched(ns, rs)
    work = torch.empty(max(256, nbytes), dtype=torch.uint8, device="cuda")
    st = b.hts_reduce_batched(red.ctx, ns, rs, dA, ns, dB, ns, b.HTS_COMP_INIT, dQ, ns, b.HTS_COMP_INIT, dZ, ns,
                              b.HTS_GEMM_FP64, params, work, work.numel())
    assert st == b.HTS_OK, b.status_string(st)
    dst, info = red.sync_status()
    assert dst == b.HTS_OK, info
    return dA, dB, dQ, dZ


def test_batched_matches_oracle(red, oracle_mod):
    from paper_2301_07964_gb300.device import to_host
    sizes = [3, 5, 32, 33, 47, 64, 65, 96, 100, 127, 150, 200, 8, 17]
    rs = [max(1, min(8, n // 8)) if n > 2 else 1 for n in sizes]
    pencils = [random_pencil(n, 500 + i) for i, n in enumerate(sizes)]
    dA, dB, dQ, dZ = _run_batch(red, pencils, rs)
    for i, ((A, B), r) in enumerate(zip(pencils, rs)):
        n = A.shape[0]
        H, T, Q, Z = (to_host(x) for x in (dA[i], dB[i], dQ[i], dZ[i]))
        c = rht_pencil_checks(A, B, H, T, Q, Z)
        assert c["H_below_hessenberg"] == 0.0 and c["T_below_diag"] == 0.0, (n, c)
        for key in ("bwd_A", "bwd_B", "orth_Q", "orth_Z"):
            assert c[key] < 1e-14 * max(n, 10), (n, c)
        if n > 2:
            Ho, To, Qo, Zo = oracle_mod.reduce(A, B, r)
            g = canonical(H, T, Q, Z, B_in=B)
            o = canonical(Ho, To, Qo, Zo, B_in=B)
            scale = max(np.abs(A).max(), np.abs(B).max())
            err = max(float(np.abs(x - y).max()) for x, y in zip(g, o)) / scale
            assert err <= 1e-12 * n, (n, r, err)


def test_batched_rejects_bad_sizes(red):
    from paper_2301_07964_gb300.device import colmajor_empty
    A = colmajor_empty(600)
    work = torch.empty(4096, dtype=torch.uint8, device="cuda")
    st = b.hts_reduce_batched(red.ctx, [600], [8], [A], [600], [A], [600], 0, None, None, 0, None, None,
                              b.HTS_GEMM_FP64, None, work, work.numel())
    assert st == b.HTS_ERR_UNSUPPORTED
    A = colmajor_empty(64)
    st = b.hts_reduce_batched(red.ctx, [64], [64], [A], [64], [A], [64], 0, None, None, 0, None, None,
                              b.HTS_GEMM_FP64, None, work, work.numel())
    assert st == b.HTS_ERR_ARG
    st = b.hts_reduce_batched(red.ctx, [64], [8], [A], [64], [A], [64], 0, None, None, 0, None, None,
                              b.HTS_GEMM_FP64, None, work, 16)
    assert st == b.HTS_ERR_WORKSPACE


def test_batch_config_4096_pencils(red, oracle_mod):
    """4096 pencils, n uniform in [32, 512], r = min(8, n // 8), A and B iid N(0, 1)."""
    from paper_2301_07964_gb300.device import to_host
    ns, rs = batch_sizes(4096, 5)
    g = np.random.Generator(np.random.PCG64(5))
    pencils = [(np.asfortranarray(g.standard_normal((n, n))), np.asfortranarray(g.standard_normal((n, n))))
               for n in ns]
    dA, dB, dQ, dZ = _run_batch(red, pencils, [int(r) for r in rs])
    worst = {"bwd_A": 0.0, "bwd_B": 0.0, "orth_Q": 0.0, "orth_Z": 0.0}
    for i, (A, B) in enumerate(pencils):
        n = A.shape[0]
        H, T, Q, Z = dA[i], dB[i], dQ[i], dZ[i]
        assert float(torch.tril(H, -2).abs().max()) == 0.0 and float(torch.tril(T, -1).abs().max()) == 0.0
        A0 = torch.from_numpy(A).cuda()
        B0 = torch.from_numpy(B).cuda()
        I = torch.eye(n, dtype=torch.float64, device="cuda")
        worst["bwd_A"] = max(worst["bwd_A"], float(torch.linalg.norm(Q @ H @ Z.T - A0) / torch.linalg.norm(A0)))
        worst["bwd_B"] = max(worst["bwd_B"], float(torch.linalg.norm(Q @ T @ Z.T - B0) / torch.linalg.norm(B0)))
        worst["orth_Q"] = max(worst["orth_Q"], float(torch.linalg.norm(Q.T @ Q - I) / n ** 0.5))
        worst["orth_Z"] = max(worst["orth_Z"], float(torch.linalg.norm(Z.T @ Z - I) / n ** 0.5))
    for key, v in worst.items():
        assert v < 1e-14 * 512, worst
    for i in (0, 1, 2, 4095, int(np.argmax(ns))):
        A, B = pencils[i]
        n = A.shape[0]
        H, T, Q, Z = (to_host(x) for x in (dA[i], dB[i], dQ[i], dZ[i]))
        Ho, To, Qo, Zo = oracle_mod.reduce(A, B, int(rs[i]))
        gg = canonical(H, T, Q, Z, B_in=B)
        oo = canonical(Ho, To, Qo, Zo, B_in=B)
        scale = max(np.abs(A).max(), np.abs(B).max())
        err = max(float(np.abs(x - y).max()) for x, y in zip(gg, oo)) / scale
        assert err <= 1e-12 * n, (i, n, err)


def test_planned_launches_and_cuda_graph_match_one_call(red):
    """hts_plan_batched once, then hts_reduce_batched_planned twice on fresh copies of the
    inputs, and the planned launch captured in a CUDA graph and replayed twice: every result
    equals the single hts_reduce_batched call's bit for bit (the same kernel on the same
    pencil, whichever block of the persistent launch takes it)."""
    from paper_2301_07964_gb300.device import colmajor_empty, to_device, to_host
    sizes = [5, 40, 64, 100, 130, 200, 33, 17, 3, 96]
    rs = [max(1, min(8, n // 8)) if n > 2 else 1 for n in sizes]
    pencils = [random_pencil(n, 700 + i) for i, n in enumerate(sizes)]
    ref = [[to_host(x) for x in mats] for mats in zip(*_run_batch(red, pencils, rs))]
    A0 = [to_device(A) for A, _ in pencils]
    B0 = [to_device(B) for _, B in pencils]
    dA, dB, dQ, dZ = ([colmajor_empty(n) for n in sizes] for _ in range(4))
    nbytes = b.hts_workspace_size_batched(sizes, rs)
    work = torch.empty(max(256, nbytes), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    st = b.hts_plan_batched(red.ctx, sizes, rs, dA, sizes, dB, sizes, b.HTS_COMP_INIT, dQ, sizes, b.HTS_COMP_INIT,
                            dZ, sizes, b.HTS_GEMM_FP64, None, work, work.numel(), stream)
    assert st == b.HTS_OK, b.status_string(st)

    def restore():
        for x, y in zip(dA + dB, A0 + B0):
            x.copy_(y)
        for x in dQ + dZ:
            x.fill_(float("nan"))   # COMP_INIT overwrites them

    def check(what):
        torch.cuda.synchronize()
        dst, info = red.sync_status()
        assert dst == b.HTS_OK, (what, info)
        for i in range(len(sizes)):
            got = [to_host(x) for x in (dA[i], dB[i], dQ[i], dZ[i])]
            for g, e, name in zip(got, ref[i], "HTQZ"):
                assert np.array_equal(g, e), (what, sizes[i], name, float(np.nanmax(np.abs(g - e))))

    for rep in range(2):
        restore()
        st = b.hts_reduce_batched_planned(red.ctx, len(sizes), work, work.numel(), stream)
        assert st == b.HTS_OK, b.status_string(st)
        check("planned launch %d" % rep)

    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        st = b.hts_reduce_batched_planned(red.ctx, len(sizes), work, work.numel(), torch.cuda.current_stream())
    assert st == b.HTS_OK, b.status_string(st)
    for rep in range(2):
        restore()
        torch.cuda.synchronize()
        graph.replay()
        check("graph replay %d" % rep)


def test_planned_launch_rejects_bad_workspace(red):
    n, r = [40, 50], [4, 4]
    need = b.hts_workspace_size_batched(n, r)
    work = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    assert b.hts_reduce_batched_planned(red.ctx, 2, None, need) == b.HTS_ERR_WORKSPACE
    assert b.hts_reduce_batched_planned(red.ctx, 2, work.data_ptr() + 8, need) == b.HTS_ERR_WORKSPACE
    assert b.hts_reduce_batched_planned(red.ctx, 2, work, 64) == b.HTS_ERR_WORKSPACE
    assert b.hts_reduce_batched_planned(red.ctx, 0, work, need) == b.HTS_ERR_ARG


def test_launch_shape_and_p(red):
    """params.tile_n (persistent blocks per SM) changes only which block takes a pencil: the
    results equal the default launch's bit for bit.  params.p changes stage 1's blocking: the
    reduction then agrees with the default one in canonical signs (the result is essentially
    unique once Q e_1 is fixed).  A negative tile_n is an argument error."""
    from paper_2301_07964_gb300.device import to_host
    sizes = [40, 64, 100, 130, 200, 17, 96, 250]
    rs = [max(1, min(8, n // 8)) for n in sizes]
    pencils = [random_pencil(n, 900 + i) for i, n in enumerate(sizes)]
    ref = [[to_host(x) for x in mats] for mats in zip(*_run_batch(red, pencils, rs))]
    for tile_n in (1, 2):
        got = [[to_host(x) for x in mats] for mats in zip(*_run_batch(red, pencils, rs, {"tile_n": tile_n}))]
        for i in range(len(sizes)):
            for g, e, name in zip(got[i], ref[i], "HTQZ"):
                assert np.array_equal(g, e), (tile_n, sizes[i], name)
    got = [[to_host(x) for x in mats] for mats in zip(*_run_batch(red, pencils, rs, {"p": 2, "tile_n": 1}))]
    for i, (n, (A, B)) in enumerate(zip(sizes, pencils)):
        scale = max(1.0, float(np.abs(A).max()), float(np.abs(B).max()))
        c_got, c_ref = canonical(*got[i]), canonical(*ref[i])
        err = max(float(np.abs(x - y).max()) for x, y in zip(c_got, c_ref))
        assert err <= 1e-12 * n * scale, (n, err)
    ns, rr = [40, 50], [4, 4]
    need = b.hts_workspace_size_batched(ns, rr)
    work = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    dA = [torch.zeros(40, 40, dtype=torch.float64, device="cuda"), torch.zeros(50, 50, dtype=torch.float64, device="cuda")]
    st = b.hts_plan_batched(red.ctx, ns, rr, dA, ns, dA, ns, b.HTS_COMP_NONE, None, None, b.HTS_COMP_NONE, None,
                            None, b.HTS_GEMM_FP64, {"tile_n": -1}, work, work.numel())
    assert st == b.HTS_ERR_ARG
