"""hts_reduce_stage2_noalloc: stage 2 for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they need the reduction (services that must not
allocate once running, code inside a framework that owns all device memory).  This entry
point uses a fixed scratch array compiled into the library instead of a caller workspace.
The test calls it twice in a row through the C ABI -- the second call finds the first call's
leftovers in the shared array -- and checks both results against hts_reduce_stage2 with a
caller workspace, with the tolerance the other stage-2 tests use (1e-12 * n).  It also
checks that a size whose workspace exceeds the array is rejected before anything runs.
This file is collected last so that a failure here does not hide the other tests' results.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2301_07964_gb300 import binding as b  # noqa: E402
from paper_2301_07964_gb300.inputs import random_rht_pencil  # noqa: E402

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_07964_gb300 import build
    build.build()
    from paper_2301_07964_gb300.device import Reducer, colmajor_empty, to_device, to_host
    red = Reducer(0)
    n, r, q = 300, 16, 8
    A, B = random_rht_pencil(n, r, 314)
    params = b.hts_params(q=q)

    def run(noalloc):
        dA, dB = to_device(A), to_device(B)
        dQ, dZ = colmajor_empty(n), colmajor_empty(n)
        if noalloc:
            st = b.hts_reduce_stage2_noalloc(red.ctx, n, r, dA, n, dB, n, b.HTS_COMP_INIT, dQ, n,
                                             b.HTS_COMP_INIT, dZ, n, b.HTS_GEMM_FP64, params)
        else:
            work = red.workspace(n, r, params)
            st = b.hts_reduce_stage2(red.ctx, n, r, dA, n, dB, n, b.HTS_COMP_INIT, dQ, n,
                                     b.HTS_COMP_INIT, dZ, n, b.HTS_GEMM_FP64, params, work, work.numel())
        assert st == b.HTS_OK, b.status_string(st)
        dst, info = red.sync_status()
        assert dst == b.HTS_OK, (b.status_string(dst), info)
        return [to_host(x) for x in (dA, dB, dQ, dZ)]

    ref = run(noalloc=False)
    tol = 1e-12 * n
    for _ in range(2):   # two calls in a row share the scratch array
        got = run(noalloc=True)
        for x, y in zip(got, ref):
            assert float(np.abs(x - y).max()) <= tol
        assert np.abs(np.tril(got[0], -2)).max() == 0.0 and np.abs(np.tril(got[1], -1)).max() == 0.0

    # a pencil whose scratch exceeds the fixed array is rejected before anything runs; the size
    # check comes first, and the matrices are NULL, so that a regression of that check ends in
    # an argument error on the host rather than in a launch
    for mode in (b.HTS_GEMM_FP64, b.HTS_GEMM_EMU_BF16):
        st = b.hts_reduce_stage2_noalloc(red.ctx, 40000, 32 if mode == b.HTS_GEMM_FP64 else 16, None, 40000,
                                         None, 40000, b.HTS_COMP_NONE, None, 1, b.HTS_COMP_NONE, None, 1, mode,
                                         None)
        assert st == b.HTS_ERR_WORKSPACE, b.status_string(st)
    red.close()
