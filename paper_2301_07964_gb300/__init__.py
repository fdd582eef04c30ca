"""GB300 (sm_103a) library for the two-stage Hessenberg-triangular reduction of a real FP64
pencil (Steel & Vandebril).  The compute runs in the CUDA library ``libhts.so`` behind the C
ABI of ``include/hts.h``; ``binding`` is its ctypes binding (same function names), and
``device`` offers small torch helpers for column-major device matrices and workspaces.
"""
from .binding import (HTS_COMP_INIT, HTS_COMP_NONE, HTS_COMP_UPDATE, HTS_ERR_ARG, HTS_ERR_CUDA,  # noqa: F401
                      HTS_ERR_TIMEOUT, HTS_ERR_UNSUPPORTED, HTS_ERR_WORKSPACE, HTS_FLAG_NO_CLEAN,
                      HTS_GEMM_EMU_BF16, HTS_GEMM_FP64, HTS_OK, HTSError, hts_create, hts_destroy,
                      hts_params, hts_reduce, hts_reduce_stage1, hts_reduce_stage2, hts_sync_status,
                      hts_workspace_size, status_string)
