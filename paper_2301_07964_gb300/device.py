"""Torch helpers around the C ABI: column-major FP64 device matrices, workspaces, and a
``Reducer`` object that owns a library context.  PyTorch provides memory and streams only.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as b


def colmajor_empty(n: int, device="cuda") -> torch.Tensor:
    """n x n FP64 tensor whose storage is column-major (stride (1, n))."""
    return torch.empty((n, n), dtype=torch.float64, device=device).t()


def to_device(M: np.ndarray, device="cuda") -> torch.Tensor:
    n = M.shape[0]
    t = colmajor_empty(n, device)
    t.copy_(torch.from_numpy(np.asarray(M, dtype=np.float64)))
    return t


def to_host(t: torch.Tensor) -> np.ndarray:
    return np.asfortranarray(t.detach().cpu().numpy())


class Reducer:
    """Owns an hts context and a workspace on one device."""

    def __init__(self, device: int = 0):
        self.device = device
        self.ctx = b.hts_create(device)
        self._work = None

    def close(self):
        if self.ctx is not None:
            b.hts_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, n: int, r: int, params=None) -> torch.Tensor:
        need = max(256, b.hts_workspace_size(n, r, params))
        if self._work is None or self._work.numel() < need:
            self._work = torch.empty(need, dtype=torch.uint8, device="cuda:%d" % self.device)
        return self._work

    def stage2(self, A: torch.Tensor, B: torch.Tensor, r: int, Q=None, Z=None,
               compq=b.HTS_COMP_UPDATE, compz=b.HTS_COMP_UPDATE, q=0, flags=0,
               mode=b.HTS_GEMM_FP64, stream=None, check=True, tile_m=0) -> int:
        n = A.shape[0]
        params = b.hts_params(q=q, flags=flags, tile_m=tile_m)
        work = self.workspace(n, r, params)
        if Q is None:
            compq = b.HTS_COMP_NONE
        if Z is None:
            compz = b.HTS_COMP_NONE
        st = b.hts_reduce_stage2(self.ctx, n, r, A, _ld(A), B, _ld(B), compq, Q, _ld(Q), compz, Z, _ld(Z),
                                 mode, params, work, work.numel(), stream)
        if check and st != b.HTS_OK:
            raise b.HTSError(st, "hts_reduce_stage2")
        return st

    def _call(self, fn, name, A, B, r, Q, Z, compq, compz, q, p, flags, mode, stream, check, tile_m=0):
        n = A.shape[0]
        params = b.hts_params(q=q, p=p, flags=flags, tile_m=tile_m)
        work = self.workspace(n, r, params)
        if Q is None:
            compq = b.HTS_COMP_NONE
        if Z is None:
            compz = b.HTS_COMP_NONE
        st = fn(self.ctx, n, r, A, _ld(A), B, _ld(B), compq, Q, _ld(Q), compz, Z, _ld(Z), mode, params, work,
                work.numel(), stream)
        if check and st != b.HTS_OK:
            raise b.HTSError(st, name)
        return st

    def stage1(self, A, B, r, Q=None, Z=None, compq=b.HTS_COMP_UPDATE, compz=b.HTS_COMP_UPDATE, p=0, flags=0,
               mode=b.HTS_GEMM_FP64, stream=None, check=True) -> int:
        return self._call(b.hts_reduce_stage1, "hts_reduce_stage1", A, B, r, Q, Z, compq, compz, 0, p, flags,
                          mode, stream, check)

    def reduce(self, A, B, r, Q=None, Z=None, compq=b.HTS_COMP_UPDATE, compz=b.HTS_COMP_UPDATE, q=0, p=0,
               flags=0, mode=b.HTS_GEMM_FP64, stream=None, check=True, tile_m=0) -> int:
        return self._call(b.hts_reduce, "hts_reduce", A, B, r, Q, Z, compq, compz, q, p, flags, mode, stream, check,
                          tile_m)

    def sync_status(self, stream=None):
        return b.hts_sync_status(self.ctx, stream)


def _ld(t):
    if t is None:
        return 1
    if t.stride(0) != 1:
        raise ValueError("matrices must be column-major (stride(0) == 1)")
    return max(1, t.stride(1))
