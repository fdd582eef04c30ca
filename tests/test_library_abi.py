"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU, exports every
function include/hts.h declares, and rejects bad arguments on the host before touching the
device."""
import ctypes
import os
import re

import pytest

from paper_2301_07964_gb300 import binding, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hts.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hts_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("hts_create", "hts_destroy", "hts_workspace_size", "hts_reduce_stage1",
                     "hts_reduce_stage2", "hts_reduce", "hts_sync_status"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(binding.LIB_PATH)
    missing = [nm for nm in _declared_functions() if not hasattr(raw, nm)]
    assert missing == []


def test_status_strings(lib):
    assert binding.status_string(binding.HTS_OK) == "HTS_OK"
    assert binding.status_string(binding.HTS_ERR_TIMEOUT) == "HTS_ERR_TIMEOUT"


def test_workspace_size_is_host_only(lib):
    w = binding.hts_workspace_size(8192, 16)
    assert w > 0 and w % 256 == 0
    assert binding.hts_workspace_size(4096, 16) < w
    with pytest.raises(binding.HTSError):
        binding.hts_workspace_size(-1, 16)
    with pytest.raises(binding.HTSError):
        binding.hts_workspace_size(100, 0)


def test_bad_arguments_rejected_on_host(lib):
    # NULL context / negative n / r < 1 / NULL matrices return HTS_ERR_ARG without any CUDA call
    args = dict(n=16, r=4, A=1 << 20, lda=16, B=1 << 21, ldb=16, compq=0, Q=None, ldq=1, compz=0,
                Z=None, ldz=1, mode=0, params=None, work=None, work_bytes=0)
    st = binding.hts_reduce_stage2(None, **args)
    assert st == binding.HTS_ERR_ARG
    for fn in (binding.hts_reduce_stage1, binding.hts_reduce_stage2, binding.hts_reduce):
        assert fn(None, **args) == binding.HTS_ERR_ARG
    assert binding.load().hts_sync_status(None, None, None) == binding.HTS_ERR_ARG
