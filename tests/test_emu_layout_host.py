"""The K order of the tcgen05 update kernel's operands (tc_kidx in
paper_2301_07964_gb300/csrc/emu_arith.cuh), from the library's own header compiled for the host
(tests/kidx_probe.cu).

A product sums over K, so the order only has to be the same in both operands; what it buys is
the store pattern. These are the properties both writers rely on."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kidx(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("kidx") / "kidx_probe")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(ROOT, "tests", "kidx_probe.cu")], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    table = dict(tuple(map(int, ln.split())) for ln in out if ln.strip())
    return [table[p] for p in range(32)]


def test_k_order_is_a_permutation(kidx):
    assert sorted(kidx) == list(range(32))


def test_a_threads_positions_are_one_8_byte_store(kidx):
    # the thread with part j holds positions 2j, 2j+1 (first half) and 16+2j, 17+2j (second half,
    # where the slide by 16 carries them): they sit at K = 4j .. 4j+3, inside one 16-byte core-matrix
    # row and 8-byte aligned
    for j in range(8):
        ks = [kidx[2 * j], kidx[2 * j + 1], kidx[16 + 2 * j], kidx[17 + 2 * j]]
        assert ks == [4 * j, 4 * j + 1, 4 * j + 2, 4 * j + 3]
        assert (ks[0] * 2) % 8 == 0 and ks[0] // 8 == ks[3] // 8


def test_adjacent_positions_stay_adjacent(kidx):
    # the block formation packs the FP16 digits of input positions 2i and 2i+1 into one 32-bit word
    for i in range(16):
        assert kidx[2 * i + 1] == kidx[2 * i] + 1 and kidx[2 * i] % 2 == 0
