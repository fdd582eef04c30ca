"""Host logic of bench.py, checked against independent counts (no GPU).

- The chase's latency floor counts, per group, the steps on the wavefront's critical path:
  the last sweep's blocks plus a lag of 3 blocks per earlier sweep.  A unit-time simulation
  of the waits the chase kernel takes (step (k, j) after step (k-1, j), and after sweep j-1
  has finished block k+2, or all of its blocks) must give the same count.
- The per-sweep direct flop count that scales the oracle sample sums to the leading-order
  closed form: about 16 n (n - j) flops for sweep j, so 8 n^3 in all (reading R7: the direct
  count is 8.1 n^3 with the lower-order terms).
- DRAM traffic from the committed ncu record is reported only while its source digest matches.
"""
import os

import numpy as np
import pytest

import bench


def _critical_path_steps(n, r, q):
    total = 0
    for j1 in range(1, n - 1, q):
        qg = min(q, n - 2 - j1 + 1)
        blocks = [2 + (n - (j1 + s) - 1) // r for s in range(qg)]
        prev = None
        for s in range(qg):
            fin = []
            for k in range(blocks[s]):
                t = fin[-1] if k else 0
                if prev is not None:
                    t = max(t, prev[min(k + 2, len(prev) - 1)])
                fin.append(t + 1)
            prev = fin
        total += prev[-1]
    return total


@pytest.mark.parametrize("n,r,q", [(64, 4, 4), (100, 8, 5), (257, 16, 16), (300, 16, 7), (1000, 16, 16)])
def test_chase_floor_counts_the_wavefronts_critical_path(n, r, q):
    steps = _critical_path_steps(n, r, q)
    mhz = 1000.0
    per_step = bench.chase_floor_ms(n, r, q, mhz) * mhz * 1e3   # cycles of all steps
    chain = (r - 1) * 332 + (2 * 24 + 18 + 39) * 64
    assert per_step == pytest.approx(steps * chain, rel=1e-12)


def test_sweep_work_sums_to_the_direct_count():
    for n in (512, 1024):
        w = bench.sweep_work(n, 16)
        assert w[0] == 0.0 and w[n - 1] == 0.0 and w[n] == 0.0
        # each sweep touches 16 n (n - j) elements' worth of flops to leading order
        j = np.arange(1, n - 1)
        assert np.allclose(w[1:n - 1] / (16.0 * n * (n - j)), 1.0, atol=0.25)
        total = w.sum() / n ** 3
        assert 7.9 < total < 8.4, total


def test_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    digest = bench.source_digest(bench.KERNEL_SOURCES["k_s2_chase16"])
    rec = tmp_path / "ncu_traffic.txt"
    rec.write_text("# kernel workload bytes digest\n"
                   "k_s2_chase16 wl_a 12345 %s\n"
                   "k_s2_chase16 wl_b 777 0000000000000000\n" % digest)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.ncu_traffic("k_s2_chase16", "wl_a") == 12345.0
    assert bench.ncu_traffic("k_s2_chase16", "wl_b") is None       # taken on another source
    assert bench.ncu_traffic("k_s2_chase16", "wl_c") is None       # no record
    monkeypatch.setattr(bench, "TRAFFIC_FILE", os.path.join(str(tmp_path), "missing.txt"))
    assert bench.ncu_traffic("k_s2_chase16", "wl_a") is None
