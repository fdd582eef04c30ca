"""Host logic of the measured choice of q (paper_2301_07964_gb300/tune.py), with an injected
timer in place of the GPU."""
import json

from paper_2301_07964_gb300 import tune


def test_candidates_cover_quarters_of_r():
    assert tune.candidates(16) == [4, 8, 12, 16]
    assert tune.candidates(8) == [2, 4, 6, 8]
    assert tune.candidates(3) == [1, 2, 3]
    assert tune.candidates(1) == [1]
    assert all(1 <= q <= r for r in range(1, 33) for q in tune.candidates(r))


def test_measure_keeps_the_fastest_after_warmup():
    calls = []
    seq = {4: [9.0, 5.0, 6.0], 8: [9.0, 3.0, 4.0]}

    def run(q):
        calls.append(q)
        return seq[q].pop(0)

    times = tune.measure(run, [4, 8], reps=2, warmup=1)
    assert times == {4: 5.0, 8: 3.0}
    assert calls == [4, 4, 4, 8, 8, 8]


def test_choose_prefers_the_larger_q_on_ties():
    assert tune.choose({4: 10.0, 8: 7.0, 12: 7.5, 16: 9.0}) == 8
    assert tune.choose({4: 7.0, 8: 7.05, 16: 7.06}) == 16      # within 1 %: fewer groups
    assert tune.choose({4: 7.0, 16: 7.2}) == 4


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert tune.load_cache(path) == {}
    key = tune._key("GPU X", 8192, 16, 1)
    tune.store_cache(path, key, 16, {16: 3.5, 8: 4.0})
    tune.store_cache(path, tune._key("GPU X", 4096, 16, 1), 8, {8: 1.0})
    data = json.load(open(path))
    assert data[key] == {"q": 16, "ms": {"16": 3.5, "8": 4.0}}
    assert len(data) == 2
    (tmp_path / "bad.json").write_text("not json")
    assert tune.load_cache(str(tmp_path / "bad.json")) == {}


def test_parameter_candidates():
    from paper_2301_07964_gb300 import binding as b
    assert tune.tile_candidates(16, b.HTS_GEMM_EMU_BF16) == [32, 64]
    assert tune.tile_candidates(16, b.HTS_GEMM_FP64) == [0]
    assert tune.tile_candidates(32, b.HTS_GEMM_EMU_BF16) == [0]
    assert tune.p_candidates(16, 128) == [2, 4, 8]
    assert tune.p_candidates(32, 128) == [2, 4]
    assert tune.p_candidates(16, 64) == [2, 4]
    assert tune.p_candidates(8, 64) == [2, 4, 8]
    assert tune.batch_shape_candidates()[0] == 0


def test_choose_with_a_preference():
    assert tune.choose({0: 7.0, 1: 7.05, 2: 9.0}, prefer=min) == 0
    assert tune.choose({0: 7.5, 1: 7.0, 2: 7.01}, prefer=min) == 1


def test_coordinate_search_one_axis_at_a_time():
    # a separable cost with its minimum at q = 12, tile = 64; each configuration runs once per
    # (warm-up + timed) call and is not run again when a later axis revisits it
    cost = {4: 10.0, 8: 6.0, 12: 4.0, 16: 4.5}
    tile_cost = {0: 0.0, 32: 0.5, 64: -0.3}
    calls = []

    def run(cfg):
        calls.append((cfg["q"], cfg["tile_m"]))
        return cost[cfg["q"]] + tile_cost[cfg["tile_m"]]

    best, seen = tune.coordinate_search(run, {"q": 16, "tile_m": 0},
                                        [("q", [4, 8, 12, 16], max), ("tile_m", [32, 64], max)], reps=1, warmup=0)
    assert best == {"q": 12, "tile_m": 64}
    assert calls == [(4, 0), (8, 0), (12, 0), (16, 0), (12, 32), (12, 64)]
    assert seen[(("q", 12), ("tile_m", 64))] == 3.7
    assert len(seen) == 6


def test_coordinate_search_ties_follow_the_preference():
    best, _ = tune.coordinate_search(lambda cfg: 5.0, {"p": 0, "tile_n": 0},
                                     [("tile_n", [0, 1, 2], min), ("p", [2, 4, 8, 0], max)], reps=1, warmup=0)
    assert best == {"p": 8, "tile_n": 0}


def test_cache_of_a_parameter_set(tmp_path):
    path = str(tmp_path / "tune.json")
    tune.store_cache(path, "k", {"q": 16, "tile_m": 64}, {(("q", 16), ("tile_m", 64)): 3.0, (("q", 8), ("tile_m", 0)): 5.0})
    data = json.load(open(path))
    assert data["k"] == {"q": 16, "tile_m": 64, "ms": {"q=16,tile_m=64": 3.0, "q=8,tile_m=0": 5.0}}


def test_default_then_largest():
    assert tune.default_then_largest([2, 4, 0, 8]) == 0
    assert tune.default_then_largest([2, 8, 4]) == 8
    assert tune.choose({0: 8.54, 2: 10.4, 4: 9.06, 8: 8.53}, prefer=tune.default_then_largest) == 0
