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
