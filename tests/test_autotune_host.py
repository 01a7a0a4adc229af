"""The autotuner's choice and cache logic, with the timing replaced by a fixed table
(no GPU): the fastest candidate wins, the choice persists in the JSON cache, a cached
shape class is not timed again, and `force` re-times it."""
import json

from paper_2207_13901_gb300 import autotune


def fake_timer(table, calls):
    def _time(self, fn, reps):
        calls.append(reps)
        return table[fn()]
    return _time


def test_fastest_candidate_is_chosen_and_cached(tmp_path, monkeypatch):
    cands = autotune.warp_candidates(True, inflight=True)
    # 4 unit sizes x 3 block sizes x 2 in-flight depths, plus the row split
    assert len(cands) == 25 and cands[-1] == {"split": "row", "tune": None}
    assert {c["tune"]["block_threads"] for c in cands[:-1]} == {128, 256, 512}
    ms = {i: 5.0 + i for i in range(len(cands))}
    ms[6] = 1.25
    calls = []
    monkeypatch.setattr(autotune.Autotuner, "_time", fake_timer(ms, calls))
    make = lambda c: (lambda i=cands.index(c): i)
    path = str(tmp_path / "tune.json")
    t = autotune.Autotuner(path=path, reps=3)
    best = t.choose("spmm|float32|k", cands, make)
    assert best["tune"] == cands[6]["tune"] and best["ms"] == 1.25
    assert len(t.last_table) == len(cands)
    assert calls.count(1) == 1 and calls.count(3) == len(cands) - 1  # the row split is timed once
    with open(path) as f:
        assert json.load(f)["spmm|float32|k"]["ms"] == 1.25
    # a second tuner reads the cache and times nothing
    calls.clear()
    t2 = autotune.Autotuner(path=path, reps=3)
    assert t2.choose("spmm|float32|k", cands, make) == best and not calls
    # force re-times and can change its mind
    ms[2] = 0.5
    best2 = t2.choose("spmm|float32|k", cands, make, force=True)
    assert best2["tune"] == cands[2]["tune"] and len(calls) == len(cands)


def test_unreadable_cache_starts_empty(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    assert autotune.Autotuner(path=str(p)).cache == {}
    assert autotune._bucket(0) == 0 and autotune._bucket(1024) == 10 and autotune._bucket(1500) == 11
