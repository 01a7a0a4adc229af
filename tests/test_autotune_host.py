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


def test_candidate_sets_per_operation(tmp_path, monkeypatch):
    """The settings each operation's tuner times: block sizes 128/256/512; for SpMM with
    narrow rows of X both lane shapes, each setting once; for bfloat16 SDDMM both forms."""
    import torch

    seen = []
    monkeypatch.setattr(autotune.Autotuner, "shape_key", staticmethod(lambda *a: "key"))
    monkeypatch.setattr(autotune.Autotuner, "choose",
                        lambda self, key, cands, make, force=False: seen.append(cands) or cands[0])

    class FakeCSR:
        shape = (10, 12)
        nnz = 30

        def __init__(self, dtype):
            self.dtype = dtype

    t = autotune.Autotuner(path=str(tmp_path / "tune.json"))
    t.spmm(FakeCSR(torch.float32), torch.zeros(12, 16), Y=torch.zeros(10, 16))  # 64-byte rows: narrow
    t.spmm(FakeCSR(torch.float32), torch.zeros(12, 128), Y=torch.zeros(10, 128))  # 512-byte rows
    narrow, wide = seen
    key = lambda c: (c["split"], json.dumps(c["tune"], sort_keys=True))
    assert len({key(c) for c in narrow}) == len(narrow) == 4 * 3 * 2 * 2 + 1
    assert {c["tune"]["lane_groups"] for c in narrow if c["tune"]} == {1, 2}
    assert len(wide) == 25 and all("lane_groups" not in (c["tune"] or {}) for c in wide)
    assert {c["tune"]["block_threads"] for c in wide if c["tune"]} == {128, 256, 512}
    seen.clear()
    monkeypatch.setattr(autotune.ops, "result_dtype", lambda dt: torch.float32)
    for dt in (torch.float32, torch.bfloat16):
        t.sddmm(FakeCSR(dt), torch.zeros(10, 32, dtype=dt), torch.zeros(12, 32, dtype=dt))
    f32, bf16 = seen
    assert len(f32) == 4 * 3 + 1 and len(bf16) == 2 * len(f32)
    assert {c["tune"]["form"] for c in bf16} == {1, 2}
