"""The multislice tuner's JSON cache (host logic, CPU): a miss measures every
row-pass variant and stores the best (batch, variant), a hit does not measure
again, entries of other grids survive, a corrupt file or an entry written
before the variant was tuned counts as a miss."""

import json

from paper_2401_15599_gb300 import tuning
import workloads as W


def _grid(n=256, ns=10):
    return W.GridSpec(n, n, n * 0.158203125, n * 0.158203125, ns, 2.0, 0.0, 200.0)


def test_miss_measures_and_hit_reuses(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def fake(grid, candidates, device="cuda", flags=0):
        calls.append((grid.nx, tuple(candidates), flags))
        t = {c: 1.0 / c + (0.5 if c == 32 else 0.0) - (0.001 if flags == 1 else 0.0) for c in candidates}
        return t, min(t, key=t.get)

    b1 = tuning.best_multislice_batch(_grid(), candidates=(8, 16, 32, 64), path=path, measure=fake)
    assert b1 == 64 and len(calls) == 2                     # 256^2: per-slice passes and the work queue
    assert {c[2] for c in calls} == {0, 4}
    b2 = tuning.best_multislice_batch(_grid(), candidates=(8, 16, 32, 64), path=path, measure=fake)
    assert b2 == 64 and len(calls) == 2                     # from the cache
    cfg = tuning.best_multislice_config(_grid(512, 101), candidates=(8, 16), path=path, measure=fake)
    assert cfg == (16, 1) and len(calls) == 7               # 512^2: four pass variants and the queue timed
    assert {c[2] for c in calls[2:]} == {0, 1, 2, 3, 4}
    assert tuning.best_multislice_config(_grid(512, 101), candidates=(8, 16), path=path, measure=fake) == (16, 1)
    data = json.load(open(path))
    assert len(calls) == 7 and len(data) == 2
    entry = data["test-device|256x256x10"]
    assert entry["batch"] == 64 and entry["flags"] == 0
    assert set(entry["ms_per_snapshot"]["0"]) == {"8", "16", "32", "64"}


def test_old_entries_are_tuned_again(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"test-device|512x512x101": {"batch": 8, "ms_per_snapshot": {"8": 1.0}}}))
    calls = []

    def fake(grid, candidates, device="cuda", flags=0):
        calls.append(flags)
        return {4: 2.0, 8: 1.0 + flags}, 8

    assert tuning.best_multislice_config(_grid(512, 101), candidates=(4, 8), path=str(path),
                                         measure=fake) == (8, 0)
    assert sorted(calls) == [0, 1, 2, 3, 4]


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    b = tuning.best_multislice_batch(_grid(), candidates=(4, 8), path=str(path),
                                     measure=lambda g, c, device="cuda", flags=0: ({4: 2.0, 8: 1.0}, 8))
    assert b == 8 and json.load(open(path))["test-device|256x256x10"]["batch"] == 8


def test_cache_path_follows_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("TACAW_TUNE_CACHE", str(tmp_path / "x.json"))
    assert tuning.cache_path() == str(tmp_path / "x.json")
