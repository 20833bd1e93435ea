"""Host logic of the schedule autotuner (no GPU): candidates outside the
item-size limits are skipped, the fastest measured schedule wins, and the
tuner caches one choice per (qubit count, circuit class, codec, bound)."""
from paper_1811_05140_gb300 import autotune


def test_valid_schedules():
    assert autotune.valid(20, 8, 4)
    assert not autotune.valid(20, 9, 4)          # c + hmax > 12
    assert not autotune.valid(6, 8, 1)           # tile larger than the state
    assert not autotune.valid(20, 11, 1)         # tile above 2^10
    assert not autotune.valid(20, 8, 0)


def test_tune_picks_the_fastest_valid_candidate(monkeypatch):
    seen = []

    def fake(n, gates, schedule, codec, eps, basis, reps):
        seen.append(schedule)
        c, hmax, depth, threads = autotune.full(schedule)
        return 1.0 + 0.01 * c + 0.001 * depth / 512 - 0.02 * hmax + 0.0001 * abs(threads - 128)

    monkeypatch.setattr(autotune, "time_schedule", fake)
    cands = [(8, 4, 512), (9, 4, 512), (7, 4, 48), (10, 2, 512), (12, 1, 512), (7, 4, 48, 128),
             (7, 4, 48, 512), (7, 4, 48, 300)]
    res = autotune.tune(20, [], candidates=cands)
    assert (9, 4, 512) not in seen and (12, 1, 512) not in seen and (7, 4, 48, 300) not in seen
    assert res["best"] == (7, 4, 48, 128)                  # the threads axis decides among equals
    secs = [row["seconds"] for row in res["table"]]
    assert secs == sorted(secs) and len(secs) == 5


def test_tuner_caches_per_key(monkeypatch):
    calls = []

    def fake(n, gates, codec="rel", eps=1e-4, basis=0, candidates=None, reps=2):
        calls.append((n, codec, eps))
        return {"best": (8, 4, 512), "table": []}

    monkeypatch.setattr(autotune, "tune", fake)
    t = autotune.Tuner()
    assert t.schedule(20, "qft", []) == (8, 4, 512)
    t.schedule(20, "qft", [])
    t.schedule(20, "grover", [])
    t.schedule(20, "qft", [], eps=1e-3)
    assert len(calls) == 3
