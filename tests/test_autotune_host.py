"""The autotuner's host logic on the CPU: the candidate grid (CTA-slot counts
capped at what can be co-resident, duplicates dropped), the choice of the
fastest median, and the JSON cache keyed by workload. The device is replaced by
a fake context whose runs take a made-up time per (window, slots)."""

import pytest

from paper_2401_12377_b300 import autotune


class FakeContext:
    made = []

    def __init__(self, window, n_streams=1, cta_slots=0, timing=False, capacity=0, **_):
        self.window, self.n_streams, self.cta_slots = window, n_streams, cta_slots
        self.kernel_ms = 0.0
        FakeContext.made.append((window, cta_slots))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def stats(self):
        cap = 296 - self.n_streams if self.window <= 32 else 200 - self.n_streams
        return {"kernel_ms": self.kernel_ms, "cta_slots": self.cta_slots or cap}


def cost(W, slots):
    # fastest at W = 16 with the most slots; a little noise per repeat below
    return 10.0 + abs(W - 16) * 0.5 + 300.0 / slots


@pytest.fixture
def fake(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune.harness, "Context", FakeContext)
    FakeContext.made = []
    return str(tmp_path / "cache.json")


def make_run(ctx):
    k = [0]

    def run():
        k[0] += 1
        ctx.kernel_ms += cost(ctx.window, ctx.cta_slots) + (0.01 if k[0] % 3 == 0 else 0.0)
        return 1000
    return run


def test_picks_the_fastest_median_and_caps_slots(fake):
    out = autotune.tune("w1", make_run, n_streams=4, windows=(8, 16, 64), slots=(64, 148, 296, 444),
                        repeats=5, path=fake)
    assert (out["window"], out["cta_slots"]) == (16, 292)     # 296 - 4 scheduler CTAs, the cap
    # slot candidates: capped and deduplicated per window
    tried = {(r["window"], r["cta_slots"]) for r in out["table"]}
    assert tried == {(8, 64), (8, 148), (8, 292), (16, 64), (16, 148), (16, 292),
                     (64, 64), (64, 148), (64, 196)}
    best = min(out["table"], key=lambda r: r["ms"])
    assert best["ms"] == out["ms"] and abs(out["ms"] - cost(16, 292)) < 0.02


def test_cache_by_workload(fake):
    a = autotune.tune("w1", make_run, n_streams=1, windows=(8, 32), slots=(64, 148), repeats=3, path=fake)
    n = len(FakeContext.made)
    b = autotune.tune("w1", make_run, n_streams=1, windows=(8, 32), slots=(64, 148), repeats=3, path=fake)
    assert b["cached"] is True and len(FakeContext.made) == n      # no context made the second time
    assert (b["window"], b["cta_slots"]) == (a["window"], a["cta_slots"])
    autotune.tune("w2", make_run, n_streams=1, windows=(8,), slots=(64,), repeats=1, path=fake)
    assert len(FakeContext.made) > n                               # another workload is tuned afresh
    assert len(autotune.load_cache(fake)) == 2


def test_unreadable_cache_is_empty(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    assert autotune.load_cache(str(p)) == {}
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
