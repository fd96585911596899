"""Host logic of the batch launch-shape autotuner: the shape-mix signature,
the choice of the fastest candidate, and the cache round trip (timing is
replaced by a fixed table, so no GPU is needed)."""
import pytest

pytest.importorskip("torch")
from paper_2402_12274_gb300 import autotune  # noqa: E402


class FakeBatch:
    def __init__(self):
        self.shapes = []

    def set_launch(self, blocks_per_sm, span_tiles):
        self.shapes.append((blocks_per_sm, span_tiles))

    def enqueue(self, stream=None):
        pass


def test_signature_depends_on_the_mix_only():
    a = [(16, 1000), (4, 70000), (16, 1020)]
    assert autotune.signature(1, a) == autotune.signature(1, list(reversed(a)))
    # same power-of-two buckets -> same signature
    assert autotune.signature(1, a) == autotune.signature(1, [(16, 1010), (4, 66000), (16, 1001)])
    assert autotune.signature(1, a) != autotune.signature(0, a)          # kind
    assert autotune.signature(1, a) != autotune.signature(1, a[:2])      # counts
    assert autotune.signature(1, a) != autotune.signature(1, [(8, 1000), (4, 70000), (16, 1020)])  # word class
    assert autotune.signature(1, a) != autotune.signature(1, [(16, 3000), (4, 70000), (16, 1020)])  # size bucket


def test_tune_applies_the_fastest_and_caches_it(tmp_path, monkeypatch):
    monkeypatch.setenv("DTE_TUNE_CACHE", str(tmp_path / "tune.json"))
    times = {c: 1.0 + 0.01 * i for i, c in enumerate(autotune.CANDIDATES)}
    best = autotune.CANDIDATES[5]
    times[best] = 0.5
    timed = []

    def fake_time(batch, stream, reps, flush):
        shape = batch.shapes[-1]
        timed.append(shape)
        return times[shape]

    monkeypatch.setattr(autotune, "time_batch", fake_time)
    b = FakeBatch()
    shapes = [(16, 4096), (2, 300)]
    choice, sec, table = autotune.tune(b, 1, shapes, stream=object())
    assert choice == best and sec == 0.5
    assert sorted(timed) == sorted(autotune.CANDIDATES)
    assert b.shapes[-1] == best
    assert set(table) == set(autotune.CANDIDATES)

    # a batch of the same mix takes the cached choice without timing anything
    def no_time(*a, **k):
        raise AssertionError("timed despite a cached choice")

    monkeypatch.setattr(autotune, "time_batch", no_time)
    b2 = FakeBatch()
    choice2, sec2, table2 = autotune.tune(b2, 1, [(16, 5000), (2, 400)], stream=object())
    assert choice2 == best and sec2 is None and table2 is None
    assert b2.shapes == [best]


def test_tune_without_cache_does_not_write(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("DTE_TUNE_CACHE", str(path))
    monkeypatch.setattr(autotune, "time_batch", lambda batch, stream, reps, flush: float(sum(batch.shapes[-1])))
    choice, _, _ = autotune.tune(FakeBatch(), 0, [(16, 64)], stream=object(), use_cache=False)
    assert choice == min(autotune.CANDIDATES, key=sum)
    assert not path.exists()
