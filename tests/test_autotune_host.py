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


# ---------------------------------------------------------------------------
# kernel plans per descriptor shape (no GPU: committed types, fake pointers,
# and a fixed timing table in place of CUDA events)
# ---------------------------------------------------------------------------
import numpy as np  # noqa: E402

import inputs  # noqa: E402
import paper_2402_12274_gb300 as dte  # noqa: E402

U, P = 1 << 20, 1 << 30  # 16-byte aligned stand-in addresses (never dereferenced)


def test_plan_abi_set_get_dup_and_errors():
    t = dte.Datatype.vector(100, 3, 7, dte.FLOAT32).commit()
    assert dte.dte_type_get_plan(t.h) == dte.PLAN_AUTO
    dte.dte_type_set_plan(t.h, dte.PLAN_SEGMENT)
    assert dte.dte_type_get_plan(t.h) == dte.PLAN_SEGMENT
    d = dte.Datatype(dte.dte_type_dup(t.h))
    assert dte.dte_type_get_plan(d.h) == dte.PLAN_SEGMENT
    with pytest.raises(dte.DteError) as e:
        dte.dte_type_set_plan(t.h, 5)
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:
        dte.dte_type_set_plan(dte.FLOAT32.h, dte.PLAN_CHUNK)
    assert e.value.code == dte.ERR_TYPE


def test_shape_query_follows_the_plan():
    rec = dte.Datatype.from_spec(inputs.record_indexed_spec(np.random.default_rng(3), 1000)).commit()
    s = dte.dte_op_shape_query(rec.h, 1, U, P)
    # 12- and 40-byte runs at a 52-byte packed stride: 4-byte words, an index
    # list of 1000 blocks, the fixed rule's segment-major kernel
    assert (s["word"], s["list"], s["max_run"]) == (4, 1, 40)
    assert s["batch_kernel"] == s["single_kernel"] == dte.PLAN_SEGMENT
    assert s["bytes"] == rec.size and s["segments"] == rec.num_segments
    dte.dte_type_set_plan(rec.h, dte.PLAN_CHUNK)
    assert dte.dte_op_shape_query(rec.h, 1, U, P)["batch_kernel"] == dte.PLAN_CHUNK
    dte.dte_type_set_plan(rec.h, dte.PLAN_CHUNK_WIDE)  # no 16-byte words: the fixed rule
    assert dte.dte_op_shape_query(rec.h, 1, U, P)["batch_kernel"] == dte.PLAN_SEGMENT
    big = dte.Datatype.hvector(64, 1, 3 * 4096, dte.Datatype.contiguous(512, dte.FLOAT64)).commit()
    s = dte.dte_op_shape_query(big.h, 1, U, P)
    assert (s["word"], s["batch_kernel"]) == (16, dte.PLAN_CHUNK)
    dte.dte_type_set_plan(big.h, dte.PLAN_CHUNK_WIDE)
    assert dte.dte_op_shape_query(big.h, 1, U, P)["batch_kernel"] == dte.PLAN_CHUNK_WIDE
    dte.dte_type_set_plan(big.h, dte.PLAN_SEGMENT)  # segment-major needs words below 16 bytes
    assert dte.dte_op_shape_query(big.h, 1, U, P)["batch_kernel"] == dte.PLAN_CHUNK
    # a misaligned user pointer lowers the copy word
    assert dte.dte_op_shape_query(big.h, 1, U + 4, P)["word"] == 4


def test_shape_keys_and_candidates():
    a = {"word": 4, "list": 1, "bytes": 1 << 20, "segments": 1 << 15, "max_run": 40}
    assert autotune.shape_key(1, a) == autotune.shape_key(1, dict(a, bytes=(1 << 20) + 7))
    assert autotune.shape_key(1, a) != autotune.shape_key(0, a)                       # direction
    assert autotune.shape_key(1, a) != autotune.shape_key(1, a, single=True)          # batch vs single
    assert autotune.shape_key(1, a) != autotune.shape_key(1, dict(a, word=8))         # copy word
    assert autotune.shape_key(1, a) != autotune.shape_key(1, dict(a, list=0))         # list or regular
    assert autotune.shape_key(1, a) != autotune.shape_key(1, dict(a, segments=1 << 10))  # mean run
    # size separates single moves only (a batch's operations share one launch)
    assert autotune.shape_key(1, a) == autotune.shape_key(1, dict(a, bytes=1 << 26, segments=1 << 21))
    assert (autotune.shape_key(1, a, single=True) !=
            autotune.shape_key(1, dict(a, bytes=1 << 26, segments=1 << 21), single=True))
    assert autotune.plan_candidates(a) == [dte.PLAN_CHUNK, dte.PLAN_SEGMENT]
    assert autotune.plan_candidates(dict(a, max_run=8192)) == [dte.PLAN_CHUNK]
    w16 = dict(a, word=16)
    assert autotune.plan_candidates(w16) == [dte.PLAN_CHUNK, dte.PLAN_CHUNK_WIDE]
    assert autotune.plan_candidates(w16, single=True) == [dte.PLAN_CHUNK, dte.PLAN_CHUNK_WIDE, dte.PLAN_BULK]


def test_tune_plans_keeps_only_switches_that_speed_up_the_whole_set(tmp_path, monkeypatch):
    monkeypatch.setenv("DTE_TUNE_CACHE", str(tmp_path / "tune.json"))
    rng = np.random.default_rng(3)
    recs = [dte.Datatype.from_spec(inputs.record_indexed_spec(rng, 500)).commit() for _ in range(3)]
    bigs = [dte.Datatype.hvector(64, 1, 3 * 4096, dte.Datatype.contiguous(512, dte.FLOAT64)).commit()
            for _ in range(2)]
    ops = [(t.h, 1, U, P) for t in recs + bigs]
    timed = []

    def fake_timer(kind, allops, stream, reps, flush, single):
        # the whole set is timed every time; its time depends on every plan
        assert len(allops) == len(ops)
        rec = {dte.dte_type_get_plan(t.h) for t in recs}
        big = {dte.dte_type_get_plan(t.h) for t in bigs}
        assert len(rec) == 1 and len(big) == 1  # a group switches as a whole
        rec, big = rec.pop(), big.pop()
        timed.append((rec, big))
        t = 10.0
        t -= 2.0 if rec == dte.PLAN_CHUNK else 0.0          # chunk-major helps the records
        t -= 0.1 if big == dte.PLAN_CHUNK_WIDE else 0.0     # the wide step: within noise
        return t

    rep = autotune.tune_plans(1, ops, stream=object(), timer=fake_timer)
    # the fixed rule first, then one switch per group (largest bytes first)
    assert timed[0] == (dte.PLAN_AUTO, dte.PLAN_AUTO) and len(timed) == 3
    picks = {v["ops"]: (v["auto"], v["pick"]) for k, v in rep.items() if not k.startswith("_")}
    assert picks == {3: ("segment", "chunk"), 2: ("chunk", "auto")}  # a 1% gain is not kept
    assert rep["_total_ms"] == {"fixed_rule": 10000.0, "tuned": 8000.0}
    assert [dte.dte_type_get_plan(t.h) for t in recs] == [dte.PLAN_CHUNK] * 3
    assert [dte.dte_type_get_plan(t.h) for t in bigs] == [dte.PLAN_AUTO] * 2

    # the same shapes later take the cached picks without timing
    def no_timer(*a):
        raise AssertionError("timed despite cached picks")

    autotune.reset_plans(ops)
    rep2 = autotune.tune_plans(1, ops, stream=object(), timer=no_timer)
    assert "_total_ms" not in rep2
    assert [dte.dte_type_get_plan(t.h) for t in recs] == [dte.PLAN_CHUNK] * 3
