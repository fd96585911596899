"""Autotuners: kernel plans per descriptor shape, and the launch shape of a
batch.

Plans (``dte_type_set_plan``): how the kernels move a type -- chunk-major
with 1 KiB or 2 KiB warp steps for 16-byte copy words, segment-major rounds
for smaller words, or TMA bulk copies for single moves of long runs.  The
library's fixed rule picks one from descriptor statistics; ``tune_plans``
measures instead.  It groups the operations of a batch (or single moves) by
shape -- direction, copy word, whether an index list is searched, the mean
run and the size, as the library reports them (``dte_op_shape_query``) --
times each candidate plan on the operations of each group, keeps the
fastest per group, and caches the pick under the shape key, so later
operations of the same shape reuse it without timing.

Launch shape (below): 

A batch runs one persistent launch per copy-word class; its shape has two
knobs (``dte_batch_set_launch``): CTAs per SM and the span of consecutive
tiles (1-2 KiB of packed data, or 32-segment rounds) a warp takes at a time.
The best choice depends on the shapes in the batch (many tiny ops favour
short spans and full occupancy; long runs over large index tables favour
longer spans).  The tuner times every
candidate on the batch itself with CUDA events, keeps the fastest, and caches
it under a signature of the batch's shape mix (per word class: count of ops
in each power-of-two size bucket), so batches of the same mix reuse it.
The cache is a JSON file (``DTE_TUNE_CACHE``, default
``~/.cache/dte_autotune.json``).
"""
from __future__ import annotations

import hashlib
import json
import math
import os

import torch

from . import (PLAN_AUTO, PLAN_BULK, PLAN_CHUNK, PLAN_CHUNK_WIDE, PLAN_SEGMENT, Batch, dte_op_shape_query,
               dte_type_get_plan, dte_type_set_plan)

CANDIDATES = [(b, s) for b in (0, 2, 3) for s in (1, 2, 4, 8)]

PLAN_NAMES = {PLAN_AUTO: "auto", PLAN_CHUNK: "chunk", PLAN_CHUNK_WIDE: "chunk_wide", PLAN_SEGMENT: "segment",
              PLAN_BULK: "bulk"}
SEG_MAX_RUN = 4096  # runs the segment-major kernels take (include/dte.h, dte_plan)


def _cache_path() -> str:
    return os.environ.get("DTE_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "dte_autotune.json"))


def _load() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache: dict) -> None:
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, p)
    except OSError:
        pass


def signature(kind: int, shapes) -> str:
    """shapes: iterable of (word_bytes, packed_bytes) per op."""
    hist = {}
    for w, nbytes in shapes:
        b = int(math.log2(max(nbytes, 1)))
        hist[f"{w}:{b}"] = hist.get(f"{w}:{b}", 0) + 1
    key = json.dumps([kind, sorted(hist.items())])
    return hashlib.sha256(key.encode()).hexdigest()[:20]


def time_batch(batch: Batch, stream, reps: int = 5, flush=None) -> float:
    """Mean seconds per launch of `batch` on `stream` (events on that stream)."""
    ev = []
    with torch.cuda.stream(stream):
        batch.enqueue(stream)
        for _ in range(reps):
            if flush is not None:
                flush()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.enqueue(stream)
            b.record(stream)
            ev.append((a, b))
    stream.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / len(ev) * 1e-3


def tune(batch: Batch, kind: int, shapes, stream=None, reps: int = 5, flush=None, use_cache: bool = True):
    """Pick and apply the fastest (blocks_per_sm, span_tiles) for `batch`.
    Returns (choice, seconds, table of all candidates)."""
    stream = stream or torch.cuda.current_stream()
    sig = signature(kind, shapes)
    cache = _load() if use_cache else {}
    if use_cache and sig in cache:
        b, s = cache[sig]
        batch.set_launch(b, s)
        return (b, s), None, None
    table = {}
    for b, s in CANDIDATES:
        batch.set_launch(b, s)
        table[(b, s)] = time_batch(batch, stream, reps, flush)
    best = min(table, key=table.get)
    batch.set_launch(*best)
    if use_cache:
        cache[sig] = list(best)
        _store(cache)
    return best, table[best], table


# ---------------------------------------------------------------------------
# kernel plans per descriptor shape
# ---------------------------------------------------------------------------
def shape_key(kind: int, shape: dict, single: bool = False) -> str:
    """Group of an operation: direction, batch or single move, copy word,
    index list or not, and mean run (a power of two); single moves also by
    size (a power of four), since a single launch's size decides how much of
    the GPU it fills, while a batch's operations share one launch."""
    mean = shape["bytes"] // max(shape["segments"], 1)
    key = f"{'s' if single else 'b'}{kind}:w{shape['word']}:l{shape['list']}:r{int(math.log2(max(mean, 1)))}"
    return key + (f":z{int(math.log2(max(shape['bytes'], 1))) // 2}" if single else "")


def plan_candidates(shape: dict, single: bool = False):
    """Plans that can differ for this shape (one entry: nothing to tune)."""
    if shape["word"] == 16:
        return [PLAN_CHUNK, PLAN_CHUNK_WIDE] + ([PLAN_BULK] if single else [])
    if shape["max_run"] <= SEG_MAX_RUN:
        return [PLAN_CHUNK, PLAN_SEGMENT]
    return [PLAN_CHUNK]


def _kernel_of(shape: dict, single: bool) -> int:
    return shape["single_kernel"] if single else shape["batch_kernel"]


def time_ops(kind: int, ops, stream, reps: int = 5, flush=None, single: bool = False) -> float:
    """Mean seconds to run `ops` (one batch, or one enqueue per op when
    `single`) on `stream`, CUDA events on that stream."""
    from . import dte_pack_enqueue, dte_unpack_enqueue
    sh = stream.cuda_stream
    if single:
        def run():
            for t, n, u, p in ops:
                if kind == 1:
                    dte_pack_enqueue(u, n, t, p, 1 << 62, 0, sh)
                else:
                    dte_unpack_enqueue(p, 1 << 62, 0, u, n, t, sh)
        b = None
    else:
        b = Batch(kind, ops)

        def run():
            b.enqueue(stream)
    ev = []
    with torch.cuda.stream(stream):
        run()
        for _ in range(reps):
            if flush is not None:
                flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            ev.append((e0, e1))
    stream.synchronize()
    if b is not None:
        b.free()
    return sum(x.elapsed_time(y) for x, y in ev) / len(ev) * 1e-3


def tune_plans(kind: int, ops, stream=None, reps: int = 20, flush=None, single: bool = False,
               use_cache: bool = True, timer=None, min_gain: float = 0.02):
    """Pick a plan per shape group for `ops` ((type, count, user, packed)
    tuples of one direction, run as one batch, or one move each when
    `single`) and set it on their types.

    Groups are judged in context: starting from the fixed rule, each group in
    turn (largest packed bytes first) is switched to each of its other
    candidate plans and the whole set of operations is timed; a switch is kept
    only if the whole set gets faster by more than `min_gain` (a group timed
    alone -- a tiny launch -- would favour whatever has the least launch
    overhead).  Returns a report {group: {"ops", "auto", "pick", "ms"}}: "auto"
    is the kernel the fixed rule takes, "ms" the whole set's time with the
    group under each candidate (absent for cached or single-candidate
    groups), plus "_total_ms": the whole set under the fixed rule and under
    the picks."""
    stream = stream or torch.cuda.current_stream()
    timer = timer or time_ops
    cache = _load() if use_cache else {}
    groups = {}
    for op in ops:
        dte_type_set_plan(op[0], PLAN_AUTO)
    for op in ops:
        shape = dte_op_shape_query(*op)
        g = groups.setdefault(shape_key(kind, shape, single), {"ops": [], "shape": shape, "bytes": 0})
        g["ops"].append(op)
        g["bytes"] += shape["bytes"]

    def set_group(g, plan):
        for op in g["ops"]:
            dte_type_set_plan(op[0], plan)

    report = {}
    todo = []
    for key, g in groups.items():
        report[key] = {"ops": len(g["ops"]), "auto": PLAN_NAMES[_kernel_of(g["shape"], single)]}
        if use_cache and key in cache:
            set_group(g, int(cache[key]))
            report[key]["pick"] = PLAN_NAMES[int(cache[key])]
        elif len(plan_candidates(g["shape"], single)) > 1:
            todo.append(key)
        else:
            report[key]["pick"] = "auto"
    t_auto = best = timer(kind, ops, stream, reps, flush, single) if todo else None
    for key in sorted(todo, key=lambda k: -groups[k]["bytes"]):
        g = groups[key]
        ms = {"auto": best}
        pick = PLAN_AUTO
        for plan in plan_candidates(g["shape"], single):
            if plan == _kernel_of(g["shape"], single):
                continue  # what the fixed rule already does
            set_group(g, plan)
            t = timer(kind, ops, stream, reps, flush, single)
            ms[PLAN_NAMES[plan]] = t
            if t < best * (1.0 - min_gain):
                best, pick = t, plan
        set_group(g, pick)
        report[key]["ms"] = {k: round(v * 1e3, 4) for k, v in ms.items()}
        report[key]["pick"] = PLAN_NAMES[pick]
        if use_cache:
            cache[key] = pick
    if todo:
        report["_total_ms"] = {"fixed_rule": round(t_auto * 1e3, 4), "tuned": round(best * 1e3, 4)}
    if use_cache:
        _store(cache)
    return report


def reset_plans(ops):
    """Put every type of `ops` back on the fixed rule."""
    for op in ops:
        dte_type_set_plan(op[0], PLAN_AUTO)
