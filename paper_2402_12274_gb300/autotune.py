"""Launch-shape autotuner for batches.

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

from . import Batch

CANDIDATES = [(b, s) for b in (0, 2, 3) for s in (1, 2, 4, 8)]


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
