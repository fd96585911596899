"""Shared test helpers: build the same spec on both sides and compare."""
import numpy as np

import oracle
import paper_2402_12274_gb300 as dte


def both(spec, commit=True):
    t = dte.Datatype.from_spec(spec)
    if t.h in {b.h for b in dte._BASIC_BY_NAME.values()}:
        t = dte.Datatype.contiguous(1, t)
    if commit:
        t.commit()
    return t, oracle.from_spec(spec)


def iov_arrays(t, offset=0, max_len=None):
    lst = t.iov(offset, max_len)
    d = np.array([a for a, _ in lst], np.int64)
    l = np.array([b for _, b in lst], np.int64)
    return d, l


def span_of(o, count):
    """(lo, hi) byte range touched by `count` elements, relative to displacement 0."""
    if o.size == 0 or count == 0:
        return 0, 0
    ends = [e * o.extent for e in (0, count - 1)]
    lo = min(e + o.true_lb for e in ends)
    hi = max(e + o.true_lb + o.true_extent for e in ends)
    return lo, hi
