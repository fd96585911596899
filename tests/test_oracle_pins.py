"""Pins for the CPU oracle: each test checks the oracle against something that
is not the oracle -- a closed form, a numpy/library routine, an invariant, or
the paper's worked example (§3.2) -- so that a dropped term, a wrong sign or a
transposed operand anywhere in the typemap walker fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle as o

GOLD = os.path.join(os.path.dirname(__file__), "golden")
F32 = lambda: o.basic(4, 4)  # noqa: E731
F64 = lambda: o.basic(8, 8)  # noqa: E731


def origins_of_packed(t, count, span, base=0):
    """Byte-marking: pack four planes whose byte i holds byte p of i, and
    reassemble the source offset of every packed byte."""
    idx = np.arange(span, dtype=np.int64) - base
    out = np.zeros(count * t.size, np.int64)
    for p in range(4):
        plane = ((idx + base) >> (8 * p)).astype(np.uint8)
        out |= t.pack(plane, count, base).astype(np.int64) << (8 * p)
    return out - base


def expand(disps, sizes):
    if len(disps) == 0:
        return np.zeros(0, np.int64)
    return np.concatenate([np.arange(d, d + s) for d, s in zip(disps, sizes)])


# --------------------------------------------------------------------------
# §3.2 worked example
# --------------------------------------------------------------------------

def test_typeiov_example_closed_form():
    g = json.load(open(os.path.join(GOLD, "typeiov.json")))
    value = o.contiguous(g["value_bytes"], o.basic(1, 1))
    vol = o.subarray(g["full_sizes"], g["sub_sizes"], g["sub_offsets"], value)
    assert vol.size == g["size"]
    assert vol.lb == g["lb"]
    assert vol.extent == g["extent"]
    assert vol.iov_len(g["max_iov_bytes"]) == (g["iov_len"], g["iov_bytes"])
    d, l = vol.iov(0, 4)
    assert [[int(a), int(b)] for a, b in zip(d, l)] == g["iov"]
    # displacement beyond 2^32: int64 arithmetic is required
    assert d[0] > 2**32


# --------------------------------------------------------------------------
# Sizes, bounds and extents: closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("c,bl,st", [(1, 1, 1), (5, 2, 3), (7, 3, 3), (4, 1, -2), (6, 2, -5), (3, 4, 2)])
def test_vector_closed_form(c, bl, st):
    v = o.vector(c, bl, st, F32())
    assert v.size == 4 * c * bl
    lo = min(0, (c - 1) * st)
    hi = max(0, (c - 1) * st) + bl
    assert v.lb == 4 * lo
    assert v.extent == 4 * (hi - lo)
    h = o.hvector(c, bl, 4 * st, F32())
    assert (h.size, h.lb, h.extent) == (v.size, v.lb, v.extent)


def test_subarray_closed_form():
    t = o.subarray([7, 5, 3], [2, 3, 1], [4, 1, 2], F64())
    assert (t.size, t.lb, t.extent) == (2 * 3 * 1 * 8, 0, 7 * 5 * 3 * 8)
    # true bounds: first element (4,1,2), last (5,3,2) in C order
    first = ((4 * 5 + 1) * 3 + 2) * 8
    last = ((5 * 5 + 3) * 3 + 2) * 8
    assert (t.true_lb, t.true_extent) == (first, last + 8 - first)


def test_resized_and_sticky_bounds():
    r = o.resized(F32(), -4, 16)
    assert (r.lb, r.extent, r.true_lb, r.true_extent, r.size) == (-4, 16, 0, 4, 4)
    c = o.contiguous(3, r)
    # copies at 0, 16, 32: explicit lb -4, explicit ub 12 + 32
    assert (c.lb, c.extent) == (-4, 48)
    # struct mixing an explicit-bound member with a plain one: only the
    # explicit bound counts for lb/ub (the plain int at -100 does not move lb)
    s = o.struct([1, 1], [0, -100], [r, o.basic(4, 4)])
    assert (s.lb, s.extent) == (-4, 16)
    assert (s.true_lb, s.true_extent) == (-100, 104)


@pytest.mark.parametrize("fields", [
    [("f8", 0), ("i1", 8)],
    [("i4", 0), ("f8", 8), ("i2", 16)],
    [("i1", 0), ("i2", 2), ("i1", 4)],
    [("f4", 0), ("f4", 4), ("i1", 8)],
])
def test_struct_padding_matches_aligned_c_layout(fields):
    # numpy's aligned structured dtype lays fields out like a C compiler;
    # its itemsize is the padded extent the MPI struct constructor produces.
    dt = np.dtype([(f"f{i}", f) for i, (f, _) in enumerate(fields)], align=True)
    offs = [dt.fields[f"f{i}"][1] for i in range(len(fields))]
    types = [o.basic(np.dtype(f).itemsize, np.dtype(f).alignment) for f, _ in fields]
    s = o.struct([1] * len(fields), offs, types)
    assert s.extent == dt.itemsize
    assert s.size == sum(np.dtype(f).itemsize for f, _ in fields)


def test_empty_types():
    e = o.contiguous(0, F32())
    assert (e.size, e.lb, e.extent, e.iov_count()) == (0, 0, 0, 0)
    s = o.struct([1, 0, 1], [8, 100, 0], [F32(), F64(), e])
    # the zero-length block and the empty member add nothing
    assert (s.size, s.lb, s.extent) == (4, 8, 4)


# --------------------------------------------------------------------------
# Typemaps against numpy views (library routines)
# --------------------------------------------------------------------------

def test_vector_matches_numpy_strided_rows():
    rng = np.random.default_rng(1)
    src = rng.random(10 * 16, dtype=np.float32)
    v = o.vector(10, 4, 16, F32())
    ref = src.reshape(10, 16)[:, :4].ravel()
    assert np.array_equal(v.pack(src, 1).view(np.float32), ref)
    # count > 1 repeats at the extent (9*16+4 floats)
    big = rng.random(3 * 148 + 16, dtype=np.float32)
    got = v.pack(big, 3).view(np.float32)
    ref = np.concatenate([big[e * 148:e * 148 + 160].reshape(10, 16)[:, :4].ravel() for e in range(3)])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("order", [o.ORDER_C, o.ORDER_F])
def test_subarray_matches_numpy_slicing(order):
    rng = np.random.default_rng(2)
    for _ in range(20):
        nd = int(rng.integers(1, 5))
        sizes = rng.integers(1, 7, nd)
        sub = np.array([rng.integers(0, s + 1) for s in sizes])
        st = np.array([rng.integers(0, s - u + 1) for s, u in zip(sizes, sub)])
        npo = "C" if order == o.ORDER_C else "F"
        arr = np.asarray(rng.random(tuple(sizes)), order=npo)
        t = o.subarray(sizes, sub, st, F64(), order)
        sl = tuple(slice(a, a + b) for a, b in zip(st, sub))
        flat = arr.ravel(order="K").view(np.uint8)
        got = t.pack(flat, 1).view(np.float64)
        assert np.array_equal(got, arr[sl].ravel(order=npo))
        assert t.extent == arr.nbytes


def test_indexed_matches_numpy_take():
    rng = np.random.default_rng(3)
    src = rng.random(400, dtype=np.float32)
    bl = rng.integers(0, 5, 30)
    disp = rng.integers(0, 390, 30)
    t = o.indexed(bl, disp, F32())
    idx = np.repeat(disp, bl) + (np.arange(bl.sum()) - np.repeat(np.cumsum(bl) - bl, bl))
    assert np.array_equal(t.pack(src, 1).view(np.float32), np.take(src, idx))
    h = o.hindexed(bl, disp * 4, F32())
    assert np.array_equal(h.pack(src, 1), t.pack(src, 1))
    ib = o.indexed_block(2, disp, F32())
    idx2 = (disp[:, None] + np.arange(2)[None, :]).ravel()
    assert np.array_equal(ib.pack(src, 1).view(np.float32), np.take(src, idx2))


def test_struct_resized_matches_numpy_record_fields():
    # struct{int32[3] @0, float64[5] @16} resized to 64 B: the record layout
    dt = np.dtype({"names": ["a", "b"], "formats": [("<i4", 3), ("<f8", 5)],
                   "offsets": [0, 16], "itemsize": 64})
    rng = np.random.default_rng(4)
    raw = rng.integers(0, 256, 64 * 9, dtype=np.uint8)
    rec = raw.view(dt)
    st = o.struct([3, 5], [0, 16], [o.basic(4, 4), F64()])
    r = o.resized(st, 0, 64)
    ref = np.hstack([rec["a"].view(np.uint8).reshape(9, 12), rec["b"].view(np.uint8).reshape(9, 40)]).ravel()
    assert np.array_equal(r.pack(raw, 9), ref)
    assert (r.size, r.extent) == (52, 64)


def test_nested_vector_of_vector_is_2d_strided_view():
    # §3: a YZ surface is a two-level nested strided vector
    nz, ny, nx = 5, 6, 7
    rng = np.random.default_rng(5)
    a = rng.random((nz, ny, nx))
    x0 = 3
    inner = o.vector(ny, 1, nx, F64())                  # one column over y
    face = o.hvector(nz, 1, nx * ny * 8, inner)          # stacked over z
    ref = a[:, :, x0].ravel()
    got = face.pack(a.ravel().view(np.uint8), 1, base_offset=8 * x0).view(np.float64)
    assert np.array_equal(got, ref)
    sub = o.subarray([nz, ny, nx], [nz, ny, 1], [0, 0, x0], F64())
    assert sub.iov_count() == ny * nz
    d1, s1 = face.typemap()
    d2, s2 = sub.typemap()
    assert np.array_equal(d1 + 8 * x0, d2) and np.array_equal(s1, s2)


def test_resized_contiguous_is_strided_view():
    src = np.arange(60, dtype=np.float32)
    r = o.resized(F32(), 0, 12)
    c = o.contiguous(20, r)
    assert np.array_equal(c.pack(src, 1).view(np.float32), src[::3])
    neg = o.hvector(5, 1, -8, F32())      # backwards stride
    got = neg.pack(src, 1, base_offset=4 * 40).view(np.float32)
    assert np.array_equal(got, src[40:30:-2])


# --------------------------------------------------------------------------
# Segments and iov queries
# --------------------------------------------------------------------------

def rle_segments(disps, sizes):
    """Run-length encode a typemap with numpy: a new segment starts wherever
    an entry does not begin at the previous entry's end."""
    if len(disps) == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    start = np.ones(len(disps), bool)
    start[1:] = disps[1:] != disps[:-1] + sizes[:-1]
    seg_id = np.cumsum(start) - 1
    lens = np.bincount(seg_id, weights=sizes).astype(np.int64)
    return disps[start], lens


def random_type(rng, depth=0):
    kinds = ["basic", "contig", "vector", "hvector", "indexed", "hindexed", "struct",
             "subarray", "resized", "indexed_block"]
    if depth >= 3:
        kinds = ["basic"]
    k = kinds[int(rng.integers(len(kinds)))] if depth > 0 else kinds[int(rng.integers(1, len(kinds)))]
    if k == "basic":
        s = int(rng.choice([1, 2, 4, 8]))
        return o.basic(s, s)
    old = random_type(rng, depth + 1)
    if k == "contig":
        return o.contiguous(int(rng.integers(0, 4)), old)
    if k == "vector":
        return o.vector(int(rng.integers(0, 4)), int(rng.integers(0, 4)), int(rng.integers(-4, 5)), old)
    if k == "hvector":
        return o.hvector(int(rng.integers(0, 4)), int(rng.integers(0, 3)), int(rng.integers(-40, 41)), old)
    if k in ("indexed", "hindexed"):
        n = int(rng.integers(0, 4))
        bl = rng.integers(0, 3, n)
        d = rng.integers(-5, 6, n) if k == "indexed" else rng.integers(-40, 41, n)
        return (o.indexed if k == "indexed" else o.hindexed)(bl, d, old)
    if k == "indexed_block":
        n = int(rng.integers(0, 4))
        return o.indexed_block(int(rng.integers(0, 3)), rng.integers(-5, 6, n), old)
    if k == "struct":
        n = int(rng.integers(1, 4))
        ts = [old] + [random_type(rng, depth + 1) for _ in range(n - 1)]
        return o.struct(rng.integers(0, 3, n), rng.integers(-40, 41, n), ts)
    if k == "subarray":
        nd = int(rng.integers(1, 3))
        sizes = rng.integers(1, 4, nd)
        sub = np.array([rng.integers(0, s + 1) for s in sizes])
        st = np.array([rng.integers(0, s - u + 1) for s, u in zip(sizes, sub)])
        return o.subarray(sizes, sub, st, old, int(rng.integers(2)))
    return o.resized(old, int(rng.integers(-8, 9)), int(rng.integers(0, 40)))


def test_random_types_segment_and_pack_invariants():
    rng = np.random.default_rng(6)
    for _ in range(300):
        t = random_type(rng)
        d, s = t.typemap()
        assert s.sum() == t.size
        # iov list = run-length encoding of the typemap, in order
        sd, sl = t.iov()
        rd, rl = rle_segments(d, s)
        assert np.array_equal(sd, rd) and np.array_equal(sl, rl)
        assert sl.sum() == t.size and t.iov_count() == len(sd)
        if t.size:
            assert t.true_lb == (d).min() and t.true_extent == (d + s).max() - d.min()
        # byte marking: every packed byte comes from the typemap byte it should
        count = int(rng.integers(1, 4))
        if t.size == 0:
            continue
        lo = min(0, t.lb, t.true_lb, (count - 1) * t.extent + t.true_lb)
        hi = max(t.true_lb + t.true_extent, (count - 1) * t.extent + t.true_lb + t.true_extent) + 1
        base = -lo
        span = hi - lo
        got = origins_of_packed(t, count, span, base)
        ref = np.concatenate([expand(d + e * t.extent, s) for e in range(count)])
        assert np.array_equal(got, ref)


def test_iov_chunks_and_offsets():
    rng = np.random.default_rng(7)
    for _ in range(100):
        t = random_type(rng)
        sd, sl = t.iov()
        n = len(sd)
        for k in [0, 1, n // 2, max(n - 1, 0), n, n + 3]:
            for m in [0, 1, 3, n + 5]:
                d, l = t.iov(k, m)
                assert np.array_equal(d, sd[k:k + m]) and np.array_equal(l, sl[k:k + m])
        with pytest.raises(ValueError):
            t.iov(-1, 2)
        # element-level list: per-element list at e*extent, nothing merged across
        ed, el = t.iov_elements(3)
        assert np.array_equal(ed, np.concatenate([sd + e * t.extent for e in range(3)]))
        assert np.array_equal(el, np.tile(sl, 3))


def test_iov_len_bisection_identity():
    rng = np.random.default_rng(8)
    for _ in range(100):
        t = random_type(rng)
        sd, sl = t.iov()
        pre = np.concatenate([[0], np.cumsum(sl)])
        n = len(sl)
        assert t.iov_len(-1) == (n, t.size)
        assert t.iov_len(t.size) == (n, t.size)
        assert t.iov_len(t.size + 17) == (n, t.size)
        assert t.iov_len(0) == (0, 0)
        for b in range(0, t.size + 1):
            k = int(np.searchsorted(pre, b, side="right") - 1)
            assert t.iov_len(b) == (k, int(pre[k]))
        with pytest.raises(ValueError):
            t.iov_len(-2)


def test_merge_rule_only_adjacent_in_order():
    f = F32()
    # entries at 4 then 0: byte-adjacent but out of order -> two segments
    t = o.hindexed([1, 1], [4, 0], f)
    assert t.iov_count() == 2
    # entries at 0 then 4: merged
    assert o.hindexed([1, 1], [0, 4], f).iov_count() == 1
    # zero-length block in the middle does not break a merge
    assert o.hindexed([1, 0, 1], [0, 100, 4], f).iov_count() == 1
    # config-1 layout: vector(1024,4,16) of float, 64 elements as one type
    v = o.vector(1024, 4, 16, f)
    assert v.iov_count() == 1024 and v.extent == 65488
    c = o.contiguous(64, v)
    assert c.iov_count() == 64 * 1024 - 63      # last/first blocks abut
    d, l = c.iov(1023, 2)
    assert list(l) == [32, 16]


def test_struct_iov_len_closed_form():
    st = o.resized(o.struct([3, 5], [0, 16], [o.basic(4, 4), F64()]), 0, 64)
    ix = o.indexed([2, 3, 1], [0, 5, 9], st)
    size = 52 * 6
    assert ix.size == size
    for b in range(size):
        e, r = divmod(b, 52)
        k = 2 * e + (r >= 12)
        assert ix.iov_len(b) == (k, 52 * e + 12 * (r >= 12))


# --------------------------------------------------------------------------
# Unpack, overlap and the adjoint
# --------------------------------------------------------------------------

def test_unpack_round_trip_and_sentinels():
    rng = np.random.default_rng(9)
    for _ in range(200):
        t = random_type(rng)
        if t.size == 0 or t.overlaps(2):
            continue
        count = 2
        lo = min(0, t.true_lb, t.extent + t.true_lb)
        hi = max(t.true_lb + t.true_extent, t.extent + t.true_lb + t.true_extent) + 1
        span, base = hi - lo, -lo
        src = rng.integers(0, 256, span, dtype=np.uint8)
        packed = t.pack(src, count, base)
        dst = np.full(span, 0xA5, np.uint8)
        t.unpack(packed, count, dst, base)
        d, s = t.typemap()
        cover = np.concatenate([expand(d + e * t.extent, s) for e in range(count)]) + base
        mask = np.zeros(span, bool)
        mask[cover] = True
        assert np.array_equal(dst[mask], src[mask])
        assert np.all(dst[~mask] == 0xA5)
        assert np.array_equal(t.pack(dst, count, base), packed)


def test_overlap_detection():
    f = F32()
    assert not o.vector(4, 2, 2, f).overlaps()
    assert o.vector(4, 3, 2, f).overlaps()
    assert o.hindexed([1, 1], [0, 2], f).overlaps()
    r = o.resized(o.contiguous(2, f), 0, 4)  # elements 8 B long at a 4 B extent
    assert not r.overlaps(1) and r.overlaps(2)


def test_adjoint_dot_product_and_multiplicity():
    rng = np.random.default_rng(10)
    f = F32()
    n = 300
    disp = rng.integers(0, n - 3, 80)
    bl = rng.integers(1, 4, 80)
    t = o.indexed(bl, disp, f)  # repeats entries
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(t.size // 4)
    px = t.pack(x, 1).view(np.float32).astype(np.float64)
    gx = t.pack_adjoint_f64(y, 1, n)
    assert abs(px @ y - x.astype(np.float64) @ gx) < 1e-9 * (1 + abs(px @ y))
    idx = np.repeat(disp, bl) + (np.arange(bl.sum()) - np.repeat(np.cumsum(bl) - bl, bl))
    counts = t.pack_adjoint_f64(np.ones(t.size // 4), 1, n)
    assert np.array_equal(counts, np.bincount(idx, minlength=n).astype(np.float64))


def _owned(g, dist, darg, p, c):
    """Global indices process coordinate c owns along one dimension, from the
    distribution's definition (block: one contiguous run of b per process;
    cyclic: blocks of b dealt round-robin; none: everything)."""
    i = np.arange(g)
    if dist == o.DIST_NONE:
        return i
    if dist == o.DIST_BLOCK:
        b = -(-g // p) if darg == o.DFLT_DARG else darg
        return i[(i >= c * b) & (i < (c + 1) * b)]
    b = 1 if darg == o.DFLT_DARG else darg
    return i[(i // b) % p == c]


def _random_darray(rng):
    nd = int(rng.integers(1, 4))
    gs = [int(x) for x in rng.integers(1, 8, nd)]
    ps, dist, dargs = [], [], []
    for g in gs:
        k = int(rng.integers(3))
        p = 1 if k == o.DIST_NONE else int(rng.integers(1, 4))
        if k == o.DIST_BLOCK:
            d = o.DFLT_DARG if rng.random() < 0.5 else -(-g // p) + int(rng.integers(0, 2))
        elif k == o.DIST_CYCLIC:
            d = o.DFLT_DARG if rng.random() < 0.5 else int(rng.integers(1, 4))
        else:
            d = o.DFLT_DARG
        ps.append(p), dist.append(k), dargs.append(d)
    return gs, ps, dist, dargs


@pytest.mark.parametrize("order", [o.ORDER_C, o.ORDER_F])
def test_darray_matches_numpy_ownership(order):
    """Every rank's darray packs exactly arr[ix_(owned per dim)] in the
    array's storage order, over a row-major process grid; its extent is the
    whole global array; and the ranks' typemaps tile the array exactly once."""
    rng = np.random.default_rng(17 + order)
    npo = "C" if order == o.ORDER_C else "F"
    for _ in range(40):
        gs, ps, dist, dargs = _random_darray(rng)
        arr = np.asarray(rng.random(tuple(gs)), order=npo)
        flat = arr.ravel(order="K").view(np.uint8)
        cover = np.zeros(arr.nbytes, np.int64)
        size = int(np.prod(ps))
        for rank in range(size):
            coords = np.unravel_index(rank, ps)  # process grid is always row-major
            t = o.darray(size, rank, gs, dist, dargs, ps, F64(), order)
            idx = [_owned(g, d, a, p, int(c)) for g, d, a, p, c in zip(gs, dist, dargs, ps, coords)]
            ref = arr[np.ix_(*idx)].ravel(order=npo)
            assert t.size == ref.nbytes
            assert (t.lb, t.extent) == (0, arr.nbytes)
            assert np.array_equal(t.pack(flat, 1).view(np.float64), ref), (gs, ps, dist, dargs, rank)
            d, sz = t.typemap()
            for a, s in zip(d, sz):
                cover[a:a + s] += 1
        assert np.all(cover == 1)


def test_darray_rejects_bad_grids():
    with pytest.raises(ValueError):  # block too small to cover the dimension
        o.darray(2, 0, [9], [o.DIST_BLOCK], [4], [2], F64())
    with pytest.raises(ValueError):  # grid does not have `size` processes
        o.darray(4, 0, [8], [o.DIST_CYCLIC], [o.DFLT_DARG], [3], F64())
    with pytest.raises(ValueError):  # undistributed dimension over 2 processes
        o.darray(2, 0, [8], [o.DIST_NONE], [o.DFLT_DARG], [2], F64())
    with pytest.raises(ValueError):  # rank out of range
        o.darray(2, 2, [8], [o.DIST_CYCLIC], [o.DFLT_DARG], [2], F64())


def _stream_addrs(t, count):
    """User byte address of every packed-stream byte, by expanding the typemap
    entry by entry (brute force, tiny types only)."""
    d, s = t.typemap()
    one = np.concatenate([np.arange(a, a + n) for a, n in zip(d, s)]) if len(d) else np.zeros(0, np.int64)
    return np.concatenate([one + e * t.extent for e in range(count)]) if count else one[:0]


def test_range_moves_follow_the_stream_byte_map():
    """Range pack / unpack move exactly the packed-stream bytes of the window:
    brute-force byte maps from the typemap, random windows (ragged, inside one
    entry, empty, whole stream), and windows that tile the stream reproduce
    the full pack and unpack."""
    rng = np.random.default_rng(23)
    for _ in range(150):
        t = random_type(rng)
        count = int(rng.integers(1, 4))
        addr = _stream_addrs(t, count)
        total = count * t.size
        assert addr.size == total
        if total == 0:
            continue
        lo = min(0, int(addr.min()))
        span = int(addr.max()) - lo + 1
        src = rng.integers(0, 256, span, dtype=np.uint8)
        for _ in range(4):
            a = int(rng.integers(0, total + 1))
            b = int(rng.integers(a, total + 1))
            got = t.pack_range(src, count, a, b - a, -lo)
            assert np.array_equal(got, src[addr[a:b] - lo])
            win = rng.integers(0, 256, b - a, dtype=np.uint8)
            dst = np.zeros(span, np.uint8)
            if not t.overlaps(count):
                t.unpack_range(win, a, count, dst, -lo)
                want = np.zeros(span, np.uint8)
                want[addr[a:b] - lo] = win
                assert np.array_equal(dst, want)
        cuts = np.unique(np.concatenate([[0, total], rng.integers(0, total + 1, 5)]))
        parts = [t.pack_range(src, count, int(x), int(y - x), -lo) for x, y in zip(cuts[:-1], cuts[1:])]
        full = t.pack(src, count, -lo)
        assert np.array_equal(np.concatenate(parts), full)
        if not t.overlaps(count):
            want = np.zeros(span, np.uint8)
            t.unpack(full, count, want, -lo)
            dst = np.zeros(span, np.uint8)
            order = rng.permutation(len(cuts) - 1)
            for i in order:
                x, y = int(cuts[i]), int(cuts[i + 1])
                t.unpack_range(full[x:y], x, count, dst, -lo)
            assert np.array_equal(dst, want)
    t = o.vector(3, 1, 2, F64())
    with pytest.raises(ValueError):
        t.pack_range(np.zeros(64, np.uint8), 1, 20, 5)
