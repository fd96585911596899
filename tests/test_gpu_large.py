"""Moves past 32-bit offsets: a packed stream longer than 4 GiB (chunk-major,
bulk-copy and record-major kernels, a range window across 2^32, a batch),
and a segment-major move of more than 2^31 segments.

The oracle walks every typemap entry, so it is run on one element and the
full-size result is checked through a property of pack, which is a byte
copy: element e's source is a seeded pattern XOR (e mod 256), so its packed
bytes are the oracle's one-element pack XOR (e mod 256).  A 32-bit truncation
of an offset would read or write another element's bytes (32 or 64 elements
away at these sizes) and fail the check.  Every output byte is compared, on
the device, in chunks of elements."""
import numpy as np
import pytest

from tests.helpers import both

torch = pytest.importorskip("torch")
import paper_2402_12274_gb300 as dte  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda"
SENT = 0xA5


def element_source(o, count, rng):
    """Device source of `count` elements: pattern XOR (e mod 256), with the
    pattern spanning one extent; also returns the pattern (host)."""
    ext = o.extent
    pattern = rng.integers(0, 256, ext, dtype=np.uint8)
    pd = torch.from_numpy(pattern).to(DEV)
    xr = (torch.arange(count, device=DEV) & 255).to(torch.uint8)
    src = torch.empty(count * ext, dtype=torch.uint8, device=DEV)
    rows = max(1, (256 << 20) // ext)
    sv = src.view(count, ext)
    for r0 in range(0, count, rows):
        r1 = min(count, r0 + rows)
        sv[r0:r1] = pd[None, :] ^ xr[r0:r1, None]
    return src, pattern


def check_rows(got, count, width, row_fn):
    """Compare got.view(count, width) with row_fn(r0, r1), chunk by chunk."""
    gv = got.view(count, width)
    rows = max(1, (256 << 20) // width)
    for r0 in range(0, count, rows):
        r1 = min(count, r0 + rows)
        assert torch.equal(gv[r0:r1], row_fn(r0, r1)), (r0, r1)


def typemap_mask(o):
    """Bool mask over one extent: True at the typemap's bytes (oracle unpack
    of zeros into 0xFF)."""
    tgt = np.full(o.extent, 0xFF, np.uint8)
    o.unpack(np.zeros(o.size, np.uint8), 1, tgt, 0)
    return torch.from_numpy(tgt == 0).to(DEV)


def big_round_trip(spec, count, rng, extra=None):
    t, o = both(spec)
    assert o.lb == 0
    src, pattern = element_source(o, count, rng)
    single = torch.from_numpy(o.pack(pattern, 1, 0)).to(DEV)
    xr = (torch.arange(count, device=DEV) & 255).to(torch.uint8)

    def packed_rows(r0, r1):
        return single[None, :] ^ xr[r0:r1, None]

    total = count * o.size
    packed = torch.empty(total, dtype=torch.uint8, device=DEV)
    s = torch.cuda.current_stream()
    assert dte.pack(src, count, t, packed, 0, s) == total
    s.synchronize()
    check_rows(packed, count, o.size, packed_rows)
    if extra is not None:
        extra(t, o, src, packed, packed_rows)
    del packed_rows
    mask = typemap_mask(o)
    dst = torch.full((count * o.extent,), SENT, dtype=torch.uint8, device=DEV)
    assert dte.unpack(packed, 0, dst, count, t, s) == total
    s.synchronize()
    del packed
    sv = src.view(count, o.extent)
    sent = torch.tensor(SENT, dtype=torch.uint8, device=DEV)
    check_rows(dst, count, o.extent, lambda r0, r1: torch.where(mask[None, :], sv[r0:r1], sent))
    assert dte.dte_device_timeouts() == 0


def test_packed_stream_beyond_4GiB_chunk_kernel():
    # 72 elements of 64 MiB in 1 KiB runs (16-byte words, mean run below the
    # bulk path's): 4.83 GB packed, element offsets up to 4.9 GB.  Also a
    # range window across packed offset 2^32 and the same move as a batch.
    rng = np.random.default_rng(901)
    spec = ("hvector", 65536, 1, 1040, ("contig", 128, ("basic", "float64")))
    count = 72

    def extra(t, o, src, packed, packed_rows):
        assert count * o.size > 1 << 32
        s = torch.cuda.current_stream()
        a, n = (1 << 32) - (1 << 20) - 48, (2 << 20) + 96
        win = torch.full((n,), SENT, dtype=torch.uint8, device=DEV)
        dte.pack_range(src, count, t, a, n, win, s)
        s.synchronize()
        r0, r1 = a // o.size, (a + n - 1) // o.size + 1
        want = packed_rows(r0, r1).reshape(-1)[a - r0 * o.size: a - r0 * o.size + n]
        assert torch.equal(win, want)
        out = torch.full_like(packed, SENT)
        b = dte.Batch(dte.BATCH_PACK, [(t.h, count, src.data_ptr(), out.data_ptr())])
        b.enqueue(s)
        s.synchronize()
        b.free()
        check_rows(out, count, o.size, packed_rows)

    big_round_trip(spec, count, rng, extra)


def test_packed_stream_beyond_4GiB_bulk_kernel():
    # 64 KiB runs in moves of 4.83 GB: the bulk-copy kernels, tile indices
    # past 2^18 and byte offsets past 2^32
    rng = np.random.default_rng(902)
    spec = ("hvector", 1024, 1, 65536 + 4096, ("contig", 8192, ("basic", "float64")))
    big_round_trip(spec, 72, rng)


def test_more_than_2_31_segments_segment_major():
    # 33 one-byte blocks at even offsets (a list of more than 32 entries, so
    # the segment-major kernel with 1-byte words): 65,075,263 elements give
    # 2,147,483,679 segments, 2.15 GB packed and 4.23 GB of element span
    rng = np.random.default_rng(903)
    spec = ("indexed", np.ones(33, np.int64), np.arange(0, 66, 2, dtype=np.int64), ("basic", "byte"))
    count = 65075263
    t, o = both(spec)
    assert o.iov_count() == 33 and count * 33 > (1 << 31)
    big_round_trip(spec, count, rng)


def test_records_beyond_4GiB_record_major():
    # an array of records under an index list of 34 entries (irregular
    # displacements, so it stays a list), each two 4-byte records 8 bytes
    # apart: the record-major kernels with their staged tiles (272 packed
    # bytes per element, a multiple of 16); 15,794,419 elements give 4.3 GB
    # packed and 10.6 GB of element span
    rng = np.random.default_rng(306)
    disp = np.concatenate([[0], np.cumsum(np.where(np.arange(33) % 2, 3, 2))]).astype(np.int64)
    spec = ("indexed", np.full(34, 2, np.int64), disp, ("resized", 0, 8, ("basic", "int32")))
    t, o = both(spec)
    assert (o.size, o.extent) == (272, 672)
    big_round_trip(spec, (1 << 32) // o.size + 4099, rng)
