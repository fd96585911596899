"""GPU parity: pack / unpack / segment enumeration through the C ABI on the
device, compared byte for byte (and index for index) with the CPU oracle on
the same seeded inputs.  Source bytes are raw random bytes, so NaN payloads
and every bit pattern must survive verbatim."""
import numpy as np
import pytest

import oracle
import inputs
from tests.helpers import both, span_of

torch = pytest.importorskip("torch")
import paper_2402_12274_gb300 as dte  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
SENT = 0xA5


def gpu_pack(t, src_np, count, base, pk_pos=0, stream=None):
    s = stream or torch.cuda.current_stream()
    d_src = torch.from_numpy(src_np).to(DEV)
    out = torch.full((pk_pos + count * t.size + 16,), SENT, dtype=torch.uint8, device=DEV)
    pos = dte.pack(d_src, count, t, out, pk_pos, s, src_offset=base)
    s.synchronize()
    assert pos == pk_pos + count * t.size
    o = out.cpu().numpy()
    assert np.all(o[:pk_pos] == SENT) and np.all(o[pos:] == SENT), "pack wrote outside its range"
    return o[pk_pos:pos]


def gpu_unpack(t, packed_np, count, span, base, pk_pos=0):
    s = torch.cuda.current_stream()
    buf = np.full(pk_pos + packed_np.size, SENT, np.uint8)
    buf[pk_pos:] = packed_np
    d_pk = torch.from_numpy(buf).to(DEV)
    d_dst = torch.full((span,), SENT, dtype=torch.uint8, device=DEV)
    pos = dte.unpack(d_pk, pk_pos, d_dst, count, t, s, dst_offset=base)
    s.synchronize()
    assert pos == pk_pos + count * t.size
    return d_dst.cpu().numpy()


def check_move(spec, count, rng, misalign=True):
    t, o = both(spec)
    if o.size == 0:
        return
    lo, hi = span_of(o, count)
    shift = int(rng.integers(0, 16)) if misalign else 0
    base = -lo + shift
    span = hi - lo + shift + 1
    src = rng.integers(0, 256, span, dtype=np.uint8)
    ref = o.pack(src, count, base)
    pk_pos = int(rng.integers(0, 20)) if misalign else 0
    got = gpu_pack(t, src, count, base, pk_pos)
    assert np.array_equal(got, ref), spec
    if o.overlaps(count):
        with pytest.raises(dte.DteError) as e:
            gpu_unpack(t, ref, count, span, base, pk_pos)
        assert e.value.code == dte.ERR_OVERLAP
        return
    want = np.full(span, SENT, np.uint8)
    o.unpack(ref, count, want, base)
    got = gpu_unpack(t, ref, count, span, base, pk_pos)
    assert np.array_equal(got, want), spec


def test_random_nests_pack_unpack():
    rng = np.random.default_rng(201)
    for i in range(600):
        check_move(inputs.random_spec(rng, big=i % 3 == 0), int(rng.integers(1, 4)), rng)


def test_merging_layouts_pack_unpack():
    rng = np.random.default_rng(202)
    for _ in range(200):
        check_move(inputs.sequential_spec(rng), int(rng.integers(1, 4)), rng)


BULK_MOVE = 72 << 20  # well above the size that gives every warp of the bulk grid six tiles


@pytest.mark.parametrize("L", [2048, 4096 + 16, 65536, 1 << 20])
def test_long_runs_take_bulk_copies(L):
    # runs of L bytes (16-byte multiples, 16-byte aligned buffers) in moves of
    # BULK_MOVE bytes and more go through the bulk-copy kernels, ragged tile
    # at the end included; no bounded wait gives up
    rng = np.random.default_rng(210)
    n = BULK_MOVE // L + 3
    spec = ("hvector", n, 1, L + 768, ("contig", L // 8, ("basic", "float64")))
    check_move(spec, 1, rng, misalign=False)
    if L == 65536:
        half = ("hvector", n // 2 + 1, 1, L + 768, ("contig", L // 8, ("basic", "float64")))
        check_move(half, 2, rng, misalign=False)
    # a struct of long and short runs still averages long runs per segment
    spec = ("struct", [1, 1], [0, BULK_MOVE + (8 << 20)],
            [("contig", BULK_MOVE // 8, ("basic", "float64")), ("vector", 64, 2, 4, ("basic", "float64"))])
    check_move(spec, 1, rng, misalign=False)
    assert dte.dte_device_timeouts() == 0


def test_long_runs_from_pinned_host_memory():
    # host buffers take the chunk kernels (bulk copies only run between
    # device buffers); results as from device memory
    rng = np.random.default_rng(211)
    spec = ("hvector", 48, 1, 64 << 10, ("contig", 4096, ("basic", "float64")))
    t, o = both(spec)
    lo, hi = span_of(o, 1)
    src = rng.integers(0, 256, hi, dtype=np.uint8)
    h_src = torch.from_numpy(src).pin_memory()
    h_pk = torch.full((o.size,), SENT, dtype=torch.uint8).pin_memory()
    s = torch.cuda.current_stream()
    dte.pack(h_src, 1, t, h_pk, 0, s)
    s.synchronize()
    assert np.array_equal(h_pk.numpy(), o.pack(src, 1))
    h_dst = torch.full((hi,), SENT, dtype=torch.uint8).pin_memory()
    dte.unpack(h_pk, 0, h_dst, 1, t, s)
    s.synchronize()
    want = np.full(hi, SENT, np.uint8)
    o.unpack(o.pack(src, 1), 1, want)
    assert np.array_equal(h_dst.numpy(), want)


@pytest.mark.parametrize("el", ["byte", "int16", "float32", "float64"])
def test_short_runs_under_index_tables(el):
    # indexed lists longer than 32 entries with short blocks take the
    # segment-major kernel (one word class per element size)
    rng = np.random.default_rng(205)
    for n in (33, 200, 3000):
        bl = rng.integers(1, 6, n)
        disp = np.cumsum(bl + rng.integers(0, 4, n)) - bl
        spec = ("indexed", bl.astype(np.int64), disp.astype(np.int64), ("basic", el))
        for count in (1, 3):
            check_move(spec, count, rng, misalign=False)
            check_move(spec, count, rng)


def test_darray_pack_unpack():
    rng = np.random.default_rng(204)
    for _ in range(200):
        check_move(inputs.random_darray_spec(rng), int(rng.integers(1, 4)), rng)
    # a 3-D block-cyclic distribution big enough to span many tiles
    spec = ("darray", 8, 5, [96, 80, 72], [0, 1, 1], [-1, 2, 3], [2, 2, 2], 0, ("basic", "float64"))
    check_move(spec, 1, rng)
    check_move(spec[:7] + (1,) + spec[8:], 2, rng)


def test_aligned_word_sizes():
    # runs whose lengths and offsets allow 16/8/4/2/1-byte words
    rng = np.random.default_rng(203)
    for el, bl, st in [("float64", 2, 6), ("float64", 1, 3), ("float32", 1, 3), ("float32", 4, 16),
                       ("bfloat16", 3, 7), ("byte", 5, 9), ("int16", 8, 8)]:
        for count in (1, 2, 7):
            for mis in (False, True):
                check_move(("vector", 37, bl, st, ("basic", el)), count, rng, misalign=mis)


def iov_check(t, o, count, first, n):
    d_iov = torch.zeros((max(n, 1), 2), dtype=torch.int64, device=DEV)
    d_act = torch.full((1,), -7, dtype=torch.int64, device=DEV)
    base = 1 << 40
    dte.dte_type_iov_async(t.h, count, first, d_iov.data_ptr(), n, d_act.data_ptr(), base,
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    od, ol = o.iov_elements(count, first, n)
    got = d_iov.cpu().numpy()[: len(od)]
    assert int(d_act.item()) == len(od)
    assert np.array_equal(got[:, 0] - base, od) and np.array_equal(got[:, 1], ol)


def test_random_nests_iov_device():
    rng = np.random.default_rng(204)
    for i in range(300):
        spec = inputs.random_spec(rng) if i % 2 else inputs.sequential_spec(rng)
        t, o = both(spec)
        count = int(rng.integers(1, 4))
        total = count * o.iov_count()
        for first in (0, total // 2):
            iov_check(t, o, count, first, total + 3)


def test_iov_len_and_at_bytes_device():
    rng = np.random.default_rng(205)
    s = torch.cuda.current_stream().cuda_stream
    for i in range(200):
        spec = inputs.random_spec(rng, big=True) if i % 2 else inputs.sequential_spec(rng)
        t, o = both(spec)
        if o.size == 0:
            continue
        budgets = np.unique(np.concatenate([rng.integers(-3, o.size + 4, 64), [-1, 0, o.size]])).astype(np.int64)
        d_b = torch.from_numpy(budgets).to(DEV)
        d_n = torch.empty_like(d_b)
        d_y = torch.empty_like(d_b)
        dte.dte_type_iov_len_async(t.h, budgets.size, d_b.data_ptr(), d_n.data_ptr(), d_y.data_ptr(), s)
        torch.cuda.synchronize()
        for b, n, y in zip(budgets, d_n.cpu().numpy(), d_y.cpu().numpy()):
            if b < -1:
                assert (n, y) == (-1, -1)
            else:
                assert (n, y) == o.iov_len(int(b)), (spec, b)
        # byte offset -> the segment containing it, and the next segments
        offs = rng.integers(-2, o.size + 2, 40).astype(np.int64)
        m = 3
        d_o = torch.from_numpy(offs).to(DEV)
        d_iov = torch.zeros((offs.size * m, 2), dtype=torch.int64, device=DEV)
        d_f = torch.empty_like(d_o)
        d_a = torch.empty_like(d_o)
        dte.dte_type_iov_at_bytes_async(t.h, offs.size, d_o.data_ptr(), m, d_iov.data_ptr(), d_f.data_ptr(),
                                        d_a.data_ptr(), 0, s)
        torch.cuda.synchronize()
        f, a, iv = d_f.cpu().numpy(), d_a.cpu().numpy(), d_iov.cpu().numpy()
        sd, sl = o.iov()
        for q, b in enumerate(offs):
            if b < 0 or b >= o.size:
                assert (f[q], a[q]) == (-1, 0)
                continue
            k = o.iov_len(int(b))[0]
            assert f[q] == k and a[q] == min(m, len(sd) - k)
            got = iv[q * m: q * m + a[q]]
            assert np.array_equal(got[:, 0], sd[k:k + a[q]]) and np.array_equal(got[:, 1], sl[k:k + a[q]])


def test_record_block_gather_layouts():
    # arrays of records whose starts are all one offset modulo 16 (record
    # extents and byte displacements multiples of 16), user buffers shifted
    # by 0-15 bytes against aligned packed buffers: the record-major kernels
    # with their staged tiles at every copy word, pack and unpack
    rng = np.random.default_rng(208)
    for _ in range(60):
        kind, lens, disp, rec = inputs.record_variety_spec(rng, int(rng.choice([40, 700, 3000])))
        ext = oracle.from_spec(rec).extent
        e16 = -(-ext // 16) * 16 + 16 * int(rng.integers(0, 2))
        rec16 = ("resized", 0, e16, rec)
        units = np.cumsum(np.concatenate([[0], lens[:-1] + 1]))  # one-record gaps keep blocks apart
        spec = ("indexed", lens, units.astype(np.int64), rec16) if kind == "indexed" else \
            ("hindexed", lens, (units * e16).astype(np.int64), rec16)
        t, o = both(spec)
        count = int(rng.integers(1, 4))
        lo, hi = span_of(o, count)
        for shift in (0, int(rng.integers(1, 16))):
            base = -lo + shift
            span = hi - lo + shift + 1
            src = rng.integers(0, 256, span, dtype=np.uint8)
            ref = o.pack(src, count, base)
            assert np.array_equal(gpu_pack(t, src, count, base, 0), ref), (spec, count, shift)
            want = np.full(span, SENT, np.uint8)
            o.unpack(ref, count, want, base)
            assert np.array_equal(gpu_unpack(t, ref, count, span, base, 0), want), (spec, count, shift)


def test_list_iov_device_rounds():
    # large index lists over one shared child (arrays of records): the iov
    # kernels decode rounds of 32 records by the warp together and write each
    # record's runs, and map byte offsets and budgets to segments directly;
    # requests and queries that start or end inside a record, windows across
    # elements, 37, 64 and 4096 segments per query, and offsets and budgets
    # outside the type
    rng = np.random.default_rng(207)
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(40):
        spec = inputs.record_variety_spec(rng, int(rng.choice([33, 300, 2000])))
        t, o = both(spec)
        count = int(rng.integers(1, 4))
        total = count * o.iov_count()
        first = int(rng.integers(0, max(1, total // 3)))
        iov_check(t, o, count, first, int(rng.integers(1, total - first + 5)))
        sd, sl = o.iov()
        budgets = np.unique(np.concatenate([rng.integers(-3, o.size + 4, 48), [-1, 0, o.size]])).astype(np.int64)
        d_b = torch.from_numpy(budgets).to(DEV)
        d_n = torch.empty_like(d_b)
        d_y = torch.empty_like(d_b)
        dte.dte_type_iov_len_async(t.h, budgets.size, d_b.data_ptr(), d_n.data_ptr(), d_y.data_ptr(), s)
        torch.cuda.synchronize()
        for b, nn, y in zip(budgets, d_n.cpu().numpy(), d_y.cpu().numpy()):
            assert (nn, y) == ((-1, -1) if b < -1 else o.iov_len(int(b))), (spec, b)
        offs = np.concatenate([rng.integers(0, o.size, 24), [-1, o.size]]).astype(np.int64)
        for m in (37, 64, 4096):
            d_o = torch.from_numpy(offs).to(DEV)
            d_iov = torch.zeros((offs.size * m, 2), dtype=torch.int64, device=DEV)
            d_f = torch.empty_like(d_o)
            d_a = torch.empty_like(d_o)
            dte.dte_type_iov_at_bytes_async(t.h, offs.size, d_o.data_ptr(), m, d_iov.data_ptr(), d_f.data_ptr(),
                                            d_a.data_ptr(), 0, s)
            torch.cuda.synchronize()
            f, a, iv = d_f.cpu().numpy(), d_a.cpu().numpy(), d_iov.cpu().numpy()
            for q, b in enumerate(offs):
                if b < 0 or b >= o.size:
                    assert (f[q], a[q]) == (-1, 0)
                    continue
                k = o.iov_len(int(b))[0]
                assert f[q] == k and a[q] == min(m, len(sd) - k)
                got = iv[q * m: q * m + a[q]]
                assert np.array_equal(got[:, 0], sd[k:k + a[q]]) and np.array_equal(got[:, 1], sl[k:k + a[q]])


# --------------------------------------------------------------------------
# workload layouts
# --------------------------------------------------------------------------
def test_strided_vector_workload():
    # vector(1024, 4, 16) of float32, 64 elements, values U[-1,1) seed 1
    spec = inputs.strided_vector_spec()
    t, o = both(spec)
    count = 64
    lo, hi = span_of(o, count)
    src = inputs.uniform_f32(hi // 4, 1).view(np.uint8)
    ref = o.pack(src, count)
    assert ref.size == 1 << 20
    got = gpu_pack(t, src, count, 0)
    assert np.array_equal(got, ref)
    want = np.full(hi, SENT, np.uint8)
    o.unpack(ref, count, want)
    assert np.array_equal(gpu_unpack(t, ref, count, hi, 0), want)
    iov_check(t, o, count, 0, count * 1024)
    d = torch.empty((count * 1024, 2), dtype=torch.int64, device=DEV)
    dte.dte_type_iov_async(t.h, count, 0, d.data_ptr(), count * 1024, 0, 0, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.all(d[:, 1].cpu().numpy() == 16)


@pytest.mark.parametrize("n", [16, 64])
def test_halo_faces_small(n):
    check_halo(n)


def check_halo(n, g=2):
    """Pack the six send faces (one struct, one launch) and unpack them into
    the same six faces of a second grid.  The faces share edge cells, so as
    one layout they overlap (rejected for unpack); as a batch of six per-face
    unpacks each op is valid and shared cells receive identical bytes."""
    send = inputs.all_faces_struct(inputs.halo_face_specs(n, g))
    recv_faces = inputs.halo_face_specs(n, g)
    ts, os_ = both(send)
    tr, or_ = both(inputs.all_faces_struct(recv_faces))
    grid = inputs.normal_f64(n ** 3, 2).view(np.uint8)
    ref = os_.pack(grid, 1)
    d_grid = torch.from_numpy(grid).to(DEV)
    d_pk = torch.empty(ts.size, dtype=torch.uint8, device=DEV)
    s = torch.cuda.current_stream()
    dte.pack(d_grid, 1, ts, d_pk, 0, s)
    d_g2 = torch.full((grid.size,), SENT, dtype=torch.uint8, device=DEV)
    with pytest.raises(dte.DteError) as e:
        dte.unpack(d_pk, 0, d_g2, 1, tr, s)
    assert e.value.code == dte.ERR_OVERLAP
    faces = [dte.Datatype.from_spec(f).commit() for f in recv_faces]
    ops, pos = [], 0
    for f in faces:
        ops.append((f.h, 1, d_g2.data_ptr(), d_pk.data_ptr() + pos))
        pos += f.size
    dte.dte_unpack_batch_enqueue(ops, s.cuda_stream)
    s.synchronize()
    assert np.array_equal(d_pk.cpu().numpy(), ref)
    want = np.full(grid.size, SENT, np.uint8)
    pos = 0
    for spec in recv_faces:
        of = oracle.from_spec(spec)
        of.unpack(ref[pos:pos + of.size], 1, want)
        pos += of.size
    assert np.array_equal(d_g2.cpu().numpy(), want)


@pytest.mark.slow
def test_halo_faces_full_size():
    check_halo(512)


@pytest.mark.parametrize("nblocks", [1 << 12, 1 << 16, 1 << 19])
def test_record_indexed_workload(nblocks):
    check_record_indexed(nblocks)


@pytest.mark.slow
def test_record_indexed_full_size():
    check_record_indexed(1 << 22)


def test_record_major_layouts():
    # arrays of records under index lists of more than 32 entries move one
    # whole record per lane (record-major): random records of 1-6 blocks and
    # single resized blocks, every copy word, 1-3 elements, aligned buffers
    # (the packed side of a round staged in shared memory where the record is
    # not a multiple of 16 bytes) and misaligned ones (not staged)
    rng = np.random.default_rng(206)
    for _ in range(150):
        spec = inputs.record_variety_spec(rng, int(rng.choice([33, 100, 1000, 5000])))
        count = int(rng.integers(1, 4))
        check_move(spec, count, rng, misalign=False)
        check_move(spec, count, rng)


def check_record_indexed(nblocks):
    rng = np.random.default_rng(3)
    spec = inputs.record_indexed_spec(rng, nblocks)
    t, o = both(spec)
    span = o.true_lb + o.true_extent
    src = inputs.random_bytes(span, 3)
    ref = o.pack(src, 1)
    got = gpu_pack(t, src, 1, 0)
    assert np.array_equal(got, ref)
    want = np.full(span, SENT, np.uint8)
    o.unpack(ref, 1, want)
    assert np.array_equal(gpu_unpack(t, ref, 1, span, 0), want)
    if nblocks <= 1 << 16:
        # the whole segment list, and a window starting inside a record
        nseg = o.iov_count()
        iov_check(t, o, 1, 0, nseg)
        iov_check(t, o, 1, nseg // 3 + 1, nseg // 2)
    # iov queried in chunks of 4096 from random packed byte offsets (each
    # oracle query re-walks the whole type, so fewer at full size)
    nq = 64 if nblocks <= 1 << 16 else 6
    offs = np.sort(rng.integers(0, o.size, nq)).astype(np.int64)
    m = 4096
    d_o = torch.from_numpy(offs).to(DEV)
    d_iov = torch.zeros((offs.size * m, 2), dtype=torch.int64, device=DEV)
    d_f = torch.empty_like(d_o)
    d_a = torch.empty_like(d_o)
    dte.dte_type_iov_at_bytes_async(t.h, offs.size, d_o.data_ptr(), m, d_iov.data_ptr(), d_f.data_ptr(),
                                    d_a.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    f, a, iv = d_f.cpu().numpy(), d_a.cpu().numpy(), d_iov.cpu().numpy()
    for q, b in enumerate(offs):
        e, r = divmod(int(b), 52)          # closed form of the record layout
        k = 2 * e + (r >= 12)
        assert f[q] == k
        od, ol = o.iov(k, m)
        assert a[q] == len(od)
        got = iv[q * m: q * m + a[q]]
        assert np.array_equal(got[:, 0], od) and np.array_equal(got[:, 1], ol)


# --------------------------------------------------------------------------
# stream semantics, lifetime and errors
# --------------------------------------------------------------------------
def test_stream_ordered_pipeline_without_host_sync():
    # produce -> pack -> unpack -> consume on one non-default stream
    spec = ("vector", 4096, 3, 7, ("basic", "float32"))
    t, o = both(spec)
    s = torch.cuda.Stream()
    n = 4096 * 7
    with torch.cuda.stream(s):
        x = torch.arange(n, dtype=torch.float32, device=DEV) * 0.5 - 3.0
        pk = torch.empty(t.size, dtype=torch.uint8, device=DEV)
        dte.pack(x, 1, t, pk, 0, s)
        y = torch.zeros(n, dtype=torch.float32, device=DEV)
        dte.unpack(pk, 0, y, 1, t, s)
        z = y * 2.0 + 1.0
    s.synchronize()
    xr = (np.arange(n, dtype=np.float32) * 0.5 - 3.0)
    yr = np.zeros(n, np.float32).view(np.uint8)
    o.unpack(o.pack(xr.view(np.uint8), 1), 1, yr)
    assert np.array_equal(z.cpu().numpy(), yr.view(np.float32) * 2.0 + 1.0)


def test_free_while_enqueued_keeps_descriptor():
    rng = np.random.default_rng(206)
    spec = inputs.record_indexed_spec(rng, 1 << 15)
    t, o = both(spec)
    span = o.true_lb + o.true_extent
    src = inputs.random_bytes(span, 4)
    d_src = torch.from_numpy(src).to(DEV)
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        torch.cuda._sleep(2_000_000)  # keep the stream busy so the packs are still queued
        for _ in range(3):
            pk = torch.empty(t.size, dtype=torch.uint8, device=DEV)
            dte.pack(d_src, 1, t, pk, 0, s)
            outs.append(pk)
    del t  # free the handle while its kernels are queued
    s.synchronize()
    ref = o.pack(src, 1)
    for pk in outs:
        assert np.array_equal(pk.cpu().numpy(), ref)


def test_enqueue_errors():
    t = dte.Datatype.vector(4, 1, 2, dte.FLOAT32)
    buf = torch.zeros(64, dtype=torch.uint8, device=DEV)
    with pytest.raises(dte.DteError) as e:
        dte.pack(buf, 1, t, buf, 0)
    assert e.value.code == dte.ERR_TYPE  # not committed
    t.commit()
    small = torch.zeros(15, dtype=torch.uint8, device=DEV)
    with pytest.raises(dte.DteError) as e:
        dte.pack(buf, 1, t, small, 0)
    assert e.value.code == dte.ERR_TRUNCATE
    with pytest.raises(dte.DteError) as e:
        dte.pack(buf, 1, t, buf, 60)
    assert e.value.code == dte.ERR_TRUNCATE
    ov = dte.Datatype.vector(4, 3, 2, dte.FLOAT32).commit()
    with pytest.raises(dte.DteError) as e:
        dte.unpack(buf, 0, buf, 1, ov)
    assert e.value.code == dte.ERR_OVERLAP
    assert dte.pack(buf, 0, t, small, 0) == 0  # empty op: nothing enqueued
    with pytest.raises(dte.DteError) as e:
        dte.dte_pack_enqueue(0, 1, t.h, buf.data_ptr(), 64, 0, 0)
    assert e.value.code == dte.ERR_ARG


# --------------------------------------------------------------------------
# batches (one persistent launch) and CUDA graph capture
# --------------------------------------------------------------------------
def make_batch_case(rng, nops, kind):
    specs = [inputs.random_spec(rng, big=True) if i % 3 else inputs.sequential_spec(rng) for i in range(nops)]
    cases = []
    for spec in specs:
        t, o = both(spec)
        count = int(rng.integers(1, 3))
        if o.size == 0 or (kind == dte.BATCH_UNPACK and o.overlaps(count)):
            continue
        lo, hi = span_of(o, count)
        shift = int(rng.integers(0, 16))
        cases.append(dict(t=t, o=o, count=count, base=-lo + shift, span=hi - lo + shift + 1))
    return cases


@pytest.mark.parametrize("kind", [1, 0])
def test_batch_matches_oracle_and_per_call(kind):
    rng = np.random.default_rng(301 + kind)
    cases = make_batch_case(rng, 120, kind)
    s = torch.cuda.current_stream()
    ops, outs, refs = [], [], []
    pk_total = sum(c["count"] * c["o"].size + 16 for c in cases)
    d_pk = torch.full((pk_total,), SENT, dtype=torch.uint8, device=DEV)
    pos = 0
    for c in cases:
        src = rng.integers(0, 256, c["span"], dtype=np.uint8)
        c["src"] = src
        ref = c["o"].pack(src, c["count"], c["base"])
        if kind == dte.BATCH_PACK:
            d_src = torch.from_numpy(src).to(DEV)
            outs.append(d_src)
            ops.append((c["t"].h, c["count"], d_src.data_ptr() + c["base"], d_pk.data_ptr() + pos))
            refs.append((pos, ref))
        else:
            d_pk[pos:pos + ref.size] = torch.from_numpy(ref).to(DEV)
            d_dst = torch.full((c["span"],), SENT, dtype=torch.uint8, device=DEV)
            outs.append(d_dst)
            ops.append((c["t"].h, c["count"], d_dst.data_ptr() + c["base"], d_pk.data_ptr() + pos))
            want = np.full(c["span"], SENT, np.uint8)
            c["o"].unpack(ref, c["count"], want, c["base"])
            refs.append(want)
        pos += ref.size + int(rng.integers(0, 17))
    b = dte.Batch(kind, ops)
    b.enqueue(s)
    s.synchronize()
    if kind == dte.BATCH_PACK:
        got = d_pk.cpu().numpy()
        for p, ref in refs:
            assert np.array_equal(got[p:p + ref.size], ref)
    else:
        for d_dst, want in zip(outs, refs):
            assert np.array_equal(d_dst.cpu().numpy(), want)
    # replay the same batch under a CUDA graph: identical bytes
    if kind == dte.BATCH_PACK:
        d_pk.fill_(SENT)
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=gs):
            b.enqueue(gs)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        got = d_pk.cpu().numpy()
        for p, ref in refs:
            assert np.array_equal(got[p:p + ref.size], ref)
    b.free()


def test_batch_rejects_bad_ops():
    t = dte.Datatype.vector(4, 3, 2, dte.FLOAT32).commit()  # overlapping
    buf = torch.zeros(256, dtype=torch.uint8, device=DEV)
    with pytest.raises(dte.DteError) as e:
        dte.dte_batch_create(dte.BATCH_UNPACK, [(t.h, 1, buf.data_ptr(), buf.data_ptr())])
    assert e.value.code == dte.ERR_OVERLAP
    u = dte.Datatype.vector(4, 1, 2, dte.FLOAT32)
    with pytest.raises(dte.DteError) as e:
        dte.dte_batch_create(dte.BATCH_PACK, [(u.h, 1, buf.data_ptr(), buf.data_ptr())])
    assert e.value.code == dte.ERR_TYPE
    with pytest.raises(dte.DteError):
        dte.dte_batch_create(7, [])
    b = dte.Batch(dte.BATCH_PACK, [])  # empty batch: enqueue is a no-op
    b.enqueue()
    b.free()


def test_per_call_enqueue_under_graph_capture():
    spec = ("vector", 1000, 2, 5, ("basic", "float64"))
    t, o = both(spec)
    span = o.true_lb + o.true_extent
    src = inputs.random_bytes(span, 9)
    d_src = torch.from_numpy(src).to(DEV)
    d_pk = torch.empty(t.size, dtype=torch.uint8, device=DEV)
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=gs):
        dte.pack(d_src, 1, t, d_pk, 0, gs)
    d_pk.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(d_pk.cpu().numpy(), o.pack(src, 1))


@pytest.fixture(scope="module")
def full_batch():
    """The 10^4-op pack batch of the batch benchmark (same generator and
    seed, 3.9 GB packed out of 6.5 GB of sources): committed types, device
    sources, and the expected packed arena computed by the oracle for every
    op (sentinel bytes in the gaps between ops), built once per module."""
    rng = np.random.default_rng(4)
    specs = inputs.batch_specs(rng, 10_000)
    types = [dte.Datatype.from_spec(sp).commit() for sp, _ in specs]
    spans = [t.true_lb + t.true_extent for t in types]
    sizes = [t.size for t in types]
    up = lambda v: (v + 255) // 256 * 256  # noqa: E731
    so = np.concatenate([[0], np.cumsum([up(v) for v in spans])])
    po = np.concatenate([[0], np.cumsum([up(v) for v in sizes])])
    gen = torch.Generator(device=DEV)
    gen.manual_seed(44)
    src = torch.randint(0, 256, (int(so[-1]),), dtype=torch.uint8, device=DEV, generator=gen)
    h_src = src.cpu().numpy()
    want = np.full(int(po[-1]), SENT, np.uint8)
    for i, (sp, _) in enumerate(specs):
        o = oracle.from_spec(sp)
        assert o.size == sizes[i]
        want[int(po[i]):int(po[i]) + sizes[i]] = o.pack(h_src[int(so[i]):int(so[i]) + spans[i]], 1)
    del h_src
    d_want = torch.from_numpy(want).to(DEV)
    del want
    yield types, so, po, src, d_want
    del d_want, src


@pytest.mark.slow
@pytest.mark.parametrize("launch", [(0, 1), (0, 8), (3, 4)])
def test_full_size_batch_against_oracle(full_batch, launch):
    # every byte of every one of the 10^4 ops, and every gap between them,
    # equals the oracle's arena, in several launch shapes
    types, so, po, src, d_want = full_batch
    pk = torch.full((int(po[-1]),), SENT, dtype=torch.uint8, device=DEV)
    b = dte.Batch(dte.BATCH_PACK, [(t.h, 1, src.data_ptr() + int(a), pk.data_ptr() + int(c))
                                   for t, a, c in zip(types, so, po)])
    b.set_launch(*launch)
    b.enqueue(torch.cuda.current_stream())
    torch.cuda.synchronize()
    if not torch.equal(pk, d_want):
        bad = (pk != d_want).nonzero()[:1]
        i = int(np.searchsorted(po, int(bad[0]), side="right")) - 1
        pytest.fail(f"byte {int(bad[0])} differs from the oracle (op {i})")
    b.free()
    del pk
