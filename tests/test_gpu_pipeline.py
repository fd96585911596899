"""GPU parity of the partial (packed-window) moves and of the windowed
send-to-self pipeline (pack -> copy -> unpack per window on one stream),
byte for byte against the oracle's range pack / unpack."""
import numpy as np
import pytest

import inputs
from tests.helpers import both, span_of

torch = pytest.importorskip("torch")
import paper_2402_12274_gb300 as dte  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
SENT = 0xA5


def windows(rng, total, k=5):
    """Random windows: ragged, empty, one byte, the whole stream."""
    out = [(0, total), (0, 0), (total, 0)]
    if total:
        out.append((total - 1, 1))
    for _ in range(k):
        a = int(rng.integers(0, total + 1))
        out.append((a, int(rng.integers(0, total - a + 1))))
    return out


def check_ranges(spec, count, rng):
    t, o = both(spec)
    total = count * o.size
    if total == 0:
        return
    lo, hi = span_of(o, count)
    shift = int(rng.integers(0, 16))
    base = -lo + shift
    span = hi - lo + shift + 1
    src = rng.integers(0, 256, span, dtype=np.uint8)
    d_src = torch.from_numpy(src).to(DEV)
    full = o.pack(src, count, base)
    overl = o.overlaps(count)
    s = torch.cuda.current_stream()
    for a, n in windows(rng, total):
        pk_pos = int(rng.integers(0, 20))
        out = torch.full((pk_pos + n + 16,), SENT, dtype=torch.uint8, device=DEV)
        dte.pack_range(d_src, count, t, a, n, out, s, src_offset=base, dst_offset=pk_pos)
        got = out.cpu().numpy()
        assert np.array_equal(got[pk_pos:pk_pos + n], full[a:a + n]), (spec, a, n)
        assert np.all(got[:pk_pos] == SENT) and np.all(got[pk_pos + n:] == SENT)
        if overl:
            continue
        want = np.full(span, SENT, np.uint8)
        o.unpack_range(full[a:a + n], a, count, want, base)
        buf = np.full(pk_pos + n, SENT, np.uint8)
        buf[pk_pos:] = full[a:a + n]
        d_dst = torch.full((span,), SENT, dtype=torch.uint8, device=DEV)
        dte.unpack_range(torch.from_numpy(buf).to(DEV), a, n, d_dst, count, t, s, src_offset=pk_pos,
                         dst_offset=base)
        assert np.array_equal(d_dst.cpu().numpy(), want), (spec, a, n)


def test_random_nests_range_moves():
    rng = np.random.default_rng(301)
    for i in range(250):
        check_ranges(inputs.random_spec(rng, big=i % 4 == 0), int(rng.integers(1, 4)), rng)


@pytest.mark.parametrize("el,bl,st", [("float64", 2, 6), ("float32", 1, 3), ("bfloat16", 3, 7),
                                      ("byte", 5, 9), ("float32", 64, 80)])
def test_range_moves_each_word_size(el, bl, st):
    # short runs in small words take the segment-major kernel (windows clip
    # its first and last segment); long runs take the chunk-major one
    rng = np.random.default_rng(302)
    for count in (1, 3):
        check_ranges(("vector", 3000, bl, st, ("basic", el)), count, rng)


@pytest.mark.parametrize("el", ["byte", "bfloat16", "float32", "float64"])
def test_range_moves_short_runs_under_index_tables(el):
    # segment-major kernel: windows clip its first and last segment
    rng = np.random.default_rng(307)
    bl = rng.integers(1, 6, 2000)
    disp = np.cumsum(bl + rng.integers(0, 4, 2000)) - bl
    spec = ("indexed", bl.astype(np.int64), disp.astype(np.int64), ("basic", el))
    for count in (1, 2):
        check_ranges(spec, count, rng)


def test_range_moves_long_runs_bulk_copies():
    # 16-byte aligned windows of 66 MiB and more over long runs take the
    # bulk-copy kernels; odd windows fall back to the chunk kernels
    rng = np.random.default_rng(308)
    spec = ("hvector", 1200, 1, 96 << 10, ("contig", 8192, ("basic", "float64")))
    t, o = both(spec)
    total = o.size
    lo, hi = span_of(o, 1)
    src = rng.integers(0, 256, hi, dtype=np.uint8)
    d_src = torch.from_numpy(src).to(DEV)
    full = o.pack(src, 1)
    s = torch.cuda.current_stream()
    big = 66 << 20
    for a, n in ((0, total), (16 * 4097, big), (16 * 12345, total - 16 * 12345 - 16 * 77),
                 (4096, big + 16), (8, big)):
        out = torch.full((n + 16,), SENT, dtype=torch.uint8, device=DEV)
        dte.pack_range(d_src, 1, t, a, n, out, s)
        got = out.cpu().numpy()
        assert np.array_equal(got[:n], full[a:a + n]) and np.all(got[n:] == SENT)
        want = np.full(hi, SENT, np.uint8)
        o.unpack_range(full[a:a + n], a, 1, want)
        d_dst = torch.full((hi,), SENT, dtype=torch.uint8, device=DEV)
        dte.unpack_range(torch.from_numpy(full[a:a + n].copy()).to(DEV), a, n, d_dst, 1, t, s)
        assert np.array_equal(d_dst.cpu().numpy(), want)
    assert dte.dte_device_timeouts() == 0


def sendrecv_case(sspec, rspec, scount, staging_bytes, rng):
    ts, os_ = both(sspec)
    tr, or_ = both(rspec)
    S = scount * os_.size
    rcount = -(-S // or_.size) if or_.size else 0
    if S == 0 or rcount == 0 or or_.overlaps(rcount):
        return False
    slo, shi = span_of(os_, scount)
    rlo, rhi = span_of(or_, rcount)
    src = rng.integers(0, 256, shi - slo + 1, dtype=np.uint8)
    msg = os_.pack(src, scount, -slo)
    want = np.full(rhi - rlo + 1, SENT, np.uint8)
    or_.unpack_range(msg, 0, rcount, want, -rlo)
    d_src = torch.from_numpy(src).to(DEV)
    d_dst = torch.full((rhi - rlo + 1,), SENT, dtype=torch.uint8, device=DEV)
    staging = torch.empty(staging_bytes, dtype=torch.uint8, device=DEV)
    dte.sendrecv(d_src, scount, ts, d_dst, rcount, tr, staging, torch.cuda.current_stream(),
                 send_offset=-slo, recv_offset=-rlo)
    assert np.array_equal(d_dst.cpu().numpy(), want), (sspec, rspec, scount, staging_bytes)
    return True


def test_random_sendrecv_pairs():
    rng = np.random.default_rng(303)
    done = 0
    for i in range(400):
        a = inputs.random_spec(rng, big=i % 5 == 0) if i % 3 else inputs.sequential_spec(rng)
        b = inputs.sequential_spec(rng) if i % 2 else inputs.random_spec(rng, big=i % 7 == 0)
        st = int(rng.choice([32, 48, 100, 1024, 4096, 1 << 20]))
        done += sendrecv_case(a, b, int(rng.integers(1, 4)), st, rng)
    assert done > 150  # pairs with a non-empty message and a non-overlapping receive layout


def test_sendrecv_larger_layout_pairs():
    rng = np.random.default_rng(306)
    rec = inputs.record_indexed_spec(rng, 1 << 12)
    vec = inputs.strided_vector_spec()
    cases = [(rec, ("contig", 1 << 20, ("basic", "byte")), 1),
             (vec, ("subarray", [256, 128], [256, 64], [0, 32], 0, ("basic", "float32")), 1),
             (("contig", 4, vec), vec, 4)]
    for sspec, rspec, sc in cases:
        size = dte.Datatype.from_spec(sspec).size * sc
        for st in (32, 4096, 65536, 1 << 24):
            if size // (st // 2) <= 20000:  # bounded number of windows
                assert sendrecv_case(sspec, rspec, sc, st, rng)


def test_sendrecv_periodic_halo_faces():
    # a periodic halo exchange with oneself: each send face of a 64^3
    # float64 grid lands in the opposite ghost face, through windows much
    # smaller than the message that end on send-side segment boundaries
    rng = np.random.default_rng(304)
    faces = inputs.halo_face_specs(64, 2)
    recv = inputs.halo_recv_face_specs(64, 2)
    for f in range(len(faces)):
        for st in (4096, 65536, 1 << 22):
            assert sendrecv_case(faces[f], recv[f ^ 1], 1, st, rng)


def test_sendrecv_stream_order_and_graph_replay():
    rng = np.random.default_rng(305)
    sspec = ("vector", 4096, 3, 7, ("basic", "float32"))
    rspec = ("subarray", [128, 160], [128, 96], [0, 40], 0, ("basic", "float32"))
    ts, os_ = both(sspec)
    tr, or_ = both(rspec)
    assert os_.size == or_.size
    n = 4096 * 7
    s = torch.cuda.Stream()
    staging = torch.empty(8192, dtype=torch.uint8, device=DEV)
    with torch.cuda.stream(s):
        torch.cuda._sleep(1_000_000)
        x = torch.arange(n, dtype=torch.float32, device=DEV) * 0.25 - 7.0
        y = torch.zeros(128 * 160, dtype=torch.float32, device=DEV)
        dte.sendrecv(x, 1, ts, y, 1, tr, staging, s)
        z = y * 2.0 + 1.0
    s.synchronize()
    xr = (np.arange(n, dtype=np.float32) * 0.25 - 7.0).view(np.uint8)
    yr = np.zeros(128 * 160, np.float32)
    or_.unpack(os_.pack(xr, 1), 1, yr.view(np.uint8))
    assert np.array_equal(z.cpu().numpy(), yr * 2.0 + 1.0)
    # captured once, replayed on new data
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream()
    y.zero_()
    with torch.cuda.graph(g, stream=gs):
        dte.sendrecv(x, 1, ts, y, 1, tr, staging, gs)
    src = rng.standard_normal(n).astype(np.float32)
    x.copy_(torch.from_numpy(src))
    g.replay()
    torch.cuda.synchronize()
    yr = np.zeros(128 * 160, np.float32)
    or_.unpack(os_.pack(src.view(np.uint8), 1), 1, yr.view(np.uint8))
    assert np.array_equal(y.cpu().numpy(), yr)


def test_sendrecv_and_range_errors():
    t, _ = both(("vector", 10, 1, 2, ("basic", "float32")))
    u, _ = both(("contig", 5, ("basic", "float32")))
    ov, _ = both(("vector", 10, 2, 1, ("basic", "float32")))  # writes bytes twice
    x = torch.zeros(64, dtype=torch.float32, device=DEV)
    y = torch.zeros(64, dtype=torch.float32, device=DEV)
    g = torch.empty(64, dtype=torch.uint8, device=DEV)
    with pytest.raises(dte.DteError) as e:  # 40 bytes into 20
        dte.sendrecv(x, 1, t, y, 1, u, g)
    assert e.value.code == dte.ERR_TRUNCATE
    with pytest.raises(dte.DteError) as e:
        dte.sendrecv(x, 1, u, y, 1, ov, g)
    assert e.value.code == dte.ERR_OVERLAP
    with pytest.raises(dte.DteError) as e:
        dte.sendrecv(x, 1, u, y, 1, t, g[:31])
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:
        dte.pack_range(x, 1, t, 30, 11, g)
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:
        dte.unpack_range(g, 0, 8, y, 1, ov)
    assert e.value.code == dte.ERR_OVERLAP
    torch.cuda.synchronize()
