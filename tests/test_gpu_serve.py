"""The device-resident request loop: requests of mixed sizes and directions
that arrive while others run are admitted and batched continuously; each
result must be byte-identical whether the request ran alone or in the mix,
and identical to the oracle's pack or unpack of the same seeded bytes (into
a sentinel-filled destination for unpacks).  Also: admission under a small
byte cap, leaving when idle and relaunching, and argument errors."""
import time

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
import paper_2402_12274_gb300 as dte  # noqa: E402

pytestmark = pytest.mark.gpu
SENT = 0x6B


def make_requests(rng, n, lo=1 << 10, hi=1 << 20):
    specs = inputs.batch_specs(rng, n, lo=lo, hi=hi)
    reqs = []
    for spec, _ in specs:
        t = dte.Datatype.from_spec(spec).commit()
        kind = dte.BATCH_PACK if rng.random() < 0.5 else dte.BATCH_UNPACK
        span = t.true_lb + t.true_extent
        user = rng.integers(0, 256, span, dtype=np.uint8)
        packed = rng.integers(0, 256, t.size, dtype=np.uint8)
        reqs.append(dict(t=t, kind=kind, user=user, packed=packed, spec=spec))
    return reqs


def buffers(reqs):
    bufs = []
    for r in reqs:
        if r["kind"] == dte.BATCH_PACK:
            u = torch.from_numpy(r["user"]).cuda()
            p = torch.full((r["t"].size,), SENT, dtype=torch.uint8, device="cuda")
        else:
            u = torch.full((r["user"].size,), SENT, dtype=torch.uint8, device="cuda")
            p = torch.from_numpy(r["packed"]).cuda()
        bufs.append((u, p))
    torch.cuda.synchronize()
    return bufs


def outputs(reqs, bufs):
    torch.cuda.synchronize()
    return [(p if r["kind"] == dte.BATCH_PACK else u).cpu().numpy() for r, (u, p) in zip(reqs, bufs)]


def reference(reqs):
    """Expected output of every request from the oracle: the packed bytes of
    a pack, the sentinel-filled user span after an unpack."""
    out = []
    for r in reqs:
        o = oracle.from_spec(r["spec"])
        assert o.size == r["t"].size
        if r["kind"] == dte.BATCH_PACK:
            out.append(o.pack(r["user"], 1))
        else:
            want = np.full(r["user"].size, SENT, np.uint8)
            o.unpack(r["packed"], 1, want)
            out.append(want)
    return out


def test_results_identical_alone_and_in_the_mix():
    rng = np.random.default_rng(601)
    reqs = make_requests(rng, 80)
    reqs += make_requests(rng, 4, lo=8 << 20, hi=16 << 20)
    ref = reference(reqs)
    srv = dte.dte_server_create()
    try:
        # alone: one request at a time
        bufs = buffers(reqs)
        for r, (u, p) in zip(reqs, bufs):
            tk = dte.dte_server_submit(srv, r["kind"], r["t"].h, 1, u.data_ptr(), p.data_ptr())
            dte.dte_server_wait(srv, tk)
        alone = outputs(reqs, bufs)
        # mixed: everything submitted back to back, with a few short pauses
        bufs = buffers(reqs)
        tickets = []
        for i, (r, (u, p)) in enumerate(zip(reqs, bufs)):
            tickets.append(dte.dte_server_submit(srv, r["kind"], r["t"].h, 1, u.data_ptr(), p.data_ptr()))
            if i % 17 == 0:
                time.sleep(0.0005)
        for tk in tickets:
            dte.dte_server_wait(srv, tk)
        mixed = outputs(reqs, bufs)
    finally:
        dte.dte_server_free(srv)
    for a, b, c in zip(ref, alone, mixed):
        assert np.array_equal(a, b)
        assert np.array_equal(a, c)
    assert dte.dte_device_timeouts() == 0


def test_admission_under_a_small_byte_cap():
    rng = np.random.default_rng(602)
    reqs = make_requests(rng, 40, lo=16 << 10, hi=64 << 10)
    ref = reference(reqs)
    srv = dte.dte_server_create(ring_slots=4, max_inflight_bytes=96 << 10)
    try:
        bufs = buffers(reqs)
        tickets = [dte.dte_server_submit(srv, r["kind"], r["t"].h, 1, u.data_ptr(), p.data_ptr())
                   for r, (u, p) in zip(reqs, bufs)]
        inflight, queued = dte.dte_server_progress(srv)
        assert inflight <= 4 and inflight + queued <= len(reqs)
        assert queued > 0  # the cap held most requests back on the host
        for tk in tickets:
            dte.dte_server_wait(srv, tk)
        assert dte.dte_server_progress(srv) == (0, 0)
        got = outputs(reqs, bufs)
    finally:
        dte.dte_server_free(srv)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_leaves_when_idle_and_relaunches():
    rng = np.random.default_rng(603)
    reqs = make_requests(rng, 6)
    ref = reference(reqs)
    srv = dte.dte_server_create(idle_exit_us=2000)
    try:
        bufs = buffers(reqs)
        for i, (r, (u, p)) in enumerate(zip(reqs, bufs)):
            tk = dte.dte_server_submit(srv, r["kind"], r["t"].h, 1, u.data_ptr(), p.data_ptr())
            dte.dte_server_wait(srv, tk)
            time.sleep(0.05)  # long enough for the loop to leave
        got = outputs(reqs, bufs)
    finally:
        dte.dte_server_free(srv)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_server_argument_errors():
    with pytest.raises(dte.DteError) as e:
        dte.dte_server_create(ring_slots=3)
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:
        dte.dte_server_create(span_tiles=1 << 17)
    assert e.value.code == dte.ERR_ARG
    srv = dte.dte_server_create()
    try:
        ov = dte.Datatype.vector(4, 3, 2, dte.FLOAT32).commit()
        buf = torch.zeros(256, dtype=torch.uint8, device="cuda")
        with pytest.raises(dte.DteError) as e:
            dte.dte_server_submit(srv, dte.BATCH_UNPACK, ov.h, 1, buf.data_ptr(), buf.data_ptr())
        assert e.value.code == dte.ERR_OVERLAP
        with pytest.raises(dte.DteError) as e:
            dte.dte_server_submit(srv, 5, ov.h, 1, buf.data_ptr(), buf.data_ptr())
        assert e.value.code == dte.ERR_ARG
        with pytest.raises(dte.DteError):
            dte.dte_server_wait(srv, 99)
        # an empty request completes too
        tk = dte.dte_server_submit(srv, dte.BATCH_PACK, ov.h, 0, 0, 0)
        dte.dte_server_wait(srv, tk, 2_000_000)
    finally:
        dte.dte_server_free(srv)


def test_over_claims_carried_across_relaunches():
    """Warps racing for a group's last tiles claim past its published end and
    keep those positions for the group's next requests, across the loop's
    exits and relaunches: small requests of one kernel variant with pauses
    longer than the idle exit between them, claims of up to 64 tiles, then
    the other direction and a burst of both."""
    rng = np.random.default_rng(604)
    spec = ("vector", 4096, 4, 8, ("basic", "float32"))  # 64 KiB packed: 64 tiles
    t = dte.Datatype.from_spec(spec).commit()
    o = oracle.from_spec(spec)
    reqs = []
    for i in range(24):
        kind = dte.BATCH_PACK if i < 10 or (i >= 16 and i % 2) else dte.BATCH_UNPACK
        span = t.true_lb + t.true_extent
        reqs.append(dict(t=t, kind=kind, spec=spec, user=rng.integers(0, 256, span, dtype=np.uint8),
                         packed=rng.integers(0, 256, t.size, dtype=np.uint8)))
    assert o.size == t.size
    ref = reference(reqs)
    srv = dte.dte_server_create(idle_exit_us=1000, span_tiles=64)
    try:
        bufs = buffers(reqs)
        tickets = []
        for i, (r, (u, p)) in enumerate(zip(reqs, bufs)):
            tickets.append(dte.dte_server_submit(srv, r["kind"], r["t"].h, 1, u.data_ptr(), p.data_ptr()))
            if i < 16:
                dte.dte_server_wait(srv, tickets[-1])
                time.sleep(0.01)  # long enough for the loop to leave
        for tk in tickets:
            dte.dte_server_wait(srv, tk)
        got = outputs(reqs, bufs)
    finally:
        dte.dte_server_free(srv)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_default_cap_from_the_environment(monkeypatch):
    """A loop created without a byte cap takes DTE_SERVE_MAX_INFLIGHT_BYTES."""
    monkeypatch.setenv("DTE_SERVE_MAX_INFLIGHT_BYTES", str(96 << 10))
    rng = np.random.default_rng(605)
    reqs = make_requests(rng, 30, lo=16 << 10, hi=64 << 10)
    ref = reference(reqs)
    srv = dte.dte_server_create(ring_slots=64)  # max_inflight_bytes 0: the default
    try:
        bufs = buffers(reqs)
        tickets = [dte.dte_server_submit(srv, r["kind"], r["t"].h, 1, u.data_ptr(), p.data_ptr())
                   for r, (u, p) in zip(reqs, bufs)]
        inflight, queued = dte.dte_server_progress(srv)
        assert queued > 0  # 96 KiB held most requests back on the host
        for tk in tickets:
            dte.dte_server_wait(srv, tk)
        got = outputs(reqs, bufs)
    finally:
        dte.dte_server_free(srv)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_reorder_stage_under_a_backlog():
    """With span_tiles 1 the reorder stage holds requests back once about
    four tiles per warp are unclaimed: a burst of mixed-variant requests then
    runs through its per-variant queues.  A 16-slot ring makes the append
    positions wrap many times, so entries are reused only after their
    requests completed.  Every result must match the oracle."""
    rng = np.random.default_rng(606)
    reqs = make_requests(rng, 120, lo=256 << 10, hi=2 << 20)
    ref = reference(reqs)
    srv = dte.dte_server_create(ring_slots=16, span_tiles=1, max_inflight_bytes=1 << 40)
    try:
        bufs = buffers(reqs)
        tickets = [dte.dte_server_submit(srv, r["kind"], r["t"].h, 1, u.data_ptr(), p.data_ptr())
                   for r, (u, p) in zip(reqs, bufs)]
        for tk in tickets:
            dte.dte_server_wait(srv, tk)
        assert dte.dte_server_progress(srv) == (0, 0)
        got = outputs(reqs, bufs)
    finally:
        dte.dte_server_free(srv)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert dte.dte_device_timeouts() == 0
