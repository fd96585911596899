"""The Python convenience layer refuses user buffers that a move's layout
would run past (the C ABI takes raw pointers and cannot check): a
ValueError before anything is enqueued.  Host-only; no call here reaches a
kernel."""
import pytest

torch = pytest.importorskip("torch")
import paper_2402_12274_gb300 as dte  # noqa: E402


def vec():
    return dte.Datatype.vector(4, 1, 2, dte.FLOAT32).commit()  # floats 0, 2, 4, 6: bytes [0, 28)


def test_pack_source_must_hold_the_layout():
    t = vec()
    buf = torch.zeros(64, dtype=torch.uint8)
    with pytest.raises(ValueError, match=r"\[0, 28\) of a 27-byte"):
        dte.pack(torch.zeros(27, dtype=torch.uint8), 1, t, buf, 0, stream=0)
    with pytest.raises(ValueError, match=r"\[-4, 24\)"):
        dte.pack(buf, 1, t, buf, 0, stream=0, src_offset=-4)
    with pytest.raises(ValueError, match=r"\[40, 96\)"):  # two elements at the 28-byte extent
        dte.pack(buf, 2, t, buf, 0, stream=0, src_offset=40)
    assert dte.pack(torch.zeros(0, dtype=torch.uint8), 0, t, buf, 0, stream=0) == 0  # nothing moved


def test_unpack_destination_must_hold_the_layout():
    t = vec()
    pk = torch.zeros(64, dtype=torch.uint8)
    with pytest.raises(ValueError, match="unpack destination"):
        dte.unpack(pk, 0, torch.zeros(20, dtype=torch.uint8), 1, t, stream=0)
    with pytest.raises(ValueError, match="unpack_range destination"):
        dte.unpack_range(pk, 0, 8, torch.zeros(20, dtype=torch.uint8), 1, t, stream=0)
    with pytest.raises(ValueError, match="pack_range source"):
        dte.pack_range(torch.zeros(20, dtype=torch.uint8), 1, t, 0, 8, pk, stream=0)


def test_sendrecv_buffers_must_hold_their_layouts():
    t = vec()
    u = dte.Datatype.contiguous(4, dte.FLOAT32).commit()
    ok = torch.zeros(64, dtype=torch.uint8)
    g = torch.zeros(64, dtype=torch.uint8)
    with pytest.raises(ValueError, match="send buffer"):
        dte.sendrecv(torch.zeros(10, dtype=torch.uint8), 1, t, ok, 1, u, g, stream=0)
    with pytest.raises(ValueError, match="receive buffer"):
        dte.sendrecv(ok, 1, t, torch.zeros(10, dtype=torch.uint8), 1, u, g, stream=0)


def test_negative_extent_runs_backwards():
    # resized to extent -4: element e starts 4e bytes before element 0
    t = dte.Datatype.resized(dte.Datatype.contiguous(1, dte.FLOAT32), 0, -4).commit()
    assert t.extent == -4
    buf = torch.zeros(12, dtype=torch.uint8)
    with pytest.raises(ValueError, match=r"\[-4, 8\)"):
        dte.pack(buf, 3, t, buf, 0, stream=0, src_offset=4)
    # three elements at displacement 8, 4, 0 fit a 12-byte buffer with origin 8
    dte._check_span("x", 12, 8, 3, t)
