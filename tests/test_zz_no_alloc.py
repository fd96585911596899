"""dte_pack_batch_enqueue_noalloc: the batched pack for callers that must not
allocate device memory while enqueueing (memory held in full by a caching
allocator, paths that cannot wait on the allocator, libraries that may not
touch the device heap).  It keeps its op table in a fixed array inside the
library instead of cudaMalloc'd memory.

Checked through the C ABI against the allocating dte_pack_batch_enqueue on
the same ops: byte-identical output (the bar every pack test here uses), on
two calls in a row with different source bytes, since every call reuses the
same array; the second call must leave the device's free memory and torch's
reserved bytes unchanged.  Also: an op of count 0 writes nothing, an empty
op list succeeds, an uncommitted type is refused, and a call under stream
capture is refused before anything is queued.  Collected last so that a
stop-at-first-failure run has already run everything else; it also passes
alone in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2402_12274_gb300 as dte  # noqa: E402
import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _cases(rng):
    specs = [inputs.random_spec(rng, big=True) for _ in range(60)]
    specs += inputs.halo_face_specs(24, 2)
    specs += [inputs.strided_vector_spec(64, 4, 16), inputs.record_indexed_spec(rng, 300),
              ("vector", 100, 3, 7, ("basic", "bfloat16"))]
    out = []
    for sp in specs:
        t = dte.Datatype.from_spec(sp)
        if t.h in {b.h for b in dte._BASIC_BY_NAME.values()}:
            t = dte.Datatype.contiguous(1, t)
        t.commit()
        if t.size == 0:
            continue
        count = int(rng.integers(1, 3))
        ends = [e * t.extent for e in (0, count - 1)]
        lo = min(e + t.true_lb for e in ends)
        hi = max(e + t.true_lb + t.true_extent for e in ends)
        shift = int(rng.integers(0, 16))
        out.append((t, count, -lo + shift, hi - lo + shift + 1))
    # an op with count 0 moves nothing (its packed bytes must stay untouched)
    out.append((out[0][0], 0, out[0][2], out[0][3]))
    return out


def test_noalloc_batch_pack_matches_batch_pack_on_two_calls():
    rng = np.random.default_rng(4242)
    cases = _cases(rng)
    assert 0 < len(cases) <= dte.NOALLOC_MAX_OPS
    s = torch.cuda.Stream()
    srcs = [torch.from_numpy(rng.integers(0, 256, span, dtype=np.uint8)).cuda() for _, _, _, span in cases]
    sizes = [t.size * c for t, c, _, _ in cases]
    offs = np.concatenate([[0], np.cumsum([z + 16 for z in sizes])])
    total = int(offs[-1])
    for call in range(2):
        if call == 1:  # new source bytes: the second call must not reuse stale state
            for x in srcs:
                x.copy_(torch.from_numpy(rng.integers(0, 256, x.numel(), dtype=np.uint8)))
        ref = torch.full((total,), 0x5A, dtype=torch.uint8, device="cuda")
        got = torch.full((total,), 0xC3 + call, dtype=torch.uint8, device="cuda")
        ops_ref = [(t.h, c, x.data_ptr() + base, ref.data_ptr() + int(o))
                   for (t, c, base, _), x, o in zip(cases, srcs, offs)]
        ops_got = [(t.h, c, x.data_ptr() + base, got.data_ptr() + int(o))
                   for (t, c, base, _), x, o in zip(cases, srcs, offs)]
        dte.dte_pack_batch_enqueue(ops_ref, s.cuda_stream)
        s.synchronize()
        if call == 1:
            # the call itself must not allocate: free device memory and torch's
            # reserved bytes are the same before and after it has run
            free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        dte.dte_pack_batch_enqueue_noalloc(ops_got, s.cuda_stream)
        s.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_reserved() == reserved0
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        for o, z in zip(offs[:-1], sizes):
            o = int(o)
            assert np.array_equal(g[o:o + z], r[o:o + z])
            assert np.all(g[o + z:o + z + 16] == 0xC3 + call)  # nothing written past each op
        # the count-0 op's slot keeps the sentinel
        assert sizes[-1] == 0 and np.all(g[int(offs[-2]):int(offs[-1])] == 0xC3 + call)


def test_noalloc_empty_list_and_refusals():
    t = dte.Datatype.vector(4, 1, 2, dte.FLOAT32).commit()
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    dte.dte_pack_batch_enqueue_noalloc([])  # nothing to do: success
    ops = [(t.h, 1, buf.data_ptr(), buf.data_ptr() + 64 * i) for i in range(dte.NOALLOC_MAX_OPS + 1)]
    with pytest.raises(dte.DteError) as e:
        dte.dte_pack_batch_enqueue_noalloc(ops)
    assert e.value.code == dte.ERR_UNSUPPORTED
    u = dte.Datatype.vector(4, 1, 2, dte.FLOAT32)  # never committed
    with pytest.raises(dte.DteError) as e:
        dte.dte_pack_batch_enqueue_noalloc([(u.h, 1, buf.data_ptr(), buf.data_ptr() + 4096)])
    assert e.value.code == dte.ERR_TYPE
    with pytest.raises(dte.DteError) as e:
        dte.dte_pack_batch_enqueue_noalloc([(t.h, -1, buf.data_ptr(), buf.data_ptr() + 4096)])
    assert e.value.code == dte.ERR_ARG
    # under stream capture the call is refused and queues nothing
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream()
    codes = []
    with torch.cuda.graph(g, stream=gs):
        try:
            dte.dte_pack_batch_enqueue_noalloc([(t.h, 1, buf.data_ptr(), buf.data_ptr() + 4096)], gs.cuda_stream)
        except dte.DteError as err:
            codes.append(err.code)
    assert codes == [dte.ERR_UNSUPPORTED]
