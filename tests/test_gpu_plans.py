"""Every kernel plan gives the oracle's bytes.  A plan only changes how the
kernels move a type (chunk-major with 1 KiB or 2 KiB steps, segment-major
rounds, TMA bulk copies), so pack, unpack, range moves and batches under
each plan are compared byte for byte with the oracle on the same seeded
inputs, including layouts where a plan does not apply (it then falls back to
the fixed rule)."""
import numpy as np
import pytest

import inputs
import oracle
from tests.helpers import both, span_of

torch = pytest.importorskip("torch")
import paper_2402_12274_gb300 as dte  # noqa: E402

pytestmark = pytest.mark.gpu
SENT = 0x3C
PLANS = [dte.PLAN_AUTO, dte.PLAN_CHUNK, dte.PLAN_CHUNK_WIDE, dte.PLAN_SEGMENT, dte.PLAN_BULK]


def _layouts(rng):
    specs = [inputs.random_spec(rng, big=True) for _ in range(40)]
    specs += inputs.halo_face_specs(24, 2) + inputs.halo_face_specs(64, 2)
    specs += [inputs.record_indexed_spec(rng, 4096), inputs.strided_vector_spec(256, 4, 16),
              ("hvector", 96, 1, 3 * 16384, ("contig", 2048, ("basic", "float64"))),
              ("vector", 500, 3, 7, ("basic", "bfloat16"))]
    out = []
    for sp in specs:
        t, o = both(sp)
        if o.size == 0:
            continue
        count = 1 if o.size > (1 << 20) else int(rng.integers(1, 3))
        lo, hi = span_of(o, count)
        out.append((t, o, count, -lo, hi - lo))
    return out


@pytest.fixture(scope="module")
def layouts():
    return _layouts(np.random.default_rng(777))


@pytest.mark.parametrize("plan", PLANS)
def test_single_moves_under_each_plan(layouts, plan):
    rng = np.random.default_rng(100 + plan)
    s = torch.cuda.current_stream()
    for t, o, count, base, span in layouts:
        dte.dte_type_set_plan(t.h, plan)
        src = rng.integers(0, 256, span, dtype=np.uint8)
        want = o.pack(src, count, base)
        d_src = torch.from_numpy(src).cuda()
        d_pk = torch.full((count * t.size + 16,), SENT, dtype=torch.uint8, device="cuda")
        dte.dte_pack_enqueue(d_src.data_ptr() + base, count, t.h, d_pk.data_ptr(), count * t.size, 0, s.cuda_stream)
        d_out = torch.full((span,), SENT, dtype=torch.uint8, device="cuda")
        if not o.overlaps(count):
            dte.dte_unpack_enqueue(d_pk.data_ptr(), count * t.size, 0, d_out.data_ptr() + base, count, t.h,
                                   s.cuda_stream)
        # a ragged window of the packed stream, 16-byte aligned at both ends
        # so that every plan can apply to it
        total = count * t.size
        a = (int(rng.integers(0, max(total // 16, 1))) * 16) if total >= 32 else 0
        b = min(total, a + 16 * int(rng.integers(1, max((total - a) // 16, 1) + 1)))
        d_win = torch.full((b - a + 16,), SENT, dtype=torch.uint8, device="cuda")
        if b > a:
            dte.dte_pack_range_enqueue(d_src.data_ptr() + base, count, t.h, a, b - a, d_win.data_ptr(), s.cuda_stream)
        s.synchronize()
        pk = d_pk.cpu().numpy()
        assert np.array_equal(pk[:total], want), (plan, t.size)
        assert np.all(pk[total:] == SENT)
        exp = np.full(span, SENT, np.uint8)
        if not o.overlaps(count):
            o.unpack(want, count, exp, base)
            assert np.array_equal(d_out.cpu().numpy(), exp), (plan, t.size)
        if b > a:
            w = d_win.cpu().numpy()
            assert np.array_equal(w[:b - a], want[a:b]) and np.all(w[b - a:] == SENT), (plan, a, b)
        dte.dte_type_set_plan(t.h, dte.PLAN_AUTO)


@pytest.mark.parametrize("plan", PLANS)
def test_batches_under_each_plan(layouts, plan):
    rng = np.random.default_rng(200 + plan)
    ops_src, ops_pk, wants, specs = [], [], [], []
    srcs, pks, dsts = [], [], []
    for t, o, count, base, span in layouts:
        dte.dte_type_set_plan(t.h, plan)
        src = rng.integers(0, 256, span, dtype=np.uint8)
        srcs.append(torch.from_numpy(src).cuda())
        pks.append(torch.full((count * t.size,), SENT, dtype=torch.uint8, device="cuda"))
        wants.append((o.pack(src, count, base), src))
    pack_ops = [(t.h, c, x.data_ptr() + base, p.data_ptr())
                for (t, o, c, base, span), x, p in zip(layouts, srcs, pks)]
    b = dte.Batch(dte.BATCH_PACK, pack_ops)
    b.enqueue(torch.cuda.current_stream())
    torch.cuda.synchronize()
    for p, (w, _) in zip(pks, wants):
        assert np.array_equal(p.cpu().numpy(), w), plan
    b.free()
    # unpack the oracle's packed bytes into sentinel-filled buffers
    un = [(t, o, c, base, span) for t, o, c, base, span in layouts if not o.overlaps(c)]
    wants_u = [w for (t, o, c, base, span), w in zip(layouts, wants) if not o.overlaps(c)]
    pk_in = [torch.from_numpy(w).cuda() for w, _ in wants_u]
    outs = [torch.full((span,), SENT, dtype=torch.uint8, device="cuda") for t, o, c, base, span in un]
    b = dte.Batch(dte.BATCH_UNPACK, [(t.h, c, d.data_ptr() + base, p.data_ptr())
                                     for (t, o, c, base, span), d, p in zip(un, outs, pk_in)])
    b.enqueue(torch.cuda.current_stream())
    torch.cuda.synchronize()
    for (t, o, c, base, span), d, (w, _) in zip(un, outs, wants_u):
        exp = np.full(span, SENT, np.uint8)
        o.unpack(w, c, exp, base)
        assert np.array_equal(d.cpu().numpy(), exp), plan
    b.free()
    for t, *_ in layouts:
        dte.dte_type_set_plan(t.h, dte.PLAN_AUTO)
