"""CPU checks of the library's type system and commit compiler against the
oracle: sizes, bounds, segment lists and iov_len (paper §3.1) for random
nests, for layouts whose segments merge across copies/entries/levels, and for
the paper's worked example.  No GPU needed: these queries run on the host
over the committed descriptor."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2402_12274_gb300 as dte
import inputs
from tests.helpers import both, iov_arrays

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dte.h")


def test_library_exports_every_declared_symbol():
    import re
    decl = set(re.findall(r"DTE_API\s+[\w\s\*]*?\b(dte_\w+)\s*\(", open(HDR).read()))
    assert len(decl) >= 25
    missing = [n for n in decl if not hasattr(dte.lib, n)]
    assert not missing, missing
    assert decl == set(dte.EXPORTED)


def compare(spec, full_iov_len=True):
    t, o = both(spec)
    assert t.size == o.size
    assert (t.lb, t.extent) == (o.lb, o.extent), spec
    if o.size:
        assert (t.true_lb, t.true_extent) == (o.true_lb, o.true_extent)
    assert t.num_segments == o.iov_count()
    d, l = iov_arrays(t)
    od, ol = o.iov()
    assert np.array_equal(d, od) and np.array_equal(l, ol), spec
    n = len(ol)
    pre = np.concatenate([[0], np.cumsum(ol)])
    if full_iov_len:
        bs = range(0, o.size + 1)
    else:  # segment starts, their predecessors, and random bytes (sampled)
        rng = np.random.default_rng(n)
        pick = rng.integers(0, n + 1, min(n + 1, 40))
        bs = np.unique(np.concatenate([pre[pick], np.maximum(pre[pick] - 1, 0),
                                       rng.integers(0, o.size + 1, 20), [0, o.size]]))
    for b in bs:
        assert t.iov_len(int(b)) == o.iov_len(int(b)), (spec, b)
    assert t.iov_len(-1) == (n, o.size)
    assert t.iov_len(o.size + 5) == (n, o.size)
    for k in (0, 1, n // 3, n - 1, n, n + 2):
        for m in (1, 3, 7):
            if k < 0:
                continue
            d, l = iov_arrays(t, k, m)
            od, ol = o.iov(k, m)
            assert np.array_equal(d, od) and np.array_equal(l, ol)


def test_random_nests_match_oracle():
    rng = np.random.default_rng(101)
    for _ in range(3000):
        compare(inputs.random_spec(rng))


def test_random_bigger_nests_match_oracle():
    rng = np.random.default_rng(102)
    for _ in range(600):
        compare(inputs.random_spec(rng, big=True), full_iov_len=False)


def test_merging_layouts_match_oracle():
    rng = np.random.default_rng(103)
    for _ in range(1000):
        compare(inputs.sequential_spec(rng))


def test_typeiov_example():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "typeiov.json")))
    value = dte.Datatype.contiguous(g["value_bytes"], dte.BYTE)
    vol = dte.Datatype.subarray(g["full_sizes"], g["sub_sizes"], g["sub_offsets"], value).commit()
    assert (vol.size, vol.lb, vol.extent) == (g["size"], g["lb"], g["extent"])
    assert vol.iov_len(g["max_iov_bytes"]) == (g["iov_len"], g["iov_bytes"])
    assert [list(x) for x in vol.iov(0, 4)] == g["iov"]


def test_workload_types_match_oracle():
    compare(inputs.strided_vector_spec(), full_iov_len=False)
    compare(("contig", 64, inputs.strided_vector_spec()), full_iov_len=False)
    for f in inputs.halo_face_specs(n=24, g=2):
        compare(f, full_iov_len=False)
    compare(inputs.all_faces_struct(inputs.halo_face_specs(n=16, g=2)), full_iov_len=False)
    rng = np.random.default_rng(3)
    compare(inputs.record_indexed_spec(rng, 200), full_iov_len=False)
    for spec, _ in inputs.batch_specs(rng, 30, lo=64, hi=4096):
        compare(spec, full_iov_len=False)
    for spec in inputs.halo_indexed_specs(rng, n=8, g=2):
        compare(spec, full_iov_len=False)


def test_halo_face_segment_counts():
    # YZ-surface rule (paper §3): faces normal to the slowest axis are one
    # contiguous run, the middle axis gives n runs of g*n, the fastest n*n runs of g
    n, g = 32, 2
    counts = [dte.Datatype.from_spec(f).num_segments for f in inputs.halo_face_specs(n, g)]
    assert counts == [1, 1, n, n, n * n, n * n]


def test_error_paths():
    with pytest.raises(dte.DteError) as e:
        dte.Datatype.vector(-1, 1, 1, dte.FLOAT32)
    assert e.value.code == dte.ERR_ARG
    t = dte.Datatype.vector(3, 1, 2, dte.FLOAT32)
    with pytest.raises(dte.DteError) as e:
        t.iov_len(-1)  # not committed
    assert e.value.code == dte.ERR_TYPE
    t.commit()
    with pytest.raises(dte.DteError) as e:
        t.iov_len(-2)
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:
        t.iov(-1, 2)
    assert e.value.code == dte.ERR_ARG
    assert t.iov(10, 2) == []
    with pytest.raises(dte.DteError) as e:
        dte.dte_type_free(dte.FLOAT32.h)
    assert e.value.code == dte.ERR_TYPE
    h = dte.dte_type_contiguous(2, dte.FLOAT32.h)
    dte.dte_type_free(h)
    with pytest.raises(dte.DteError) as e:
        dte.dte_type_size(h)
    assert e.value.code == dte.ERR_TYPE
    with pytest.raises(dte.DteError) as e:
        dte.Datatype.subarray([4], [3], [2], dte.FLOAT32)
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:  # count * size overflows int64
        big = dte.Datatype.contiguous(1 << 40, dte.FLOAT64)
        dte.Datatype.contiguous(1 << 40, big)
    assert e.value.code == dte.ERR_OVERFLOW
    assert dte.dte_pack_size(5, t.h) == 5 * 12


def test_inputs_freed_after_construction():
    a = dte.Datatype.vector(4, 1, 3, dte.INT32)
    b = dte.Datatype.contiguous(2, a)
    del a
    b.commit()
    o = oracle.contiguous(2, oracle.vector(4, 1, 3, oracle.basic(4, 4)))
    assert b.size == o.size and b.num_segments == o.iov_count()
    c = b.dup()
    del b
    assert c.size == o.size and c.iov_len(-1) == (o.iov_count(), o.size)


def test_server_needs_a_device_and_valid_settings():
    # no CUDA device in a CPU-only run: creation reports it instead of failing later
    import torch
    with pytest.raises(dte.DteError) as e:
        dte.dte_server_create(ring_slots=3)
    assert e.value.code == dte.ERR_ARG
    if not torch.cuda.is_available():
        with pytest.raises(dte.DteError) as e:
            dte.dte_server_create()
        assert e.value.code in (dte.ERR_NODEVICE, dte.ERR_CUDA)


def test_random_darrays_match_oracle():
    rng = np.random.default_rng(104)
    for _ in range(400):
        compare(inputs.random_darray_spec(rng))
    # darray nested inside other constructors, and other constructors inside it
    for _ in range(100):
        d = inputs.random_darray_spec(rng)
        compare(("contig", 2, d))
        compare(("darray",) + d[1:8] + (("resized", -4, 12, ("basic", "int32")),))


def test_darray_errors():
    with pytest.raises(dte.DteError) as e:  # block size too small to cover
        dte.Datatype.darray(2, 0, [9], [dte.DISTRIBUTE_BLOCK], [4], [2], dte.FLOAT64)
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:  # grid of 3 for a size of 4
        dte.Datatype.darray(4, 0, [8], [dte.DISTRIBUTE_CYCLIC], [dte.DISTRIBUTE_DFLT_DARG], [3], dte.FLOAT64)
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:  # undistributed dimension split over two processes
        dte.Datatype.darray(2, 0, [8], [dte.DISTRIBUTE_NONE], [dte.DISTRIBUTE_DFLT_DARG], [2], dte.FLOAT64)
    assert e.value.code == dte.ERR_ARG
    with pytest.raises(dte.DteError) as e:
        dte.Datatype.darray(2, 2, [8], [dte.DISTRIBUTE_CYCLIC], [dte.DISTRIBUTE_DFLT_DARG], [2], dte.FLOAT64)
    assert e.value.code == dte.ERR_ARG


def test_range_and_sendrecv_argument_checks():
    # these checks run before any device work, so they hold without a GPU
    t = dte.Datatype.vector(10, 1, 2, dte.FLOAT32).commit()
    u = dte.Datatype.contiguous(5, dte.FLOAT32).commit()
    for first, n in ((-1, 4), (0, -4), (30, 11), (41, 0)):
        with pytest.raises(dte.DteError) as e:
            dte.dte_pack_range_enqueue(16, 1, t.h, first, n, 16)
        assert e.value.code == dte.ERR_ARG
        with pytest.raises(dte.DteError) as e:
            dte.dte_unpack_range_enqueue(16, first, n, 16, 1, t.h)
        assert e.value.code == dte.ERR_ARG
    dte.dte_pack_range_enqueue(16, 1, t.h, 40, 0, 16)  # empty window at the end: nothing to do
    with pytest.raises(dte.DteError) as e:  # 40-byte message into a 20-byte receive
        dte.dte_sendrecv_enqueue(16, 1, t.h, 16, 1, u.h, 16, 64)
    assert e.value.code == dte.ERR_TRUNCATE
    with pytest.raises(dte.DteError) as e:
        dte.dte_sendrecv_enqueue(16, 1, u.h, 16, 2, t.h, 16, -1)
    assert e.value.code == dte.ERR_ARG
    v = dte.Datatype.vector(3, 1, 2, dte.FLOAT32)  # not committed
    with pytest.raises(dte.DteError) as e:
        dte.dte_sendrecv_enqueue(16, 1, v.h, 16, 1, u.h, 16, 64)
    assert e.value.code == dte.ERR_TYPE
    dte.dte_sendrecv_enqueue(16, 0, u.h, 16, 0, t.h, 16, 64)  # empty message


def test_descriptor_sizes_stay_compact():
    # strided and subarray layouts commit to a few hundred bytes whatever
    # their size; an index table costs about its entries
    rng = np.random.default_rng(105)
    vec = dte.Datatype.vector(1 << 20, 4, 16, dte.FLOAT32).commit()
    assert vec.descriptor_bytes <= 1024
    faces = [dte.Datatype.from_spec(f).commit() for f in inputs.halo_face_specs(512, 2)]
    assert max(f.descriptor_bytes for f in faces) <= 2048
    rec = dte.Datatype.from_spec(inputs.record_indexed_spec(rng, 1 << 12)).commit()
    assert 16 * 4096 <= rec.descriptor_bytes <= 64 * 4096
    with pytest.raises(dte.DteError) as e:
        dte.Datatype.vector(3, 1, 2, dte.FLOAT32).descriptor_bytes
    assert e.value.code == dte.ERR_TYPE
