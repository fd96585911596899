"""The seeded input generators follow the stated workload recipe: record
layout (Geometric block lengths and gaps, sorted non-overlapping blocks, the
64-byte record), the batch mix (kinds, element types, log-uniform sizes),
the halo faces and their repeated-entry variant; and each generator is a
pure function of its seed."""
import numpy as np

import oracle
import inputs


def test_record_layout_recipe():
    rng = np.random.default_rng(3)
    spec = inputs.record_indexed_spec(rng, 1 << 16)
    kind, bl, disp, rec = spec
    assert kind == "indexed" and bl.size == disp.size == 1 << 16
    # block lengths Geometric(mean 8) on {1, 2, ...}
    assert bl.min() >= 1 and abs(bl.mean() - 8.0) < 0.15
    # sorted, non-overlapping, first block at 0; gaps Geometric(mean 1) on {0, 1, ...}
    assert disp[0] == 0
    gaps = disp[1:] - (disp[:-1] + bl[:-1])
    assert gaps.min() >= 0 and abs(gaps.mean() - 1.0) < 0.05
    assert np.mean(gaps == 0) > 0.45  # P(0) = 1/2 for mean 1
    # the record: int32[3] at 0 and float64[5] at 16, resized to 64 bytes
    o = oracle.from_spec(rec)
    assert (o.size, o.lb, o.extent) == (52, 0, 64)
    d, l = o.iov()
    assert d.tolist() == [0, 16] and l.tolist() == [12, 40]


def test_record_variety_recipe():
    # records of 1-6 blocks (or one block) at a grain of 1-8 bytes, under an
    # index list of sorted, non-overlapping blocks of whole records
    rng = np.random.default_rng(206)
    seen = set()
    for _ in range(200):
        kind, bl, disp, rec = inputs.record_variety_spec(rng, 100)
        assert kind in ("indexed", "hindexed") and bl.size == disp.size == 100 and bl.min() >= 1
        r = oracle.from_spec(rec)
        assert r.size > 0 and r.lb == 0 and r.true_lb == 0 and r.extent >= r.true_extent
        d, l = r.iov()
        assert d.size <= 6 and np.all(d[1:] >= d[:-1] + l[:-1])  # runs in order, disjoint
        ext = r.extent if kind == "indexed" else 1
        lo = disp * ext
        hi = lo + (bl - 1) * r.extent + r.true_extent
        assert np.all(lo[1:] >= hi[:-1])  # whole records never overlap
        seen.add((kind, rec[0], int(np.gcd.reduce(np.concatenate([d, l, [r.extent]])) % 16)))
    assert {k for k, _, _ in seen} == {"indexed", "hindexed"}
    assert {c for _, c, _ in seen} == {"struct", "resized", "contig"}
    assert {g for _, _, g in seen} >= {1, 2, 4, 8}


def test_batch_mix_recipe():
    rng = np.random.default_rng(4)
    specs = inputs.batch_specs(rng, 3000)
    kinds = np.array([s[0] for s, _ in specs])
    for k in ("vector", "indexed", "subarray"):
        assert abs(np.mean(kinds == k) - 1 / 3) < 0.04
    elems = np.array([(s[-1] if s[0] != "indexed" else s[3])[1] for s, _ in specs])
    assert set(elems) == {"float32", "bfloat16"} and abs(np.mean(elems == "float32") - 0.5) < 0.04
    # target sizes log-uniform on [64 B, 4 MiB]
    t = np.array([n for _, n in specs], np.float64)
    assert t.min() >= 64 and t.max() <= 4 << 20
    u = (np.log(t) - np.log(64)) / (np.log(4 << 20) - np.log(64))
    assert abs(u.mean() - 0.5) < 0.03 and abs(np.mean(u < 0.25) - 0.25) < 0.04
    # the layouts' packed sizes track the targets (indexed layouts of a few
    # Geometric blocks can land well away from theirs)
    ratio = np.array([oracle.from_spec(s).size / n for s, n in specs[:400]])
    assert 0.95 < np.median(ratio) <= 1.0
    assert np.mean((ratio > 0.5) & (ratio < 2.0)) > 0.9


def test_halo_faces_recipe():
    n, g = 12, 2
    faces = inputs.halo_face_specs(n, g)
    assert len(faces) == 6
    for i, (kind, sizes, sub, start, order, child) in enumerate(faces):
        axis, hi = divmod(i, 2)
        assert kind == "subarray" and order == 0 and child == ("basic", "float64")
        assert sizes.tolist() == [n, n, n]
        assert sub.tolist() == [g if a == axis else n for a in range(3)]
        assert start.tolist() == [(n - 2 * g if hi else g) if a == axis else 0 for a in range(3)]
    recv = inputs.halo_recv_face_specs(n, g)
    for i, f in enumerate(recv):
        axis, hi = divmod(i, 2)
        assert f[3][axis] == (n - g if hi else 0)


def test_repeated_entry_faces_recipe():
    rng = np.random.default_rng(5)
    n, g = 10, 2
    plain = inputs.halo_indexed_specs(np.random.default_rng(0), n=n, g=g, repeat_frac=0.0)
    rep = inputs.halo_indexed_specs(rng, n=n, g=g, repeat_frac=0.10)
    for p, r in zip(plain, rep):
        base, idx = p[2], r[2]
        k = int(round(0.10 * base.size))
        assert idx.size == base.size + k
        # every entry is a cell of the face; the extra entries are k distinct cells
        assert set(idx.tolist()) == set(base.tolist())
        vals, counts = np.unique(idx, return_counts=True)
        assert counts.max() == 2 and int(np.sum(counts == 2)) == k
        # the face's own list is kept, in order, around the inserted copies
        j = 0
        for v in idx.tolist():
            if j < base.size and v == base[j]:
                j += 1
        assert j == base.size


def test_generators_are_pure_functions_of_the_seed():
    def same(a, b):
        if isinstance(a, np.ndarray):
            return np.array_equal(a, b)
        if isinstance(a, (tuple, list)):
            return len(a) == len(b) and all(same(x, y) for x, y in zip(a, b))
        return a == b

    for f in (lambda r: inputs.record_indexed_spec(r, 100), lambda r: inputs.batch_specs(r, 50),
              lambda r: inputs.halo_indexed_specs(r, n=6, g=2), lambda r: [inputs.random_spec(r) for _ in range(20)],
              lambda r: [inputs.random_darray_spec(r) for _ in range(20)],
              lambda r: [inputs.record_variety_spec(r, 40) for _ in range(20)]):
        assert same(f(np.random.default_rng(11)), f(np.random.default_rng(11)))
    assert np.array_equal(inputs.random_bytes(1000, 7), inputs.random_bytes(1000, 7))
