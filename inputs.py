"""Seeded synthetic inputs: datatype specs and source buffers.

This module holds no datatype arithmetic -- no typemap expansion, no sizes,
no segment logic.  It only draws parameters and bytes from seeded numpy
generators and writes them down as *specs*, plain nested tuples that both the
library binding (``Datatype.from_spec``) and the test oracle turn into types
with their own constructors:

    ("basic", name)
    ("contig", count, child)
    ("vector", count, bl, stride, child)
    ("hvector", count, bl, stride_bytes, child)
    ("indexed", bl[], disp[], child)
    ("hindexed", bl[], disp_bytes[], child)
    ("indexed_block", bl, disp[], child)
    ("hindexed_block", bl, disp_bytes[], child)
    ("struct", bl[], disp_bytes[], [children])
    ("subarray", sizes[], subsizes[], starts[], order, child)   # order 0 = C, 1 = Fortran
    ("resized", lb, extent, child)
    ("darray", size, rank, gsizes[], distribs[], dargs[], psizes[], order, child)
                                            # distribs: 0 block, 1 cyclic, 2 none; darg -1 = default

Workload shapes follow the benchmark configurations: a strided vector of
float32, the six ghost faces of a 3-D float64 grid, a struct/indexed nest
with geometric block lengths, a batch of mixed small/large layouts, and
halo faces as element-granular indexed types with repeated entries.
"""
from __future__ import annotations

import numpy as np

BASIC_NAMES = ("byte", "int8", "uint8", "int16", "uint16", "int32", "uint32", "int64", "uint64",
               "float16", "bfloat16", "float32", "float64")


# ---------------------------------------------------------------------------
# random tiny nests (fuzzing)
# ---------------------------------------------------------------------------
def random_spec(rng: np.random.Generator, depth: int = 0, max_depth: int = 3, big: bool = False):
    """A random nested spec with small parameters (big=True: larger counts).
    Counts and block lengths are zero with probability 0.08 each."""
    kinds = ["basic", "contig", "vector", "hvector", "indexed", "hindexed", "struct",
             "subarray", "resized", "indexed_block", "hindexed_block"]
    if depth >= max_depth:
        kinds = ["basic"]
    k = kinds[int(rng.integers(len(kinds)))] if depth > 0 else kinds[int(rng.integers(1, len(kinds)))]
    m = 9 if big else 4

    def cnt(hi):
        return 0 if rng.random() < 0.08 else int(rng.integers(1, hi + 1))

    if k == "basic":
        return ("basic", str(rng.choice(["byte", "int16", "float32", "float64", "bfloat16", "int32"])))
    child = random_spec(rng, depth + 1, max_depth, big)
    if k == "contig":
        return ("contig", cnt(m), child)
    if k == "vector":
        return ("vector", cnt(m), cnt(3), int(rng.integers(-5, 6)), child)
    if k == "hvector":
        return ("hvector", cnt(m), cnt(2), int(rng.integers(-48, 49)), child)
    if k in ("indexed", "hindexed"):
        n = cnt(m)
        bl = np.array([cnt(2) for _ in range(n)], np.int64)
        d = rng.integers(-6, 7, n) if k == "indexed" else rng.integers(-48, 49, n)
        return (k, bl, d.astype(np.int64), child)
    if k in ("indexed_block", "hindexed_block"):
        n = cnt(m)
        d = rng.integers(-6, 7, n) if k == "indexed_block" else rng.integers(-48, 49, n)
        return (k, cnt(2), d.astype(np.int64), child)
    if k == "struct":
        n = int(rng.integers(1, 4))
        kids = [child] + [random_spec(rng, depth + 1, max_depth, big) for _ in range(n - 1)]
        bl = np.array([cnt(2) for _ in range(n)], np.int64)
        return ("struct", bl, rng.integers(-48, 49, n).astype(np.int64), kids)
    if k == "subarray":
        nd = int(rng.integers(1, 4))
        sizes = rng.integers(1, 5, nd)
        sub = np.array([0 if rng.random() < 0.05 else rng.integers(1, s + 1) for s in sizes], np.int64)
        st = np.array([rng.integers(0, s - u + 1) for s, u in zip(sizes, sub)], np.int64)
        return ("subarray", sizes.astype(np.int64), sub, st, int(rng.integers(2)), child)
    return ("resized", int(rng.integers(-8, 9)), int(rng.integers(0, 48)), child)


def random_darray_spec(rng: np.random.Generator):
    """A random distributed-array spec over a small global array."""
    nd = int(rng.integers(1, 4))
    gs = rng.integers(1, 9, nd).astype(np.int64)
    ps = np.array([rng.integers(1, 4) for _ in range(nd)], np.int64)
    dist, dargs = [], []
    for d in range(nd):
        kind = int(rng.integers(3))
        if kind == 2:
            ps[d] = 1
        dist.append(kind)
        if kind == 0:  # block: default, or a block size big enough to cover
            dargs.append(-1 if rng.random() < 0.5 else int(-(-gs[d] // ps[d]) + rng.integers(0, 3)))
        elif kind == 1:
            dargs.append(-1 if rng.random() < 0.5 else int(rng.integers(1, 4)))
        else:
            dargs.append(-1)
    size = int(np.prod(ps))
    rank = int(rng.integers(size))
    child = ("basic", str(rng.choice(["int32", "float64", "bfloat16"])))
    if rng.random() < 0.3:
        child = ("vector", 2, 1, 2, child)
    return ("darray", size, rank, gs, dist, np.array(dargs, np.int64), ps, int(rng.integers(2)), child)


def sequential_spec(rng: np.random.Generator):
    """Random specs biased toward layouts whose segments merge across copies,
    entries and levels (abutting blocks, strides equal to block sizes)."""
    base = ("basic", str(rng.choice(["byte", "int32", "float64"])))
    n = int(rng.integers(2, 7))
    choice = int(rng.integers(6))
    if choice == 0:  # hindexed with some abutting blocks
        bl = rng.integers(1, 3, n).astype(np.int64)
        gaps = rng.integers(0, 2, n).astype(np.int64)
        return ("contig", int(rng.integers(1, 4)), ("indexed", bl, np.cumsum(bl + gaps) - bl - gaps[0], base))
    if choice == 1:  # vector whose blocks touch across the element boundary
        return ("contig", int(rng.integers(2, 5)), ("vector", n, 2, 4, ("resized", 0, 1, ("basic", "byte"))))
    if choice == 2:  # struct of pieces that may chain together
        pieces = [("basic", "int32"), ("vector", 2, 1, 2, ("basic", "int32")), ("contig", 2, ("basic", "int32"))]
        kids = [pieces[int(rng.integers(3))] for _ in range(n)]
        d = np.cumsum(rng.choice([4, 8, 12], n)).astype(np.int64) - 4
        return ("struct", np.ones(n, np.int64), d, kids)
    if choice == 3:  # resized struct whose last run reaches the next element
        inner = ("struct", np.array([1, 1], np.int64), np.array([0, 8], np.int64),
                 [("basic", "int32"), ("basic", "int32")])
        return ("contig", n, ("resized", 0, 12, inner))
    if choice == 4:  # subarray with full rows
        return ("subarray", np.array([3, n], np.int64), np.array([2, n], np.int64),
                np.array([1, 0], np.int64), 0, base)
    return ("hindexed_block", 1, (np.arange(n) * 8).astype(np.int64),
            ("struct", np.array([1, 1], np.int64), np.array([0, 4], np.int64),
             [("basic", "int32"), ("resized", 0, 4, ("basic", "int16"))]))


# ---------------------------------------------------------------------------
# benchmark-shaped workloads
# ---------------------------------------------------------------------------
def strided_vector_spec(count: int = 1024, bl: int = 4, stride: int = 16):
    """vector(count, bl, stride) of float32."""
    return ("vector", count, bl, stride, ("basic", "float32"))


def halo_face_specs(n: int = 512, g: int = 2, elem: str = "float64"):
    """The six send faces of an n^3 row-major grid with ghost thickness g:
    the owned layers next to the ghosts, g cells thick, full n along the
    other two axes.  Index (i0, i1, i2), i2 fastest."""
    faces = []
    for axis in range(3):
        for start in (g, n - 2 * g):
            sub = [n, n, n]
            st = [0, 0, 0]
            sub[axis] = g
            st[axis] = start
            faces.append(("subarray", np.array([n, n, n], np.int64), np.array(sub, np.int64),
                          np.array(st, np.int64), 0, ("basic", elem)))
    return faces


def halo_recv_face_specs(n: int = 512, g: int = 2, elem: str = "float64"):
    """The six ghost (receive) faces: the outermost g layers."""
    faces = []
    for axis in range(3):
        for start in (0, n - g):
            sub = [n, n, n]
            st = [0, 0, 0]
            sub[axis] = g
            st[axis] = start
            faces.append(("subarray", np.array([n, n, n], np.int64), np.array(sub, np.int64),
                          np.array(st, np.int64), 0, ("basic", elem)))
    return faces


def all_faces_struct(face_specs):
    """One struct holding every face at displacement 0: packing it packs the
    faces one after another into one contiguous buffer."""
    k = len(face_specs)
    return ("struct", np.ones(k, np.int64), np.zeros(k, np.int64), list(face_specs))


def record_indexed_spec(rng: np.random.Generator, nblocks: int, mean_len: float = 8.0, mean_gap: float = 1.0):
    """struct{int32[3] @0, float64[5] @16} resized to 64 B, inside an indexed
    type of `nblocks` blocks with Geometric(mean_len) lengths on {1,2,...} and
    sorted non-overlapping displacements separated by Geometric(mean_gap)
    gaps on {0,1,...} (in 64-byte records)."""
    rec = ("resized", 0, 64, ("struct", np.array([3, 5], np.int64), np.array([0, 16], np.int64),
                              [("basic", "int32"), ("basic", "float64")]))
    bl = rng.geometric(1.0 / mean_len, nblocks).astype(np.int64)
    gaps = (rng.geometric(1.0 / (mean_gap + 1.0), nblocks) - 1).astype(np.int64)
    disp = np.cumsum(gaps + bl) - bl
    if nblocks:
        disp -= disp[0]
    return ("indexed", bl, disp.astype(np.int64), rec)


def record_variety_spec(rng: np.random.Generator, nblocks: int):
    """An array of records under an index list, with the record drawn at
    random.  A grain g of 1, 2, 4 or 8 bytes is drawn first; the record is a
    struct of 1-6 blocks (1-5 elements each) of basic types at least g bytes
    wide, at increasing displacements 0-12 bytes apart in multiples of g, or a
    single block of one such type, and is resized with probability 0.7 to its
    extent plus 0-12 bytes (a multiple of g).  It sits inside an indexed type
    (displacements in records, sorted, Geometric(mean) block lengths with mean
    1, 3 or 8 and Geometric(1/2) gaps on {0,1,...}) or a hindexed type (the
    same displacements in bytes, shifted by a multiple of g in [-64, 64])."""
    sizes = {"byte": 1, "int16": 2, "bfloat16": 2, "int32": 4, "float32": 4, "float64": 8}
    g = int(rng.choice([1, 2, 4, 8]))
    names = [n for n, z in sizes.items() if z >= g]

    def pad():
        return g * int(rng.integers(0, 12 // g + 1))

    if rng.random() < 0.2:
        el = str(rng.choice(names))
        rec = ("contig", int(rng.integers(1, 9)), ("basic", el))
        span = sizes[el] * rec[1]
    else:
        nb = int(rng.integers(1, 7))
        kids = [("basic", str(rng.choice(names))) for _ in range(nb)]
        bl = rng.integers(1, 6, nb).astype(np.int64)
        d, at = [], 0
        for kid, b in zip(kids, bl):
            s = sizes[kid[1]]
            at = -(-at // s) * s  # natural alignment of the block's element
            d.append(at)
            at += int(b) * s + pad()
        rec = ("struct", bl, np.array(d, np.int64), kids)
        span = at
    if rng.random() < 0.7:
        rec = ("resized", 0, span + pad(), rec)
    mean = float(rng.choice([1.0, 3.0, 8.0]))
    lens = rng.geometric(1.0 / mean, nblocks).astype(np.int64)
    gaps = (rng.geometric(0.5, nblocks) - 1).astype(np.int64)
    disp = np.cumsum(gaps + lens) - lens
    disp -= disp[0]
    if rng.random() < 0.5:
        return ("indexed", lens, disp.astype(np.int64), rec)
    ext = span + 16  # byte displacements: records at least this far apart
    shift = g * int(rng.integers(-64 // g, 64 // g + 1))
    return ("hindexed", lens, (disp * ext + shift).astype(np.int64), rec)


def batch_specs(rng: np.random.Generator, nops: int, lo: int = 64, hi: int = 4 << 20):
    """`nops` independent layouts of float32 or bfloat16 with packed sizes
    log-uniform in [lo, hi] bytes: kind uniform over vector, indexed and
    subarray.  Returns a list of (spec, approx_packed_bytes)."""
    out = []
    for _ in range(nops):
        elem = "float32" if rng.random() < 0.5 else "bfloat16"
        es = 4 if elem == "float32" else 2
        target = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        n_el = max(1, target // es)
        kind = int(rng.integers(3))
        if kind == 0:
            bl = int(rng.choice([1, 2, 3, 4, 8, 16, 32, 64, 256, 1024]))
            bl = min(bl, n_el)
            cnt = max(1, n_el // bl)
            stride = bl + int(rng.integers(0, 2 * bl + 1))
            spec = ("vector", cnt, bl, stride, ("basic", elem))
        elif kind == 1:
            mean = float(rng.choice([2, 8, 64, 512]))
            nb = max(1, int(n_el / mean))
            bl = rng.geometric(1.0 / mean, nb).astype(np.int64)
            gaps = rng.integers(0, int(mean) + 1, nb).astype(np.int64)
            disp = np.cumsum(gaps + bl) - bl - gaps[0]
            spec = ("indexed", bl, disp.astype(np.int64), ("basic", elem))
        else:
            d1 = max(1, int(np.sqrt(n_el)))
            d0 = max(1, n_el // d1)
            full = [d0 + int(rng.integers(0, 3)), d1 + int(rng.integers(0, d1 + 1))]
            st = [int(rng.integers(0, full[0] - d0 + 1)), int(rng.integers(0, full[1] - d1 + 1))]
            spec = ("subarray", np.array(full, np.int64), np.array([d0, d1], np.int64),
                    np.array(st, np.int64), 0, ("basic", elem))
        out.append((spec, target))
    return out


def halo_indexed_specs(rng: np.random.Generator, n: int = 256, g: int = 2, repeat_frac: float = 0.10):
    """Six faces of an n^3 float32 grid as element-granular indexed types
    (one float per entry); in each face a `repeat_frac` share of the entries,
    drawn without replacement, is duplicated and the copies are inserted at
    random positions of that face's list."""
    specs = []
    for axis in range(3):
        for start in (g, n - 2 * g):
            ranges = [np.arange(n), np.arange(n), np.arange(n)]
            ranges[axis] = np.arange(start, start + g)
            i0, i1, i2 = np.meshgrid(*ranges, indexing="ij")
            idx = ((i0 * n + i1) * n + i2).ravel().astype(np.int64)
            if repeat_frac > 0:
                k = int(round(repeat_frac * idx.size))
                dup = rng.choice(idx, size=k, replace=False)
                pos = np.sort(rng.integers(0, idx.size + 1, k))
                idx = np.insert(idx, pos, dup)
            specs.append(("indexed_block", 1, idx, ("basic", "float32")))
    return specs


# ---------------------------------------------------------------------------
# source bytes
# ---------------------------------------------------------------------------
def uniform_f32(nbytes_or_n: int, seed: int, as_bytes: bool = False):
    rng = np.random.default_rng(seed)
    n = nbytes_or_n // 4 if as_bytes else nbytes_or_n
    return rng.uniform(-1.0, 1.0, n).astype(np.float32)


def normal_f64(n: int, seed: int):
    return np.random.default_rng(seed).standard_normal(n)


def random_bytes(n: int, seed: int):
    """Raw random bytes (every bit pattern, NaN payloads included)."""
    return np.random.default_rng(seed).integers(0, 256, n, dtype=np.uint8)
