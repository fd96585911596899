"""ctypes wrapper around the plain-C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this module to compute expected values.  The product
library never imports it.

The oracle walks the typemap of an MPI-style derived datatype one basic entry
at a time (paper §3, §3.1) and implements pack/unpack/iov/iov_len on that walk.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORDER_C = 0
ORDER_F = 1

_i64 = C.c_int64
_p = C.c_void_p
_pi64 = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host C compiler (no GPU involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        for name, args in {
            "or_basic": [_i64, _i64],
            "or_contiguous": [_i64, _p],
            "or_vector": [_i64, _i64, _i64, _p],
            "or_hvector": [_i64, _i64, _i64, _p],
            "or_indexed": [_i64, _pi64, _pi64, _p],
            "or_hindexed": [_i64, _pi64, _pi64, _p],
            "or_indexed_block": [_i64, _i64, _pi64, _p],
            "or_hindexed_block": [_i64, _i64, _pi64, _p],
            "or_struct": [_i64, _pi64, _pi64, C.POINTER(_p)],
            "or_subarray": [C.c_int, _pi64, _pi64, _pi64, C.c_int, _p],
            "or_resized": [_p, _i64, _i64],
            "or_darray": [C.c_int, C.c_int, C.c_int, _pi64, C.POINTER(C.c_int), _pi64, _pi64, C.c_int, _p],
        }.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _p
        L.or_free.argtypes = [_p]
        L.or_free.restype = None
        for name in ("or_size", "or_lb", "or_extent", "or_true_lb", "or_true_extent",
                     "or_typemap_len", "or_iov_count"):
            getattr(L, name).argtypes = [_p]
            getattr(L, name).restype = _i64
        L.or_typemap.argtypes = [_p, _pi64, _pi64]
        L.or_typemap.restype = None
        L.or_iov.argtypes = [_p, _i64, _i64, _pi64, _pi64]
        L.or_iov.restype = _i64
        L.or_iov_elements.argtypes = [_p, _i64, _i64, _i64, _pi64, _pi64]
        L.or_iov_elements.restype = _i64
        L.or_iov_len.argtypes = [_p, _i64, _pi64, _pi64]
        L.or_iov_len.restype = C.c_int
        L.or_pack.argtypes = [_p, _i64, _p, _p]
        L.or_pack.restype = C.c_int
        L.or_unpack.argtypes = [_p, _i64, _p, _p]
        L.or_pack_range.argtypes = [_p, _i64, _p, _i64, _i64, _p]
        L.or_pack_range.restype = C.c_int
        L.or_unpack_range.argtypes = [_p, _i64, _i64, _i64, _p, _p]
        L.or_unpack_range.restype = C.c_int
        L.or_unpack.restype = C.c_int
        L.or_overlaps.argtypes = [_p, _i64]
        L.or_overlaps.restype = C.c_int
        L.or_pack_adjoint_f64.argtypes = [_p, _i64, _p, _p, _i64]
        L.or_pack_adjoint_f64.restype = C.c_int
        _lib = L
    return _lib


def _arr(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
    return a, a.ctypes.data_as(_pi64)


class OType:
    """One oracle datatype handle (reference counted on the C side)."""

    __slots__ = ("h",)

    def __init__(self, h):
        if not h:
            raise ValueError("oracle rejected the constructor arguments")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_free(self.h)
            self.h = None

    # ---- attributes ----
    @property
    def size(self) -> int:
        return lib().or_size(self.h)

    @property
    def lb(self) -> int:
        return lib().or_lb(self.h)

    @property
    def extent(self) -> int:
        return lib().or_extent(self.h)

    @property
    def true_lb(self) -> int:
        return lib().or_true_lb(self.h)

    @property
    def true_extent(self) -> int:
        return lib().or_true_extent(self.h)

    # ---- typemap and segments ----
    def typemap(self):
        n = lib().or_typemap_len(self.h)
        d = np.zeros(n, np.int64)
        s = np.zeros(n, np.int64)
        lib().or_typemap(self.h, d.ctypes.data_as(_pi64), s.ctypes.data_as(_pi64))
        return d, s

    def iov_count(self) -> int:
        return lib().or_iov_count(self.h)

    def iov(self, offset: int = 0, max_len: int | None = None):
        if max_len is None:
            max_len = self.iov_count()
        d = np.zeros(max(max_len, 0), np.int64)
        l = np.zeros(max(max_len, 0), np.int64)
        got = lib().or_iov(self.h, offset, max_len, d.ctypes.data_as(_pi64), l.ctypes.data_as(_pi64))
        if got < 0:
            raise ValueError("oracle iov: bad argument")
        return d[:got], l[:got]

    def iov_elements(self, count: int, offset: int = 0, max_len: int | None = None):
        if max_len is None:
            max_len = count * self.iov_count()
        d = np.zeros(max(max_len, 0), np.int64)
        l = np.zeros(max(max_len, 0), np.int64)
        got = lib().or_iov_elements(self.h, count, offset, max_len,
                                    d.ctypes.data_as(_pi64), l.ctypes.data_as(_pi64))
        if got < 0:
            raise ValueError("oracle iov_elements: bad argument")
        return d[:got], l[:got]

    def iov_len(self, max_bytes: int):
        n = _i64(0)
        b = _i64(0)
        rc = lib().or_iov_len(self.h, max_bytes, C.byref(n), C.byref(b))
        if rc != 0:
            raise ValueError("oracle iov_len: bad argument")
        return n.value, b.value

    # ---- data movement ----
    def pack(self, origin: np.ndarray, count: int, base_offset: int = 0) -> np.ndarray:
        """Pack `count` elements whose displacement 0 is origin[base_offset]."""
        buf = np.ascontiguousarray(origin).view(np.uint8).reshape(-1)
        out = np.empty(count * self.size, np.uint8)
        rc = lib().or_pack(buf.ctypes.data + base_offset, count, self.h, out.ctypes.data)
        if rc != 0:
            raise ValueError("oracle pack failed")
        return out

    def unpack(self, packed: np.ndarray, count: int, origin: np.ndarray, base_offset: int = 0):
        """Unpack into `origin` (modified in place) with displacement 0 at base_offset."""
        pk = np.ascontiguousarray(packed).view(np.uint8).reshape(-1)
        assert pk.size >= count * self.size
        buf = origin.view(np.uint8).reshape(-1)
        assert buf.flags.c_contiguous
        rc = lib().or_unpack(pk.ctypes.data, count, self.h, buf.ctypes.data + base_offset)
        if rc != 0:
            raise ValueError("oracle unpack failed")
        return origin

    def pack_range(self, origin: np.ndarray, count: int, first: int, nbytes: int,
                   base_offset: int = 0) -> np.ndarray:
        """Bytes [first, first + nbytes) of the packed stream of `count` elements."""
        buf = np.ascontiguousarray(origin).view(np.uint8).reshape(-1)
        out = np.empty(nbytes, np.uint8)
        rc = lib().or_pack_range(buf.ctypes.data + base_offset, count, self.h, first, nbytes, out.ctypes.data)
        if rc != 0:
            raise ValueError("oracle pack_range: bad argument")
        return out

    def unpack_range(self, packed: np.ndarray, first: int, count: int, origin: np.ndarray,
                     base_offset: int = 0):
        """Unpack packed-stream bytes [first, first + packed.size) into `origin` (in place)."""
        pk = np.ascontiguousarray(packed).view(np.uint8).reshape(-1)
        buf = origin.view(np.uint8).reshape(-1)
        assert buf.flags.c_contiguous
        rc = lib().or_unpack_range(pk.ctypes.data, first, pk.size, count, self.h, buf.ctypes.data + base_offset)
        if rc != 0:
            raise ValueError("oracle unpack_range: bad argument")
        return origin

    def overlaps(self, count: int = 1) -> bool:
        return bool(lib().or_overlaps(self.h, count))

    def pack_adjoint_f64(self, gy: np.ndarray, count: int, gx_len: int):
        """FP64 adjoint of the float32 pack: gx[i] = sum of gy[k] over packed k taken from float i."""
        gy = np.ascontiguousarray(gy, dtype=np.float64)
        gx = np.zeros(gx_len, np.float64)
        rc = lib().or_pack_adjoint_f64(gy.ctypes.data, count, self.h, gx.ctypes.data, gx_len)
        if rc != 0:
            raise ValueError("oracle adjoint: entries must be aligned float32 inside gx")
        return gx


# ---- constructors ----
def basic(size: int, align: int | None = None) -> OType:
    return OType(lib().or_basic(size, size if align is None else align))


def types():
    """The basic types the library exposes, as oracle handles (size, alignment)."""
    return {
        "byte": basic(1, 1), "int8": basic(1, 1), "uint8": basic(1, 1),
        "int16": basic(2, 2), "uint16": basic(2, 2), "int32": basic(4, 4),
        "uint32": basic(4, 4), "int64": basic(8, 8), "uint64": basic(8, 8),
        "float16": basic(2, 2), "bfloat16": basic(2, 2), "float32": basic(4, 4),
        "float64": basic(8, 8),
    }


def contiguous(count, old: OType) -> OType:
    return OType(lib().or_contiguous(count, old.h))


def vector(count, bl, stride, old: OType) -> OType:
    return OType(lib().or_vector(count, bl, stride, old.h))


def hvector(count, bl, stride_bytes, old: OType) -> OType:
    return OType(lib().or_hvector(count, bl, stride_bytes, old.h))


def indexed(bls, disps, old: OType) -> OType:
    b, pb = _arr(bls)
    d, pd = _arr(disps)
    assert b.size == d.size
    return OType(lib().or_indexed(b.size, pb, pd, old.h))


def hindexed(bls, disps_bytes, old: OType) -> OType:
    b, pb = _arr(bls)
    d, pd = _arr(disps_bytes)
    assert b.size == d.size
    return OType(lib().or_hindexed(b.size, pb, pd, old.h))


def indexed_block(bl, disps, old: OType) -> OType:
    d, pd = _arr(disps)
    return OType(lib().or_indexed_block(d.size, bl, pd, old.h))


def hindexed_block(bl, disps_bytes, old: OType) -> OType:
    d, pd = _arr(disps_bytes)
    return OType(lib().or_hindexed_block(d.size, bl, pd, old.h))


def struct(bls, disps_bytes, types_: list) -> OType:
    b, pb = _arr(bls)
    d, pd = _arr(disps_bytes)
    hs = (_p * max(len(types_), 1))(*[t.h for t in types_])
    return OType(lib().or_struct(b.size, pb, pd, hs))


def subarray(sizes, subsizes, starts, old: OType, order: int = ORDER_C) -> OType:
    s, ps = _arr(sizes)
    u, pu = _arr(subsizes)
    t, pt = _arr(starts)
    return OType(lib().or_subarray(s.size, ps, pu, pt, order, old.h))


DIST_BLOCK, DIST_CYCLIC, DIST_NONE = 0, 1, 2
DFLT_DARG = -1


def darray(size, rank, gsizes, distribs, dargs, psizes, old: OType, order: int = ORDER_C) -> OType:
    g, pg = _arr(gsizes)
    a, pa = _arr(dargs)
    ps, pps = _arr(psizes)
    dist = (C.c_int * len(distribs))(*[int(x) for x in distribs])
    return OType(lib().or_darray(size, rank, g.size, pg, dist, pa, pps, order, old.h))


def resized(old: OType, lb: int, extent: int) -> OType:
    return OType(lib().or_resized(old.h, lb, extent))


_BASIC = {"byte": (1, 1), "int8": (1, 1), "uint8": (1, 1), "int16": (2, 2), "uint16": (2, 2),
          "int32": (4, 4), "uint32": (4, 4), "int64": (8, 8), "uint64": (8, 8),
          "float16": (2, 2), "bfloat16": (2, 2), "float32": (4, 4), "float64": (8, 8)}


def from_spec(spec) -> OType:
    """Build an oracle type from a nested spec tuple (see the package's inputs module)."""
    k = spec[0]
    if k == "basic":
        return basic(*_BASIC[spec[1]])
    if k == "contig":
        return contiguous(spec[1], from_spec(spec[2]))
    if k == "vector":
        return vector(spec[1], spec[2], spec[3], from_spec(spec[4]))
    if k == "hvector":
        return hvector(spec[1], spec[2], spec[3], from_spec(spec[4]))
    if k == "indexed":
        return indexed(spec[1], spec[2], from_spec(spec[3]))
    if k == "hindexed":
        return hindexed(spec[1], spec[2], from_spec(spec[3]))
    if k == "indexed_block":
        return indexed_block(spec[1], spec[2], from_spec(spec[3]))
    if k == "hindexed_block":
        return hindexed_block(spec[1], spec[2], from_spec(spec[3]))
    if k == "struct":
        return struct(spec[1], spec[2], [from_spec(c) for c in spec[3]])
    if k == "subarray":
        return subarray(spec[1], spec[2], spec[3], from_spec(spec[5]), spec[4])
    if k == "resized":
        return resized(from_spec(spec[3]), spec[1], spec[2])
    if k == "darray":
        _, size, rank, gs, dist, dargs, ps, order, child = spec
        return darray(size, rank, gs, dist, dargs, ps, from_spec(child), order)
    raise ValueError(f"unknown spec kind {k!r}")
