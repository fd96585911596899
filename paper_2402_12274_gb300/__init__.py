"""GB300 datatype engine: Python binding of ``libdte.so``.

The functions named ``dte_*`` are one-to-one wrappers of the C ABI declared in
``include/dte.h`` (argument marshalling only: every byte is moved and every
segment enumerated by the library's CUDA kernels or its committed
descriptor).  They raise :class:`DteError` instead of returning an error code,
and return out-parameters as Python values.

:class:`Datatype` is a small convenience handle on top of them, and
:func:`pack` / :func:`unpack` accept torch tensors (device memory and streams
come from PyTorch; nothing else does).

The library must have been built (``paper_2402_12274_gb300.build.build()`` or
``__graft_entry__.build()``); importing this module without it raises
ImportError -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

__all__ = [
    "DteError", "Datatype", "pack", "unpack", "lib", "ORDER_C", "ORDER_FORTRAN",
    "BYTE", "INT8", "UINT8", "INT16", "UINT16", "INT32", "UINT32", "INT64", "UINT64",
    "FLOAT16", "BFLOAT16", "FLOAT32", "FLOAT64",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
# DTE_LIBRARY selects another build of the same library (e.g. one compiled
# with different tuning constants); default: the in-tree build.
LIB_PATH = os.environ.get("DTE_LIBRARY") or os.path.join(_HERE, "libdte.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it first with "
        "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc); "
        "the datatype engine has no CPU fallback"
    )

lib = C.CDLL(LIB_PATH)

_i64 = C.c_int64
_pi64 = C.POINTER(C.c_int64)
_p = C.c_void_p
_pp = C.POINTER(C.c_void_p)


class dte_iov(C.Structure):
    _fields_ = [("iov_base", C.c_void_p), ("iov_len", C.c_int64)]


class dte_op(C.Structure):
    _fields_ = [("type", C.c_void_p), ("count", C.c_int64), ("user", C.c_void_p), ("packed", C.c_void_p)]


BATCH_UNPACK, BATCH_PACK = 0, 1


class dte_op_shape(C.Structure):
    _fields_ = [("word", C.c_int32), ("list", C.c_int32), ("single_kernel", C.c_int32),
                ("batch_kernel", C.c_int32), ("bytes", C.c_int64), ("segments", C.c_int64),
                ("max_run", C.c_int64)]


# kernel plans (include/dte.h, enum dte_plan)
PLAN_AUTO, PLAN_CHUNK, PLAN_CHUNK_WIDE, PLAN_SEGMENT, PLAN_BULK = range(5)


class dte_server_config(C.Structure):
    _fields_ = [("ring_slots", C.c_int64), ("max_inflight_bytes", C.c_int64), ("ctas_per_sm", C.c_int32),
                ("span_tiles", C.c_int32), ("idle_exit_us", C.c_int64)]


# error codes (include/dte.h)
SUCCESS, ERR_ARG, ERR_TYPE, ERR_OVERFLOW, ERR_TRUNCATE, ERR_OVERLAP, ERR_NOMEM, ERR_CUDA, \
    ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_NODEVICE = range(11)
ORDER_C, ORDER_FORTRAN = 0, 1


class DteError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        msg = lib.dte_error_string(code).decode()
        super().__init__(f"{where}: {msg} (code {code})" if where else f"{msg} (code {code})")


_SIGS = {
    "dte_error_string": ([C.c_int], C.c_char_p),
    "dte_type_basic": ([C.c_int, _pp], C.c_int),
    "dte_type_contiguous": ([_i64, _p, _pp], C.c_int),
    "dte_type_vector": ([_i64, _i64, _i64, _p, _pp], C.c_int),
    "dte_type_hvector": ([_i64, _i64, _i64, _p, _pp], C.c_int),
    "dte_type_indexed": ([_i64, _pi64, _pi64, _p, _pp], C.c_int),
    "dte_type_hindexed": ([_i64, _pi64, _pi64, _p, _pp], C.c_int),
    "dte_type_indexed_block": ([_i64, _i64, _pi64, _p, _pp], C.c_int),
    "dte_type_hindexed_block": ([_i64, _i64, _pi64, _p, _pp], C.c_int),
    "dte_type_struct": ([_i64, _pi64, _pi64, _pp, _pp], C.c_int),
    "dte_type_subarray": ([C.c_int, _pi64, _pi64, _pi64, C.c_int, _p, _pp], C.c_int),
    "dte_type_resized": ([_p, _i64, _i64, _pp], C.c_int),
    "dte_type_darray": ([C.c_int, C.c_int, C.c_int, _pi64, C.POINTER(C.c_int), _pi64, _pi64, C.c_int, _p, _pp],
                        C.c_int),
    "dte_type_dup": ([_p, _pp], C.c_int),
    "dte_type_commit": ([_pp], C.c_int),
    "dte_type_free": ([_pp], C.c_int),
    "dte_type_size": ([_p, _pi64], C.c_int),
    "dte_type_get_extent": ([_p, _pi64, _pi64], C.c_int),
    "dte_type_get_true_extent": ([_p, _pi64, _pi64], C.c_int),
    "dte_type_num_segments": ([_p, _pi64], C.c_int),
    "dte_type_descriptor_bytes": ([_p, _pi64], C.c_int),
    "dte_type_set_plan": ([_p, C.c_int], C.c_int),
    "dte_type_get_plan": ([_p, C.POINTER(C.c_int)], C.c_int),
    "dte_op_shape_query": ([C.POINTER(dte_op), C.POINTER(dte_op_shape)], C.c_int),
    "dte_type_iov_len": ([_p, _i64, _pi64, _pi64], C.c_int),
    "dte_type_iov": ([_p, _i64, C.POINTER(dte_iov), _i64, _pi64], C.c_int),
    "dte_type_iov_len_async": ([_p, _i64, _p, _p, _p, _p], C.c_int),
    "dte_type_iov_async": ([_p, _i64, _i64, _p, _i64, _p, _p, _p], C.c_int),
    "dte_type_iov_at_bytes_async": ([_p, _i64, _p, _i64, _p, _p, _p, _p, _p], C.c_int),
    "dte_pack_size": ([_i64, _p, _pi64], C.c_int),
    "dte_pack_enqueue": ([_p, _i64, _p, _p, _i64, _pi64, _p], C.c_int),
    "dte_unpack_enqueue": ([_p, _i64, _pi64, _p, _i64, _p, _p], C.c_int),
    "dte_pack_range_enqueue": ([_p, _i64, _p, _i64, _i64, _p, _p], C.c_int),
    "dte_unpack_range_enqueue": ([_p, _i64, _i64, _p, _i64, _p, _p], C.c_int),
    "dte_sendrecv_enqueue": ([_p, _i64, _p, _p, _i64, _p, _p, _i64, _p], C.c_int),
    "dte_device_timeouts": ([_pi64], C.c_int),
    "dte_batch_create": ([C.c_int, _i64, C.POINTER(dte_op), _pp], C.c_int),
    "dte_batch_set_launch": ([_p, C.c_int, _i64], C.c_int),
    "dte_batch_enqueue": ([_p, _p], C.c_int),
    "dte_batch_free": ([_pp], C.c_int),
    "dte_pack_batch_enqueue": ([_i64, C.POINTER(dte_op), _p], C.c_int),
    "dte_unpack_batch_enqueue": ([_i64, C.POINTER(dte_op), _p], C.c_int),
    "dte_pack_batch_enqueue_noalloc": ([_i64, C.POINTER(dte_op), _p], C.c_int),
    "dte_pack_adjoint_f32_enqueue": ([_p, _i64, _p, _p, _p], C.c_int),
    "dte_server_create": ([C.POINTER(dte_server_config), _pp], C.c_int),
    "dte_server_submit": ([_p, C.c_int, C.POINTER(dte_op), _pi64], C.c_int),
    "dte_server_progress": ([_p, _pi64, _pi64], C.c_int),
    "dte_server_test": ([_p, _i64, C.POINTER(C.c_int)], C.c_int),
    "dte_server_wait": ([_p, _i64, _i64], C.c_int),
    "dte_server_free": ([_pp], C.c_int),
}
NOALLOC_MAX_OPS = 256  # DTE_NOALLOC_MAX_OPS in include/dte.h
for _n, (_a, _r) in _SIGS.items():
    _f = getattr(lib, _n)
    _f.argtypes = _a
    _f.restype = _r

EXPORTED = tuple(_SIGS)


def _ck(rc: int, where: str):
    if rc != 0:
        raise DteError(rc, where)


def _arr64(values):
    a = (C.c_int64 * max(len(values), 1))(*[int(v) for v in values])
    return a


# ---------------------------------------------------------------------------
# one-to-one wrappers (handles are plain ints)
# ---------------------------------------------------------------------------
def dte_type_basic(which: int) -> int:
    out = C.c_void_p()
    _ck(lib.dte_type_basic(which, C.byref(out)), "dte_type_basic")
    return out.value


def _ctor(name, *args) -> int:
    out = C.c_void_p()
    _ck(getattr(lib, name)(*args, C.byref(out)), name)
    return out.value


def dte_type_contiguous(count: int, old: int) -> int:
    return _ctor("dte_type_contiguous", count, old)


def dte_type_vector(count: int, bl: int, stride: int, old: int) -> int:
    return _ctor("dte_type_vector", count, bl, stride, old)


def dte_type_hvector(count: int, bl: int, stride_bytes: int, old: int) -> int:
    return _ctor("dte_type_hvector", count, bl, stride_bytes, old)


def _int64_ptr(a):
    """Host int64 array argument: a sequence or a numpy int64 array."""
    try:
        import numpy as np
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.int64)
            return a, a.ctypes.data_as(_pi64), a.size
    except ImportError:  # pragma: no cover
        pass
    arr = _arr64(list(a))
    return arr, C.cast(arr, _pi64), len(a)


def dte_type_indexed(bl, disp, old: int) -> int:
    kb, pb, n = _int64_ptr(bl)
    kd, pd, m = _int64_ptr(disp)
    if n != m:
        raise ValueError("bl and disp differ in length")
    return _ctor("dte_type_indexed", n, pb, pd, old)


def dte_type_hindexed(bl, disp_bytes, old: int) -> int:
    kb, pb, n = _int64_ptr(bl)
    kd, pd, m = _int64_ptr(disp_bytes)
    if n != m:
        raise ValueError("bl and disp differ in length")
    return _ctor("dte_type_hindexed", n, pb, pd, old)


def dte_type_indexed_block(bl: int, disp, old: int) -> int:
    kd, pd, n = _int64_ptr(disp)
    return _ctor("dte_type_indexed_block", n, bl, pd, old)


def dte_type_hindexed_block(bl: int, disp_bytes, old: int) -> int:
    kd, pd, n = _int64_ptr(disp_bytes)
    return _ctor("dte_type_hindexed_block", n, bl, pd, old)


def dte_type_struct(bl, disp_bytes, types) -> int:
    kb, pb, n = _int64_ptr(bl)
    kd, pd, m = _int64_ptr(disp_bytes)
    if not (n == m == len(types)):
        raise ValueError("struct arrays differ in length")
    ts = (C.c_void_p * max(n, 1))(*[int(t) for t in types])
    return _ctor("dte_type_struct", n, pb, pd, ts)


def dte_type_subarray(sizes, subsizes, starts, order: int, old: int) -> int:
    ks, ps, n = _int64_ptr(sizes)
    ku, pu, n2 = _int64_ptr(subsizes)
    kt, pt, n3 = _int64_ptr(starts)
    if not (n == n2 == n3):
        raise ValueError("subarray arrays differ in length")
    return _ctor("dte_type_subarray", n, ps, pu, pt, order, old)


DISTRIBUTE_BLOCK, DISTRIBUTE_CYCLIC, DISTRIBUTE_NONE = 0, 1, 2
DISTRIBUTE_DFLT_DARG = -1


def dte_type_darray(size: int, rank: int, gsizes, distribs, dargs, psizes, order: int, old: int) -> int:
    kg, pg, n = _int64_ptr(gsizes)
    ka, pa, n2 = _int64_ptr(dargs)
    kp, pp, n3 = _int64_ptr(psizes)
    if not (n == n2 == n3 == len(distribs)):
        raise ValueError("darray arrays differ in length")
    dist = (C.c_int * max(n, 1))(*[int(x) for x in distribs])
    return _ctor("dte_type_darray", size, rank, n, pg, dist, pa, pp, order, old)


def dte_type_resized(old: int, lb: int, extent: int) -> int:
    out = C.c_void_p()
    _ck(lib.dte_type_resized(old, lb, extent, C.byref(out)), "dte_type_resized")
    return out.value


def dte_type_dup(old: int) -> int:
    out = C.c_void_p()
    _ck(lib.dte_type_dup(old, C.byref(out)), "dte_type_dup")
    return out.value


def dte_type_commit(t: int) -> int:
    h = C.c_void_p(t)
    _ck(lib.dte_type_commit(C.byref(h)), "dte_type_commit")
    return h.value


def dte_type_free(t: int) -> None:
    h = C.c_void_p(t)
    _ck(lib.dte_type_free(C.byref(h)), "dte_type_free")


def _q1(name, t):
    v = C.c_int64()
    _ck(getattr(lib, name)(t, C.byref(v)), name)
    return v.value


def _q2(name, t):
    a, b = C.c_int64(), C.c_int64()
    _ck(getattr(lib, name)(t, C.byref(a), C.byref(b)), name)
    return a.value, b.value


def dte_type_size(t: int) -> int:
    return _q1("dte_type_size", t)


def dte_type_get_extent(t: int):
    return _q2("dte_type_get_extent", t)


def dte_type_get_true_extent(t: int):
    return _q2("dte_type_get_true_extent", t)


def dte_type_num_segments(t: int) -> int:
    return _q1("dte_type_num_segments", t)


def dte_type_descriptor_bytes(t: int) -> int:
    return _q1("dte_type_descriptor_bytes", t)


def dte_type_set_plan(t: int, plan: int) -> None:
    _ck(lib.dte_type_set_plan(t, plan), "dte_type_set_plan")


def dte_type_get_plan(t: int) -> int:
    v = C.c_int()
    _ck(lib.dte_type_get_plan(t, C.byref(v)), "dte_type_get_plan")
    return v.value


def dte_op_shape_query(t: int, count: int, user: int, packed: int) -> dict:
    """The shape of one operation as the kernels see it (dte_op_shape)."""
    op = dte_op(t, count, user, packed)
    out = dte_op_shape()
    _ck(lib.dte_op_shape_query(C.byref(op), C.byref(out)), "dte_op_shape_query")
    return {f: getattr(out, f) for f, _ in dte_op_shape._fields_}


def dte_type_iov_len(t: int, max_iov_bytes: int):
    n, b = C.c_int64(), C.c_int64()
    _ck(lib.dte_type_iov_len(t, max_iov_bytes, C.byref(n), C.byref(b)), "dte_type_iov_len")
    return n.value, b.value


def dte_type_iov(t: int, iov_offset: int, max_iov_len: int):
    """Returns a list of (iov_base as int displacement, iov_len)."""
    buf = (dte_iov * max(max_iov_len, 1))()
    got = C.c_int64()
    _ck(lib.dte_type_iov(t, iov_offset, buf, max_iov_len, C.byref(got)), "dte_type_iov")
    out = []
    for i in range(got.value):
        base = buf[i].iov_base or 0
        if base >= 1 << 63:
            base -= 1 << 64
        out.append((base, buf[i].iov_len))
    return out


def dte_type_iov_len_async(t: int, n: int, d_budget: int, d_iov_len: int, d_iov_bytes: int, stream: int = 0):
    _ck(lib.dte_type_iov_len_async(t, n, d_budget, d_iov_len, d_iov_bytes, stream), "dte_type_iov_len_async")


def dte_type_iov_async(t: int, count: int, iov_offset: int, d_iov: int, max_iov_len: int,
                       d_actual: int, base: int, stream: int = 0):
    _ck(lib.dte_type_iov_async(t, count, iov_offset, d_iov, max_iov_len, d_actual, base, stream),
        "dte_type_iov_async")


def dte_type_iov_at_bytes_async(t: int, n: int, d_offset: int, max_iov_len: int, d_iov: int,
                                d_first: int, d_actual: int, base: int, stream: int = 0):
    _ck(lib.dte_type_iov_at_bytes_async(t, n, d_offset, max_iov_len, d_iov, d_first, d_actual, base, stream),
        "dte_type_iov_at_bytes_async")


def dte_pack_size(incount: int, t: int) -> int:
    v = C.c_int64()
    _ck(lib.dte_pack_size(incount, t, C.byref(v)), "dte_pack_size")
    return v.value


def dte_pack_enqueue(inbuf: int, incount: int, t: int, outbuf: int, outsize: int, position: int,
                     stream: int = 0) -> int:
    """Returns the advanced position."""
    pos = C.c_int64(position)
    _ck(lib.dte_pack_enqueue(inbuf, incount, t, outbuf, outsize, C.byref(pos), stream), "dte_pack_enqueue")
    return pos.value


def dte_unpack_enqueue(inbuf: int, insize: int, position: int, outbuf: int, outcount: int, t: int,
                       stream: int = 0) -> int:
    """Returns the advanced position."""
    pos = C.c_int64(position)
    _ck(lib.dte_unpack_enqueue(inbuf, insize, C.byref(pos), outbuf, outcount, t, stream),
        "dte_unpack_enqueue")
    return pos.value


def dte_pack_range_enqueue(inbuf: int, incount: int, t: int, first: int, nbytes: int, outbuf: int,
                           stream: int = 0) -> None:
    _ck(lib.dte_pack_range_enqueue(inbuf, incount, t, first, nbytes, outbuf, stream), "dte_pack_range_enqueue")


def dte_unpack_range_enqueue(inbuf: int, first: int, nbytes: int, outbuf: int, outcount: int, t: int,
                             stream: int = 0) -> None:
    _ck(lib.dte_unpack_range_enqueue(inbuf, first, nbytes, outbuf, outcount, t, stream),
        "dte_unpack_range_enqueue")


def dte_sendrecv_enqueue(sendbuf: int, sendcount: int, sendtype: int, recvbuf: int, recvcount: int,
                         recvtype: int, staging: int, staging_bytes: int, stream: int = 0) -> None:
    _ck(lib.dte_sendrecv_enqueue(sendbuf, sendcount, sendtype, recvbuf, recvcount, recvtype, staging,
                                 staging_bytes, stream), "dte_sendrecv_enqueue")


def dte_device_timeouts() -> int:
    n = C.c_int64()
    _ck(lib.dte_device_timeouts(C.byref(n)), "dte_device_timeouts")
    return n.value


def _ops_array(ops):
    """ops: iterable of (type handle, count, user ptr, packed ptr)."""
    ops = list(ops)
    arr = (dte_op * max(len(ops), 1))()
    for i, (t, n, u, p) in enumerate(ops):
        arr[i].type = int(t)
        arr[i].count = int(n)
        arr[i].user = int(u)
        arr[i].packed = int(p)
    return arr, len(ops)


def dte_batch_create(kind: int, ops) -> int:
    arr, n = _ops_array(ops)
    out = C.c_void_p()
    _ck(lib.dte_batch_create(kind, n, arr, C.byref(out)), "dte_batch_create")
    return out.value


def dte_batch_set_launch(batch: int, blocks_per_sm: int, span_tiles: int = 1):
    _ck(lib.dte_batch_set_launch(batch, blocks_per_sm, span_tiles), "dte_batch_set_launch")


def dte_batch_enqueue(batch: int, stream: int = 0):
    _ck(lib.dte_batch_enqueue(batch, stream), "dte_batch_enqueue")


def dte_batch_free(batch: int):
    h = C.c_void_p(batch)
    _ck(lib.dte_batch_free(C.byref(h)), "dte_batch_free")


def dte_pack_batch_enqueue(ops, stream: int = 0):
    arr, n = _ops_array(ops)
    _ck(lib.dte_pack_batch_enqueue(n, arr, stream), "dte_pack_batch_enqueue")


def dte_unpack_batch_enqueue(ops, stream: int = 0):
    arr, n = _ops_array(ops)
    _ck(lib.dte_unpack_batch_enqueue(n, arr, stream), "dte_unpack_batch_enqueue")


def dte_pack_adjoint_f32_enqueue(gy: int, count: int, t: int, gx: int, stream: int = 0):
    """gx[src(k)] += gy[k] for the float32 pack of `count` elements of t."""
    _ck(lib.dte_pack_adjoint_f32_enqueue(gy, count, t, gx, stream), "dte_pack_adjoint_f32_enqueue")


def dte_server_create(ring_slots: int = 1024, max_inflight_bytes: int = 0, ctas_per_sm: int = 4,
                      span_tiles: int = 4, idle_exit_us: int = 50000) -> int:
    cfg = dte_server_config(ring_slots, max_inflight_bytes, ctas_per_sm, span_tiles, idle_exit_us)
    out = C.c_void_p()
    _ck(lib.dte_server_create(C.byref(cfg), C.byref(out)), "dte_server_create")
    return out.value


def dte_server_submit(server: int, kind: int, t: int, count: int, user: int, packed: int) -> int:
    op = dte_op(t, count, user, packed)
    ticket = C.c_int64()
    _ck(lib.dte_server_submit(server, kind, C.byref(op), C.byref(ticket)), "dte_server_submit")
    return ticket.value


def dte_server_progress(server: int):
    a, b = C.c_int64(), C.c_int64()
    _ck(lib.dte_server_progress(server, C.byref(a), C.byref(b)), "dte_server_progress")
    return a.value, b.value


def dte_server_test(server: int, ticket: int) -> bool:
    d = C.c_int()
    _ck(lib.dte_server_test(server, ticket, C.byref(d)), "dte_server_test")
    return bool(d.value)


def dte_server_wait(server: int, ticket: int, timeout_us: int = 10_000_000):
    _ck(lib.dte_server_wait(server, ticket, timeout_us), "dte_server_wait")


def dte_server_free(server: int):
    h = C.c_void_p(server)
    _ck(lib.dte_server_free(C.byref(h)), "dte_server_free")


def dte_pack_batch_enqueue_noalloc(ops, stream: int = 0):
    """Batched pack into a fixed in-library op table (no device allocation);
    see include/dte.h for its limits."""
    arr, n = _ops_array(ops)
    _ck(lib.dte_pack_batch_enqueue_noalloc(n, arr, stream), "dte_pack_batch_enqueue_noalloc")


class Batch:
    """Owning wrapper of a dte_batch (a reusable persistent launch)."""

    def __init__(self, kind: int, ops):
        self.h = dte_batch_create(kind, ops)

    def enqueue(self, stream=None):
        dte_batch_enqueue(self.h, _stream_handle(stream))

    def set_launch(self, blocks_per_sm: int, span_tiles: int = 1):
        dte_batch_set_launch(self.h, blocks_per_sm, span_tiles)

    def free(self):
        if self.h:
            dte_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# convenience layer
# ---------------------------------------------------------------------------
class Datatype:
    """Owning wrapper of a dte_type handle."""

    __slots__ = ("h", "_owned")

    def __init__(self, h: int, owned: bool = True):
        self.h = h
        self._owned = owned

    def __int__(self):
        return int(self.h)

    def __del__(self):
        if getattr(self, "_owned", False) and self.h:
            try:
                dte_type_free(self.h)
            except Exception:
                pass
            self.h = None

    def commit(self) -> "Datatype":
        dte_type_commit(self.h)
        return self

    @property
    def size(self) -> int:
        return dte_type_size(self.h)

    @property
    def lb(self) -> int:
        return dte_type_get_extent(self.h)[0]

    @property
    def extent(self) -> int:
        return dte_type_get_extent(self.h)[1]

    @property
    def true_lb(self) -> int:
        return dte_type_get_true_extent(self.h)[0]

    @property
    def true_extent(self) -> int:
        return dte_type_get_true_extent(self.h)[1]

    @property
    def num_segments(self) -> int:
        return dte_type_num_segments(self.h)

    @property
    def descriptor_bytes(self) -> int:
        return dte_type_descriptor_bytes(self.h)

    def iov_len(self, max_iov_bytes: int):
        return dte_type_iov_len(self.h, max_iov_bytes)

    def iov(self, offset: int = 0, max_len: int | None = None):
        if max_len is None:
            max_len = self.num_segments
        return dte_type_iov(self.h, offset, max_len)

    # constructors
    @staticmethod
    def contiguous(count, old): return Datatype(dte_type_contiguous(count, int(old)))
    @staticmethod
    def vector(count, bl, stride, old): return Datatype(dte_type_vector(count, bl, stride, int(old)))
    @staticmethod
    def hvector(count, bl, stride_bytes, old): return Datatype(dte_type_hvector(count, bl, stride_bytes, int(old)))
    @staticmethod
    def indexed(bl, disp, old): return Datatype(dte_type_indexed(bl, disp, int(old)))
    @staticmethod
    def hindexed(bl, disp_bytes, old): return Datatype(dte_type_hindexed(bl, disp_bytes, int(old)))
    @staticmethod
    def indexed_block(bl, disp, old): return Datatype(dte_type_indexed_block(bl, disp, int(old)))
    @staticmethod
    def hindexed_block(bl, disp_bytes, old): return Datatype(dte_type_hindexed_block(bl, disp_bytes, int(old)))
    @staticmethod
    def struct(bl, disp_bytes, types): return Datatype(dte_type_struct(bl, disp_bytes, [int(t) for t in types]))
    @staticmethod
    def subarray(sizes, subsizes, starts, old, order=ORDER_C):
        return Datatype(dte_type_subarray(sizes, subsizes, starts, order, int(old)))
    @staticmethod
    def resized(old, lb, extent): return Datatype(dte_type_resized(int(old), lb, extent))

    @staticmethod
    def darray(size, rank, gsizes, distribs, dargs, psizes, old, order=ORDER_C):
        return Datatype(dte_type_darray(size, rank, gsizes, distribs, dargs, psizes, order, int(old)))

    def dup(self): return Datatype(dte_type_dup(self.h))

    @staticmethod
    def from_spec(spec) -> "Datatype":
        """Build a (not yet committed) type from a nested spec tuple
        (``inputs`` module format) by calling the constructors."""
        k = spec[0]
        if k == "basic":
            return _BASIC_BY_NAME[spec[1]]
        f = Datatype.from_spec
        if k == "contig":
            return Datatype.contiguous(spec[1], f(spec[2]))
        if k == "vector":
            return Datatype.vector(spec[1], spec[2], spec[3], f(spec[4]))
        if k == "hvector":
            return Datatype.hvector(spec[1], spec[2], spec[3], f(spec[4]))
        if k == "indexed":
            return Datatype.indexed(spec[1], spec[2], f(spec[3]))
        if k == "hindexed":
            return Datatype.hindexed(spec[1], spec[2], f(spec[3]))
        if k == "indexed_block":
            return Datatype.indexed_block(spec[1], spec[2], f(spec[3]))
        if k == "hindexed_block":
            return Datatype.hindexed_block(spec[1], spec[2], f(spec[3]))
        if k == "struct":
            return Datatype.struct(spec[1], spec[2], [f(c) for c in spec[3]])
        if k == "subarray":
            return Datatype.subarray(spec[1], spec[2], spec[3], f(spec[5]), spec[4])
        if k == "resized":
            return Datatype.resized(f(spec[3]), spec[1], spec[2])
        if k == "darray":
            _, size, rank, gs, dist, dargs, ps, order, child = spec
            return Datatype.darray(size, rank, gs, dist, dargs, ps, f(child), order)
        raise ValueError(f"unknown spec kind {k!r}")


def _basic(i):
    return Datatype(dte_type_basic(i), owned=False)


BYTE, INT8, UINT8, INT16, UINT16, INT32, UINT32, INT64, UINT64, FLOAT16, BFLOAT16, FLOAT32, FLOAT64 = \
    [_basic(i) for i in range(13)]
_BASIC_BY_NAME = dict(zip(("byte", "int8", "uint8", "int16", "uint16", "int32", "uint32", "int64", "uint64",
                           "float16", "bfloat16", "float32", "float64"),
                          (BYTE, INT8, UINT8, INT16, UINT16, INT32, UINT32, INT64, UINT64,
                           FLOAT16, BFLOAT16, FLOAT32, FLOAT64)))


def _ptr_nbytes(x):
    """(device pointer, byte size) of a tensor or a raw (ptr, nbytes) pair."""
    if isinstance(x, tuple):
        return int(x[0]), int(x[1])
    return x.data_ptr(), x.numel() * x.element_size()


def _check_span(what: str, nbytes: int, offset: int, count: int, dtype: "Datatype") -> None:
    """`count` elements of `dtype` with displacement 0 at byte `offset` of a
    buffer of `nbytes` bytes must touch only bytes inside it: the kernels
    take raw pointers and cannot check.  Raises ValueError before anything
    is enqueued."""
    if count <= 0 or dtype.size == 0:
        return
    ends = (0, (count - 1) * dtype.extent)
    lo = offset + min(ends) + dtype.true_lb
    hi = offset + max(ends) + dtype.true_lb + dtype.true_extent
    if lo < 0 or hi > nbytes:
        raise ValueError(f"{what}: {count} element(s) of the layout touch bytes [{lo}, {hi}) "
                         f"of a {nbytes}-byte buffer")


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def pack(src, count: int, dtype: Datatype, dst, position: int = 0, stream=None, src_offset: int = 0) -> int:
    """Enqueue a pack of `count` elements of `dtype` whose displacement 0 is
    src + src_offset bytes, into dst at byte `position`.  Returns the new
    position."""
    sp, sn = _ptr_nbytes(src)
    dp, dn = _ptr_nbytes(dst)
    _check_span("pack source", sn, src_offset, count, dtype)
    return dte_pack_enqueue(sp + src_offset, count, dtype.h, dp, dn, position, _stream_handle(stream))


def unpack(src, position: int, dst, count: int, dtype: Datatype, stream=None, dst_offset: int = 0) -> int:
    """Enqueue an unpack from src at byte `position` into `count` elements of
    `dtype` whose displacement 0 is dst + dst_offset bytes.  Returns the new
    position."""
    sp, sn = _ptr_nbytes(src)
    dp, dn = _ptr_nbytes(dst)
    _check_span("unpack destination", dn, dst_offset, count, dtype)
    return dte_unpack_enqueue(sp, sn, position, dp + dst_offset, count, dtype.h, _stream_handle(stream))


def pack_range(src, count: int, dtype: Datatype, first: int, nbytes: int, dst, stream=None,
               src_offset: int = 0, dst_offset: int = 0) -> None:
    """Enqueue packed-stream bytes [first, first + nbytes) of `count` elements
    (displacement 0 at src + src_offset) into dst + dst_offset."""
    sp, sn = _ptr_nbytes(src)
    dp, dn = _ptr_nbytes(dst)
    if dst_offset < 0 or dst_offset + nbytes > dn:
        raise ValueError("pack_range: destination too small")
    _check_span("pack_range source", sn, src_offset, count, dtype)
    dte_pack_range_enqueue(sp + src_offset, count, dtype.h, first, nbytes, dp + dst_offset,
                           _stream_handle(stream))


def unpack_range(src, first: int, nbytes: int, dst, count: int, dtype: Datatype, stream=None,
                 src_offset: int = 0, dst_offset: int = 0) -> None:
    """Enqueue the unpack of packed-stream bytes [first, first + nbytes), read
    from src + src_offset, into `count` elements at dst + dst_offset."""
    sp, sn = _ptr_nbytes(src)
    dp, dn = _ptr_nbytes(dst)
    if src_offset < 0 or src_offset + nbytes > sn:
        raise ValueError("unpack_range: source too small")
    _check_span("unpack_range destination", dn, dst_offset, count, dtype)
    dte_unpack_range_enqueue(sp + src_offset, first, nbytes, dp + dst_offset, count, dtype.h,
                             _stream_handle(stream))


def sendrecv(send, sendcount: int, sendtype: Datatype, recv, recvcount: int, recvtype: Datatype, staging,
             stream=None, send_offset: int = 0, recv_offset: int = 0) -> None:
    """Enqueue the windowed send-to-self pipeline (pack -> copy -> unpack per
    window) from `send` to `recv` through the device buffer `staging`."""
    sp, sn = _ptr_nbytes(send)
    rp, rn = _ptr_nbytes(recv)
    gp, gn = _ptr_nbytes(staging)
    _check_span("sendrecv send buffer", sn, send_offset, sendcount, sendtype)
    _check_span("sendrecv receive buffer", rn, recv_offset, recvcount, recvtype)
    dte_sendrecv_enqueue(sp + send_offset, sendcount, sendtype.h, rp + recv_offset, recvcount, recvtype.h,
                         gp, gn, _stream_handle(stream))
