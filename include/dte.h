/*
 * dte.h -- GB300 datatype engine: the C ABI.
 *
 * A derived datatype describes a memory layout (arxiv 2402.12274, §3
 * "Derived Datatypes").  This library builds such types with MPI-style
 * constructors, commits them into a compact device descriptor, answers the
 * paper's segment ("iov") queries (§3.1 MPIX_Type_iov_len / MPIX_Type_iov)
 * and packs / unpacks non-contiguous buffers with sm_103a kernels that are
 * enqueued on a caller-supplied CUDA stream (the stream-enqueue semantics of
 * §5: work is ordered by the stream, nothing synchronises the host).
 *
 * Conventions for every call below:
 *   - Every call returns an int: DTE_SUCCESS (0) or one of DTE_ERR_*.  No
 *     call aborts; out-parameters are written only on success.
 *   - Counts, sizes, displacements, strides and offsets are int64_t byte
 *     counts unless the parameter says "in extents of old".
 *   - dte_type handles are opaque, library owned and reference counted.
 *     Constructors return a new, uncommitted handle in *out; release it with
 *     dte_type_free.  A constructed type keeps what it needs from its inputs,
 *     so the inputs may be freed right after the constructor returns.
 *     Predefined (basic) handles from dte_type_basic are never freed.
 *   - Buffers are caller owned.  Device buffers must stay valid until the
 *     stream has executed the enqueued operation (CUDA stream semantics).
 *   - Streams are CUDA runtime streams (cudaStream_t); NULL is the legacy
 *     default stream.  Enqueue calls return as soon as the work is queued.
 *   - Thread safety: distinct handles may be used from distinct threads;
 *     concurrent calls on one handle must be serialised by the caller.
 */
#ifndef DTE_H
#define DTE_H

#include <stdint.h>

#if defined(__GNUC__)
#define DTE_API __attribute__((visibility("default")))
#else
#define DTE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                         /* == cudaStream_t's pointee */
typedef struct CUstream_st *dte_stream_t;   /* interchangeable with cudaStream_t */

typedef struct dte_type_s *dte_type;

/* One segment: a base address and a byte length.  Same layout as
 * struct iovec and MPIX_Iov (§3.1). */
typedef struct dte_iov {
    void *iov_base;
    int64_t iov_len;
} dte_iov;

enum dte_error {
    DTE_SUCCESS = 0,
    DTE_ERR_ARG = 1,          /* null pointer, negative count, bad enum, ... */
    DTE_ERR_TYPE = 2,         /* freed/invalid handle, or not committed      */
    DTE_ERR_OVERFLOW = 3,     /* a byte count or displacement exceeds int64   */
    DTE_ERR_TRUNCATE = 4,     /* output buffer smaller than the data         */
    DTE_ERR_OVERLAP = 5,      /* unpack target layout writes a byte twice    */
    DTE_ERR_NOMEM = 6,        /* host or device allocation failed            */
    DTE_ERR_CUDA = 7,         /* a CUDA runtime call failed                  */
    DTE_ERR_TIMEOUT = 8,      /* a bounded device wait gave up               */
    DTE_ERR_UNSUPPORTED = 9,  /* a limit of this implementation was exceeded */
    DTE_ERR_NODEVICE = 10     /* the call needs a CUDA device and none exists */
};

/* Basic types: (size, natural alignment) in bytes. */
enum dte_basic {
    DTE_BYTE = 0,      /* 1, 1 */
    DTE_INT8,          /* 1, 1 */
    DTE_UINT8,         /* 1, 1 */
    DTE_INT16,         /* 2, 2 */
    DTE_UINT16,        /* 2, 2 */
    DTE_INT32,         /* 4, 4 */
    DTE_UINT32,        /* 4, 4 */
    DTE_INT64,         /* 8, 8 */
    DTE_UINT64,        /* 8, 8 */
    DTE_FLOAT16,       /* 2, 2 (not an MPI type; moved as bytes) */
    DTE_BFLOAT16,      /* 2, 2 (not an MPI type; moved as bytes) */
    DTE_FLOAT32,       /* 4, 4 */
    DTE_FLOAT64,       /* 8, 8 */
    DTE_NBASIC
};

enum dte_order { DTE_ORDER_C = 0, DTE_ORDER_FORTRAN = 1 };
enum dte_distribute { DTE_DISTRIBUTE_BLOCK = 0, DTE_DISTRIBUTE_CYCLIC = 1, DTE_DISTRIBUTE_NONE = 2 };
#define DTE_DISTRIBUTE_DFLT_DARG (-1)

/* Human-readable name of an error code (static storage, never NULL). */
DTE_API const char *dte_error_string(int code);

/* ------------------------------------------------------------------------
 * Type constructors (§3: types nest arbitrarily, carry offsets and may
 * overlap; the paper's example uses contiguous and subarray, §3.2).
 * Typemap order and lb/ub follow the MPI constructor definitions; a
 * constructed type's lb/ub is the min/max over its copies of (copy
 * displacement + child lb/ub), where explicit bounds (resized, subarray)
 * take precedence, and a struct without an explicit ub has its extent
 * rounded up to its largest basic alignment.
 * ------------------------------------------------------------------------ */

/* Predefined handle for a basic type (DTE_ERR_ARG if `which` is invalid). */
DTE_API int dte_type_basic(int which, dte_type *out);

/* count copies of old, each at i * extent(old). */
DTE_API int dte_type_contiguous(int64_t count, dte_type old, dte_type *out);

/* count blocks of bl copies of old; block i starts at i*stride extents of
 * old (stride may be negative or zero). */
DTE_API int dte_type_vector(int64_t count, int64_t bl, int64_t stride, dte_type old, dte_type *out);

/* as vector, but stride_bytes is a byte stride. */
DTE_API int dte_type_hvector(int64_t count, int64_t bl, int64_t stride_bytes, dte_type old, dte_type *out);

/* count blocks; block i is bl[i] copies of old starting at disp[i] extents
 * of old.  bl[] and disp[] are host arrays of `count` entries, read during
 * the call only. */
DTE_API int dte_type_indexed(int64_t count, const int64_t *bl, const int64_t *disp,
                     dte_type old, dte_type *out);

/* as indexed, with byte displacements. */
DTE_API int dte_type_hindexed(int64_t count, const int64_t *bl, const int64_t *disp_bytes,
                      dte_type old, dte_type *out);

/* as indexed with every block length equal to bl. */
DTE_API int dte_type_indexed_block(int64_t count, int64_t bl, const int64_t *disp,
                           dte_type old, dte_type *out);

/* as hindexed with every block length equal to bl. */
DTE_API int dte_type_hindexed_block(int64_t count, int64_t bl, const int64_t *disp_bytes,
                            dte_type old, dte_type *out);

/* count blocks; block i is bl[i] copies of types[i] at byte disp[i]. */
DTE_API int dte_type_struct(int64_t count, const int64_t *bl, const int64_t *disp_bytes,
                    const dte_type *types, dte_type *out);

/* An ndims-dimensional sub-block (subsizes at starts) of a full array
 * (sizes) of old, in C (last index fastest) or Fortran order; lb = 0 and
 * extent = prod(sizes) * extent(old).  ndims <= 32. */
DTE_API int dte_type_subarray(int ndims, const int64_t *sizes, const int64_t *subsizes,
                      const int64_t *starts, int order, dte_type old, dte_type *out);

/* Distributed array (MPI's darray): the part of an ndims-dimensional global
 * array (gsizes, elements of old) owned by process `rank` of a row-major
 * process grid psizes (prod(psizes) == size).  Per dimension, distribs[d] is
 * DTE_DISTRIBUTE_BLOCK (one block of dargs[d] indices, default
 * ceil(g/p)), DTE_DISTRIBUTE_CYCLIC (blocks of dargs[d], default 1, dealt
 * round-robin) or DTE_DISTRIBUTE_NONE (the whole dimension; psizes[d] must
 * be 1); DTE_DISTRIBUTE_DFLT_DARG selects the default.  Elements follow the
 * array order (C or Fortran); lb = 0, extent = prod(gsizes)*extent(old). */
DTE_API int dte_type_darray(int size, int rank, int ndims, const int64_t *gsizes, const int *distribs,
                            const int64_t *dargs, const int64_t *psizes, int order, dte_type old,
                            dte_type *out);

/* Same typemap as old with lb and extent replaced. */
DTE_API int dte_type_resized(dte_type old, int64_t lb, int64_t extent, dte_type *out);

/* A new handle for the same type (committed if old is). */
DTE_API int dte_type_dup(dte_type old, dte_type *out);

/* Commit (MPI_Type_commit, which the paper's §3.2 example calls before its
 * iov queries; §3 notes that a type describes its layout in O(1) where an
 * explicit iovec list costs one entry per segment): lower the type into its
 * device descriptor (merged contiguous runs, per-level counts and strides,
 * index tables with prefix sums) and upload it to the current CUDA device
 * when one exists (other devices are uploaded on first use).  *type is the
 * handle to commit (unchanged on return).  Required before any query or data
 * movement.  Idempotent.  DTE_ERR_ARG for a NULL pointer, DTE_ERR_TYPE for an
 * invalid handle, DTE_ERR_NOMEM / DTE_ERR_CUDA if the upload fails. */
DTE_API int dte_type_commit(dte_type *type);

/* Release a handle and set *type = NULL (MPI_Type_free, the last call of the
 * §3.2 example; under §5's stream-enqueue semantics a free must not cut short
 * work already queued on a stream).  Device memory of the descriptor is kept
 * until every operation enqueued with the type has completed (checked with
 * CUDA events); for a type used inside CUDA graph capture it is kept until
 * process exit.  Freeing a predefined handle is DTE_ERR_TYPE; a NULL pointer
 * is DTE_ERR_ARG. */
DTE_API int dte_type_free(dte_type *type);

/* ------------------------------------------------------------------------
 * Attributes (committed or not).  §3.1 defines the iov queries in terms of
 * a type's bytes (iov_len counts segment bytes up to the type's size), and
 * the typemap bounds that place consecutive elements come from the MPI
 * constructor rules the paper builds on (§3).  Each call writes host int64
 * out-parameters; DTE_ERR_ARG for NULL out-pointers, DTE_ERR_TYPE for an
 * invalid handle.
 * ------------------------------------------------------------------------ */
/* Bytes of data in one element (sum of its typemap entries' sizes). */
DTE_API int dte_type_size(dte_type type, int64_t *size);
/* lb and extent = ub - lb: element e of a count starts at e*extent. */
DTE_API int dte_type_get_extent(dte_type type, int64_t *lb, int64_t *extent);
/* Lowest byte touched and the span up to one past the highest, ignoring
 * explicit (resized/subarray) bounds. */
DTE_API int dte_type_get_true_extent(dte_type type, int64_t *true_lb, int64_t *true_extent);
/* Number of merged segments of one element (the total of §3.1 iov_len). */
DTE_API int dte_type_num_segments(dte_type type, int64_t *nseg);
/* Bytes of the committed device descriptor (one copy per device that used
 * the type).  DTE_ERR_TYPE if the type is not committed. */
DTE_API int dte_type_descriptor_bytes(dte_type type, int64_t *bytes);

/* ------------------------------------------------------------------------
 * Segment queries, §3.1.  A segment is a maximal run of typemap entries
 * each starting exactly where the previous one ends, in typemap order.
 * ------------------------------------------------------------------------ */

/* MPIX_Type_iov_len: *iov_len = number of whole segments, counted from the
 * first, whose bytes fit in max_iov_bytes; *actual_iov_bytes = their bytes.
 * max_iov_bytes == -1 or >= size gives every segment.  Values below -1 are
 * DTE_ERR_ARG.  Runs on the host over the committed descriptor, O(depth *
 * log(entries)). */
DTE_API int dte_type_iov_len(dte_type type, int64_t max_iov_bytes, int64_t *iov_len,
                     int64_t *actual_iov_bytes);

/* MPIX_Type_iov: segments [iov_offset, iov_offset + max_iov_len) of one
 * element, written to the host array iov[]; iov_base is the segment's byte
 * displacement from the buffer origin, cast to a pointer.  An offset at or
 * past the end gives *actual_iov_len = 0.  Negative arguments: DTE_ERR_ARG. */
DTE_API int dte_type_iov(dte_type type, int64_t iov_offset, dte_iov *iov, int64_t max_iov_len,
                 int64_t *actual_iov_len);

/* Device form of MPIX_Type_iov_len for a batch of n byte budgets: d_budget,
 * d_iov_len and d_iov_bytes are device arrays of n int64.  A budget below -1
 * yields -1 in both outputs.  Enqueued on `stream`. */
DTE_API int dte_type_iov_len_async(dte_type type, int64_t n, const int64_t *d_budget,
                           int64_t *d_iov_len, int64_t *d_iov_bytes, dte_stream_t stream);

/* Device form of MPIX_Type_iov over `count` elements laid out at the extent
 * (element e's segments shifted by e*extent, nothing merged across
 * elements): writes segments [iov_offset, iov_offset + max_iov_len) to the
 * device array d_iov with iov_base = base + displacement, and the number
 * written to the device int64 *d_actual_iov_len (may be NULL).  `base` is
 * only added, never dereferenced.  Enqueued on `stream`. */
DTE_API int dte_type_iov_async(dte_type type, int64_t count, int64_t iov_offset, dte_iov *d_iov,
                       int64_t max_iov_len, int64_t *d_actual_iov_len, const void *base,
                       dte_stream_t stream);

/* Device form of the byte-offset lookup the paper suggests doing with
 * iov_len (§3.1, "bisect the byte offset of an arbitrary segment"): for each
 * of n packed byte offsets d_offset[q] (0 <= offset < size of one element),
 * write up to max_iov_len segments starting with the segment that contains
 * that byte to d_iov[q * max_iov_len ...], the starting segment index to
 * d_first[q] and the number written to d_actual[q].  Out-of-range offsets
 * give d_first[q] = -1 and d_actual[q] = 0.  Enqueued on `stream`. */
DTE_API int dte_type_iov_at_bytes_async(dte_type type, int64_t n, const int64_t *d_offset,
                                int64_t max_iov_len, dte_iov *d_iov, int64_t *d_first,
                                int64_t *d_actual, const void *base, dte_stream_t stream);

/* ------------------------------------------------------------------------
 * Data movement (the datatype-engine half of §5.2's stream-enqueued
 * send/recv of (buf, count, datatype)).
 * ------------------------------------------------------------------------ */

/* Bytes needed to pack incount elements: incount * size. */
DTE_API int dte_pack_size(int64_t incount, dte_type type, int64_t *size);

/* Gather incount elements of `type` (element e at inbuf + e*extent) into the
 * contiguous outbuf at byte *position, then advance *position (on the host,
 * at enqueue time).  inbuf/outbuf are device (or device-accessible pinned
 * host) pointers; *position is a host int64.  DTE_ERR_TRUNCATE if
 * outsize - *position < incount*size.  Bytes are copied verbatim (no value
 * conversion).  Enqueued on `stream`; returns without waiting. */
DTE_API int dte_pack_enqueue(const void *inbuf, int64_t incount, dte_type type, void *outbuf,
                     int64_t outsize, int64_t *position, dte_stream_t stream);

/* Scatter outcount elements from inbuf at byte *position into outbuf
 * (element e at outbuf + e*extent), then advance *position.
 * DTE_ERR_TRUNCATE if insize - *position < outcount*size; DTE_ERR_OVERLAP if
 * two typemap bytes of the outcount elements coincide.  Enqueued on
 * `stream`. */
DTE_API int dte_unpack_enqueue(const void *inbuf, int64_t insize, int64_t *position, void *outbuf,
                       int64_t outcount, dte_type type, dte_stream_t stream);

/* Partial movement: only bytes [first, first + nbytes) of the packed stream
 * of incount (outcount) elements, i.e. what a full pack would write at those
 * positions (§3.1: the iov queries address a typemap by packed byte offset).
 * outbuf (pack) / inbuf (unpack) holds just the nbytes window, packed byte
 * `first` at offset 0.  A window may start and end anywhere, inside a
 * segment too; windows that tile [0, count*size) in any order reproduce the
 * full pack or unpack.  DTE_ERR_ARG for negative arguments or a window past
 * count*size; DTE_ERR_OVERLAP (unpack) as for dte_unpack_enqueue.  Device
 * pointers, enqueued on `stream`, no host synchronisation. */
DTE_API int dte_pack_range_enqueue(const void *inbuf, int64_t incount, dte_type type, int64_t first,
                                   int64_t nbytes, void *outbuf, dte_stream_t stream);
DTE_API int dte_unpack_range_enqueue(const void *inbuf, int64_t first, int64_t nbytes, void *outbuf,
                                     int64_t outcount, dte_type type, dte_stream_t stream);

/* Send-to-self through the enqueue path of §5.2 (MPIX_Send_enqueue paired
 * with MPIX_Recv_enqueue, here on one GPU and one stream): the message
 * packed from (sendbuf, sendcount, sendtype) is delivered into (recvbuf,
 * recvcount, recvtype) -- the first sendcount*size(sendtype) bytes of the
 * receive stream, the rest of recvbuf untouched.  The message moves in
 * windows of W = (staging_bytes / 2) rounded down to 16 bytes, each cut at
 * the last segment boundary of the send layout within W (the byte form of
 * the iov-length query, §3.1) unless one segment is longer than W; every
 * window is packed into staging[0, W), copied to staging[W, 2W) (the
 * transfer) and unpacked from there, in stream order.  `staging` is a
 * caller-owned device buffer of staging_bytes (>= 32) that must not be used
 * by other work until the stream passes this call.  DTE_ERR_TRUNCATE if the
 * receive side holds fewer bytes than the message; DTE_ERR_OVERLAP if the
 * receive layout writes a byte twice; DTE_ERR_ARG for negative counts, null
 * pointers or staging_bytes < 32. */
DTE_API int dte_sendrecv_enqueue(const void *sendbuf, int64_t sendcount, dte_type sendtype, void *recvbuf,
                                 int64_t recvcount, dte_type recvtype, void *staging, int64_t staging_bytes,
                                 dte_stream_t stream);

/* Adjoint of a float32 pack (the backward of `packed = pack(x)` in a
 * differentiable solver's halo gather; overlapping layouts are describable,
 * §3): for every packed float k read from float src(k) of the user layout,
 * gx[src(k)] += gy[k].  gy holds count*size/4 floats; gx is the user-layout
 * origin (element e at gx + e*extent), both device pointers, 4-byte aligned,
 * and every run of the type must be whole floats (DTE_ERR_ARG otherwise).
 * Layouts without repeated bytes scatter-add one term per destination
 * (bit-exact: gx + gy[k]).  Layouts that repeat bytes sum each
 * destination's terms in packed order in FP64 and add the rounded sum
 * (deterministic; the inverse is built on the host and uploaded on first use
 * for a given (type, count, device) and cached with the type).  Enqueued on
 * `stream`. */
DTE_API int dte_pack_adjoint_f32_enqueue(const void *gy, int64_t count, dte_type type, void *gx,
                                         dte_stream_t stream);

/* ------------------------------------------------------------------------
 * Batches: many independent pack (or unpack) operations in one persistent
 * kernel launch.  The paper's motivation for stream-enqueued operations is
 * to take launch and synchronisation cost off the critical path (§4, §5);
 * a batch removes the per-operation launch as well.
 * ------------------------------------------------------------------------ */

/* One operation of a batch.  `user` is the user-layout origin (element e at
 * user + e*extent): the source of a pack, the destination of an unpack.
 * `packed` is the contiguous side with any byte position already applied:
 * it receives (pack) or supplies (unpack) count*size bytes. */
typedef struct dte_op {
    dte_type type;     /* committed */
    int64_t count;     /* elements, >= 0 */
    void *user;
    void *packed;
} dte_op;

typedef struct dte_batch_s *dte_batch;
enum dte_batch_kind { DTE_BATCH_UNPACK = 0, DTE_BATCH_PACK = 1 };

/* Validate `nops` operations, resolve their descriptors on the current
 * device and upload the op table (device memory owned by the batch).  The
 * ops array is read during the call only; the types may be freed afterwards
 * (the batch keeps their descriptors).  Unpack batches reject an op whose own
 * target layout overlaps (DTE_ERR_OVERLAP).  Ops of one batch run
 * concurrently: their output ranges must not overlap, except where they write
 * identical bytes. */
DTE_API int dte_batch_create(int kind, int64_t nops, const dte_op *ops, dte_batch *out);

/* Launch shape of a batch: at most blocks_per_sm CTAs of 256 threads per SM
 * (0 = as many as fit), and span_tiles consecutive tiles (1 KiB of packed data
 * for 16-byte copy words, 2 KiB otherwise, or 32-segment rounds) taken by a
 * warp at a time (warps take spans in a spread order).  Used by the autotuner;
 * the defaults are (0, 1).  DTE_ERR_ARG for negative/zero values. */
DTE_API int dte_batch_set_launch(dte_batch batch, int blocks_per_sm, int64_t span_tiles);

/* Enqueue every operation of the batch as one kernel on `stream`.  Performs
 * no allocation or host copy, so it may be captured into a CUDA graph and
 * replayed; a batch used under capture is kept until process exit. */
DTE_API int dte_batch_enqueue(dte_batch batch, dte_stream_t stream);

/* Release a batch and set *batch = NULL; device memory is kept until the
 * enqueued launches have completed. */
DTE_API int dte_batch_free(dte_batch *batch);

/* One-shot forms: create, enqueue on `stream`, free. */
DTE_API int dte_pack_batch_enqueue(int64_t nops, const dte_op *ops, dte_stream_t stream);
DTE_API int dte_unpack_batch_enqueue(int64_t nops, const dte_op *ops, dte_stream_t stream);

/* ------------------------------------------------------------------------
 * Kernel plans.  The paper's §5 enqueues (buf, count, datatype) operations
 * and leaves how the datatype engine moves them to the implementation; a
 * plan picks among this library's ways of moving one type.  A batch or a
 * single move reads the plan of each operation's type when it is created or
 * enqueued.  The default, DTE_PLAN_AUTO, is a fixed rule: segment-major for
 * copy words below 16 bytes with runs of at most 4 KiB and a mean run of at
 * most 512 bytes under an index list of more than 32 entries; TMA bulk
 * copies for single moves of runs averaging at least 2 KiB with 16-byte
 * words between device buffers, large enough to give every warp of a
 * one-CTA-per-SM grid six 16 KiB tiles; chunk-major otherwise.  An
 * autotuner that measures layouts of each shape picks a plan per type.  A
 * plan that does not apply to a move (segment-major with 16-byte words or
 * runs over 4 KiB, the wide step with smaller words, bulk copies inside
 * batches or outside device memory) leaves that move to the fixed rule.
 * ------------------------------------------------------------------------ */
enum dte_plan {
    DTE_PLAN_AUTO = 0,        /* the fixed rule above */
    DTE_PLAN_CHUNK = 1,       /* chunk-major: 16-byte packed chunks, 1 KiB warp steps for 16-byte words */
    DTE_PLAN_CHUNK_WIDE = 2,  /* chunk-major with 2 KiB warp steps for 16-byte words */
    DTE_PLAN_SEGMENT = 3,     /* segment-major: rounds of 32 runs, one descriptor walk per run */
    DTE_PLAN_BULK = 4         /* TMA bulk copies of 16 KiB tiles (single moves between device buffers) */
};

/* Set the plan of a type handle (any DTE_PLAN_*; DTE_ERR_ARG otherwise;
 * DTE_ERR_TYPE for a predefined handle).  Affects moves enqueued and
 * batches created afterwards; dte_type_dup copies it.  A type starts with
 * DTE_PLAN_AUTO, or with the plan named by the environment variable
 * DTE_PLAN (auto, chunk, chunk_wide, segment or bulk; read once per process)
 * when it is committed with DTE_PLAN_AUTO still set. */
DTE_API int dte_type_set_plan(dte_type type, int plan);
DTE_API int dte_type_get_plan(dte_type type, int *plan);

/* The shape of one operation as the kernels see it, for tuners that group
 * operations by shape. */
typedef struct dte_op_shape {
    int32_t word;          /* copy word in bytes: 16, 8, 4, 2 or 1 */
    int32_t list;          /* 1 if the layout has an index list of more than 32 entries */
    int32_t single_kernel; /* DTE_PLAN_CHUNK, _CHUNK_WIDE, _SEGMENT or _BULK: what a single move takes now */
    int32_t batch_kernel;  /* DTE_PLAN_CHUNK, _CHUNK_WIDE or _SEGMENT: what it takes inside a batch */
    int64_t bytes;         /* packed bytes (count * size) */
    int64_t segments;      /* runs over the count elements (count * segments of one element) */
    int64_t max_run;       /* longest run in bytes */
} dte_op_shape;

/* Describe `op` (a committed type, count, user and packed pointers as in a
 * batch; the pointers are only inspected, never dereferenced, except that a
 * bulk-copy decision asks the CUDA runtime whether both are device memory).
 * DTE_ERR_TYPE for an invalid or uncommitted type, DTE_ERR_ARG for NULL
 * pointers or a negative count. */
DTE_API int dte_op_shape_query(const dte_op *op, dte_op_shape *out);

/* Largest nops accepted by dte_pack_batch_enqueue_noalloc. */
#define DTE_NOALLOC_MAX_OPS 256

/* Batched pack that allocates no device memory.  This entry point has no
 * counterpart in the paper; it exists for callers that must not allocate
 * while they enqueue work -- code whose device memory is already reserved in
 * full by a caching allocator, latency-bound or signal-driven paths that
 * cannot wait on the allocator, libraries handed a stream but not allowed to
 * touch the device heap.  Same result as dte_pack_batch_enqueue.
 *
 * The op table goes into one fixed array of about 45 KB inside the library
 * (held on every GPU that loads the library until the process exits)
 * instead of memory from cudaMalloc.  Limits and rules:
 *   - nops <= DTE_NOALLOC_MAX_OPS, else DTE_ERR_UNSUPPORTED (nothing queued);
 *   - every type must be committed with the current device current (commit
 *     uploads its descriptor; an op whose descriptor is not yet on this device
 *     gives DTE_ERR_TYPE instead of an upload);
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and should come before any stream capture;
 *   - a call made while `stream` is being captured returns
 *     DTE_ERR_UNSUPPORTED and queues nothing: the table is copied from a host
 *     array that the next call rewrites, so a recorded copy would later read
 *     the wrong table;
 *   - devices 0..63 only (the per-device address cache has 64 entries); a
 *     higher device index gives DTE_ERR_UNSUPPORTED;
 *   - all calls on a device share the array and it keeps the last call's
 *     table: two calls whose work overlaps on the GPU (different streams, or
 *     a call issued before the previous one's kernels have read their table)
 *     race -- serialise them on one stream.  The call writes every entry its
 *     kernels read, so nothing needs clearing beforehand;
 *   - the types must stay alive until the stream has executed the call (no
 *     completion events are recorded, as creating them could allocate).
 * Returns as soon as the work is queued on `stream`. */
DTE_API int dte_pack_batch_enqueue_noalloc(int64_t nops, const dte_op *ops, dte_stream_t stream);

/* Number of bounded device waits that gave up on the current device since
 * the library was loaded.  The bulk-copy kernels wait on shared-memory
 * barriers with a time budget of about a second; a wait that runs out is
 * counted here and the kernel drains what it issued and returns instead of
 * hanging.  A request-loop warp whose tile search keeps finding nothing for
 * the loop's idle budget is counted too (it keeps its claim for the next
 * launch and leaves).  Synchronises with the device.  Expected to stay 0. */
DTE_API int dte_device_timeouts(int64_t *count);

/* ------------------------------------------------------------------------
 * Request loop: a device-resident stand-in for the progress engine (§7
 * general progress, §2 polled generalized requests, §5 work executed in the
 * GPU's own context).  One persistent kernel keeps taking pack/unpack
 * requests as the host admits them, so requests of mixed sizes that arrive
 * while others are running are batched continuously instead of launched one
 * by one.  Admission is first-come first-served under a byte cap and a ring
 * of device slots.  On the device, requests are queued by direction and
 * kernel variant, and the loop's warps drain one such group at a time, so
 * requests admitted together may finish out of submission order.  Requests run without stream ordering: their inputs must
 * be ready (e.g. the producing stream synchronised) when submitted, and
 * their buffers and types must stay valid until they complete.  The loop
 * leaves after `idle_exit_us` without work and is relaunched by the next
 * submit/progress call; every device wait is bounded.
 * ------------------------------------------------------------------------ */
typedef struct dte_server_s *dte_server;

typedef struct dte_server_config {
    int64_t ring_slots;          /* requests admitted at once; power of two <= 2^20 (default 1024) */
    int64_t max_inflight_bytes;  /* cap on moved bytes (2*count*size) of admitted, unfinished
                                    requests; a larger request is admitted alone.  0 = the
                                    default: DTE_SERVE_MAX_INFLIGHT_BYTES from the environment
                                    (a positive integer) if set, else 8 GiB */
    int32_t ctas_per_sm;         /* persistent CTAs per SM, 1 to 4 (default 4) */
    int32_t span_tiles;          /* fewest tiles (1-2 KiB, or 32-segment rounds) a warp claims at once,
                                    1..65536; claims grow to 64 while many published tiles are
                                    unclaimed (default 4) */
    int64_t idle_exit_us;        /* empty-poll budget before the loop leaves (default 50000) */
} dte_server_config;

/* Create a request loop on the current device (cfg NULL = defaults).  Allocates
 * the ring and control words in pinned host memory, a small device state,
 * and its own non-blocking stream.  DTE_ERR_ARG for invalid settings. */
DTE_API int dte_server_create(const dte_server_config *cfg, dte_server *out);

/* Queue one request (kind DTE_BATCH_PACK or DTE_BATCH_UNPACK, one dte_op) and
 * return its ticket (tickets count up from 0 in submission order).  Admits it
 * at once if capacity allows, else keeps it queued on the host.  Never
 * blocks.  Unpack requests into an overlapping layout: DTE_ERR_OVERLAP; a
 * request of more than 2^30 tiles: DTE_ERR_UNSUPPORTED. */
DTE_API int dte_server_submit(dte_server s, int kind, const dte_op *op, int64_t *ticket);

/* Account completions, admit queued requests, relaunch the loop if needed;
 * report requests on the device (*inflight) and queued on the host (*queued).
 * Either pointer may be NULL. */
DTE_API int dte_server_progress(dte_server s, int64_t *inflight, int64_t *queued);

/* *done = 1 if the ticket's request has completed (its bytes are in place). */
DTE_API int dte_server_test(dte_server s, int64_t ticket, int *done);

/* Drive progress until the ticket completes or timeout_us elapses
 * (DTE_ERR_TIMEOUT). */
DTE_API int dte_server_wait(dte_server s, int64_t ticket, int64_t timeout_us);

/* Stop the loop (it leaves at its next poll), wait for it, release
 * everything and set *s = NULL.  Requests not yet completed are abandoned. */
DTE_API int dte_server_free(dte_server *s);

#ifdef __cplusplus
}
#endif
#endif /* DTE_H */
