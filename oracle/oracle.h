/*
 * oracle.h -- plain CPU reference for the derived-datatype engine.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct typemap
 * walker that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or includes anything from here, and
 * nothing here includes anything from the product library.
 *
 * What it computes (paper §3 "Derived Datatypes", §3.1 "Extension"):
 *   - the typemap of a derived datatype built from the MPI constructors the
 *     paper uses (contiguous, subarray) and the usual companions (vector,
 *     hvector, indexed, hindexed, indexed_block, hindexed_block, struct,
 *     resized, darray), expanded one basic entry at a time in constructor
 *     order;
 *   - size, lb/ub/extent and true lb/extent by the MPI constructor rules;
 *   - the segment ("iov") list: the typemap walked in order, an entry merged
 *     into the current segment only when it starts exactly where that segment
 *     ends (never reordered);
 *   - MPIX_Type_iov_len / MPIX_Type_iov semantics (§3.1);
 *   - pack / unpack of `count` elements laid out at the type's extent
 *     (the data movement behind the stream-enqueued send/recv of §5.2);
 *   - the FP64 adjoint of a typed float32 pack (a summing scatter).
 *
 * All sizes and displacements are int64 byte counts.  Functions that can
 * fail return 0 on success and a negative code otherwise.
 */
#ifndef DTE_ORACLE_H
#define DTE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_type or_type;

enum { OR_OK = 0, OR_EARG = -1, OR_ENOMEM = -2, OR_EOVERLAP = -3 };
enum { OR_ORDER_C = 0, OR_ORDER_F = 1 };
enum { OR_DIST_BLOCK = 0, OR_DIST_CYCLIC = 1, OR_DIST_NONE = 2 };
#define OR_DFLT_DARG (-1)

/* Constructors.  Each returns NULL on an invalid argument.  Children are
 * reference counted: a constructor takes a reference on each old type, and
 * or_free drops one.  Displacements of indexed/vector are in units of the
 * old type's extent; h* variants and struct take bytes. */
or_type *or_basic(int64_t size, int64_t align);
or_type *or_contiguous(int64_t count, or_type *old);
or_type *or_vector(int64_t count, int64_t bl, int64_t stride, or_type *old);
or_type *or_hvector(int64_t count, int64_t bl, int64_t stride_bytes, or_type *old);
or_type *or_indexed(int64_t count, const int64_t *bl, const int64_t *disp, or_type *old);
or_type *or_hindexed(int64_t count, const int64_t *bl, const int64_t *disp_bytes, or_type *old);
or_type *or_indexed_block(int64_t count, int64_t bl, const int64_t *disp, or_type *old);
or_type *or_hindexed_block(int64_t count, int64_t bl, const int64_t *disp_bytes, or_type *old);
or_type *or_struct(int64_t count, const int64_t *bl, const int64_t *disp_bytes, or_type *const *types);
or_type *or_subarray(int ndims, const int64_t *sizes, const int64_t *subsizes,
                     const int64_t *starts, int order, or_type *old);
or_type *or_darray(int size, int rank, int ndims, const int64_t *gsizes, const int *distribs,
                   const int64_t *dargs, const int64_t *psizes, int order, or_type *old);
or_type *or_resized(or_type *old, int64_t lb, int64_t extent);
void or_free(or_type *t);

/* Queries. */
int64_t or_size(const or_type *t);
int64_t or_lb(const or_type *t);
int64_t or_extent(const or_type *t);
int64_t or_true_lb(const or_type *t);
int64_t or_true_extent(const or_type *t);

/* Expanded typemap: number of basic entries, and the entries themselves. */
int64_t or_typemap_len(const or_type *t);
void or_typemap(const or_type *t, int64_t *disps, int64_t *sizes);

/* Segment list of one element. */
int64_t or_iov_count(const or_type *t);
int64_t or_iov(const or_type *t, int64_t iov_offset, int64_t max_iov_len,
               int64_t *disps, int64_t *lens);
int or_iov_len(const or_type *t, int64_t max_iov_bytes, int64_t *iov_len,
               int64_t *actual_iov_bytes);
/* Segment list of `count` elements at the type's extent: element e's list
 * shifted by e*extent, nothing merged across elements. */
int64_t or_iov_elements(const or_type *t, int64_t count, int64_t iov_offset,
                        int64_t max_iov_len, int64_t *disps, int64_t *lens);

/* Data movement.  `origin` is the buffer address that displacement 0 refers
 * to; `packed` is count*size contiguous bytes. */
int or_pack(const void *origin, int64_t count, const or_type *t, void *packed);
int or_unpack(const void *packed, int64_t count, const or_type *t, void *origin);
/* The same movement restricted to bytes [first, first + nbytes) of the
 * packed stream of `count` elements; `packed` holds just those bytes.  The
 * typemap is walked in order and every byte outside the window is skipped,
 * so a sequence of windows covering the stream equals one full pack. */
int or_pack_range(const void *origin, int64_t count, const or_type *t, int64_t first, int64_t nbytes,
                  void *packed);
int or_unpack_range(const void *packed, int64_t first, int64_t nbytes, int64_t count, const or_type *t,
                    void *origin);
/* 1 if two typemap entries of `count` elements share a byte, else 0. */
int or_overlaps(const or_type *t, int64_t count);

/* Adjoint of the typed float32 pack: for every packed float k taken from
 * float index src_index(k) of the origin, gx[src_index(k)] += gy[k], summed
 * in FP64.  The type's entries must all be 4-byte, 4-aligned. */
int or_pack_adjoint_f64(const double *gy, int64_t count, const or_type *t,
                        double *gx, int64_t gx_len);

#ifdef __cplusplus
}
#endif
#endif
