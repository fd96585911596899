/*
 * oracle.c -- plain CPU reference for the derived-datatype engine.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Deliberately slow: every query
 * re-walks the typemap one basic entry at a time, in constructor order, with
 * no descriptor, no merging shortcut and no blocking.  The goal is that a
 * reader can check each constructor against its MPI definition by eye.
 *
 * Paper anchors (arxiv 2402.12274):
 *   §3      a datatype describes a layout; types nest, carry offsets and may
 *           overlap; a YZ surface of an Nx*Ny*Nz array is Ny*Nz segments.
 *   §3.1    MPIX_Type_iov_len / MPIX_Type_iov / MPIX_Iov semantics.
 *   §3.2    the typeiov example (contiguous(16, BYTE) inside a 3-D subarray).
 *   §5.2    send/recv of (buf, count, datatype) enqueued on a GPU stream:
 *           the pack/unpack data movement below.
 * The lb/ub/extent rules are the MPI standard's, which the paper uses without
 * restating them; the readings taken where it is silent are:
 *   - lb/ub of a constructed type: the minimum/maximum over its copies of
 *     (copy displacement + child lb/ub); when any copy carries an explicit
 *     bound (from resized or subarray), only the copies with an explicit bound
 *     take part for that bound ("sticky" bounds).
 *   - struct only: with no explicit ub, the extent is rounded up to a multiple
 *     of the largest basic alignment in the struct.
 *   - subarray: lb = 0 and extent = prod(sizes) * extent(old), both explicit.
 *   - a segment absorbs the next typemap entry only if that entry starts
 *     exactly at the segment's end; zero-length blocks contribute nothing.
 *   - iov_len: a budget of -1 or any budget >= size gives every segment; a
 *     budget below -1 is an error.  iov: an offset past the end returns zero
 *     segments; negative offset/length is an error.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

enum {
    K_BASIC, K_CONTIG, K_VECTOR, K_HVECTOR, K_INDEXED, K_HINDEXED,
    K_STRUCT, K_SUBARRAY, K_RESIZED, K_DARRAY
};

#define OR_MAXDIMS 32

struct or_type {
    int refs;
    int kind;
    /* constructor arguments */
    int64_t count, bl, stride;           /* contig/vector/hvector */
    int64_t *bls, *disps;                /* indexed/hindexed/struct */
    or_type **types;                     /* struct */
    or_type *old;                        /* everything but basic/struct */
    int ndims, order;                    /* subarray */
    int64_t sizes[OR_MAXDIMS], subsizes[OR_MAXDIMS], starts[OR_MAXDIMS];
    int64_t *owned[OR_MAXDIMS], nowned[OR_MAXDIMS];   /* darray: owned indices per dim */
    int64_t basic_size;
    /* derived attributes */
    int64_t size, nbasic, lb, ub, true_lb, true_ub, align;
    int lb_explicit, ub_explicit, nonempty;
};

static int64_t ext_of(const or_type *t) { return t->ub - t->lb; }

/* ------------------------------------------------------------------------ */
/* Copies: every constructor is a list of (displacement, child type) pairs.  */
/* ------------------------------------------------------------------------ */

typedef void (*copy_fn)(void *ctx, int64_t disp, const or_type *child);

static void for_each_copy(const or_type *t, copy_fn fn, void *ctx)
{
    int64_t i, j;
    switch (t->kind) {
    case K_CONTIG: /* count copies at i * extent(old) */
        for (i = 0; i < t->count; i++)
            fn(ctx, i * ext_of(t->old), t->old);
        break;
    case K_VECTOR: /* (i*stride + j) * extent(old) */
        for (i = 0; i < t->count; i++)
            for (j = 0; j < t->bl; j++)
                fn(ctx, (i * t->stride + j) * ext_of(t->old), t->old);
        break;
    case K_HVECTOR: /* i*stride_bytes + j*extent(old) */
        for (i = 0; i < t->count; i++)
            for (j = 0; j < t->bl; j++)
                fn(ctx, i * t->stride + j * ext_of(t->old), t->old);
        break;
    case K_INDEXED: /* (disp[i] + j) * extent(old) */
        for (i = 0; i < t->count; i++)
            for (j = 0; j < t->bls[i]; j++)
                fn(ctx, (t->disps[i] + j) * ext_of(t->old), t->old);
        break;
    case K_HINDEXED: /* disp_bytes[i] + j*extent(old) */
        for (i = 0; i < t->count; i++)
            for (j = 0; j < t->bls[i]; j++)
                fn(ctx, t->disps[i] + j * ext_of(t->old), t->old);
        break;
    case K_STRUCT: /* disp_bytes[i] + j*extent(types[i]) */
        for (i = 0; i < t->count; i++)
            for (j = 0; j < t->bls[i]; j++)
                fn(ctx, t->disps[i] + j * ext_of(t->types[i]), t->types[i]);
        break;
    case K_SUBARRAY: {
        /* Elements of the sub-block in C order (last index fastest) or
         * Fortran order (first index fastest); element idx sits at the
         * linear index of (starts + idx) in the full array, times
         * extent(old). */
        int n = t->ndims, d;
        int64_t idx[OR_MAXDIMS];
        for (d = 0; d < n; d++) {
            if (t->subsizes[d] == 0) return;
            idx[d] = 0;
        }
        for (;;) {
            int64_t lin = 0;
            if (t->order == OR_ORDER_C) {
                for (d = 0; d < n; d++)
                    lin = lin * t->sizes[d] + (t->starts[d] + idx[d]);
            } else {
                for (d = n - 1; d >= 0; d--)
                    lin = lin * t->sizes[d] + (t->starts[d] + idx[d]);
            }
            fn(ctx, lin * ext_of(t->old), t->old);
            /* advance the multi-index */
            if (t->order == OR_ORDER_C) {
                for (d = n - 1; d >= 0; d--) {
                    if (++idx[d] < t->subsizes[d]) break;
                    idx[d] = 0;
                }
            } else {
                for (d = 0; d < n; d++) {
                    if (++idx[d] < t->subsizes[d]) break;
                    idx[d] = 0;
                }
                if (d == n) d = -1;
            }
            if (d < 0) return;
        }
        break;
    }
    case K_DARRAY: {
        /* Owned elements of the global array in C or Fortran order; element
         * idx sits at the linear index of (owned[0][idx0], ...) in the global
         * array, times extent(old). */
        int n = t->ndims, d;
        int64_t idx[OR_MAXDIMS];
        for (d = 0; d < n; d++) {
            if (t->nowned[d] == 0) return;
            idx[d] = 0;
        }
        for (;;) {
            int64_t lin = 0;
            if (t->order == OR_ORDER_C) {
                for (d = 0; d < n; d++) lin = lin * t->sizes[d] + t->owned[d][idx[d]];
            } else {
                for (d = n - 1; d >= 0; d--) lin = lin * t->sizes[d] + t->owned[d][idx[d]];
            }
            fn(ctx, lin * ext_of(t->old), t->old);
            if (t->order == OR_ORDER_C) {
                for (d = n - 1; d >= 0; d--) {
                    if (++idx[d] < t->nowned[d]) break;
                    idx[d] = 0;
                }
            } else {
                for (d = 0; d < n; d++) {
                    if (++idx[d] < t->nowned[d]) break;
                    idx[d] = 0;
                }
                if (d == n) d = -1;
            }
            if (d < 0) return;
        }
        break;
    }
    case K_RESIZED:
        fn(ctx, 0, t->old);
        break;
    default:
        break;
    }
}

/* ------------------------------------------------------------------------ */
/* Attribute computation from the copies.                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t size, nbasic, align;
    int any, any_lb_x, any_ub_x, any_data;
    int64_t lb_all, ub_all, lb_x, ub_x, tlb, tub;
} attr_acc;

static void attr_copy(void *vctx, int64_t d, const or_type *c)
{
    attr_acc *a = (attr_acc *)vctx;
    /* a copy with no typemap entries and no explicit bound adds nothing */
    if (!c->nonempty && !c->lb_explicit && !c->ub_explicit) return;
    a->size += c->size;
    a->nbasic += c->nbasic;
    if (c->align > a->align) a->align = c->align;
    if (!a->any || d + c->lb < a->lb_all) a->lb_all = d + c->lb;
    if (!a->any || d + c->ub > a->ub_all) a->ub_all = d + c->ub;
    a->any = 1;
    if (c->lb_explicit) {
        if (!a->any_lb_x || d + c->lb < a->lb_x) a->lb_x = d + c->lb;
        a->any_lb_x = 1;
    }
    if (c->ub_explicit) {
        if (!a->any_ub_x || d + c->ub > a->ub_x) a->ub_x = d + c->ub;
        a->any_ub_x = 1;
    }
    if (c->nonempty) {
        if (!a->any_data || d + c->true_lb < a->tlb) a->tlb = d + c->true_lb;
        if (!a->any_data || d + c->true_ub > a->tub) a->tub = d + c->true_ub;
        a->any_data = 1;
    }
}

static void finish_attrs(or_type *t)
{
    attr_acc a;
    memset(&a, 0, sizeof a);
    a.align = 1;
    for_each_copy(t, attr_copy, &a);
    t->size = a.size;
    t->nbasic = a.nbasic;
    t->align = a.align;
    t->nonempty = a.any_data;
    t->true_lb = a.any_data ? a.tlb : 0;
    t->true_ub = a.any_data ? a.tub : 0;
    t->lb = a.any_lb_x ? a.lb_x : (a.any ? a.lb_all : 0);
    t->ub = a.any_ub_x ? a.ub_x : (a.any ? a.ub_all : 0);
    t->lb_explicit = a.any_lb_x;
    t->ub_explicit = a.any_ub_x;
    if (t->kind == K_STRUCT && !a.any_ub_x && a.any) {
        int64_t ext = t->ub - t->lb;
        int64_t r = ext % t->align;
        if (r < 0) r += t->align;
        if (r) t->ub += t->align - r;
    }
}

static or_type *new_type(int kind)
{
    or_type *t = (or_type *)calloc(1, sizeof(or_type));
    if (t) { t->refs = 1; t->kind = kind; }
    return t;
}

static int64_t *dup_i64(const int64_t *a, int64_t n)
{
    int64_t *r = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (r && n > 0) memcpy(r, a, (size_t)n * sizeof(int64_t));
    return r;
}

/* ------------------------------------------------------------------------ */
/* Constructors                                                              */
/* ------------------------------------------------------------------------ */

or_type *or_basic(int64_t size, int64_t align)
{
    or_type *t;
    if (size <= 0 || align <= 0) return NULL;
    t = new_type(K_BASIC);
    if (!t) return NULL;
    t->basic_size = size;
    t->size = size;
    t->nbasic = 1;
    t->lb = 0;
    t->ub = size;
    t->true_lb = 0;
    t->true_ub = size;
    t->align = align;
    t->nonempty = 1;
    return t;
}

or_type *or_contiguous(int64_t count, or_type *old)
{
    or_type *t;
    if (count < 0 || !old) return NULL;
    t = new_type(K_CONTIG);
    if (!t) return NULL;
    t->count = count;
    t->old = old; old->refs++;
    finish_attrs(t);
    return t;
}

static or_type *mk_vec(int kind, int64_t count, int64_t bl, int64_t stride, or_type *old)
{
    or_type *t;
    if (count < 0 || bl < 0 || !old) return NULL;
    t = new_type(kind);
    if (!t) return NULL;
    t->count = count; t->bl = bl; t->stride = stride;
    t->old = old; old->refs++;
    finish_attrs(t);
    return t;
}

or_type *or_vector(int64_t count, int64_t bl, int64_t stride, or_type *old)
{ return mk_vec(K_VECTOR, count, bl, stride, old); }

or_type *or_hvector(int64_t count, int64_t bl, int64_t stride_bytes, or_type *old)
{ return mk_vec(K_HVECTOR, count, bl, stride_bytes, old); }

static or_type *mk_idx(int kind, int64_t count, const int64_t *bl, const int64_t *disp, or_type *old)
{
    or_type *t;
    int64_t i;
    if (count < 0 || !old || (count > 0 && (!bl || !disp))) return NULL;
    for (i = 0; i < count; i++)
        if (bl[i] < 0) return NULL;
    t = new_type(kind);
    if (!t) return NULL;
    t->count = count;
    t->bls = dup_i64(bl, count);
    t->disps = dup_i64(disp, count);
    t->old = old; old->refs++;
    finish_attrs(t);
    return t;
}

or_type *or_indexed(int64_t count, const int64_t *bl, const int64_t *disp, or_type *old)
{ return mk_idx(K_INDEXED, count, bl, disp, old); }

or_type *or_hindexed(int64_t count, const int64_t *bl, const int64_t *disp_bytes, or_type *old)
{ return mk_idx(K_HINDEXED, count, bl, disp_bytes, old); }

static or_type *mk_idx_block(int kind, int64_t count, int64_t bl, const int64_t *disp, or_type *old)
{
    or_type *t;
    int64_t i, *bls;
    if (count < 0 || bl < 0) return NULL;
    bls = (int64_t *)malloc((size_t)(count > 0 ? count : 1) * sizeof(int64_t));
    if (!bls) return NULL;
    for (i = 0; i < count; i++) bls[i] = bl;
    t = mk_idx(kind, count, bls, disp, old);
    free(bls);
    return t;
}

or_type *or_indexed_block(int64_t count, int64_t bl, const int64_t *disp, or_type *old)
{ return mk_idx_block(K_INDEXED, count, bl, disp, old); }

or_type *or_hindexed_block(int64_t count, int64_t bl, const int64_t *disp_bytes, or_type *old)
{ return mk_idx_block(K_HINDEXED, count, bl, disp_bytes, old); }

or_type *or_struct(int64_t count, const int64_t *bl, const int64_t *disp_bytes, or_type *const *types)
{
    or_type *t;
    int64_t i;
    if (count < 0 || (count > 0 && (!bl || !disp_bytes || !types))) return NULL;
    for (i = 0; i < count; i++)
        if (bl[i] < 0 || !types[i]) return NULL;
    t = new_type(K_STRUCT);
    if (!t) return NULL;
    t->count = count;
    t->bls = dup_i64(bl, count);
    t->disps = dup_i64(disp_bytes, count);
    t->types = (or_type **)malloc((size_t)(count > 0 ? count : 1) * sizeof(or_type *));
    for (i = 0; i < count; i++) { t->types[i] = types[i]; types[i]->refs++; }
    finish_attrs(t);
    return t;
}

or_type *or_subarray(int ndims, const int64_t *sizes, const int64_t *subsizes,
                     const int64_t *starts, int order, or_type *old)
{
    or_type *t;
    int d;
    int64_t full = 1;
    if (ndims <= 0 || ndims > OR_MAXDIMS || !old) return NULL;
    if (order != OR_ORDER_C && order != OR_ORDER_F) return NULL;
    for (d = 0; d < ndims; d++) {
        if (sizes[d] <= 0 || subsizes[d] < 0 || starts[d] < 0) return NULL;
        if (starts[d] + subsizes[d] > sizes[d]) return NULL;
        full *= sizes[d];
    }
    t = new_type(K_SUBARRAY);
    if (!t) return NULL;
    t->ndims = ndims;
    t->order = order;
    for (d = 0; d < ndims; d++) {
        t->sizes[d] = sizes[d];
        t->subsizes[d] = subsizes[d];
        t->starts[d] = starts[d];
    }
    t->old = old; old->refs++;
    finish_attrs(t);
    /* the subarray type spans the whole array: lb 0, explicit bounds */
    t->lb = 0;
    t->ub = full * ext_of(old);
    t->lb_explicit = t->ub_explicit = 1;
    return t;
}

/* Distributed array: the block of a global array (gsizes) that process
 * `rank` of a row-major process grid (psizes) owns, per dimension BLOCK
 * (block size darg, default ceil(g/p)), CYCLIC (blocks of darg, default 1,
 * dealt round-robin) or NONE (whole dimension, p must be 1). */
or_type *or_darray(int size, int rank, int ndims, const int64_t *gsizes, const int *distribs,
                   const int64_t *dargs, const int64_t *psizes, int order, or_type *old)
{
    or_type *t;
    int d;
    int64_t full = 1, nproc = 1, r, coord[OR_MAXDIMS];
    if (ndims <= 0 || ndims > OR_MAXDIMS || !old || size <= 0 || rank < 0 || rank >= size) return NULL;
    if (order != OR_ORDER_C && order != OR_ORDER_F) return NULL;
    for (d = 0; d < ndims; d++) {
        if (gsizes[d] <= 0 || psizes[d] <= 0) return NULL;
        nproc *= psizes[d];
        full *= gsizes[d];
    }
    if (nproc != size) return NULL;
    r = rank;
    for (d = ndims - 1; d >= 0; d--) {  /* process grid is row-major */
        coord[d] = r % psizes[d];
        r /= psizes[d];
    }
    t = new_type(K_DARRAY);
    if (!t) return NULL;
    t->ndims = ndims;
    t->order = order;
    for (d = 0; d < ndims; d++) {
        int64_t g = gsizes[d], p = psizes[d], c = coord[d], b, i, n = 0;
        t->sizes[d] = g;
        t->owned[d] = (int64_t *)malloc((size_t)g * sizeof(int64_t));
        if (!t->owned[d]) { or_free(t); return NULL; }
        if (distribs[d] == OR_DIST_NONE) {
            if (p != 1) { or_free(t); return NULL; }
            for (i = 0; i < g; i++) t->owned[d][n++] = i;
        } else if (distribs[d] == OR_DIST_BLOCK) {
            b = dargs[d] == OR_DFLT_DARG ? (g + p - 1) / p : dargs[d];
            if (b <= 0 || b * p < g) { or_free(t); return NULL; }
            for (i = c * b; i < c * b + b && i < g; i++) t->owned[d][n++] = i;
        } else if (distribs[d] == OR_DIST_CYCLIC) {
            b = dargs[d] == OR_DFLT_DARG ? 1 : dargs[d];
            if (b <= 0) { or_free(t); return NULL; }
            for (i = 0; i < g; i++)
                if ((i / b) % p == c) t->owned[d][n++] = i;
        } else {
            or_free(t);
            return NULL;
        }
        t->nowned[d] = n;
    }
    t->old = old; old->refs++;
    finish_attrs(t);
    t->lb = 0;
    t->ub = full * ext_of(old);
    t->lb_explicit = t->ub_explicit = 1;
    return t;
}

or_type *or_resized(or_type *old, int64_t lb, int64_t extent)
{
    or_type *t;
    if (!old) return NULL;
    t = new_type(K_RESIZED);
    if (!t) return NULL;
    t->old = old; old->refs++;
    finish_attrs(t);
    t->lb = lb;
    t->ub = lb + extent;
    t->lb_explicit = t->ub_explicit = 1;
    return t;
}

void or_free(or_type *t)
{
    int64_t i;
    if (!t || --t->refs > 0) return;
    if (t->old) or_free(t->old);
    if (t->types) {
        for (i = 0; i < t->count; i++) or_free(t->types[i]);
        free(t->types);
    }
    free(t->bls);
    free(t->disps);
    for (i = 0; i < OR_MAXDIMS; i++) free(t->owned[i]);
    free(t);
}

int64_t or_size(const or_type *t) { return t->size; }
int64_t or_lb(const or_type *t) { return t->lb; }
int64_t or_extent(const or_type *t) { return ext_of(t); }
int64_t or_true_lb(const or_type *t) { return t->true_lb; }
int64_t or_true_extent(const or_type *t) { return t->true_ub - t->true_lb; }

/* ------------------------------------------------------------------------ */
/* The typemap walk: visit every basic entry (displacement, size) in order.  */
/* ------------------------------------------------------------------------ */

typedef void (*entry_fn)(void *ctx, int64_t disp, int64_t size);

typedef struct {
    entry_fn fn;
    void *ctx;
    int64_t base;
} walk_ctx;

static void walk(const or_type *t, int64_t disp, entry_fn fn, void *ctx);

static void walk_copy(void *vctx, int64_t d, const or_type *c)
{
    walk_ctx *w = (walk_ctx *)vctx;
    walk(c, w->base + d, w->fn, w->ctx);
}

static void walk(const or_type *t, int64_t disp, entry_fn fn, void *ctx)
{
    walk_ctx w;
    if (t->kind == K_BASIC) {
        fn(ctx, disp, t->basic_size);
        return;
    }
    w.fn = fn;
    w.ctx = ctx;
    w.base = disp;
    for_each_copy(t, walk_copy, &w);
}

int64_t or_typemap_len(const or_type *t) { return t->nbasic; }

typedef struct { int64_t *d, *s, n; } tm_ctx;

static void tm_entry(void *vctx, int64_t disp, int64_t size)
{
    tm_ctx *c = (tm_ctx *)vctx;
    c->d[c->n] = disp;
    c->s[c->n] = size;
    c->n++;
}

void or_typemap(const or_type *t, int64_t *disps, int64_t *sizes)
{
    tm_ctx c;
    c.d = disps; c.s = sizes; c.n = 0;
    walk(t, 0, tm_entry, &c);
}

/* ------------------------------------------------------------------------ */
/* Segments: merge an entry into the open segment iff it starts at its end.  */
/* ------------------------------------------------------------------------ */

typedef void (*seg_fn)(void *ctx, int64_t index, int64_t disp, int64_t len);

typedef struct {
    int open;
    int64_t start, len, index;
    seg_fn emit;
    void *ctx;
} merge_ctx;

static void merge_entry(void *vctx, int64_t disp, int64_t size)
{
    merge_ctx *m = (merge_ctx *)vctx;
    if (m->open && disp == m->start + m->len) {
        m->len += size;
        return;
    }
    if (m->open) {
        m->emit(m->ctx, m->index, m->start, m->len);
        m->index++;
    }
    m->open = 1;
    m->start = disp;
    m->len = size;
}

static void merge_flush(merge_ctx *m)
{
    if (m->open) {
        m->emit(m->ctx, m->index, m->start, m->len);
        m->index++;
        m->open = 0;
    }
}

/* Walk the segments of one element, shifted by `base`. */
static int64_t walk_segments(const or_type *t, int64_t base, seg_fn emit, void *ctx)
{
    merge_ctx m;
    memset(&m, 0, sizeof m);
    m.emit = emit;
    m.ctx = ctx;
    walk(t, base, merge_entry, &m);
    merge_flush(&m);
    return m.index;
}

static void seg_ignore(void *ctx, int64_t i, int64_t d, int64_t l)
{ (void)ctx; (void)i; (void)d; (void)l; }

int64_t or_iov_count(const or_type *t)
{
    return walk_segments(t, 0, seg_ignore, NULL);
}

typedef struct {
    int64_t first, max, got, shift;
    int64_t *d, *l;
} range_ctx;

static void range_seg(void *vctx, int64_t i, int64_t d, int64_t l)
{
    range_ctx *r = (range_ctx *)vctx;
    i += r->shift;
    if (i >= r->first && i < r->first + r->max) {
        r->d[i - r->first] = d;
        r->l[i - r->first] = l;
        r->got++;
    }
}

/* §3.1 MPIX_Type_iov: segments [iov_offset, iov_offset + max_iov_len). */
int64_t or_iov(const or_type *t, int64_t iov_offset, int64_t max_iov_len,
               int64_t *disps, int64_t *lens)
{
    range_ctx r;
    if (iov_offset < 0 || max_iov_len < 0) return OR_EARG;
    r.first = iov_offset; r.max = max_iov_len; r.got = 0; r.shift = 0;
    r.d = disps; r.l = lens;
    walk_segments(t, 0, range_seg, &r);
    return r.got;
}

int64_t or_iov_elements(const or_type *t, int64_t count, int64_t iov_offset,
                        int64_t max_iov_len, int64_t *disps, int64_t *lens)
{
    range_ctx r;
    int64_t e, per;
    if (count < 0 || iov_offset < 0 || max_iov_len < 0) return OR_EARG;
    r.first = iov_offset; r.max = max_iov_len; r.got = 0; r.shift = 0;
    r.d = disps; r.l = lens;
    for (e = 0; e < count; e++) {
        per = walk_segments(t, e * ext_of(t), range_seg, &r);
        r.shift += per;
    }
    return r.got;
}

typedef struct {
    int64_t budget, n, bytes, stop;
} len_ctx;

static void len_seg(void *vctx, int64_t i, int64_t d, int64_t l)
{
    len_ctx *c = (len_ctx *)vctx;
    (void)i; (void)d;
    if (c->stop) return;
    if (c->bytes + l <= c->budget) {
        c->n++;
        c->bytes += l;
    } else {
        c->stop = 1;
    }
}

/* §3.1 MPIX_Type_iov_len: the number of whole segments that fit in the
 * byte budget and their bytes; -1 or a budget above the size means all. */
int or_iov_len(const or_type *t, int64_t max_iov_bytes, int64_t *iov_len,
               int64_t *actual_iov_bytes)
{
    len_ctx c;
    if (max_iov_bytes < -1) return OR_EARG;
    c.budget = (max_iov_bytes == -1 || max_iov_bytes > t->size) ? t->size : max_iov_bytes;
    c.n = 0; c.bytes = 0; c.stop = 0;
    walk_segments(t, 0, len_seg, &c);
    *iov_len = c.n;
    *actual_iov_bytes = c.bytes;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Pack / unpack: element e of the user buffer starts at e * extent.         */
/* ------------------------------------------------------------------------ */

typedef struct {
    const unsigned char *src;
    unsigned char *dst;
    int64_t pos;
    int to_packed;
    int64_t lo, hi;  /* packed-stream window moved by the range variants */
} move_ctx;

static void move_entry(void *vctx, int64_t disp, int64_t size)
{
    move_ctx *m = (move_ctx *)vctx;
    if (m->to_packed)
        memcpy(m->dst + m->pos, m->src + disp, (size_t)size);
    else
        memcpy(m->dst + disp, m->src + m->pos, (size_t)size);
    m->pos += size;
}

/* Like move_entry, but only the bytes whose packed-stream position lies in
 * [lo, hi) move, and packed byte `lo` sits at offset 0 of the packed buffer. */
static void move_entry_range(void *vctx, int64_t disp, int64_t size)
{
    move_ctx *m = (move_ctx *)vctx;
    int64_t a = m->pos > m->lo ? m->pos : m->lo;
    int64_t b = m->pos + size < m->hi ? m->pos + size : m->hi;
    if (a < b) {
        int64_t ud = disp + (a - m->pos);
        if (m->to_packed)
            memcpy(m->dst + (a - m->lo), m->src + ud, (size_t)(b - a));
        else
            memcpy(m->dst + ud, m->src + (a - m->lo), (size_t)(b - a));
    }
    m->pos += size;
}

static int move_range(const void *src, void *dst, int to_packed, int64_t count, const or_type *t,
                      int64_t first, int64_t nbytes)
{
    move_ctx m;
    int64_t e;
    if (count < 0 || first < 0 || nbytes < 0 || first + nbytes > count * t->size) return OR_EARG;
    m.src = (const unsigned char *)src;
    m.dst = (unsigned char *)dst;
    m.pos = 0;
    m.to_packed = to_packed;
    m.lo = first;
    m.hi = first + nbytes;
    for (e = 0; e < count && m.pos < m.hi; e++)
        walk(t, e * ext_of(t), move_entry_range, &m);
    return OR_OK;
}

int or_pack_range(const void *origin, int64_t count, const or_type *t, int64_t first, int64_t nbytes,
                  void *packed)
{
    return move_range(origin, packed, 1, count, t, first, nbytes);
}

int or_unpack_range(const void *packed, int64_t first, int64_t nbytes, int64_t count, const or_type *t,
                    void *origin)
{
    return move_range(packed, origin, 0, count, t, first, nbytes);
}

int or_pack(const void *origin, int64_t count, const or_type *t, void *packed)
{
    move_ctx m;
    int64_t e;
    if (count < 0) return OR_EARG;
    m.src = (const unsigned char *)origin;
    m.dst = (unsigned char *)packed;
    m.pos = 0;
    m.to_packed = 1;
    for (e = 0; e < count; e++)
        walk(t, e * ext_of(t), move_entry, &m);
    return OR_OK;
}

int or_unpack(const void *packed, int64_t count, const or_type *t, void *origin)
{
    move_ctx m;
    int64_t e;
    if (count < 0) return OR_EARG;
    m.src = (const unsigned char *)packed;
    m.dst = (unsigned char *)origin;
    m.pos = 0;
    m.to_packed = 0;
    for (e = 0; e < count; e++)
        walk(t, e * ext_of(t), move_entry, &m);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Overlap: expand, sort by displacement, look for a shared byte.           */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t d, s; } ds_pair;

static int cmp_pair(const void *a, const void *b)
{
    const ds_pair *x = (const ds_pair *)a, *y = (const ds_pair *)b;
    return (x->d > y->d) - (x->d < y->d);
}

typedef struct { ds_pair *p; int64_t n; } ov_ctx;

static void ov_entry(void *vctx, int64_t disp, int64_t size)
{
    ov_ctx *c = (ov_ctx *)vctx;
    c->p[c->n].d = disp;
    c->p[c->n].s = size;
    c->n++;
}

int or_overlaps(const or_type *t, int64_t count)
{
    ov_ctx c;
    int64_t e, i, end;
    int hit = 0;
    if (count <= 0 || t->nbasic == 0) return 0;
    c.p = (ds_pair *)malloc((size_t)(count * t->nbasic) * sizeof(ds_pair));
    if (!c.p) return OR_ENOMEM;
    c.n = 0;
    for (e = 0; e < count; e++)
        walk(t, e * ext_of(t), ov_entry, &c);
    qsort(c.p, (size_t)c.n, sizeof(ds_pair), cmp_pair);
    end = c.p[0].d + c.p[0].s;
    for (i = 1; i < c.n && !hit; i++) {
        if (c.p[i].d < end) hit = 1;
        if (c.p[i].d + c.p[i].s > end) end = c.p[i].d + c.p[i].s;
    }
    free(c.p);
    return hit;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the float32 pack, accumulated in FP64.                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *gy;
    double *gx;
    int64_t gx_len, k;
    int bad;
} adj_ctx;

static void adj_entry(void *vctx, int64_t disp, int64_t size)
{
    adj_ctx *a = (adj_ctx *)vctx;
    int64_t idx;
    if (size != 4 || disp % 4 != 0) { a->bad = 1; a->k++; return; }
    idx = disp / 4;
    if (idx < 0 || idx >= a->gx_len) { a->bad = 1; a->k++; return; }
    a->gx[idx] += a->gy[a->k];
    a->k++;
}

int or_pack_adjoint_f64(const double *gy, int64_t count, const or_type *t,
                        double *gx, int64_t gx_len)
{
    adj_ctx a;
    int64_t e;
    if (count < 0) return OR_EARG;
    a.gy = gy; a.gx = gx; a.gx_len = gx_len; a.k = 0; a.bad = 0;
    for (e = 0; e < count; e++)
        walk(t, e * ext_of(t), adj_entry, &a);
    return a.bad ? OR_EARG : OR_OK;
}
