// kernels.cu -- sm_103a pack / unpack / segment-enumeration kernels and the
// stream-enqueue entry points of the GB300 datatype engine.
//
// Paper anchors (arxiv 2402.12274): §5 (operations on a GPU-stream-backed
// context are queued and run in stream order; no host synchronisation,
// §5.3), §5.2 (send/recv of (buf, count, datatype)), §3.1 (iov queries).
//
// Data movement design (pure data movement, no tensor cores):
//  * The packed side is contiguous, so work is split in packed space into
//    warp steps of 16-byte chunks: 1 KiB for 16-byte copy words (lane l
//    handles chunks l and l+32), 2 KiB otherwise (chunks l, l+32, l+64,
//    l+96).  Every packed-side access of a warp is one coalesced 512-byte
//    transaction, and all of a lane's loads are in flight before its stores
//    (an unpack issues its packed loads before walking the descriptor).
//    Warps take spans of steps in a spread order (Spread, move.cuh).
//  * Each chunk maps back to the user layout through the committed descriptor
//    (desc.h: REG levels by fast invariant division, LIST levels by a search
//    that gallops from the step's previous position).  Descriptors of up to
//    16 KiB are staged whole in shared memory; larger ones stage their node
//    table and read index arrays through L1/L2.
//  * W, the copy word, is the largest power of two <= 16 dividing every run
//    length and displacement of the type and both buffer addresses; a word
//    never straddles two runs, so W = 16 moves each chunk with one 16-byte
//    load and one 16-byte store.  Smaller W assembles the chunk run by run
//    from W-byte words.
//  * Short runs under large index tables move segment-major (seg_kernel);
//    whole moves of arrays of short records (an index list over one struct
//    of a few runs) move record-major, a record per lane with the packed
//    side staged in shared memory (rec_kernel); long runs with W = 16 in
//    moves large enough to give every warp of the bulk grid several 16 KiB
//    tiles move by TMA bulk copies (bulk_kernel, bulk.cuh).
//  * A warp whose search position is far from its target (a new span of the
//    spread or strided work order, a new query) searches by the warp: 32
//    probes a step (warp_find_le), then gallops from there.
//  * Bytes are moved verbatim through integer registers: no value is ever
//    converted, so NaN payloads survive.
//  * Batches: many independent operations (different types, buffers and
//    sizes) run in one persistent launch over a global list of tiles (warp
//    steps, or rounds of 32 segments);
//    the launch reads only a device-resident op table, so it can be captured
//    in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstring>
#include <numeric>
#include <vector>

#include "bulk.cuh"
#include "internal.h"
#include "move.cuh"

namespace dte {

// Warps take spans of `span` chunks (a multiple of the step) in the spread
// order (see Spread), so costly and cheap regions of a layout are worked on
// at the same time, while a span keeps consecutive steps together for the
// search hints.
template <int W, bool PACK, bool PK16, bool WIDE = false>
__global__ void __launch_bounds__(kThreads, kMinBlocks) move_kernel(Desc d, Op op, int64_t nchunks, int64_t span,
                                                                   Spread sp)
{
    extern __shared__ uint4 smem[];
    __shared__ uint4 scratch[kScratch<W>];
    char *scr = reinterpret_cast<char *>(&scratch[W < 16 ? threadIdx.x : 0]);
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    allow_dependents();
    prior_grids_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    Hint h{-1, 0};
    int64_t p = spread_first(sp, warp);
    for (int64_t j = warp; j < sp.nspans; j += nwarps) {
        const int64_t c0 = p * span;
        const int64_t c1 = min(c0 + span, nchunks);
        if (kSeedHint) seed_root_hint(op, nodes, blob, c0 * 16, h, lane);  // spans lie far apart
        for (int64_t base = c0; base < c1; base += kStepOf<W, WIDE>)
            warp_step<W, PACK, PK16, WIDE>(op, nodes, blob, base, c1, lane, h, scr);
        p += sp.inc;
        if (p >= sp.nspans) p -= sp.nspans;
    }
}

// Segment-major movement for short runs (words of fewer than 16 bytes) under
// a large index table.  Each lane walks the descriptor once per round for one
// whole segment (a direct table lookup instead of a search per run end inside
// a chunk), then the warp moves the packed range its 32 segments cover
// together: lane l takes words l, l+32, l+64, l+96 of each 128-word slice and
// finds the segment of each word from a bit mask of the segment starts in its
// 32-word window (seg_round), so packed-side accesses stay coalesced.
// Segments [seg0, seg0 + nsegs) of the count-level segment list are moved;
// a range move clips the first and last of them to its packed window.
template <int W, bool PACK>
__global__ void __launch_bounds__(kThreads, kMinBlocks) seg_kernel(Desc d, Op op, int64_t nseg_elem, FastDiv div_nseg,
                                                                  int64_t seg0, int64_t nsegs, int64_t span)
{
    extern __shared__ uint4 smem[];
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    allow_dependents();
    prior_grids_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kWarps * span;
    Hint h{-1, 0}, rh{-1, 0};
    for (int64_t s0 = warp * span; s0 < nsegs; s0 += stride) {
        const int64_t s1 = min(s0 + span, nsegs);
        rh = Hint{-1, 0};  // spans lie far apart: start each with a search by the warp
        for (int64_t base = s0; base < s1; base += 32)
            seg_round<W, PACK, true, kSegWide>(op, nodes, blob, nseg_elem, div_nseg, seg0 + base, seg0 + s1, lane, h,
                                               rh);
    }
}

// Record-major movement (rec_round): whole moves of an index list over a
// short child table of runs, one record per lane per round of 32 records.
// Warps take spans of `span` consecutive rounds (the search position carries
// from one round to the next).  STAGE routes the packed side through
// per-warp shared-memory tiles; a staged unpack keeps two, so that the next
// round's packed bytes are fetched while the current round is scattered.
// CTAs per SM the record-major kernels are built for, by direction (records
// of 2^22 blocks: pack 3.74 / 3.96 / 3.30 TB/s at 4 / 6 / 8 CTAs on one box,
// 4.12 at 5 against 3.96-3.99 at 6 on another; unpack, with its two tiles,
// 2.27-2.28 at 4 and 2.22 at 5 or 6).
#ifndef DTE_REC_MB_PACK
#define DTE_REC_MB_PACK 5
#endif
#ifndef DTE_REC_MB_UNPACK
#define DTE_REC_MB_UNPACK 4
#endif
constexpr int kRecMinBlocksPack = DTE_REC_MB_PACK;
constexpr int kRecMinBlocksUnpack = DTE_REC_MB_UNPACK;
template <int W, bool PACK, bool STAGE>
__global__ void __launch_bounds__(kThreads, PACK ? kRecMinBlocksPack : kRecMinBlocksUnpack)
    rec_kernel(Desc d, Op op, int64_t nrec_elem, int64_t rounds_elem, FastDiv div_rounds, int64_t nrounds, int64_t span)
{
    constexpr int kTilesPerWarp = STAGE ? (PACK ? 1 : 2) : 0;
    extern __shared__ uint4 smem[];
    __shared__ uint4 tiles[STAGE ? kWarps * kTilesPerWarp * kRecTile / 16 : 1];
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    allow_dependents();
    prior_grids_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kWarps * span;
    char *tile = reinterpret_cast<char *>(&tiles[STAGE ? (threadIdx.x >> 5) * (kTilesPerWarp * kRecTile / 16) : 0]);
    Hint rh{-1, 0};
    for (int64_t q0 = warp * span; q0 < nrounds; q0 += stride) {
        const int64_t q1 = min(q0 + span, nrounds);
        rh = Hint{-1, 0};  // spans lie far apart: start each with a search by the warp
        if (STAGE && !PACK) {
            rec_unpack_rounds<W>(op, nodes, blob, nrec_elem, rounds_elem, div_rounds, q0, q1, lane, rh, tile);
        } else {
            for (int64_t q = q0; q < q1; q++)
                rec_round<W, PACK, STAGE>(op, nodes, blob, nrec_elem, rounds_elem, div_rounds, q, lane, rh, tile);
        }
    }
}

// ---------------------------------------------------------------------------
// batched movement: one persistent launch over many independent operations
// ---------------------------------------------------------------------------
// One launch per copy-word class present in a batch: ops are grouped by
// (W, packed side 16-aligned) so each kernel is specialised like move_kernel.
// tile0: nops+1 prefix of the tiles (warp steps) per op of the group.  Warps take spans
// of `span` consecutive tiles in the spread order.  When the group's descriptors fit
// in shared memory together (`image`, image_bytes > 0) they are staged once
// per CTA and every op with soff >= 0 walks its staged copy.
template <int W, bool PACK, bool PK16, bool WIDE = false>
__global__ void __launch_bounds__(kThreads, kMinBlocks) batch_kernel(const BatchOp *ops, const int64_t *tile0, int64_t nops,
                                                         int64_t ntiles, int64_t span, const char *image,
                                                         int64_t image_bytes, Spread sp)
{
    extern __shared__ uint4 smem[];
    __shared__ Op wop[kWarps];  // the op each warp is working on
    __shared__ uint4 scratch[kScratch<W>];
    char *scr = reinterpret_cast<char *>(&scratch[W < 16 ? threadIdx.x : 0]);
    const int wid = threadIdx.x >> 5;
    if (image_bytes > 0) {
        const uint4 *s = reinterpret_cast<const uint4 *>(image);
        int nw = (int)(image_bytes / 16);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) smem[i] = s[i];
        __syncthreads();
    }
    allow_dependents();
    prior_grids_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    Hint oh{-1, 0};
    Hint h{-1, 0};
    int64_t cur = -1;
    int64_t p = spread_first(sp, warp);
    for (int64_t j = warp; j < sp.nspans; j += nwarps, p = p + sp.inc >= sp.nspans ? p + sp.inc - sp.nspans : p + sp.inc) {
        const int64_t s0 = p * span;
        const int64_t s1 = min(s0 + span, ntiles);
        oh = Hint{-1, 0};  // spans lie far apart: find each span's first op by the warp
        for (int64_t t = s0; t < s1; t++) {
            int64_t i = warp_find_le_hint(tile0, nops, t, oh, 0, lane);
            const BatchOp *b = ops + i;
            if (i != cur) {
                h = Hint{-1, 0};
                cur = i;
                load_op(wop[wid], b->op, lane);
            }
            const int soff = b->soff;
            const char *blob = soff >= 0 ? reinterpret_cast<const char *>(smem) + soff : b->d.blob;
            const DNode *nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
            int64_t base = (t - tile0[i]) * kStepOf<W, WIDE>;
            warp_step<W, PACK, PK16, WIDE>(wop[wid], nodes, blob, base, b->nchunks, lane, h, scr);
        }
    }
}

// Segment-major batch variant: a tile of a segment-major op is one round of
// 32 segments.
template <int W, bool PACK>
__global__ void __launch_bounds__(kThreads, kMinBlocks) batch_seg_kernel(const BatchOp *ops, const int64_t *tile0,
                                                                        int64_t nops, int64_t ntiles, int64_t span,
                                                                        const char *image, int64_t image_bytes,
                                                                        Spread sp)
{
    extern __shared__ uint4 smem[];
    __shared__ Op wop[kWarps];  // the op each warp is working on
    const int wid = threadIdx.x >> 5;
    if (image_bytes > 0) {
        const uint4 *s = reinterpret_cast<const uint4 *>(image);
        int nw = (int)(image_bytes / 16);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) smem[i] = s[i];
        __syncthreads();
    }
    allow_dependents();
    prior_grids_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    Hint oh{-1, 0};
    Hint h{-1, 0}, rh{-1, 0};
    int64_t cur = -1;
    int64_t p = spread_first(sp, warp);
    for (int64_t j = warp; j < sp.nspans; j += nwarps, p = p + sp.inc >= sp.nspans ? p + sp.inc - sp.nspans : p + sp.inc) {
        const int64_t s0 = p * span;
        const int64_t s1 = min(s0 + span, ntiles);
        oh = Hint{-1, 0};  // spans lie far apart: find each span's first op by the warp
        for (int64_t t = s0; t < s1; t++) {
            int64_t i = warp_find_le_hint(tile0, nops, t, oh, 0, lane);
            const BatchOp *b = ops + i;
            if (i != cur) {
                h = Hint{-1, 0};
                rh = Hint{-1, 0};
                cur = i;
                load_op(wop[wid], b->op, lane);
            }
            const int soff = b->soff;
            const char *blob = soff >= 0 ? reinterpret_cast<const char *>(smem) + soff : b->d.blob;
            const DNode *nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
            const int64_t base = (t - tile0[i]) * 32;
            seg_round<W, PACK, false>(wop[wid], nodes, blob, b->nseg_elem, b->div_nseg, base, b->nsegs, lane, h, rh);
        }
    }
}

typedef void (*BatchKernel)(const BatchOp *, const int64_t *, int64_t, int64_t, int64_t, const char *, int64_t,
                            Spread);

template <bool PACK>
static BatchKernel pick_batch(int wsel)
{
    switch (wsel) {
    case 9: return batch_seg_kernel<8, PACK>;
    case 10: return batch_seg_kernel<4, PACK>;
    case 11: return batch_seg_kernel<2, PACK>;
    case 12: return batch_seg_kernel<1, PACK>;
    case kWideClass: return batch_kernel<16, PACK, true, true>;
    case 0: return batch_kernel<16, PACK, true>;
    case 1: return batch_kernel<8, PACK, true>;
    case 2: return batch_kernel<8, PACK, false>;
    case 3: return batch_kernel<4, PACK, true>;
    case 4: return batch_kernel<4, PACK, false>;
    case 5: return batch_kernel<2, PACK, true>;
    case 6: return batch_kernel<2, PACK, false>;
    case 7: return batch_kernel<1, PACK, true>;
    default: return batch_kernel<1, PACK, false>;
    }
}

// ---------------------------------------------------------------------------
// segment enumeration (§3.1 MPIX_Type_iov, device form)
// ---------------------------------------------------------------------------
struct IovArgs {
    dte_iov *out;
    int64_t *actual;
    const char *base;
    int64_t first;      // first segment index (over count elements)
    int64_t n;          // segments to write
    int64_t nseg;       // per element
    FastDiv div_nseg;
    int64_t extent;
    int64_t per_warp;
    // record-major lists (arrays of short records, rec_shape): runs per
    // record (0: off), records per element and their rounds of 32, and the
    // request's first round; per_warp then counts rounds
    int64_t rec_runs;
    int64_t nrec_elem;
    int64_t rounds_elem;
    FastDiv div_rounds;
    int64_t q_first;
    int64_t nrounds;
};

// Segments s0 .. s0 + nvalid - 1 (warp-uniform, 1 <= nvalid <= 32) of the
// count-level segment list: lane l < nvalid gets the displacement and length
// of segment s0 + l.  A round inside one element of a root index list over
// one shared child is decoded by the warp together (shared_list_round: one
// search, coalesced entry loads, shuffles); other rounds lane by lane.
__device__ __forceinline__ void iov_round(const Op &op, const DNode *nodes, const char *blob, int64_t nseg,
                                          const FastDiv &div_nseg, int64_t s0, int nvalid, int lane, Hint &h,
                                          Hint &rh, int64_t &disp, int64_t &len)
{
    const DNode &R = nodes[op.root];
    const int64_t e0 = fdiv(s0, div_nseg);
    const int64_t local0 = s0 - e0 * nseg;
    disp = 0;
    len = 0;
    if (shared_list_root(R) && local0 + nvalid <= nseg) {
        int64_t ps;
        shared_list_round(op, nodes, blob, R, e0, local0, nvalid, lane, rh, h, disp, len, ps);
    } else if (lane < nvalid) {
        const int64_t sl = s0 + lane;
        const int64_t e = fdiv(sl, div_nseg);
        disp = e * op.extent;
        decode_seg(nodes, blob, op.root, sl - e * nseg, disp, len, h);
    }
}

// Only the fields iov_round reads: the root and the element stride.
__device__ __forceinline__ Op iov_op(int32_t root, int64_t extent)
{
    Op op = {};
    op.root = root;
    op.extent = extent;
    return op;
}

// Warp w writes segments [w * per_warp, (w + 1) * per_warp) of the request
// (per_warp a multiple of 32) in rounds of 32 consecutive segments.
__global__ void __launch_bounds__(kThreads) iov_kernel(Desc d, IovArgs a)
{
    extern __shared__ uint4 smem[];
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t k0 = warp * a.per_warp;
    const int64_t k1 = min(k0 + a.per_warp, a.n);
    const Op op = iov_op(d.root, a.extent);
    Hint h{-1, 0}, rh{-1, 0};
    if (a.rec_runs > 0) {
        // one record per lane per round of 32 records (rec_locate); segment
        // k of the list is run k % runs of record k / runs
        const DNode &R = nodes[d.root];
        const DNode &C = nodes[R.child];
        const int64_t *cpb = C.kind == NK_RUN ? nullptr : arr<int64_t>(blob, C.a_pbytes);
        const int64_t *cdv = C.kind == NK_RUN ? nullptr : arr<int64_t>(blob, C.a_disp);
        const int64_t q0 = a.q_first + warp * a.per_warp;
        const int64_t q1 = min(q0 + a.per_warp, a.q_first + a.nrounds);
        for (int64_t q = q0; q < q1; q++) {
            const RecPlace at = rec_place(op, C, a.nrec_elem, a.rounds_elem, a.div_rounds, q);
            const int64_t ud = rec_locate(op, R, C, blob, at, lane, rh);
            if (lane >= at.nvalid) continue;
            const int64_t k0r = (at.e * a.nrec_elem + at.local0 + lane) * a.rec_runs - a.first;
#pragma unroll 1
            for (int j = 0; j < (int)a.rec_runs; j++) {
                const int64_t k = k0r + j;
                if (k < 0 || k >= a.n) continue;
                dte_iov v;
                v.iov_base = (void *)(a.base + ud + (cdv ? cdv[j] : 0));
                v.iov_len = cpb ? cpb[j + 1] - cpb[j] : C.len;
                a.out[k] = v;
            }
        }
        if (a.actual && blockIdx.x == 0 && threadIdx.x == 0) *a.actual = a.n;
        return;
    }
    for (int64_t kb = k0; kb < k1; kb += 32) {
        const int nvalid = (int)min((int64_t)32, k1 - kb);
        int64_t dd, len;
        iov_round(op, nodes, blob, a.nseg, a.div_nseg, a.first + kb, nvalid, lane, h, rh, dd, len);
        if (lane < nvalid) {
            dte_iov v;
            v.iov_base = (void *)(a.base + dd);
            v.iov_len = len;
            a.out[kb + lane] = v;
        }
    }
    if (a.actual && blockIdx.x == 0 && threadIdx.x == 0) *a.actual = a.n;
}

// Packed byte P (0 <= P < size) of one element of an array of short records
// (the rec_kernel shapes: `runs` runs per record, none merged) -> the index
// of its segment and the packed offset where that segment starts, without a
// search: records are contiguous in packed space, so P lies in record
// P / size(record), in the last run of it that starts at or before P.
__device__ __forceinline__ void rec_pos(const DNode *nodes, const char *blob, int root, int64_t runs, int64_t P,
                                        int64_t &k, int64_t &start)
{
    const DNode &C = nodes[nodes[root].child];
    const int64_t r = fdiv(P, C.div_size);
    const int64_t o = P - r * C.size;
    int64_t j = 0, pj = 0;
    if (C.kind != NK_RUN) {
        const int64_t *cpb = arr<int64_t>(blob, C.a_pbytes);
        while (j + 1 < runs && cpb[j + 1] <= o) j++;
        pj = cpb[j];
    }
    k = r * runs + j;
    start = r * C.size + pj;
}

// §3.1 MPIX_Type_iov_len for a batch of budgets
__global__ void __launch_bounds__(kThreads) iov_len_kernel(Desc d, int64_t nq, const int64_t *budget,
                                                           int64_t *out_len, int64_t *out_bytes, int64_t size,
                                                           int64_t nseg, int64_t rec_runs)
{
    extern __shared__ uint4 smem[];
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t B = budget[q];
        int64_t k, st;
        if (B < -1) {
            k = -1;
            st = -1;
        } else if (B == -1 || B >= size) {
            k = nseg;
            st = size;
        } else if (rec_runs > 0) {
            rec_pos(nodes, blob, d.root, rec_runs, B, k, st);
        } else {
            decode_pos(nodes, blob, d.root, B, k, st);
        }
        out_len[q] = k;
        out_bytes[q] = st;
    }
}

// byte offset -> first segment index and count (first pass of iov_at_bytes)
__global__ void __launch_bounds__(kThreads) at_bytes_first_kernel(Desc d, int64_t nq, const int64_t *off,
                                                                  int64_t maxlen, int64_t *first,
                                                                  int64_t *actual, int64_t size, int64_t nseg,
                                                                  int64_t rec_runs)
{
    extern __shared__ uint4 smem[];
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t B = off[q];
        if (B < 0 || B >= size) {
            first[q] = -1;
            actual[q] = 0;
            continue;
        }
        int64_t k, st;
        if (rec_runs > 0) rec_pos(nodes, blob, d.root, rec_runs, B, k, st);
        else decode_pos(nodes, blob, d.root, B, k, st);
        first[q] = k;
        actual[q] = min(maxlen, nseg - k);
    }
}

// Second pass: item it of the nq x maxlen output is segment first[q] + i of
// query q = it / maxlen (one element: segments below nseg).  Warp w fills
// items [w * per_warp, (w + 1) * per_warp) (per_warp a multiple of 32) in
// rounds of 32: a round inside one query is 32 consecutive segments and goes
// through iov_round; a round across two queries is decoded lane by lane.  A
// grid-wide stride would instead send every lookup to another query and
// search the index table from far away.
__global__ void __launch_bounds__(kThreads) at_bytes_fill_kernel(Desc d, int64_t nq, int64_t maxlen,
                                                                 FastDiv div_max, const int64_t *first,
                                                                 const int64_t *actual, dte_iov *out,
                                                                 const char *base, int64_t nseg, FastDiv div_nseg,
                                                                 int64_t per_warp)
{
    extern __shared__ uint4 smem[];
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t total = nq * maxlen;
    const int64_t i0 = warp * per_warp;
    const int64_t i1 = min(i0 + per_warp, total);
    const Op op = iov_op(d.root, 0);
    Hint h{-1, 0}, rh{-1, 0};
    for (int64_t ib = i0; ib < i1; ib += 32) {
        const int n = (int)min((int64_t)32, i1 - ib);
        const int64_t qb = fdiv(ib, div_max);
        const int64_t jb = ib - qb * maxlen;
        if (jb + n <= maxlen) {
            // one query: segments first[qb] + jb onward, cut at its count
            const int nv = (int)max((int64_t)0, min((int64_t)n, actual[qb] - jb));
            if (nv == 0) continue;
            int64_t dd, len;
            iov_round(op, nodes, blob, nseg, div_nseg, first[qb] + jb, nv, lane, h, rh, dd, len);
            if (lane < nv) {
                dte_iov v;
                v.iov_base = (void *)(base + dd);
                v.iov_len = len;
                out[ib + lane] = v;
            }
            continue;
        }
        const int64_t it = ib + lane;
        if (lane >= n) continue;
        const int64_t q = fdiv(it, div_max);
        const int64_t i = it - q * maxlen;
        if (i >= actual[q]) continue;
        int64_t dd = 0, len = 0;
        decode_seg(nodes, blob, d.root, first[q] + i, dd, len, h);
        dte_iov v;
        v.iov_base = (void *)(base + dd);
        v.iov_len = len;
        out[it] = v;
    }
}

// Second pass for arrays of short records (the rec_kernel shapes, one
// element: segment k is run k % runs of record k / runs).  Query q's
// segments first[q] .. first[q] + actual[q] - 1 lie in rounds of 32 records;
// task t = q * cpq + c (a warp each, grid-stride) takes rounds c * kRecIovSpan
// onward of its query, one record per lane, and writes the record's runs that
// fall inside the query.
constexpr int64_t kRecIovSpan = 16;  // rounds of 32 records per task

__global__ void __launch_bounds__(kThreads) at_bytes_fill_rec_kernel(Desc d, int64_t nq, int64_t maxlen,
                                                                     const int64_t *first, const int64_t *actual,
                                                                     dte_iov *out, const char *base, int64_t runs,
                                                                     int64_t nrec, FastDiv div_rounds, int64_t cpq)
{
    extern __shared__ uint4 smem[];
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    const DNode &R = nodes[d.root];
    const DNode &C = nodes[R.child];
    const int64_t *cpb = C.kind == NK_RUN ? nullptr : arr<int64_t>(blob, C.a_pbytes);
    const int64_t *cdv = C.kind == NK_RUN ? nullptr : arr<int64_t>(blob, C.a_disp);
    const Op op = iov_op(d.root, 0);
    const int64_t rounds_elem = (nrec + 31) / 32;
    Hint rh{-1, 0};
    for (int64_t t = warp; t < nq * cpq; t += nwarps) {
        const int64_t q = t / cpq;
        const int64_t c = t - q * cpq;
        const int64_t f = first[q], cnt = actual[q];
        if (cnt <= 0) continue;
        rh = Hint{-1, 0};  // queries land anywhere: a cold search by the warp
        const int64_t qa = f / runs / 32, qb = (f + cnt - 1) / runs / 32;  // the query's rounds
        const int64_t q0 = qa + c * kRecIovSpan;
        const int64_t q1 = min(q0 + kRecIovSpan, qb + 1);
        dte_iov *o = out + q * maxlen;
        for (int64_t rq = q0; rq < q1; rq++) {
            const RecPlace at = rec_place(op, C, nrec, rounds_elem, div_rounds, rq);
            const int64_t ud = rec_locate(op, R, C, blob, at, lane, rh);
            if (lane >= at.nvalid) continue;
            const int64_t k0 = (at.local0 + lane) * runs - f;
#pragma unroll 1
            for (int j = 0; j < (int)runs; j++) {
                const int64_t k = k0 + j;
                if (k < 0 || k >= cnt) continue;
                dte_iov v;
                v.iov_base = (void *)(base + ud + (cdv ? cdv[j] : 0));
                v.iov_len = cpb ? cpb[j + 1] - cpb[j] : C.len;
                o[k] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// adjoint of the typed float32 pack: gx[src(k)] += gy[k]
// ---------------------------------------------------------------------------
// Layouts without repeated bytes: every destination float receives exactly
// one term, so a scatter with a float add (gx usually zero) reproduces the
// adjoint exactly.  Same work split as move_kernel with 4-byte words.
template <bool PK16>
__global__ void __launch_bounds__(kThreads, kMinBlocks) adjoint_kernel(Desc d, Op op, int64_t nchunks, int64_t span)
{
    extern __shared__ uint4 smem[];
    __shared__ uint4 scratch[kThreads];
    char *scr = reinterpret_cast<char *>(&scratch[threadIdx.x]);
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kWarps * span;
    Hint h{-1, 0};
    for (int64_t c0 = warp * span; c0 < nchunks; c0 += stride) {
        const int64_t c1 = min(c0 + span, nchunks);
        for (int64_t base = c0; base < c1; base += kStep) {
            uint4 v[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) {
                int64_t c = base + u * 32 + lane;
                if (c < c1) {
                    int nb = (int)(op.total - c * 16 < 16 ? op.total - c * 16 : 16);
                    v[u] = load_packed<4, PK16>(op.packed_in + c * 16, nb);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; u++) {
                int64_t c = base + u * 32 + lane;
                if (c < c1) {
                    int64_t P = c * 16;
                    int nb = (int)(op.total - P < 16 ? op.total - P : 16);
                    // one descriptor walk per run (see gather_chunk)
                    *reinterpret_cast<uint4 *>(scr) = v[u];
                    int got = 0;
#pragma unroll 1
                    while (got < nb) {
                        int64_t dd, rem;
                        locate(op, nodes, blob, P + got, dd, rem, h);
                        const int take = rem < (int64_t)(nb - got) ? (int)rem : nb - got;
                        float *p = reinterpret_cast<float *>(op.user_out + dd);
#pragma unroll
                        for (int k = 0; k < 4; k++)
                            if (k * 4 < take) p[k] = p[k] + *reinterpret_cast<const float *>(scr + got + 4 * k);
                        got += take;
                    }
                }
            }
        }
    }
}

// Layouts that repeat entries: one thread per destination float sums its
// sources in packed order in FP64 (deterministic), then adds the rounded sum.
__global__ void __launch_bounds__(kThreads) adjoint_csr_kernel(const int64_t *rows, const int64_t *dest,
                                                               const int64_t *cols, int64_t ndest, const float *gy,
                                                               float *gx)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < ndest;
         u += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t j = rows[u]; j < rows[u + 1]; j++) s += (double)__ldg(gy + cols[j]);
        float *p = gx + dest[u];
        *p = *p + (float)s;
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
typedef void (*MoveKernel)(Desc, Op, int64_t, int64_t, Spread);



template <bool PACK>
static MoveKernel pick_move(int W, bool pk16, bool wide)
{
    switch (W) {
    case 16: return wide ? move_kernel<16, PACK, true, true> : move_kernel<16, PACK, true>;
    case 8: return pk16 ? move_kernel<8, PACK, true> : move_kernel<8, PACK, false>;
    case 4: return pk16 ? move_kernel<4, PACK, true> : move_kernel<4, PACK, false>;
    case 2: return pk16 ? move_kernel<2, PACK, true> : move_kernel<2, PACK, false>;
    default: return pk16 ? move_kernel<1, PACK, true> : move_kernel<1, PACK, false>;
    }
}

typedef void (*RecKernelFn)(Desc, Op, int64_t, int64_t, FastDiv, int64_t, int64_t);

template <int W, bool PACK>
static RecKernelFn pick_rec_w(bool stage)
{
    return stage ? rec_kernel<W, PACK, true> : rec_kernel<W, PACK, false>;
}

static RecKernelFn pick_rec(int W, bool pack, bool stage)
{
    switch (W) {
    case 8: return pack ? pick_rec_w<8, true>(stage) : pick_rec_w<8, false>(stage);
    case 4: return pack ? pick_rec_w<4, true>(stage) : pick_rec_w<4, false>(stage);
    case 2: return pack ? pick_rec_w<2, true>(stage) : pick_rec_w<2, false>(stage);
    default: return pack ? pick_rec_w<1, true>(stage) : pick_rec_w<1, false>(stage);
    }
}

// The bulk kernels use more than the default 48 KiB of dynamic shared
// memory (stages + staged descriptor); raised once per device.
static void allow_bulk_smem(int dev)
{
    static std::atomic<bool> done[64];
    if (done[dev & 63].load(std::memory_order_acquire)) return;
    const int bytes = (int)(kSmemBlob + 128 + kBulkSmem);
    cudaFuncSetAttribute(bulk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(bulk_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaGetLastError();
    done[dev & 63].store(true, std::memory_order_release);
}

// The bulk copies are used only between buffers in device memory; pinned or
// managed host memory (which the other kernels read and write directly)
// keeps the chunk-major path.
static bool device_memory(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}

// Count-level index of the segment holding packed-stream byte B (< count*size).
static int64_t segment_of(const Committed &c, int64_t B)
{
    int64_t e = B / c.size, k = 0, start = 0;
    decode_pos(c.nodes(), c.blob(), c.root, B - e * c.size, k, start);
    return e * c.nseg + k;
}

// Move packed-stream bytes [first, first + nbytes) of `count` elements
// (nbytes > 0); `packed` holds just those bytes.  A whole move is
// first = 0, nbytes = count * size.
static int launch_move(bool pack, dte_type t, const char *dblob, const void *user, void *packed, int64_t count,
                       int64_t first, int64_t nbytes, cudaStream_t stream, int dev)
{
    Committed &c = *t->desc;
    Op op = make_op(c, t->extent(), user, packed, count);
    op.pbase = first;
    op.total = nbytes;
    if (op.total == 0) return DTE_SUCCESS;
    int W = word_of(c, t->extent(), count, user, packed);
    if (first != 0 || nbytes != count * c.size) W = (int)std::min<int64_t>(W, std::min(p2v(first), p2v(nbytes)));
    const int plan = t->plan;
    bool pk16 = p2addr(packed) >= 16;
    const bool wide = plan_wide(W, plan);
    MoveKernel k = pack ? pick_move<true>(W, pk16, wide) : pick_move<false>(W, pk16, wide);
    size_t smem = 0;
    Desc d = make_desc(c, dblob, &smem);
    // occupancy per (device, direction, variant, staging mode); the staged
    // blob is sized for its upper bound
    static thread_local int occ_cache[64][2][kNumClasses][3];
    int &occ = occ_cache[dev & 63][pack ? 1 : 0][wide ? kWideClass : wsel_of(W, pk16)][d.stage];
    if (occ == 0) occ = occupancy(k, d.stage == STAGE_BLOB ? (size_t)kSmemBlob : smem);
    int64_t max_blocks = (int64_t)sm_count(dev) * occ;
    int64_t max_warps = max_blocks * kWarps;
    int64_t rec_size = 0;
    if (plan_seg(c, W, plan) && kRec && first == 0 && nbytes == count * c.size && rec_shape(c, &rec_size)) {
        // an array of short records under a large index list: one record
        // per lane per round
        const int64_t nrec = c.size / rec_size;
        const int64_t rounds_elem = (nrec + 31) / 32;
        const int64_t nrounds = count * rounds_elem;
        const bool stage = kRecStage && rec_size % 16 != 0 && rec_size <= kRecStageMaxSize &&
                           p2addr(packed) >= 16 && (count == 1 || c.size % 16 == 0);
        RecKernelFn rk = pick_rec(W, pack, stage);
        static thread_local int rocc_cache[64][2][4][2][3];
        int &rocc = rocc_cache[dev & 63][pack ? 1 : 0][W == 8 ? 0 : W == 4 ? 1 : W == 2 ? 2 : 3][stage ? 1 : 0]
                              [d.stage];
        if (rocc == 0) rocc = occupancy(rk, d.stage == STAGE_BLOB ? (size_t)kSmemBlob : smem);
        const int64_t slots = (int64_t)sm_count(dev) * rocc * kWarps;
        const int64_t span_rounds = std::max<int64_t>(1, std::min<int64_t>(8, nrounds / slots));
        const int64_t units = (nrounds + span_rounds - 1) / span_rounds;
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((units + kWarps - 1) / kWarps,
                                                                      (int64_t)sm_count(dev) * rocc));
        if (launch_overlapped(rk, (unsigned)blocks, kThreads, smem, stream, d, op, nrec, rounds_elem,
                              make_div(rounds_elem), nrounds, span_rounds) != cudaSuccess) {
            cudaGetLastError();
            return DTE_ERR_CUDA;
        }
        return DTE_SUCCESS;
    }
    if (plan_seg(c, W, plan)) {
        // short runs, small words: one decode per segment, cooperative copy
        typedef void (*SegKernel)(Desc, Op, int64_t, FastDiv, int64_t, int64_t, int64_t);
        SegKernel sk;
        switch (W) {
        case 8: sk = pack ? seg_kernel<8, true> : seg_kernel<8, false>; break;
        case 4: sk = pack ? seg_kernel<4, true> : seg_kernel<4, false>; break;
        case 2: sk = pack ? seg_kernel<2, true> : seg_kernel<2, false>; break;
        default: sk = pack ? seg_kernel<1, true> : seg_kernel<1, false>; break;
        }
        static thread_local int socc_cache[64][2][4][3];
        int &socc = socc_cache[dev & 63][pack ? 1 : 0][W == 8 ? 0 : W == 4 ? 1 : W == 2 ? 2 : 3][d.stage];
        if (socc == 0) socc = occupancy(sk, d.stage == STAGE_BLOB ? (size_t)kSmemBlob : smem);
        int64_t seg0 = first == 0 ? 0 : segment_of(c, first);
        int64_t nsegs = (first + nbytes == count * c.size ? count * c.nseg : segment_of(c, first + nbytes - 1) + 1) - seg0;
        int64_t rounds = (nsegs + 31) / 32;
        int64_t span_rounds = std::max<int64_t>(1, std::min<int64_t>(8, rounds / ((int64_t)sm_count(dev) * socc * kWarps)));
        int64_t units = (rounds + span_rounds - 1) / span_rounds;
        int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((units + kWarps - 1) / kWarps,
                                                                (int64_t)sm_count(dev) * socc));
        if (launch_overlapped(sk, (unsigned)blocks, kThreads, smem, stream, d, op, c.nseg,
                              c.nodes()[c.root].div_nseg, seg0, nsegs, (int64_t)32 * span_rounds) != cudaSuccess) {
            cudaGetLastError();
            return DTE_ERR_CUDA;
        }
        return DTE_SUCCESS;
    }
    const bool bulk_rule = plan == DTE_PLAN_BULK ||
                           (plan == DTE_PLAN_AUTO && kBulk &&
                            nbytes >= kBulkMinTilesPerWarp * kBulkWarps * kBulkTile * sm_count(dev) &&
                            c.nseg > 0 && c.size / c.nseg >= kBulkMinRun);
    if (bulk_rule && W == 16 && c.nseg > 0 && device_memory(user) && device_memory(packed)) {
        // long runs: bulk copies by the copy engine of each SM (bulk.cuh)
        allow_bulk_smem(dev);
        const int64_t buf_off = ((int64_t)smem + 127) & ~(int64_t)127;
        const int64_t ntiles = (nbytes + kBulkTile - 1) / kBulkTile;
        const int64_t blocks =
            std::max<int64_t>(1, std::min<int64_t>((ntiles + kBulkWarps - 1) / kBulkWarps, sm_count(dev)));
        auto bk = pack ? bulk_kernel<true> : bulk_kernel<false>;
        if (launch_overlapped(bk, (unsigned)blocks, kBulkWarps * 32, (size_t)(buf_off + kBulkSmem), stream, d, op,
                              ntiles, (int32_t)buf_off) != cudaSuccess) {
            cudaGetLastError();
            return DTE_ERR_CUDA;
        }
        return DTE_SUCCESS;
    }
    int64_t nchunks = (op.total + 15) / 16;
    const int64_t step = step_of_word(W, wide);
    int64_t steps = (nchunks + step - 1) / step;
    // span: one step when the descriptor sits in shared memory; up to eight
    // when index tables are searched in global memory (consecutive steps
    // reuse the search position), but never so many that warps go idle
    int64_t span_steps = d.stage == STAGE_BLOB ? 1 : std::max<int64_t>(1, std::min<int64_t>(8, steps / max_warps));
    int64_t units = (steps + span_steps - 1) / span_steps;
    int64_t blocks = std::min<int64_t>((units + kWarps - 1) / kWarps, max_blocks);
    if (blocks < 1) blocks = 1;
    if (launch_overlapped(k, (unsigned)blocks, kThreads, smem, stream, d, op, nchunks, span_steps * step,
                          make_spread(units, blocks * kWarps)) != cudaSuccess) {
        cudaGetLastError();
        return DTE_ERR_CUDA;
    }
    return DTE_SUCCESS;
}

}  // namespace dte

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
namespace dte {
struct BatchGroup {     // ops of one copy-word class, launched together
    int wsel;
    int64_t op0, nops;  // range in the (grouped) op table
    int64_t t0;         // offset of this group's tile prefix in the prefix table
    int64_t ntiles;
    int occ;
    int64_t image_off;  // staged descriptor image (bytes into the batch image)
    int64_t image_bytes;  // 0: descriptors are read from global memory
};
}  // namespace dte

struct dte_batch_s {
    int kind = 0;  // DTE_BATCH_PACK or DTE_BATCH_UNPACK
    int device = -1;
    int64_t nops = 0, ntiles = 0;
    char *dmem = nullptr;  // BatchOp[nops] followed by the groups' int64 tile prefixes
    dte::BatchOp *d_ops = nullptr;
    int64_t *d_tile0 = nullptr;
    char *d_image = nullptr;
    std::vector<dte::BatchGroup> groups;
    std::vector<std::shared_ptr<dte::Committed>> keep;  // descriptors in use
    std::vector<std::pair<void *, void *>> uses;        // (stream, event)
    bool captured = false;
    int blocks_per_sm = 0;          // 0: occupancy limit
    int64_t span_tiles = 1;         // consecutive tiles a warp takes at a time
};

namespace dte {

static std::mutex g_bmu;
static std::vector<dte_batch> *g_bdeferred = new std::vector<dte_batch>();
static std::vector<dte_batch> *g_blive = new std::vector<dte_batch>();

static bool batch_idle(dte_batch b)
{
    if (b->captured) return false;
    for (auto &u : b->uses)
        if (cudaEventQuery((cudaEvent_t)u.second) == cudaErrorNotReady) return false;
    return true;
}

static void batch_destroy(dte_batch b)
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (b->device >= 0) cudaSetDevice(b->device);
    for (auto &u : b->uses) cudaEventDestroy((cudaEvent_t)u.second);
    if (b->dmem) cudaFree(b->dmem);
    if (cur >= 0) cudaSetDevice(cur);
    delete b;
}

static void reap_batches()
{
    std::vector<dte_batch> done;
    {
        std::lock_guard<std::mutex> g(g_bmu);
        auto &v = *g_bdeferred;
        for (size_t i = 0; i < v.size();) {
            if (batch_idle(v[i])) {
                done.push_back(v[i]);
                v[i] = v.back();
                v.pop_back();
            } else {
                i++;
            }
        }
    }
    for (auto b : done) batch_destroy(b);
}

static bool batch_valid(dte_batch b)
{
    std::lock_guard<std::mutex> g(g_bmu);
    return b && std::find(g_blive->begin(), g_blive->end(), b) != g_blive->end();
}

}  // namespace dte

using namespace dte;

extern "C" {

int dte_pack_enqueue(const void *inbuf, int64_t incount, dte_type type, void *outbuf, int64_t outsize,
                     int64_t *position, dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_pack_enqueue");
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (!position || incount < 0 || outsize < 0 || *position < 0 || *position > outsize)
            return DTE_ERR_ARG;
        int64_t need;
        if (__builtin_mul_overflow(incount, type->size, &need)) return DTE_ERR_OVERFLOW;
        if (outsize - *position < need) return DTE_ERR_TRUNCATE;
        if (need == 0) return DTE_SUCCESS;
        if (!inbuf || !outbuf) return DTE_ERR_ARG;
        const char *blob;
        int dev;
        if (int rc = prep(type, stream, &blob, &dev)) return rc;
        int rc = launch_move(true, type, blob, inbuf, (char *)outbuf + *position, incount, 0, need,
                             (cudaStream_t)stream, dev);
        if (rc) return rc;
        note_use(type, dev, stream);
        *position += need;
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

int dte_unpack_enqueue(const void *inbuf, int64_t insize, int64_t *position, void *outbuf, int64_t outcount,
                       dte_type type, dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_unpack_enqueue");
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (!position || outcount < 0 || insize < 0 || *position < 0 || *position > insize)
            return DTE_ERR_ARG;
        int64_t need;
        if (__builtin_mul_overflow(outcount, type->size, &need)) return DTE_ERR_OVERFLOW;
        if (insize - *position < need) return DTE_ERR_TRUNCATE;
        if (need == 0) return DTE_SUCCESS;
        if (!inbuf || !outbuf) return DTE_ERR_ARG;
        if (committed_overlaps(*type->desc, outcount, type->extent())) return DTE_ERR_OVERLAP;
        const char *blob;
        int dev;
        if (int rc = prep(type, stream, &blob, &dev)) return rc;
        int rc = launch_move(false, type, blob, outbuf, (char *)inbuf + *position, outcount, 0, need,
                             (cudaStream_t)stream, dev);
        if (rc) return rc;
        note_use(type, dev, stream);
        *position += need;
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

int dte_pack_range_enqueue(const void *inbuf, int64_t incount, dte_type type, int64_t first, int64_t nbytes,
                           void *outbuf, dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_pack_range_enqueue");
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (incount < 0 || first < 0 || nbytes < 0) return DTE_ERR_ARG;
        int64_t total, end;
        if (__builtin_mul_overflow(incount, type->size, &total)) return DTE_ERR_OVERFLOW;
        if (__builtin_add_overflow(first, nbytes, &end) || end > total) return DTE_ERR_ARG;
        if (nbytes == 0) return DTE_SUCCESS;
        if (!inbuf || !outbuf) return DTE_ERR_ARG;
        const char *blob;
        int dev;
        if (int rc = prep(type, stream, &blob, &dev)) return rc;
        if (int rc = launch_move(true, type, blob, inbuf, outbuf, incount, first, nbytes, (cudaStream_t)stream, dev))
            return rc;
        note_use(type, dev, stream);
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

int dte_unpack_range_enqueue(const void *inbuf, int64_t first, int64_t nbytes, void *outbuf, int64_t outcount,
                             dte_type type, dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_unpack_range_enqueue");
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (outcount < 0 || first < 0 || nbytes < 0) return DTE_ERR_ARG;
        int64_t total, end;
        if (__builtin_mul_overflow(outcount, type->size, &total)) return DTE_ERR_OVERFLOW;
        if (__builtin_add_overflow(first, nbytes, &end) || end > total) return DTE_ERR_ARG;
        if (nbytes == 0) return DTE_SUCCESS;
        if (!inbuf || !outbuf) return DTE_ERR_ARG;
        if (committed_overlaps(*type->desc, outcount, type->extent())) return DTE_ERR_OVERLAP;
        const char *blob;
        int dev;
        if (int rc = prep(type, stream, &blob, &dev)) return rc;
        if (int rc = launch_move(false, type, blob, outbuf, const_cast<void *>(inbuf), outcount, first, nbytes,
                                 (cudaStream_t)stream, dev))
            return rc;
        note_use(type, dev, stream);
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

// Send-to-self pipeline (§5.2's enqueued send and receive on one stream):
// the message is cut into windows that end on segment boundaries of the send
// layout (the byte-window form of the iov-length query, §3.1) unless a
// single segment is longer than the window; each window is packed into the
// sender half of `staging`, copied to the receiver half (the transfer), and
// unpacked from there, all in stream order.
int dte_sendrecv_enqueue(const void *sendbuf, int64_t sendcount, dte_type sendtype, void *recvbuf,
                         int64_t recvcount, dte_type recvtype, void *staging, int64_t staging_bytes,
                         dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_sendrecv_enqueue");
    try {
        if (!handle_valid(sendtype) || !handle_valid(recvtype)) return DTE_ERR_TYPE;
        if (!sendtype->committed || !recvtype->committed) return DTE_ERR_TYPE;
        if (sendcount < 0 || recvcount < 0 || staging_bytes < 0) return DTE_ERR_ARG;
        int64_t S, R;
        if (__builtin_mul_overflow(sendcount, sendtype->size, &S) ||
            __builtin_mul_overflow(recvcount, recvtype->size, &R))
            return DTE_ERR_OVERFLOW;
        if (S > R) return DTE_ERR_TRUNCATE;
        if (S == 0) return DTE_SUCCESS;
        const int64_t window = (staging_bytes / 2) & ~(int64_t)15;
        if (!sendbuf || !recvbuf || !staging || window <= 0) return DTE_ERR_ARG;
        if (committed_overlaps(*recvtype->desc, recvcount, recvtype->extent())) return DTE_ERR_OVERLAP;
        const char *sblob, *rblob;
        int dev, rdev;
        if (int rc = prep(sendtype, stream, &sblob, &dev)) return rc;
        if (int rc = prep(recvtype, stream, &rblob, &rdev)) return rc;
        char *tx = (char *)staging, *rx = (char *)staging + window;
        const Committed &sc = *sendtype->desc;
        const cudaStream_t st = (cudaStream_t)stream;
        for (int64_t off = 0; off < S;) {
            int64_t end = std::min(S, off + window);
            if (end < S) {
                int64_t e = end / sc.size, k = 0, start = 0;
                decode_pos(sc.nodes(), sc.blob(), sc.root, end - e * sc.size, k, start);
                if (e * sc.size + start > off) end = e * sc.size + start;
            }
            const int64_t n = end - off;
            if (int rc = launch_move(true, sendtype, sblob, sendbuf, tx, sendcount, off, n, st, dev)) return rc;
            if (cudaMemcpyAsync(rx, tx, (size_t)n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                cudaGetLastError();
                return DTE_ERR_CUDA;
            }
            if (int rc = launch_move(false, recvtype, rblob, recvbuf, rx, recvcount, off, n, st, rdev)) return rc;
            off = end;
        }
        note_use(sendtype, dev, stream);
        note_use(recvtype, rdev, stream);
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

int dte_batch_create(int kind, int64_t nops, const dte_op *ops, dte_batch *out)
{
    dte_batch b = nullptr;
    try {
        if (!out || nops < 0 || (nops > 0 && !ops)) return DTE_ERR_ARG;
        if (kind != DTE_BATCH_PACK && kind != DTE_BATCH_UNPACK) return DTE_ERR_ARG;
        reap_batches();
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return DTE_ERR_NODEVICE;
        }
        std::vector<BatchOp> hops((size_t)nops);
        std::vector<const Committed *> hc((size_t)nops, nullptr);
        b = new dte_batch_s();
        b->kind = kind;
        b->device = dev;
        int rc = DTE_SUCCESS;
        for (int64_t i = 0; i < nops && rc == DTE_SUCCESS; i++) {
            const dte_op &o = ops[i];
            BatchOp &h = hops[(size_t)i];
            std::memset(&h, 0, sizeof h);
            if (!handle_valid(o.type) || !o.type->committed) { rc = DTE_ERR_TYPE; break; }
            if (o.count < 0) { rc = DTE_ERR_ARG; break; }
            int64_t total;
            if (__builtin_mul_overflow(o.count, o.type->size, &total)) { rc = DTE_ERR_OVERFLOW; break; }
            if (total > 0) {
                if (!o.user || !o.packed) { rc = DTE_ERR_ARG; break; }
                if (kind == DTE_BATCH_UNPACK && committed_overlaps(*o.type->desc, o.count, o.type->extent())) {
                    rc = DTE_ERR_OVERLAP;
                    break;
                }
                const char *dblob;
                int d2;
                if ((rc = device_blob(o.type, &dblob, &d2)) != DTE_SUCCESS) break;
                Committed &c = *o.type->desc;
                hc[(size_t)i] = &c;
                fill_batch_op(h, c, o.type->extent(), o, dblob, o.type->plan);
                b->keep.push_back(o.type->desc);
            }
        }
        if (rc != DTE_SUCCESS) {
            delete b;
            return rc;
        }
        // group the non-empty ops by kernel variant, keeping their order
        std::vector<BatchOp> grouped;
        std::vector<const Committed *> gc;
        std::vector<int64_t> prefix;
        std::vector<char> image;  // staged descriptor images of all groups
        grouped.reserve((size_t)nops);
        for (int w = 0; w < kNumClasses; w++) {
            BatchGroup g{w, (int64_t)grouped.size(), 0, (int64_t)prefix.size(), 0, 0, 0, 0};
            prefix.push_back(0);
            for (size_t i = 0; i < hops.size(); i++) {
                const BatchOp &h = hops[i];
                if (h.nchunks == 0 || h.wsel != w) continue;
                grouped.push_back(h);
                gc.push_back(hc[i]);
                prefix.push_back(prefix.back() + op_tiles(h));
            }
            g.nops = (int64_t)grouped.size() - g.op0;
            if (g.nops == 0) {
                prefix.pop_back();
                continue;
            }
            g.ntiles = prefix.back();
            // stage the group's distinct descriptors together if they fit
            std::vector<std::pair<const Committed *, int64_t>> at;
            int64_t img = 0;
            for (int64_t i = g.op0; i < g.op0 + g.nops; i++) {
                bool found = false;
                for (auto &p : at) found = found || p.first == gc[(size_t)i];
                if (!found) {
                    at.push_back({gc[(size_t)i], img});
                    img += (gc[(size_t)i]->bytes + 15) & ~(int64_t)15;
                }
                if (img > kSmemBlob) break;
            }
            if (img <= kSmemBlob) {
                g.image_off = (int64_t)image.size();
                g.image_bytes = img;
                image.resize(image.size() + (size_t)img, 0);
                for (auto &p : at) std::memcpy(image.data() + g.image_off + p.second, p.first->blob(), p.first->bytes);
                for (int64_t i = g.op0; i < g.op0 + g.nops; i++)
                    for (auto &p : at)
                        if (p.first == gc[(size_t)i]) grouped[(size_t)i].soff = (int32_t)p.second;
            }
            BatchKernel k = kind == DTE_BATCH_PACK ? pick_batch<true>(w) : pick_batch<false>(w);
            g.occ = occupancy(k, (size_t)g.image_bytes);
            b->groups.push_back(g);
            b->ntiles += g.ntiles;
        }
        b->nops = (int64_t)grouped.size();
        size_t ops_bytes = (grouped.size() * sizeof(BatchOp) + 15) & ~(size_t)15;
        size_t pre_bytes = ((prefix.size() + 1) * sizeof(int64_t) + 15) & ~(size_t)15;
        size_t bytes = ops_bytes + pre_bytes + image.size();
        if (cudaMalloc(&b->dmem, bytes) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return DTE_ERR_NOMEM;
        }
        b->d_ops = reinterpret_cast<BatchOp *>(b->dmem);
        b->d_tile0 = reinterpret_cast<int64_t *>(b->dmem + ops_bytes);
        b->d_image = b->dmem + ops_bytes + pre_bytes;
        if ((!grouped.empty() && cudaMemcpy(b->d_ops, grouped.data(), grouped.size() * sizeof(BatchOp),
                                            cudaMemcpyHostToDevice) != cudaSuccess) ||
            (!prefix.empty() && cudaMemcpy(b->d_tile0, prefix.data(), prefix.size() * sizeof(int64_t),
                                           cudaMemcpyHostToDevice) != cudaSuccess) ||
            (!image.empty() &&
             cudaMemcpy(b->d_image, image.data(), image.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
            batch_destroy(b);
            return DTE_ERR_CUDA;
        }
        std::sort(b->keep.begin(), b->keep.end());
        b->keep.erase(std::unique(b->keep.begin(), b->keep.end()), b->keep.end());
        {
            std::lock_guard<std::mutex> g(g_bmu);
            g_blive->push_back(b);
        }
        *out = b;
        return DTE_SUCCESS;
    } catch (const Error &e) {
        delete b;
        return e.code;
    } catch (...) {
        delete b;
        return DTE_ERR_NOMEM;
    }
}

int dte_batch_set_launch(dte_batch batch, int blocks_per_sm, int64_t span_tiles)
{
    if (!batch_valid(batch) || blocks_per_sm < 0 || span_tiles < 1) return DTE_ERR_ARG;
    batch->blocks_per_sm = blocks_per_sm;
    batch->span_tiles = span_tiles;
    return DTE_SUCCESS;
}

int dte_batch_enqueue(dte_batch b, dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_batch_enqueue");
    if (!batch_valid(b)) return DTE_ERR_ARG;
    if (b->ntiles == 0) return DTE_SUCCESS;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return DTE_ERR_ARG;
    for (const BatchGroup &g : b->groups) {
        int per_sm = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, g.occ) : g.occ;
        int64_t max_blocks = (int64_t)sm_count(dev) * per_sm;
        int64_t span = b->span_tiles;
        int64_t units = (g.ntiles + span - 1) / span;
        int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((units + kWarps - 1) / kWarps, max_blocks));
        BatchKernel k = b->kind == DTE_BATCH_PACK ? pick_batch<true>(g.wsel) : pick_batch<false>(g.wsel);
        if (launch_overlapped(k, (unsigned)blocks, kThreads, (size_t)g.image_bytes, (cudaStream_t)stream,
                              (const BatchOp *)(b->d_ops + g.op0), (const int64_t *)(b->d_tile0 + g.t0), g.nops,
                              g.ntiles, span, (const char *)(b->d_image + g.image_off), g.image_bytes,
                              make_spread(units, blocks * kWarps)) != cudaSuccess) {
            cudaGetLastError();
            return DTE_ERR_CUDA;
        }
        if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
    }
    if (capturing(stream)) {
        b->captured = true;
        return DTE_SUCCESS;
    }
    for (auto &u : b->uses) {
        if (u.first == (void *)stream) {
            cudaEventRecord((cudaEvent_t)u.second, (cudaStream_t)stream);
            return DTE_SUCCESS;
        }
    }
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ev, (cudaStream_t)stream);
        b->uses.push_back({(void *)stream, (void *)ev});
    }
    return DTE_SUCCESS;
}

int dte_batch_free(dte_batch *batch)
{
    if (!batch || !batch_valid(*batch)) return DTE_ERR_ARG;
    dte_batch b = *batch;
    bool idle;
    {
        std::lock_guard<std::mutex> g(g_bmu);
        g_blive->erase(std::find(g_blive->begin(), g_blive->end(), b));
        idle = batch_idle(b);
        if (!idle) g_bdeferred->push_back(b);
    }
    if (idle) batch_destroy(b);
    *batch = nullptr;
    reap_batches();
    return DTE_SUCCESS;
}

static int batch_once(int kind, int64_t nops, const dte_op *ops, dte_stream_t stream)
{
    dte_batch b = nullptr;
    int rc = dte_batch_create(kind, nops, ops, &b);
    if (rc) return rc;
    rc = dte_batch_enqueue(b, stream);
    int rc2 = dte_batch_free(&b);
    return rc ? rc : rc2;
}

int dte_pack_batch_enqueue(int64_t nops, const dte_op *ops, dte_stream_t stream)
{
    return batch_once(DTE_BATCH_PACK, nops, ops, stream);
}

int dte_unpack_batch_enqueue(int64_t nops, const dte_op *ops, dte_stream_t stream)
{
    return batch_once(DTE_BATCH_UNPACK, nops, ops, stream);
}

// Runs per record when a type is an array of short records whose every run
// is its own segment (the shapes the record-major kernels take), else 0.
static int64_t rec_runs_of(const Committed &c)
{
    int64_t rsz = 0;
    if (!kRec || !rec_shape(c, &rsz)) return 0;
    const DNode &C = c.nodes()[c.nodes()[c.root].child];
    const int64_t runs = C.kind == NK_RUN ? 1 : C.count;
    return (c.size / rsz) * runs == c.nseg ? runs : 0;
}

int dte_type_iov_async(dte_type type, int64_t count, int64_t iov_offset, dte_iov *d_iov, int64_t max_iov_len,
                       int64_t *d_actual_iov_len, const void *base, dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_type_iov_async");
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (count < 0 || iov_offset < 0 || max_iov_len < 0 || (max_iov_len > 0 && !d_iov))
            return DTE_ERR_ARG;
        Committed &c = *type->desc;
        int64_t total;
        if (__builtin_mul_overflow(count, c.nseg, &total)) return DTE_ERR_OVERFLOW;
        int64_t n = iov_offset >= total ? 0 : std::min(max_iov_len, total - iov_offset);
        const char *blob;
        int dev;
        if (int rc = prep(type, stream, &blob, &dev)) return rc;
        if (n == 0) {
            if (d_actual_iov_len &&
                cudaMemsetAsync(d_actual_iov_len, 0, sizeof(int64_t), (cudaStream_t)stream) != cudaSuccess)
                return DTE_ERR_CUDA;
            return DTE_SUCCESS;
        }
        size_t smem;
        Desc d = make_desc(c, blob, &smem);
        IovArgs a;
        a.out = d_iov;
        a.actual = d_actual_iov_len;
        a.base = (const char *)base;
        a.first = iov_offset;
        a.n = n;
        a.nseg = c.nseg;
        a.div_nseg = c.nodes()[c.root].div_nseg;
        a.extent = type->extent();
        int64_t max_blocks = (int64_t)sm_count(dev) * 4;
        a.rec_runs = 0;
        a.nrec_elem = a.rounds_elem = a.q_first = a.nrounds = 0;
        a.div_rounds = make_div(1);
        if (const int64_t runs = rec_runs_of(c)) {
            const int64_t nrec = c.nseg / runs;
            a.rec_runs = runs;
            a.nrec_elem = nrec;
            a.rounds_elem = (nrec + 31) / 32;
            a.div_rounds = make_div(a.rounds_elem);
            const int64_t r0 = iov_offset / runs, r1 = (iov_offset + n - 1) / runs;  // records touched
            const int64_t e0 = r0 / nrec, e1 = r1 / nrec;
            a.q_first = e0 * a.rounds_elem + (r0 - e0 * nrec) / 32;
            a.nrounds = e1 * a.rounds_elem + (r1 - e1 * nrec) / 32 - a.q_first + 1;
        }
        int64_t blocks, per_warp;
        if (a.rec_runs > 0) {
            // a few rounds per warp, as many warps as there are rounds
            blocks = std::max<int64_t>(1, std::min<int64_t>((a.nrounds + 4 * kWarps - 1) / (4 * kWarps), max_blocks));
            per_warp = (a.nrounds + blocks * kWarps - 1) / (blocks * kWarps);
        } else {
            int64_t warps_needed = (n + 127) / 128;
            blocks = std::max<int64_t>(1, std::min<int64_t>((warps_needed + kWarps - 1) / kWarps, max_blocks));
            per_warp = (n + blocks * kWarps - 1) / (blocks * kWarps);
            per_warp = (per_warp + 31) / 32 * 32;
        }
        a.per_warp = per_warp;
        iov_kernel<<<(unsigned)blocks, kThreads, smem, (cudaStream_t)stream>>>(d, a);
        if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
        note_use(type, dev, stream);
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

int dte_type_iov_len_async(dte_type type, int64_t n, const int64_t *d_budget, int64_t *d_iov_len,
                           int64_t *d_iov_bytes, dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_type_iov_len_async");
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (n < 0 || (n > 0 && (!d_budget || !d_iov_len || !d_iov_bytes))) return DTE_ERR_ARG;
        if (n == 0) return DTE_SUCCESS;
        const char *blob;
        int dev;
        if (int rc = prep(type, stream, &blob, &dev)) return rc;
        Committed &c = *type->desc;
        size_t smem;
        Desc d = make_desc(c, blob, &smem);
        int64_t blocks = std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)sm_count(dev) * 4);
        iov_len_kernel<<<(unsigned)blocks, kThreads, smem, (cudaStream_t)stream>>>(d, n, d_budget, d_iov_len,
                                                                                  d_iov_bytes, c.size, c.nseg,
                                                                                  rec_runs_of(c));
        if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
        note_use(type, dev, stream);
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

int dte_type_iov_at_bytes_async(dte_type type, int64_t n, const int64_t *d_offset, int64_t max_iov_len,
                                dte_iov *d_iov, int64_t *d_first, int64_t *d_actual, const void *base,
                                dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_type_iov_at_bytes_async");
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (n < 0 || max_iov_len < 0) return DTE_ERR_ARG;
        if (n == 0) return DTE_SUCCESS;
        if (!d_offset || !d_first || !d_actual || (max_iov_len > 0 && !d_iov)) return DTE_ERR_ARG;
        int64_t total;
        if (__builtin_mul_overflow(n, max_iov_len, &total)) return DTE_ERR_OVERFLOW;
        const char *blob;
        int dev;
        if (int rc = prep(type, stream, &blob, &dev)) return rc;
        Committed &c = *type->desc;
        size_t smem;
        Desc d = make_desc(c, blob, &smem);
        int64_t sms = sm_count(dev);
        int64_t b1 = std::min<int64_t>((n + kThreads - 1) / kThreads, sms * 4);
        at_bytes_first_kernel<<<(unsigned)b1, kThreads, smem, (cudaStream_t)stream>>>(
            d, n, d_offset, max_iov_len, d_first, d_actual, c.size, c.nseg, rec_runs_of(c));
        if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
        if (total > 0) {
            if (const int64_t runs = rec_runs_of(c)) {
                const int64_t nrec = c.nseg / runs;
                // tasks of kRecIovSpan rounds; a query's records r0 .. r1
                // have r1 - r0 <= (max_iov_len - 1) / runs + 1, so they
                // span at most (r1 - r0) / 32 + 2 rounds
                const int64_t max_rounds = ((max_iov_len - 1) / runs + 1) / 32 + 2;
                const int64_t cpq = (max_rounds + kRecIovSpan - 1) / kRecIovSpan;
                const int64_t tasks = n * cpq;
                const int64_t b2 = std::max<int64_t>(1, std::min<int64_t>((tasks + kWarps - 1) / kWarps, sms * 4));
                at_bytes_fill_rec_kernel<<<(unsigned)b2, kThreads, smem, (cudaStream_t)stream>>>(
                    d, n, max_iov_len, d_first, d_actual, d_iov, (const char *)base, runs, nrec,
                    make_div((nrec + 31) / 32), cpq);
                if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
                note_use(type, dev, stream);
                return DTE_SUCCESS;
            }
            FastDiv dm = make_div(max_iov_len);
            const int64_t warps_needed = (total + 127) / 128;
            const int64_t b2 = std::max<int64_t>(1, std::min<int64_t>((warps_needed + kWarps - 1) / kWarps, sms * 4));
            int64_t per_warp = (total + b2 * kWarps - 1) / (b2 * kWarps);
            per_warp = (per_warp + 31) / 32 * 32;
            at_bytes_fill_kernel<<<(unsigned)b2, kThreads, smem, (cudaStream_t)stream>>>(
                d, n, max_iov_len, dm, d_first, d_actual, d_iov, (const char *)base, c.nseg,
                c.nodes()[c.root].div_nseg, per_warp);
            if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
        }
        note_use(type, dev, stream);
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

// The kernel class a single move and a batch op of `op` take (the same
// decisions as launch_move and fill_batch_op).
int dte_op_shape_query(const dte_op *op, dte_op_shape *out)
{
    try {
        if (!op || !out) return DTE_ERR_ARG;
        if (!handle_valid(op->type)) return DTE_ERR_TYPE;
        if (!op->type->committed) return DTE_ERR_TYPE;
        if (op->count < 0) return DTE_ERR_ARG;
        const Committed &c = *op->type->desc;
        const int64_t ext = op->type->extent();
        int64_t bytes, segs;
        if (__builtin_mul_overflow(op->count, c.size, &bytes) || __builtin_mul_overflow(op->count, c.nseg, &segs))
            return DTE_ERR_OVERFLOW;
        const int plan = op->type->plan;
        const int W = word_of(c, ext, op->count, op->user, op->packed);
        dte_op_shape r;
        r.word = W;
        r.list = c.big_list ? 1 : 0;
        r.bytes = bytes;
        r.segments = segs;
        r.max_run = c.maxrun;
        const int batch = plan_seg(c, W, plan) ? DTE_PLAN_SEGMENT : plan_wide(W, plan) ? DTE_PLAN_CHUNK_WIDE
                                                                                        : DTE_PLAN_CHUNK;
        r.batch_kernel = batch;
        r.single_kernel = batch;
        if (batch != DTE_PLAN_SEGMENT && W == 16 && c.nseg > 0) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) {
                cudaGetLastError();
                dev = -1;
            }
            const bool rule = plan == DTE_PLAN_BULK ||
                              (plan == DTE_PLAN_AUTO && kBulk && dev >= 0 &&
                               bytes >= kBulkMinTilesPerWarp * kBulkWarps * kBulkTile * sm_count(dev) &&
                               c.size / c.nseg >= kBulkMinRun);
            if (rule && dev >= 0 && device_memory(op->user) && device_memory(op->packed))
                r.single_kernel = DTE_PLAN_BULK;
        }
        *out = r;
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched pack that allocates nothing.
//
// For callers that must not allocate device memory while enqueueing work:
// code running inside a memory budget that a caching allocator has already
// reserved in full, real-time or signal-driven paths that cannot take the
// allocator's locks or its latency, and libraries that are handed a stream
// but forbidden to touch the device heap.  The regular batch keeps its op
// table in memory it allocates with cudaMalloc; this variant writes the table
// into a fixed array that is part of the library image instead.
//
// The array is `static __device__`: every GPU that loads the library holds
// it until the process exits, and every call on a device shares it.  Host
// code must not pass the array's name to a kernel (on the host that name is
// only a stand-in), so its device address is looked up once per device with
// cudaGetSymbolAddress -- on the first call made while that device is
// current -- and that address is what the kernels receive.
// ---------------------------------------------------------------------------
namespace dte {

constexpr int64_t kNoAllocMaxOps = DTE_NOALLOC_MAX_OPS;

struct NoAllocTable {
    BatchOp ops[kNoAllocMaxOps];
    int64_t prefix[kNoAllocMaxOps + kNumClasses];  // per-group tile prefixes
};

static __device__ __align__(256) char g_noalloc_scratch[sizeof(NoAllocTable)];

static std::mutex g_noalloc_mu;
static char *g_noalloc_addr[64];

static int noalloc_scratch(int dev, char **out)
{
    if (dev < 0 || dev >= 64) return DTE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DTE_ERR_CUDA;
        }
        g_noalloc_addr[dev] = static_cast<char *>(p);
    }
    *out = g_noalloc_addr[dev];
    return DTE_SUCCESS;
}

}  // namespace dte

extern "C" int dte_pack_batch_enqueue_noalloc(int64_t nops, const dte_op *ops, dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_pack_batch_enqueue_noalloc");
    try {
        if (nops < 0 || (nops > 0 && !ops)) return DTE_ERR_ARG;
        if (nops > kNoAllocMaxOps) return DTE_ERR_UNSUPPORTED;
        // the op table is copied from a host array that the next call
        // rewrites, so a copy recorded now and replayed later would read the
        // wrong table: refuse before anything is queued
        if (capturing(stream)) return DTE_ERR_UNSUPPORTED;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return DTE_ERR_NODEVICE;
        }
        char *scratch = nullptr;
        if (int rc = noalloc_scratch(dev, &scratch)) return rc;

        // host image of the table: thread-local, so the call itself allocates nothing
        static thread_local NoAllocTable table;
        static thread_local BatchOp staged[kNoAllocMaxOps];
        for (int64_t i = 0; i < nops; i++) {
            const dte_op &o = ops[i];
            BatchOp &h = staged[i];
            std::memset(&h, 0, sizeof h);
            if (!handle_valid(o.type) || !o.type->committed) return DTE_ERR_TYPE;
            if (o.count < 0) return DTE_ERR_ARG;
            int64_t total;
            if (__builtin_mul_overflow(o.count, o.type->size, &total)) return DTE_ERR_OVERFLOW;
            if (total == 0) continue;
            if (!o.user || !o.packed) return DTE_ERR_ARG;
            const char *dblob;
            // the descriptor must already be on this device (commit uploads it)
            if (int rc = device_blob_resident(o.type, dev, &dblob)) return rc;
            fill_batch_op(h, *o.type->desc, o.type->extent(), o, dblob, o.type->plan);
        }
        // group by kernel variant exactly like the allocating batch
        struct G { int wsel; int64_t op0, nops, t0, ntiles; };
        G groups[kNumClasses];
        int ng = 0;
        int64_t n = 0, np = 0;
        for (int w = 0; w < kNumClasses; w++) {
            G g{w, n, 0, np, 0};
            table.prefix[np++] = 0;
            for (int64_t i = 0; i < nops; i++) {
                if (staged[i].nchunks == 0 || staged[i].wsel != w) continue;
                table.ops[n++] = staged[i];
                table.prefix[np] = table.prefix[np - 1] + op_tiles(staged[i]);
                np++;
            }
            g.nops = n - g.op0;
            if (g.nops == 0) {
                np--;
                continue;
            }
            g.ntiles = table.prefix[np - 1];
            groups[ng++] = g;
        }
        if (ng == 0) return DTE_SUCCESS;
        BatchOp *d_ops = reinterpret_cast<BatchOp *>(scratch + offsetof(NoAllocTable, ops));
        int64_t *d_prefix = reinterpret_cast<int64_t *>(scratch + offsetof(NoAllocTable, prefix));
        // pageable source: the copy is staged before cudaMemcpyAsync returns,
        // so the thread-local image may be rewritten by the next call
        if (cudaMemcpyAsync(d_ops, table.ops, (size_t)n * sizeof(BatchOp), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream) != cudaSuccess ||
            cudaMemcpyAsync(d_prefix, table.prefix, (size_t)np * sizeof(int64_t), cudaMemcpyHostToDevice,
                            (cudaStream_t)stream) != cudaSuccess) {
            cudaGetLastError();
            return DTE_ERR_CUDA;
        }
        static thread_local int occ_cache[64][kNumClasses];
        for (int gi = 0; gi < ng; gi++) {
            const G &g = groups[gi];
            BatchKernel k = pick_batch<true>(g.wsel);
            int &occ = occ_cache[dev & 63][g.wsel];
            if (occ == 0) occ = occupancy(k, 0);
            int64_t max_blocks = (int64_t)sm_count(dev) * occ;
            int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((g.ntiles + kWarps - 1) / kWarps, max_blocks));
            k<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(d_ops + g.op0, d_prefix + g.t0, g.nops,
                                                                      g.ntiles, 1, nullptr, 0,
                                                                      make_spread(g.ntiles, blocks * kWarps));
            if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
        }
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_ARG;
    }
}

// ---------------------------------------------------------------------------
// Adjoint of the typed float32 pack (differentiable halo gathers).
// ---------------------------------------------------------------------------
namespace dte {

// Build (once per type, count and device) the destination-major inverse of
// the pack: for every destination float the packed floats that read it, in
// packed order.
static int adjoint_inverse(dte_type t, int64_t count, int dev, AdjointInverse *out)
{
    Committed &c = *t->desc;
    std::lock_guard<std::mutex> g(c.mu);
    for (auto &a : c.adj) {
        if (a.device == dev && a.count == count) {
            *out = a;
            return DTE_SUCCESS;
        }
    }
    int64_t nsrc = count * (c.size / 4);
    std::vector<int64_t> dst((size_t)nsrc);
    int64_t p = 0;
    Hint h{-1, 0};
    const int64_t ext = t->extent();
    for (int64_t e = 0; e < count; e++) {
        for (int64_t k = 0; k < c.nseg; k++) {
            int64_t d = 0, len = 0;
            decode_seg(c.nodes(), c.blob(), c.root, k, d, len, h);
            d += e * ext;
            for (int64_t f = 0; f < len / 4; f++) dst[(size_t)p++] = d / 4 + f;
        }
    }
    std::vector<int64_t> order((size_t)nsrc);
    std::iota(order.begin(), order.end(), (int64_t)0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return dst[(size_t)a] < dst[(size_t)b]; });
    std::vector<int64_t> rows, dest;
    rows.reserve((size_t)nsrc + 1);
    dest.reserve((size_t)nsrc);
    for (int64_t j = 0; j < nsrc; j++) {
        if (j == 0 || dst[(size_t)order[(size_t)j]] != dst[(size_t)order[(size_t)j - 1]]) {
            rows.push_back(j);
            dest.push_back(dst[(size_t)order[(size_t)j]]);
        }
    }
    rows.push_back(nsrc);
    AdjointInverse a;
    a.device = dev;
    a.count = count;
    a.ndest = (int64_t)dest.size();
    a.nsrc = nsrc;
    size_t bytes = sizeof(int64_t) * (rows.size() + dest.size() + order.size());
    if (cudaMalloc(&a.dmem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return DTE_ERR_NOMEM;
    }
    char *q = a.dmem;
    if (cudaMemcpy(q, rows.data(), rows.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(q + rows.size() * 8, dest.data(), dest.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(q + (rows.size() + dest.size()) * 8, order.data(), order.size() * 8, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaFree(a.dmem);
        return DTE_ERR_CUDA;
    }
    c.adj.push_back(a);
    *out = a;
    return DTE_SUCCESS;
}

}  // namespace dte

extern "C" int dte_pack_adjoint_f32_enqueue(const void *gy, int64_t count, dte_type type, void *gx,
                                            dte_stream_t stream)
{
    DTE_NVTX_RANGE("dte_pack_adjoint_f32_enqueue");
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (count < 0) return DTE_ERR_ARG;
        int64_t need;
        if (__builtin_mul_overflow(count, type->size, &need)) return DTE_ERR_OVERFLOW;
        if (need == 0) return DTE_SUCCESS;
        if (!gy || !gx) return DTE_ERR_ARG;
        Committed &c = *type->desc;
        const int64_t ext = type->extent();
        if (c.align < 4 || (count > 1 && ext % 4 != 0) || ((uintptr_t)gy & 3) || ((uintptr_t)gx & 3))
            return DTE_ERR_ARG;
        const char *blob;
        int dev;
        if (int rc = prep(type, stream, &blob, &dev)) return rc;
        if (!committed_overlaps(c, count, ext)) {
            Op op = make_op(c, ext, gx, const_cast<void *>(gy), count);
            size_t smem;
            Desc d = make_desc(c, blob, &smem);
            bool pk16 = p2addr(gy) >= 16;
            int64_t nchunks = (op.total + 15) / 16;
            int64_t span_steps = d.stage == STAGE_BLOB ? 1 : 8;
            int64_t units = (nchunks + span_steps * kStep - 1) / (span_steps * kStep);
            auto k = pk16 ? adjoint_kernel<true> : adjoint_kernel<false>;
            static thread_local int occ_cache[64][2][3];
            int &occ = occ_cache[dev & 63][pk16 ? 1 : 0][d.stage];
            if (occ == 0) occ = occupancy(k, d.stage == STAGE_BLOB ? (size_t)kSmemBlob : smem);
            int64_t blocks = std::max<int64_t>(
                1, std::min<int64_t>((units + kWarps - 1) / kWarps, (int64_t)sm_count(dev) * occ));
            k<<<(unsigned)blocks, kThreads, smem, (cudaStream_t)stream>>>(d, op, nchunks, span_steps * kStep);
        } else {
            AdjointInverse a;
            if (int rc = adjoint_inverse(type, count, dev, &a)) return rc;
            const int64_t *rows = reinterpret_cast<const int64_t *>(a.dmem);
            const int64_t *dest = rows + a.ndest + 1;
            const int64_t *cols = dest + a.ndest;
            int64_t blocks = std::max<int64_t>(
                1, std::min<int64_t>((a.ndest + kThreads - 1) / kThreads, (int64_t)sm_count(dev) * 8));
            adjoint_csr_kernel<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(
                rows, dest, cols, a.ndest, static_cast<const float *>(gy), static_cast<float *>(gx));
        }
        if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
        note_use(type, dev, stream);
        return DTE_SUCCESS;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

// Bounded device waits that gave up (bulk kernels and the request loop), on
// the current device.
extern "C" int dte_device_timeouts(int64_t *count)
{
    if (!count) return DTE_ERR_ARG;
    unsigned long long v = 0, sv = 0;
    if (cudaMemcpyFromSymbol(&v, dte::g_bulk_timeouts, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return DTE_ERR_CUDA;
    }
    if (int rc = dte::serve_timeouts(&sv)) return rc;
    *count = (int64_t)(v + sv);
    return DTE_SUCCESS;
}
