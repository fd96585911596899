// move.cuh -- building blocks shared by the data-movement kernels (single
// operations, batches, the request loop): launch constants, the records a
// kernel needs for one operation, the warp-level chunk and segment steps,
// and the host helpers that choose a kernel variant for an operation.
// See kernels.cu for the design of the two work splits (chunk-major and
// segment-major).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace dte {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
#ifndef DTE_KU
#define DTE_KU 4
#endif
constexpr int kU = DTE_KU;            // chunks per lane per step
constexpr int kStep = 32 * kU;        // chunks per warp step (2 KiB)
// 16-byte moves take half-size steps (1 KiB: two chunks per lane): each
// chunk is one load and one store, so finer steps balance the warps better
// at the end of a launch; the sub-16-byte paths keep four chunks per lane to
// overlap their per-run descriptor walks.
#ifndef DTE_KU16
#define DTE_KU16 2
#endif
// The wide plan (DTE_PLAN_CHUNK_WIDE) gives 16-byte moves 2 KiB steps (four
// chunks per lane) instead.
template <int W, bool WIDE = false>
constexpr int kUOf = W == 16 ? (WIDE ? 4 : DTE_KU16) : kU;
template <int W, bool WIDE = false>
constexpr int kStepOf = 32 * kUOf<W, WIDE>;
static inline int64_t step_of_word(int W, bool wide = false)
{
    return W == 16 ? (wide ? kStepOf<16, true> : kStepOf<16>) : kStep;
}
#ifndef DTE_MINBLOCKS
#define DTE_MINBLOCKS 4
#endif
constexpr int kMinBlocks = DTE_MINBLOCKS;  // CTAs per SM the data kernels are sized for (<= 64 regs)
constexpr int64_t kSmemBlob = 16384;  // stage descriptors up to this size whole
// Segment-major movement pays off for short runs under a large index table
// (one direct table lookup per segment instead of a search per run); for
// strided layouts (divisions only) the chunk-major kernel is faster even
// with short runs.  Mixed run lengths take it while the mean run is short
// and no run is long enough to hold a warp's round up for long.
#ifndef DTE_SEGMAXRUN
#define DTE_SEGMAXRUN 4096
#endif
constexpr int64_t kSegMaxRun = DTE_SEGMAXRUN;   // longest run
constexpr int64_t kSegMaxMean = 512;            // mean run (size / segments)

static bool use_seg_major(const Committed &c, int W)
{
    return W < 16 && c.big_list && c.maxrun <= kSegMaxRun && c.nseg > 0 && c.size / c.nseg <= kSegMaxMean;
}

// Kernel class of a move under a type's plan (include/dte.h, dte_plan): the
// fixed rule above for DTE_PLAN_AUTO; otherwise the plan where it applies --
// segment-major needs a copy word below 16 bytes and runs of at most
// kSegMaxRun, the wide step a 16-byte word -- and the fixed rule's choice
// where it does not.
static bool plan_seg(const Committed &c, int W, int plan)
{
    if (plan == DTE_PLAN_CHUNK) return false;
    if (plan == DTE_PLAN_SEGMENT && W < 16 && c.nseg > 0 && c.maxrun <= kSegMaxRun) return true;
    return use_seg_major(c, W);  // the fixed rule: AUTO, and plans that do not apply
}
static bool plan_wide(int W, int plan) { return W == 16 && plan == DTE_PLAN_CHUNK_WIDE; }
constexpr int kMaxSmemNodes = 64;

enum : int { STAGE_NONE = 0, STAGE_NODES = 1, STAGE_BLOB = 2 };

// What a kernel needs to walk one committed type.
struct Desc {
    const char *blob;
    int64_t blob_bytes;
    int32_t root;
    int32_t nnodes;
    int32_t stage;
    int32_t pad_;
};

// One data movement: element e of the user layout starts at user + e*extent.
struct Op {
    const char *user_in;    // pack source
    char *user_out;         // unpack destination
    const char *packed_in;  // unpack source (position applied)
    char *packed_out;       // pack destination (position applied)
    int64_t total;          // bytes moved
    int64_t pbase;          // packed-stream offset of packed byte 0 (range moves; else 0)
    int64_t esize;          // element size
    int64_t extent;         // element stride
    FastDiv ediv;           // / esize
    int32_t root;
    int32_t pad_;
};

__device__ __forceinline__ void stage_desc(const Desc &d, uint4 *smem, const char *&blob,
                                           const DNode *&nodes)
{
    const DNode *g = reinterpret_cast<const DNode *>(d.blob + sizeof(BlobHeader));
    if (d.stage == STAGE_BLOB) {
        const uint4 *s = reinterpret_cast<const uint4 *>(d.blob);
        int nw = (int)(d.blob_bytes / 16);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) smem[i] = s[i];
        __syncthreads();
        blob = reinterpret_cast<const char *>(smem);
        nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
    } else if (d.stage == STAGE_NODES) {
        const uint4 *s = reinterpret_cast<const uint4 *>(g);
        int nw = d.nnodes * (int)(sizeof(DNode) / 16);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) smem[i] = s[i];
        __syncthreads();
        blob = d.blob;
        nodes = reinterpret_cast<const DNode *>(smem);
    } else {
        blob = d.blob;
        nodes = g;
    }
}

template <int W> struct Word;
template <> struct Word<1> { using T = uint8_t; };
template <> struct Word<2> { using T = uint16_t; };
template <> struct Word<4> { using T = uint32_t; };
template <> struct Word<8> { using T = unsigned long long; };
template <> struct Word<16> { using T = uint4; };

template <int W>
union Chunk {
    uint4 v;
    typename Word<W>::T w[16 / W];
};

// Order in which warps visit spans.  The j-th span a launch hands out
// (j = warp, warp + nwarps, ...) is span (j * mult) mod nspans, with mult
// coprime to nspans (a bijection) and close to nspans / phi: the spans in
// flight at any moment are spread over the whole packed range, so regions
// of a layout that are slow per byte (short runs far apart) run side by side
// with fast ones instead of being left to the end of the launch.
struct Spread {
    int64_t nspans;
    int64_t mult;
    int64_t inc;  // (nwarps * mult) mod nspans
    FastDiv div;  // / nspans
};

// The first span warp `warp` takes: (warp * mult) mod nspans, by invariant
// division (a 64-bit % is a long software routine at the head of every warp).
__device__ __forceinline__ int64_t spread_first(const Spread &sp, int64_t warp)
{
    if (warp >= sp.nspans) return 0;
    const int64_t x = warp * sp.mult;
    return x - fdiv(x, sp.div) * sp.nspans;
}

// Programmatic dependent launch: the kernels that move user data are
// launched so that they may start while the previous kernel of the stream
// drains.  Before the wait a kernel touches only its own descriptor (staged
// into shared memory); the wait returns once the previous grids have
// completed and their writes are visible.  Without such a launch both
// instructions do nothing.
__device__ __forceinline__ void prior_grids_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_overlapped(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                                     cudaStream_t stream, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Copy an op record (global) into the warp's shared slot; the kernels that
// walk many ops read the fields from there instead of holding them in
// registers.  Synchronised on both sides within the warp.
__device__ __forceinline__ void load_op(Op &dst, const Op &src, int lane)
{
    static_assert(sizeof(Op) % 8 == 0 && sizeof(Op) / 8 <= 32, "Op is copied one word per lane");
    __syncwarp();
    if (lane < (int)(sizeof(Op) / 8))
        reinterpret_cast<unsigned long long *>(&dst)[lane] = reinterpret_cast<const unsigned long long *>(&src)[lane];
    __syncwarp();
}

// packed offset P (of this op's packed buffer) -> user displacement and
// bytes left in that run
__device__ __forceinline__ void locate(const Op &op, const DNode *nodes, const char *blob, int64_t P,
                                       int64_t &d, int64_t &rem, Hint &h)
{
    P += op.pbase;
    int64_t e = fdiv(P, op.ediv);
    d = e * op.extent;
    decode_bytes(nodes, blob, op.root, P - e * op.esize, d, rem, h);
}

template <int W>
__device__ __forceinline__ typename Word<W>::T ldw(const char *p)
{
    return __ldg(reinterpret_cast<const typename Word<W>::T *>(p));
}

template <int W>
__device__ __forceinline__ void stw(char *p, typename Word<W>::T v)
{
    *reinterpret_cast<typename Word<W>::T *>(p) = v;
}

// gather the nb (<= 16) packed bytes starting at P from the user layout.
// With W < 16 the chunk is assembled run by run in the thread's 16-byte
// shared scratch `scr`: one descriptor walk per run, in a rolled loop, so
// the walk is inlined once per chunk slot (inlining it once per word made
// the kernels large enough to stall on instruction fetch).
#ifndef DTE_CHUNK_WIDEN_GATHER
#define DTE_CHUNK_WIDEN_GATHER 0
#endif
#ifndef DTE_CHUNK_WIDEN_SCATTER
#define DTE_CHUNK_WIDEN_SCATTER 1
#endif
// Whether the W < 16 chunk paths move a run piece in wider words than W
// where the piece's user address, its offset in the chunk and its length all
// allow them (up to one 16-byte access for a chunk inside one run).  Measured
// on the 10^4-op batch: unpack 5.48 -> 5.10 ms with it, pack 4.77 -> 5.28 ms,
// so only the scatter (unpack) side takes it.
constexpr bool kChunkWidenGather = DTE_CHUNK_WIDEN_GATHER != 0;
constexpr bool kChunkWidenScatter = DTE_CHUNK_WIDEN_SCATTER != 0;

// The widest word, from W up to 16 bytes, dividing a piece's user address,
// its chunk offset and its length.
template <int W>
__device__ __forceinline__ int piece_word(const char *p, int got, int take)
{
    const unsigned a = (unsigned)(uintptr_t)p | (unsigned)got | (unsigned)take;
    const int wd = (a & 15) == 0 ? 16 : (a & 7) == 0 ? 8 : (a & 3) == 0 ? 4 : (a & 1) == 0 ? 2 : 1;
    return wd > W ? wd : W;
}

// Copy `take` bytes between user memory and the chunk scratch in words of
// V bytes (V divides the address, the offset and the length).
template <int V, bool IN>
__device__ __forceinline__ void piece_copy(char *user, char *scr, int take)
{
    using U = typename Word<V>::T;
#pragma unroll
    for (int k = 0; k < 16 / V; k++)
        if (k * V < take) {
            if (IN) *reinterpret_cast<U *>(scr + k * V) = ldw<V>(user + k * V);
            else stw<V>(user + k * V, *reinterpret_cast<const U *>(scr + k * V));
        }
}

template <int W>
__device__ __forceinline__ uint4 gather_chunk(const Op &op, const DNode *nodes, const char *blob, int64_t P,
                                              int nb, Hint &h, char *scr)
{
    using T = typename Word<W>::T;
    if (W == 16) {
        int64_t d, rem;
        locate(op, nodes, blob, P, d, rem, h);
        return ldw<16>(op.user_in + d);
    }
    int got = 0;
#pragma unroll 1
    while (got < nb) {
        int64_t d, rem;
        locate(op, nodes, blob, P + got, d, rem, h);
        const int take = rem < (int64_t)(nb - got) ? (int)rem : nb - got;
        const char *src = op.user_in + d;
        const int wd = kChunkWidenGather ? piece_word<W>(src, got, take) : W;
        if (wd == 16) return ldw<16>(src);  // the whole chunk from one run
        if (W < 8 && wd == 8) piece_copy<8, true>(const_cast<char *>(src), scr + got, take);
        else if (W < 4 && wd == 4) piece_copy<4, true>(const_cast<char *>(src), scr + got, take);
        else {
#pragma unroll
            for (int k = 0; k < 16 / W; k++)
                if (k * W < take) *reinterpret_cast<T *>(scr + got + k * W) = ldw<W>(src + k * W);
        }
        got += take;
    }
    return *reinterpret_cast<const uint4 *>(scr);
}

template <int W>
__device__ __forceinline__ void scatter_chunk(const Op &op, const DNode *nodes, const char *blob, int64_t P,
                                              int nb, uint4 v, Hint &h, char *scr)
{
    using T = typename Word<W>::T;
    if (W == 16) {
        int64_t d, rem;
        locate(op, nodes, blob, P, d, rem, h);
        *reinterpret_cast<uint4 *>(op.user_out + d) = v;
        return;
    }
    *reinterpret_cast<uint4 *>(scr) = v;
    int got = 0;
#pragma unroll 1
    while (got < nb) {
        int64_t d, rem;
        locate(op, nodes, blob, P + got, d, rem, h);
        const int take = rem < (int64_t)(nb - got) ? (int)rem : nb - got;
        char *dst = op.user_out + d;
        const int wd = kChunkWidenScatter ? piece_word<W>(dst, got, take) : W;
        if (wd == 16) {  // the whole chunk into one run
            *reinterpret_cast<uint4 *>(dst) = v;
            return;
        }
        if (W < 8 && wd == 8) piece_copy<8, false>(dst, scr + got, take);
        else if (W < 4 && wd == 4) piece_copy<4, false>(dst, scr + got, take);
        else {
#pragma unroll
            for (int k = 0; k < 16 / W; k++)
                if (k * W < take) stw<W>(dst + k * W, *reinterpret_cast<const T *>(scr + got + k * W));
        }
        got += take;
    }
}

template <int W, bool PK16>
__device__ __forceinline__ uint4 load_packed(const char *p, int nb)
{
    if (W == 16 || (PK16 && nb == 16)) return __ldg(reinterpret_cast<const uint4 *>(p));
    Chunk<W> c;
    c.v = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int s = 0; s < 16 / W; s++)
        if (s * W < nb) c.w[s] = ldw<W>(p + s * W);
    return c.v;
}

template <int W, bool PK16>
__device__ __forceinline__ void store_packed(char *p, uint4 v, int nb)
{
    if (W == 16 || (PK16 && nb == 16)) {
        *reinterpret_cast<uint4 *>(p) = v;
        return;
    }
    Chunk<W> c;
    c.v = v;
#pragma unroll
    for (int s = 0; s < 16 / W; s++)
        if (s * W < nb) stw<W>(p + s * W, c.w[s]);
}

// The per-thread 16-byte scratch of the W < 16 chunk paths (a kernel
// declares `__shared__ uint4 name[kScratch<W>]` and passes its slot).
template <int W>
constexpr int kScratch = W < 16 ? kThreads : 1;

// One warp step, 16-byte words, U chunks per lane: a lane's chunks sit 512
// bytes apart, so when the run found for its first chunk extends past a later
// chunk, that chunk's user address follows without walking the descriptor
// again.
template <bool PACK, int U>
__device__ __forceinline__ void warp_step16(const Op &op, const DNode *nodes, const char *blob, int64_t base,
                                            int64_t end, int lane, Hint &h)
{
    uint4 v[U];
    int64_t d[U];
    int64_t d0 = 0, rem0 = 0;
    if (!PACK) {
        // the packed side is addressed by position alone: its loads go out
        // before the descriptor walks, whose latency they then cover
#pragma unroll
        for (int u = 0; u < U; u++) {
            int64_t c = base + u * 32 + lane;
            if (c < end) v[u] = __ldg(reinterpret_cast<const uint4 *>(op.packed_in + c * 16));
        }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        int64_t c = base + u * 32 + lane;
        if (c < end) {
            if (u > 0 && rem0 >= (int64_t)u * 512 + 16) {
                d[u] = d0 + u * 512;
            } else {
                int64_t rem;
                locate(op, nodes, blob, c * 16, d[u], rem, h);
                if (u == 0) {
                    d0 = d[u];
                    rem0 = rem;
                }
            }
            if (PACK) v[u] = __ldg(reinterpret_cast<const uint4 *>(op.user_in + d[u]));
        }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        int64_t c = base + u * 32 + lane;
        if (c < end) {
            if (PACK) *reinterpret_cast<uint4 *>(op.packed_out + c * 16) = v[u];
            else *reinterpret_cast<uint4 *>(op.user_out + d[u]) = v[u];
        }
    }
}

// One warp step: chunks [base, base + kStepOf<W, WIDE>) clipped to `end`.
template <int W, bool PACK, bool PK16, bool WIDE = false>
__device__ __forceinline__ void warp_step(const Op &op, const DNode *nodes, const char *blob, int64_t base,
                                          int64_t end, int lane, Hint &h, char *scr)
{
    if constexpr (W == 16) {
        warp_step16<PACK, kUOf<16, WIDE>>(op, nodes, blob, base, end, lane, h);
    } else {
        uint4 v[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            int64_t c = base + u * 32 + lane;
            if (c < end) {
                int64_t P = c * 16;
                int nb = (int)(op.total - P < 16 ? op.total - P : 16);
                if (PACK) v[u] = gather_chunk<W>(op, nodes, blob, P, nb, h, scr);
                else v[u] = load_packed<W, PK16>(op.packed_in + P, nb);
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            int64_t c = base + u * 32 + lane;
            if (c < end) {
                int64_t P = c * 16;
                int nb = (int)(op.total - P < 16 ? op.total - P : 16);
                if (PACK) store_packed<W, PK16>(op.packed_out + P, v[u], nb);
                else scatter_chunk<W>(op, nodes, blob, P, nb, v[u], h, scr);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// segment-major round
// ---------------------------------------------------------------------------
// Largest b in [0, n) with a[b] <= x (a sorted, a[0] <= x), found by the warp
// together: every step the 32 lanes probe 32 evenly spaced entries of the
// remaining range and one ballot keeps the last probe at or below x, so a
// table of 2^22 entries takes 5 dependent loads instead of 22.  Warp-uniform
// arguments; every lane returns the same b.
__device__ __forceinline__ int64_t warp_find_le(const int64_t *a, int64_t n, int64_t x, int lane)
{
    const unsigned FULL = 0xffffffffu;
    int64_t lo = 0, hi = n;  // a[lo] <= x, and the answer is below hi
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t i = lo + lane * step;
        const unsigned le = __ballot_sync(FULL, i < hi && a[i] <= x);
        const int k = 31 - __clz(le);  // lane 0 probes lo itself, so le != 0
        lo += k * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// The same lookup with a warp's search position h (warp-uniform): a search
// by the warp when h is cold (h.node != node), else find_le galloping from h.
__device__ __forceinline__ int64_t warp_find_le_hint(const int64_t *a, int64_t n, int64_t x, Hint &h, int node,
                                                     int lane)
{
    if (h.node != node) {
        const int64_t b = warp_find_le(a, n, x, lane);
        h.node = node;
        h.b = b;
        return b;
    }
    return find_le(a, n, x, h, node);
}

// Seed a lane's search position for a warp step that starts at packed
// offset P (warp-uniform): when the layout's root is a list of more than 32
// entries (the one list the chunk decode searches with a position), the warp
// finds the entry of P together and every lane starts from it, so the lanes'
// own searches only gallop over the few entries one step covers.  Single
// moves seed at every span (indexed layouts of 2^18 blocks with 1 KiB runs:
// 5-8% faster); the batch kernels do not (a seed per small op cost the
// 10^4-op batch 1-2%).
#ifndef DTE_SEED_HINT
#define DTE_SEED_HINT 1
#endif
constexpr bool kSeedHint = DTE_SEED_HINT != 0;

__device__ __forceinline__ void seed_root_hint(const Op &op, const DNode *nodes, const char *blob, int64_t P,
                                               Hint &h, int lane)
{
    const DNode &R = nodes[op.root];
    if (R.kind != NK_LIST || R.count <= 32) return;
    const int64_t Pg = op.pbase + P;
    const int64_t e = fdiv(Pg, op.ediv);
    h.b = warp_find_le(arr<int64_t>(blob, R.a_pbytes), R.count, Pg - e * op.esize, lane);
    h.node = op.root;
}

// Whether a round can be decoded by shared_list_round: the element's root is
// a large index list whose entries all repeat one child at one stride (an
// indexed or hindexed type of any old type) with no segment merging across
// or inside entries, so entry b starts at segment (pbytes[b] / child size) *
// child segments and every entry has at least one segment.
__device__ __forceinline__ bool shared_list_root(const DNode &R)
{
    return R.kind == NK_LIST && (R.flags & NF_SHARED) &&
           !(R.flags & (NF_RUNS | NF_PSEGS | NF_XMERGE | NF_EMERGE)) && R.a_eflags == 0 && R.count > 32;
}

// Decode of a round's segments local0 .. local0 + nvalid - 1 (all of element
// e0) under such a root, by the warp together.  Those segments lie in at most
// 32 consecutive entries starting with b0, the entry of the first one (one
// warp-uniform search from the warp's hint rh, which each round leaves at the
// entry of its last segment).  Lane j loads entry b0 + j's packed prefix and
// displacement (coalesced) and computes its first segment; one OR-reduction
// marks where entries start inside the round, so lane l's entry is b0 plus the
// number of entries starting in (local0, local0 + l], and lane l takes that
// entry's values by shuffle.  Only the child (the entry's repeated type) is
// walked per lane.  Same results as decode_seg on the root.
__device__ __forceinline__ void shared_list_round(const Op &op, const DNode *nodes, const char *blob, const DNode &R,
                                                  int64_t e0, int64_t local0, int nvalid, int lane, Hint &rh,
                                                  Hint &h, int64_t &disp, int64_t &len, int64_t &ps)
{
    const unsigned FULL = 0xffffffffu;
    const DNode &C = nodes[R.child];
    const int64_t *pb = arr<int64_t>(blob, R.a_pbytes);
    const int64_t *dv = arr<int64_t>(blob, R.a_disp);
    const int64_t b0 = warp_find_le_hint(pb, R.count, fdiv(local0, C.div_nseg) * C.size, rh, op.root, lane);
    const int64_t bj = b0 + lane;
    const int64_t pbj = bj <= R.count ? pb[bj] : INT64_MAX;
    const int64_t dj = bj < R.count ? dv[bj] : 0;
    const int64_t sj = bj <= R.count ? fdiv(pbj, C.div_size) * C.nseg : INT64_MAX;
    const int64_t o = sj - local0;
    const unsigned starts = __reduce_or_sync(FULL, (lane > 0 && o > 0 && o < 32) ? 1u << (int)o : 0u);
    const int jl = __popc(starts & (0xffffffffu >> (31 - lane)));
    const int64_t pbe = __shfl_sync(FULL, pbj, jl);
    const int64_t de = __shfl_sync(FULL, dj, jl);
    const int64_t se = __shfl_sync(FULL, sj, jl);
    rh.b = b0 + __shfl_sync(FULL, jl, nvalid - 1);
    if (lane < nvalid) {
        const int64_t local = local0 + lane - se;
        const int64_t i = fdiv(local, C.div_nseg);
        const int64_t j = local - i * C.nseg;
        disp = e0 * op.extent + R.base + de + i * R.stride;
        ps = e0 * op.esize + pbe + i * C.size;
        if (C.kind == NK_LIST && (C.flags & NF_RUNS)) {
            // a child that is a table of runs (a struct of basic blocks):
            // run j directly
            const int64_t *cp = arr<int64_t>(blob, C.a_pbytes);
            disp += C.base + arr<int64_t>(blob, C.a_disp)[j];
            ps += cp[j];
            len = cp[j + 1] - cp[j];
        } else if (C.kind == NK_RUN) {
            disp += C.base;
            len = C.len;
        } else {
            int64_t pc;
            decode_seg(nodes, blob, R.child, j, disp, len, pc, h);
            ps += pc;
        }
    }
}

#ifndef DTE_SEG_RUNU
#define DTE_SEG_RUNU 4
#endif
constexpr int kSegRunU = DTE_SEG_RUNU;  // words in flight per lane in a round's run-by-run copy
#ifndef DTE_SEG_WIDE
#define DTE_SEG_WIDE 16
#endif
// Widest user-side access (8 or 16 bytes; 0 = none) the single-move
// segment-major kernel's run-by-run copy of 4-byte words takes where the
// user side is aligned for it.
constexpr int kSegWide = DTE_SEG_WIDE;

// One round: segments [base, base + 32) clipped to s1 (warp-uniform args).
// `rh` is the warp's search position in a root index list.  LISTDEC enables
// the warp decode of shared-child root lists (the batch kernels leave it out:
// under their 64-register budget the extra path costs the common layouts
// more than it gives the rare index-of-struct ones).  WIDEUSER (8 or 16)
// lets the run-by-run copy of 4-byte words take user-side accesses that wide
// where the user side is aligned (the batch kernels leave it at 0: their
// short runs of 2- and 4-byte elements got slower with it).
template <int W, bool PACK, bool LISTDEC = true, int WIDEUSER = 0>
__device__ __forceinline__ void seg_round(const Op &op, const DNode *nodes, const char *blob, int64_t nseg_elem,
                                          const FastDiv &div_nseg, int64_t base, int64_t s1, int lane, Hint &h,
                                          Hint &rh)
{
    using T = typename Word<W>::T;
    const unsigned FULL = 0xffffffffu;
    const int nvalid = (int)min((int64_t)32, s1 - base);
    int64_t disp = 0, len = 0, ps = 0;
    const DNode &R = nodes[op.root];
    const int64_t e0 = fdiv(base, div_nseg);
    const int64_t local0 = base - e0 * nseg_elem;
    if (LISTDEC && shared_list_root(R) && local0 + nvalid <= nseg_elem) {
        shared_list_round(op, nodes, blob, R, e0, local0, nvalid, lane, rh, h, disp, len, ps);
    } else if (lane < nvalid) {
        const int64_t k = base + lane;
        const int64_t e = fdiv(k, div_nseg);
        disp = e * op.extent;
        decode_seg(nodes, blob, op.root, k - e * nseg_elem, disp, len, ps, h);
        ps += e * op.esize;
    }
    // packed-stream range of the 32 segments, clipped to the op's window
    // (a range move may start or end inside a segment)
    const int64_t p0 = max(__shfl_sync(FULL, ps, 0), op.pbase);
    const int64_t p1 = min(__shfl_sync(FULL, ps + len, nvalid - 1), op.pbase + op.total);
    // Rounds whose runs are balanced (the longest at most four times the
    // mean) move run by run: each lane copies its own run in W-byte words,
    // four loads in flight.  That costs a few instructions per word where the
    // cooperative loop below pays a segment lookup per word; a round with one
    // run much longer than the rest keeps the cooperative loop, which spreads
    // the round's bytes (not its runs) over the lanes.
    const unsigned maxlen = __reduce_max_sync(FULL, (unsigned)len);  // runs are <= kSegMaxRun
    if ((int64_t)maxlen * nvalid <= 4 * (p1 - p0)) {
        if (lane < nvalid) {
            const int64_t a = max(ps, p0), e = min(ps + len, p1);
            const char *src = PACK ? op.user_in + disp + (a - ps) : op.packed_in - op.pbase + a;
            char *dst = PACK ? op.packed_out - op.pbase + a : op.user_out + disp + (a - ps);
            const int n = (int)(e - a);
            const uintptr_t ua = (uintptr_t)(PACK ? src : dst);
            if (WIDEUSER >= 8 && W == 4 && (ua & 7) == 0) {
                // the user side takes wider accesses: 16 bytes where it is
                // 16-byte aligned, else 8, then one more pair and a last
                // word; the packed side keeps 4-byte words
                int o = 0;
                if (WIDEUSER >= 16 && (ua & 15) == 0) {
                    for (; o + 16 <= n; o += 16) {
                        if (PACK) {
                            const uint4 x = ldw<16>(src + o);
                            stw<4>(dst + o, x.x);
                            stw<4>(dst + o + 4, x.y);
                            stw<4>(dst + o + 8, x.z);
                            stw<4>(dst + o + 12, x.w);
                        } else {
                            uint4 x;
                            x.x = ldw<4>(src + o);
                            x.y = ldw<4>(src + o + 4);
                            x.z = ldw<4>(src + o + 8);
                            x.w = ldw<4>(src + o + 12);
                            stw<16>(dst + o, x);
                        }
                    }
                }
                for (; o + 16 <= n; o += 16) {
                    if (PACK) {
                        const unsigned long long x = ldw<8>(src + o), y = ldw<8>(src + o + 8);
                        stw<4>(dst + o, (uint32_t)x);
                        stw<4>(dst + o + 4, (uint32_t)(x >> 32));
                        stw<4>(dst + o + 8, (uint32_t)y);
                        stw<4>(dst + o + 12, (uint32_t)(y >> 32));
                    } else {
                        const uint32_t x0 = ldw<4>(src + o), x1 = ldw<4>(src + o + 4);
                        const uint32_t y0 = ldw<4>(src + o + 8), y1 = ldw<4>(src + o + 12);
                        stw<8>(dst + o, (unsigned long long)x1 << 32 | x0);
                        stw<8>(dst + o + 8, (unsigned long long)y1 << 32 | y0);
                    }
                }
                if (o + 8 <= n) {
                    if (PACK) {
                        const unsigned long long x = ldw<8>(src + o);
                        stw<4>(dst + o, (uint32_t)x);
                        stw<4>(dst + o + 4, (uint32_t)(x >> 32));
                    } else {
                        const uint32_t x0 = ldw<4>(src + o), x1 = ldw<4>(src + o + 4);
                        stw<8>(dst + o, (unsigned long long)x1 << 32 | x0);
                    }
                    o += 8;
                }
                if (o < n) stw<4>(dst + o, ldw<4>(src + o));  // lengths are multiples of W
            } else {
                for (int o = 0; o < n; o += kSegRunU * W) {
                    T v[kSegRunU];
#pragma unroll
                    for (int u = 0; u < kSegRunU; u++)
                        if (o + u * W < n) v[u] = ldw<W>(src + o + u * W);
#pragma unroll
                    for (int u = 0; u < kSegRunU; u++)
                        if (o + u * W < n) stw<W>(dst + o + u * W, v[u]);
                }
            }
        }
        return;
    }
    const int64_t nwords = (p1 - p0) / W;
    const char *pk_in = op.packed_in - op.pbase;  // indexed by stream offset
    char *pk_out = op.packed_out - op.pbase;
    // Per lane, once per round: the first word of its segment relative to p0
    // (lanes past the last segment never start one), and its user
    // displacement minus its stream offset, so a word's user address is that
    // of its segment's lane plus the word's own stream offset.
    const int64_t pw = lane < nvalid ? (ps - p0) / W : INT64_MAX;
    const int64_t dd = disp - ps;
    const unsigned upto = 0xffffffffu >> (31 - lane);
    // segments that start before the current window, minus one (the window
    // walks forward one 32-word window at a time)
    int before = __popc(__ballot_sync(FULL, pw < 0)) - 1;
    for (int64_t w0 = 0; w0 < nwords; w0 += 32 * kU) {
        T v[kU];
        int64_t ud[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            // segment of each word of this 32-word window: the segments that
            // start before the window, plus those starting in it up to the
            // word (a bit mask of start positions, one OR-reduction)
            const int64_t wb = w0 + u * 32;
            const int64_t rw = pw - wb;
            const unsigned starts = __reduce_or_sync(FULL, (uint64_t)rw < 32 ? 1u << (int)rw : 0u);
            const int lo = before + __popc(starts & upto);
            before += __popc(starts);
            const int64_t q = p0 + (wb + lane) * W;
            ud[u] = __shfl_sync(FULL, dd, lo) + q;
            if (wb + lane < nwords) {
                if (PACK) v[u] = ldw<W>(op.user_in + ud[u]);
                else v[u] = ldw<W>(pk_in + q);
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const int64_t wi = w0 + u * 32 + lane;
            if (wi < nwords) {
                if (PACK) stw<W>(pk_out + p0 + wi * W, v[u]);
                else stw<W>(op.user_out + ud[u], v[u]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// record-major round
// ---------------------------------------------------------------------------
// A record is one copy of the child that a large index list repeats, when
// that child is a short table of runs or a single run: an indexed or hindexed
// type of a struct of basic blocks (or of a resized block), the
// array-of-records layout.  Record-major movement gives each lane one whole
// record per round of 32 records.  The warp finds the entries of the round's
// records together, as shared_list_round does for segments, and then every
// lane moves run j of its own record at the same time: the run lengths are
// the same on every lane, so no lane waits on another's longer run, and the
// per-round decode is shared by 32 records instead of 32 runs.
#ifndef DTE_REC
#define DTE_REC 1
#endif
constexpr bool kRec = DTE_REC != 0;     // build-time switch for the path
constexpr int kRecMaxRuns = 16;         // runs of the child table
constexpr int64_t kRecMaxSize = 256;    // packed bytes of one record
// The packed side of a round (32 records, contiguous) can go through a
// per-warp shared-memory tile: the lanes write their records into the tile
// in copy words, then the warp moves the tile to or from global memory in
// coalesced 16-byte accesses.  Used where the record's packed size is not a
// multiple of 16 bytes (otherwise a lane's own accesses are already aligned)
// and the round's packed start is 16-byte aligned.
#ifndef DTE_REC_STAGE
#define DTE_REC_STAGE 1
#endif
constexpr bool kRecStage = DTE_REC_STAGE != 0;
constexpr int kRecStageMaxSize = 64;    // packed bytes of a record staged in the tile
constexpr int kRecTile = 32 * kRecStageMaxSize;

// Move one V-byte user word (V >= W) of a run: the user side takes one
// V-byte access, the packed side (global memory, or the warp's shared tile
// when PKSH) V/W words of W bytes.
template <int V, int W, bool PACK, bool PKSH>
__device__ __forceinline__ void rec_word(char *user, char *pk)
{
    using T = typename Word<W>::T;
    union {
        typename Word<V>::T v;
        T w[V / W];
    } x;
    if (PACK) {
        x.v = ldw<V>(user);
#pragma unroll
        for (int k = 0; k < V / W; k++) *reinterpret_cast<T *>(pk + k * W) = x.w[k];
    } else {
#pragma unroll
        for (int k = 0; k < V / W; k++)
            x.w[k] = PKSH ? *reinterpret_cast<const T *>(pk + k * W) : ldw<W>(pk + k * W);
        *reinterpret_cast<typename Word<V>::T *>(user) = x.v;
    }
}

// Move one run of n bytes (a multiple of W) between the user layout and the
// packed side: the user side in the widest words its address allows (16,
// then 8, 4 and 2 bytes while they fit), the packed side in W-byte words.
template <int W, bool PACK, bool PKSH>
__device__ __forceinline__ void rec_run(char *user, char *pk, int n)
{
    const unsigned ua = (unsigned)(uintptr_t)user;
    int o = 0;
    if (W < 16 && (ua & 15) == 0)
        for (; o + 16 <= n; o += 16) rec_word<16, W, PACK, PKSH>(user + o, pk + o);
    if (W < 8 && (ua & 7) == 0)
        for (; o + 8 <= n; o += 8) rec_word<8, W, PACK, PKSH>(user + o, pk + o);
    if (W < 4 && (ua & 3) == 0)
        for (; o + 4 <= n; o += 4) rec_word<4, W, PACK, PKSH>(user + o, pk + o);
    if (W < 2 && (ua & 1) == 0)
        for (; o + 2 <= n; o += 2) rec_word<2, W, PACK, PKSH>(user + o, pk + o);
    for (; o < n; o += W) rec_word<W, W, PACK, PKSH>(user + o, pk + o);
}

// Move nb packed bytes (a multiple of W) between global memory g (16-byte
// aligned) and the warp's tile t: 16-byte accesses, then W-byte words for
// the tail.
template <int W, bool TO_GLOBAL>
__device__ __forceinline__ void rec_tile_move(char *g, char *t, int nb, int lane)
{
    using T = typename Word<W>::T;
    const int n16 = nb & ~15;
    for (int o = lane * 16; o < n16; o += 512) {
        if (TO_GLOBAL) *reinterpret_cast<uint4 *>(g + o) = *reinterpret_cast<const uint4 *>(t + o);
        else *reinterpret_cast<uint4 *>(t + o) = ldw<16>(g + o);
    }
    for (int o = n16 + lane * W; o < nb; o += 32 * W) {
        if (TO_GLOBAL) *reinterpret_cast<T *>(g + o) = *reinterpret_cast<const T *>(t + o);
        else *reinterpret_cast<T *>(t + o) = ldw<W>(g + o);
    }
}

// Where round q of a whole move (never a packed window) sits: records
// local0 .. local0 + 31 of element e, where q = e * rounds_elem + local0 / 32,
// clipped to the element's nrec_elem records.
struct RecPlace {
    int64_t e;
    int64_t local0;
    int64_t pround;  // packed stream offset of the round's first byte
    int nvalid;      // records in the round
};

__device__ __forceinline__ RecPlace rec_place(const Op &op, const DNode &C, int64_t nrec_elem, int64_t rounds_elem,
                                              const FastDiv &div_rounds, int64_t q)
{
    RecPlace r;
    r.e = fdiv(q, div_rounds);
    r.local0 = (q - r.e * rounds_elem) * 32;
    r.nvalid = (int)min((int64_t)32, nrec_elem - r.local0);
    r.pround = r.e * op.esize + r.local0 * C.size;
    return r;
}

// User displacement of the lane's record in round `at` (lanes past nvalid
// get a value that is never used).  Entry b of the root holds records
// pbytes[b] / size(child) onward (every entry has at least one record and
// nothing merges), so lane j loads entry b0 + j's prefix and displacement,
// one OR-reduction marks the entries that start inside the round, and lane l
// takes its entry's values by shuffle.  `rh` is the warp's search position
// in the root list.
__device__ __forceinline__ int64_t rec_locate(const Op &op, const DNode &R, const DNode &C, const char *blob,
                                              const RecPlace &at, int lane, Hint &rh)
{
    const unsigned FULL = 0xffffffffu;
    const int64_t *pb = arr<int64_t>(blob, R.a_pbytes);
    const int64_t *dv = arr<int64_t>(blob, R.a_disp);
    const int64_t b0 = warp_find_le_hint(pb, R.count, at.local0 * C.size, rh, op.root, lane);
    const int64_t bj = b0 + lane;
    const int64_t sj = bj <= R.count ? fdiv(pb[bj], C.div_size) : INT64_MAX;  // first record of entry bj
    const int64_t dj = bj < R.count ? dv[bj] : 0;
    const int64_t o = sj - at.local0;
    const unsigned starts = __reduce_or_sync(FULL, (lane > 0 && o > 0 && o < 32) ? 1u << (int)o : 0u);
    const int jl = __popc(starts & (FULL >> (31 - lane)));
    const int64_t de = __shfl_sync(FULL, dj, jl);
    const int64_t se = __shfl_sync(FULL, sj, jl);
    rh.b = b0 + __shfl_sync(FULL, jl, at.nvalid - 1);
    return at.e * op.extent + R.base + de + (at.local0 + lane - se) * R.stride + C.base;
}

// Move the runs of the lane's record between the user layout (user: the
// record's child copy) and its packed bytes pk (global memory, or the warp's
// tile when PKSH), run j of every lane at the same time.
template <int W, bool PACK, bool PKSH>
__device__ __forceinline__ void rec_runs(const DNode &C, const char *blob, char *user, char *pk, bool live)
{
    if (C.kind == NK_RUN) {
        if (live) rec_run<W, PACK, PKSH>(user, pk, (int)C.len);
        return;
    }
    const int64_t *cpb = arr<int64_t>(blob, C.a_pbytes);
    const int64_t *cdv = arr<int64_t>(blob, C.a_disp);
#pragma unroll 1
    for (int j = 0; j < (int)C.count; j++) {
        const int64_t p = cpb[j];
        const int n = (int)(cpb[j + 1] - p);
        if (live) rec_run<W, PACK, PKSH>(user + cdv[j], pk + p, n);
    }
}

// One round, moved directly (no tile), or staged through the warp's tile
// `tile` when STAGE.
template <int W, bool PACK, bool STAGE>
__device__ __forceinline__ void rec_round(const Op &op, const DNode *nodes, const char *blob, int64_t nrec_elem,
                                          int64_t rounds_elem, const FastDiv &div_rounds, int64_t q, int lane,
                                          Hint &rh, char *tile)
{
    const DNode &R = nodes[op.root];
    const DNode &C = nodes[R.child];
    const RecPlace at = rec_place(op, C, nrec_elem, rounds_elem, div_rounds, q);
    const int64_t ud = rec_locate(op, R, C, blob, at, lane, rh);
    const int csize = (int)C.size;
    const int nb = at.nvalid * csize;
    char *user = (PACK ? const_cast<char *>(op.user_in) : op.user_out) + ud;
    char *gpk = (PACK ? op.packed_out : const_cast<char *>(op.packed_in)) + at.pround;
    char *pk = STAGE ? tile + lane * csize : gpk + lane * csize;
    if (STAGE && !PACK) {
        rec_tile_move<W, false>(gpk, tile, nb, lane);
        __syncwarp();
    }
    rec_runs<W, PACK, STAGE>(C, blob, user, pk, lane < at.nvalid);
    if (STAGE) {
        __syncwarp();
        if (PACK) rec_tile_move<W, true>(gpk, tile, nb, lane);
        __syncwarp();  // the tile is refilled by the next round
    }
}

// Asynchronous 16-byte copies from global into shared memory (cp.async;
// completion per thread by commit and wait groups).
__device__ __forceinline__ void cp_async16(char *sdst, const char *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// The 16-byte part of a round's packed bytes (global, 16-byte aligned) into
// a tile, asynchronously; the tail (nb not a multiple of 16) is loaded when
// the round is scattered.
__device__ __forceinline__ void rec_tile_fetch(const char *g, char *t, int nb, int lane)
{
    const int n16 = nb & ~15;
    for (int o = lane * 16; o < n16; o += 512) cp_async16(t + o, g + o);
}

// Staged unpack of the warp's rounds [q0, q1) with two tiles: the packed
// bytes of the next round are in flight (cp.async) while the entries of the
// current round are searched and its records scattered.  A round's packed
// bytes depend on its position alone, so the copy can start before the
// search.
template <int W>
__device__ __forceinline__ void rec_unpack_rounds(const Op &op, const DNode *nodes, const char *blob,
                                                  int64_t nrec_elem, int64_t rounds_elem, const FastDiv &div_rounds,
                                                  int64_t q0, int64_t q1, int lane, Hint &rh, char *tiles)
{
    using T = typename Word<W>::T;
    const DNode &R = nodes[op.root];
    const DNode &C = nodes[R.child];
    const int csize = (int)C.size;
    {
        const RecPlace first = rec_place(op, C, nrec_elem, rounds_elem, div_rounds, q0);
        rec_tile_fetch(op.packed_in + first.pround, tiles, first.nvalid * csize, lane);
    }
    cp_async_commit();
    for (int64_t q = q0; q < q1; q++) {
        char *tile = tiles + ((q - q0) & 1) * kRecTile;
        if (q + 1 < q1) {
            const RecPlace nx = rec_place(op, C, nrec_elem, rounds_elem, div_rounds, q + 1);
            rec_tile_fetch(op.packed_in + nx.pround, tiles + ((q + 1 - q0) & 1) * kRecTile, nx.nvalid * csize, lane);
        }
        cp_async_commit();  // an empty group when there is no next round
        const RecPlace at = rec_place(op, C, nrec_elem, rounds_elem, div_rounds, q);
        const int64_t ud = rec_locate(op, R, C, blob, at, lane, rh);
        const int nb = at.nvalid * csize;
        const char *g = op.packed_in + at.pround;
        for (int o = (nb & ~15) + lane * W; o < nb; o += 32 * W)
            *reinterpret_cast<T *>(tile + o) = ldw<W>(g + o);
        cp_async_wait_prev();  // this round's tile has landed
        __syncwarp();
        rec_runs<W, false, true>(C, blob, op.user_out + ud, tile + lane * csize, lane < at.nvalid);
        __syncwarp();  // the tile is refilled two rounds on
    }
}

// ---------------------------------------------------------------------------
// batch op records
// ---------------------------------------------------------------------------
struct BatchOp {
    Desc d;
    Op op;
    int64_t nchunks;
    int32_t wsel;   // kernel variant (see wsel_of / kSegClass)
    int32_t soff;   // offset of the descriptor in the group's staged image, or -1
    // segment-major variants only
    int64_t nseg_elem;
    int64_t nsegs;
    FastDiv div_nseg;
};

constexpr int kNumClasses = 14;  // 9 chunk-major word classes + 4 segment-major + wide 16-byte steps
constexpr int kWideClass = 13;

__host__ __device__ constexpr int wsel_of(int W, bool pk16)
{
    return W == 16 ? 0 : W == 8 ? (pk16 ? 1 : 2) : W == 4 ? (pk16 ? 3 : 4) : W == 2 ? (pk16 ? 5 : 6)
                                                                                 : (pk16 ? 7 : 8);
}

// segment-major classes: 9 + (W = 8, 4, 2, 1)
__host__ __device__ constexpr int seg_class(int W)
{
    return 9 + (W == 8 ? 0 : W == 4 ? 1 : W == 2 ? 2 : 3);
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
static int sm_count(int dev)
{
    static int cache[64];
    int &c = cache[dev & 63];
    if (c == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        c = v > 0 ? v : 1;
    }
    return c;
}

template <typename K>
static int occupancy(K kernel, size_t smem)
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, kThreads, smem) != cudaSuccess ||
        blocks <= 0) {
        cudaGetLastError();
        blocks = 1;
    }
    return blocks;
}

static Desc make_desc(const Committed &c, const char *dblob, size_t *smem)
{
    Desc d;
    d.blob = dblob;
    d.blob_bytes = c.bytes;
    d.root = c.root;
    d.nnodes = c.nnodes;
    d.pad_ = 0;
    if (c.bytes <= kSmemBlob) {
        d.stage = STAGE_BLOB;
        *smem = (size_t)c.bytes;
    } else if (c.nnodes <= kMaxSmemNodes) {
        d.stage = STAGE_NODES;
        *smem = (size_t)c.nnodes * sizeof(DNode);
    } else {
        d.stage = STAGE_NONE;
        *smem = 0;
    }
    return d;
}

static int64_t p2addr(const void *p)
{
    uintptr_t u = (uintptr_t)p;
    if (u == 0) return 16;
    uintptr_t low = u & (~u + 1);
    return low >= 16 ? 16 : (int64_t)low;
}

static int64_t p2v(int64_t v)
{
    if (v == 0) return 16;
    uint64_t u = (uint64_t)v;
    uint64_t low = u & (~u + 1);
    return low >= 16 ? 16 : (int64_t)low;
}

// copy word for one operation
static int word_of(const Committed &c, int64_t extent, int64_t count, const void *user, const void *packed)
{
    int64_t W = std::min<int64_t>(c.align, std::min(p2addr(user), p2addr(packed)));
    if (count > 1) W = std::min(W, p2v(extent));
    return (int)W;
}

// Whether whole moves of a type can go record-major (rec_round): its root is
// a large index list of one shared child with no merging (the conditions of
// shared_list_root), and that child is a table of at most kRecMaxRuns runs,
// or one run, of at most kRecMaxSize packed bytes.  *child_size: packed bytes
// of one record.
static bool rec_shape(const Committed &c, int64_t *child_size)
{
    const DNode *n = c.nodes();
    const DNode &R = n[c.root];
    if (R.kind != NK_LIST || !(R.flags & NF_SHARED) || (R.flags & (NF_RUNS | NF_PSEGS | NF_XMERGE | NF_EMERGE)) ||
        R.a_eflags != 0 || R.count <= 32 || R.child < 0)
        return false;
    const DNode &C = n[R.child];
    const bool table = C.kind == NK_LIST && (C.flags & NF_RUNS) && C.count >= 1 && C.count <= kRecMaxRuns;
    if (!(table || C.kind == NK_RUN) || C.size <= 0 || C.size > kRecMaxSize) return false;
    *child_size = C.size;
    return true;
}

static Op make_op(const Committed &c, int64_t extent, const void *user, void *packed, int64_t count)
{
    Op op;
    op.user_in = (const char *)user;
    op.user_out = (char *)user;
    op.packed_in = (const char *)packed;
    op.packed_out = (char *)packed;
    op.total = count * c.size;
    op.pbase = 0;
    op.esize = c.size;
    op.extent = extent;
    op.ediv = c.nodes()[c.root].div_size;
    op.root = c.root;
    op.pad_ = 0;
    return op;
}

static Spread make_spread(int64_t nspans, int64_t nwarps)
{
    Spread sp;
    sp.nspans = nspans;
    sp.mult = 1;
    if (nspans > 2) {
        int64_t m = (int64_t)((double)nspans * 0.6180339887498949);
        if (m < 1) m = 1;
        while (std::gcd(m, nspans) != 1) m++;
        sp.mult = m;
    }
    sp.inc = nspans > 0 ? (int64_t)(((__int128)nwarps * sp.mult) % nspans) : 0;
    sp.div = make_div(nspans);
    return sp;
}

static bool capturing(dte_stream_t stream)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Resolve the device descriptor; frees finished deferred descriptors unless
// the stream is being captured (no event polling inside a capture).
static int prep(dte_type t, dte_stream_t stream, const char **blob, int *dev)
{
    if (!handle_valid(t)) return DTE_ERR_TYPE;
    if (!t->committed) return DTE_ERR_TYPE;
    if (!capturing(stream)) reap_deferred();
    return device_blob(t, blob, dev);
}

// Fill one op record: copy word, kernel variant (segment-major by the same
// rule as single ops, under the type's plan) and its work size.  A batch has
// no bulk-copy variant: DTE_PLAN_BULK takes the fixed rule there.
static void fill_batch_op(BatchOp &h, const Committed &c, int64_t extent, const dte_op &o, const char *dblob,
                          int plan)
{
    size_t smem;
    h.d = make_desc(c, dblob, &smem);
    h.soff = -1;
    h.op = make_op(c, extent, o.user, o.packed, o.count);
    h.nchunks = (h.op.total + 15) / 16;
    int W = word_of(c, extent, o.count, o.user, o.packed);
    if (plan_seg(c, W, plan)) {
        h.wsel = seg_class(W);
        h.nseg_elem = c.nseg;
        h.nsegs = o.count * c.nseg;
        h.div_nseg = c.nodes()[c.root].div_nseg;
    } else if (plan_wide(W, plan)) {
        h.wsel = kWideClass;
    } else {
        h.wsel = wsel_of(W, p2addr(o.packed) >= 16);
    }
}

// tiles of an op: warp steps (1 KiB for 16-byte words, 2 KiB for the wide
// class and the sub-16-byte words) or rounds of 32 segments
static int64_t op_tiles(const BatchOp &h)
{
    if (h.wsel >= 9 && h.wsel < kWideClass) return (h.nsegs + 31) / 32;
    const int64_t st = h.wsel == 0 ? kStepOf<16> : h.wsel == kWideClass ? kStepOf<16, true> : kStep;
    return (h.nchunks + st - 1) / st;
}

}  // namespace dte
