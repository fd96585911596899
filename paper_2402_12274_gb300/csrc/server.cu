// server.cu -- a device-resident request loop for pack/unpack requests.
//
// The paper's progress extension (§7) and generalized-request polling (§2)
// let asynchronous work advance without the caller blocking; its offloading
// section (§5) runs communication inside a GPU stream context.  The request
// loop below is the single-GPU stand-in for that progress engine: a
// persistent kernel that keeps taking work as the host admits it, so pack and
// unpack requests of mixed sizes run continuously batched instead of one
// launch each.
//
//   host                                   device (persistent kernel)
//   ----                                   ---------------------------
//   submit -> FIFO; admit while ring       one warp mirrors newly published
//   slots and the byte cap allow: write    requests into device memory and
//   the record, then publish (release)     appends their tiles to one global
//                                          tile sequence: at once while its
//                                          unclaimed backlog is short, else
//                                          from per-variant queues, one
//                                          variant at a time; the other warps
//                                          claim ranges of the sequence with
//                                          one fetch-add on a single counter,
//                                          sized by the tiles still unclaimed
//   progress: read the completion queue    the warp that finishes a request's
//   (acquire), free capacity, admit more   last tile appends it to the queue
//
// Every device wait is bounded: a warp that finds nothing to do polls with
// __nanosleep and leaves after `idle_limit` of empty polls (a claim it still
// holds is kept in device memory for the same warp of the next launch, and so
// are the mirroring warp's queues); the host relaunches the loop while
// requests are outstanding.  A host stop flag ends it at once.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <climits>
#include <cstdlib>
#include <deque>
#include <vector>

#include "internal.h"
#include "move.cuh"

namespace dte {

struct SlotRec {       // one admitted request (pinned host memory)
    BatchOp op;
    int32_t kind;      // DTE_BATCH_PACK or DTE_BATCH_UNPACK
    int32_t pad_;
    int64_t ntiles;
};

struct Ctrl {          // pinned host control block
    int64_t published; // requests visible to the device
    int64_t stop;      // host asks the loop to leave
    int64_t pad_[6];
};


__device__ __forceinline__ int64_t ld_acquire_sys(const int64_t *p)
{
    int64_t v;
    asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int64_t ld_relaxed_sys(const int64_t *p)
{
    int64_t v;
    asm volatile("ld.relaxed.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys(int64_t *p, int64_t v)
{
    asm volatile("st.release.sys.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One claimed span of tiles [t, t + k) of a request, out of line (one copy of
// each variant for the whole loop, one call per claim).  The search hint h
// is the warp's, kept while it works on the same request, so consecutive
// tiles of a large index table continue the search where it stopped.  The
// spans work on a copy of it in registers: a hint reached through the
// reference would live in local memory, and every descriptor walk reads and
// writes it.
template <int W, bool PACK, bool PK16, bool WIDE = false>
__device__ __noinline__ void serve_chunk_span(const BatchOp *b, int64_t t, int64_t k, int lane, char *scr, Hint &h)
{
    const char *blob = b->d.blob;
    const DNode *nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
    Hint hr = h;
    for (int64_t tt = t; tt < t + k; tt++)
        warp_step<W, PACK, PK16, WIDE>(b->op, nodes, blob, tt * kStepOf<W, WIDE>, b->nchunks, lane, hr, scr);
    h = hr;
}

template <int W, bool PACK>
__device__ __noinline__ void serve_seg_span(const BatchOp *b, int64_t t, int64_t k, int lane, Hint &h)
{
    const char *blob = b->d.blob;
    const DNode *nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
    Hint hr = h, rh{-1, 0};
    for (int64_t tt = t; tt < t + k; tt++)
        seg_round<W, PACK>(b->op, nodes, blob, b->nseg_elem, b->div_nseg, tt * 32, b->nsegs, lane, hr, rh);
    h = hr;
}

template <bool PACK>
__device__ __forceinline__ void serve_span_dir(const BatchOp *b, int64_t t, int64_t k, int lane, char *scr, Hint &h)
{
    switch (b->wsel) {
    case kWideClass: serve_chunk_span<16, PACK, true, true>(b, t, k, lane, scr, h); break;
    case 0: serve_chunk_span<16, PACK, true>(b, t, k, lane, scr, h); break;
    case 1: serve_chunk_span<8, PACK, true>(b, t, k, lane, scr, h); break;
    case 2: serve_chunk_span<8, PACK, false>(b, t, k, lane, scr, h); break;
    case 3: serve_chunk_span<4, PACK, true>(b, t, k, lane, scr, h); break;
    case 4: serve_chunk_span<4, PACK, false>(b, t, k, lane, scr, h); break;
    case 5: serve_chunk_span<2, PACK, true>(b, t, k, lane, scr, h); break;
    case 6: serve_chunk_span<2, PACK, false>(b, t, k, lane, scr, h); break;
    case 7: serve_chunk_span<1, PACK, true>(b, t, k, lane, scr, h); break;
    case 8: serve_chunk_span<1, PACK, false>(b, t, k, lane, scr, h); break;
    case 9: serve_seg_span<8, PACK>(b, t, k, lane, h); break;
    case 10: serve_seg_span<4, PACK>(b, t, k, lane, h); break;
    case 11: serve_seg_span<2, PACK>(b, t, k, lane, h); break;
    default: serve_seg_span<1, PACK>(b, t, k, lane, h); break;
    }
}

__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Device state of the loop (device memory, zero at creation).  The claim
// counter sits alone on its own 128-byte line: every claim is a fetch-add on
// it, while the words the mirroring warp publishes are read by every warp.
struct alignas(128) ClaimLine {
    unsigned long long next;   // next unclaimed tile of the global sequence
};
struct alignas(128) PubLine {
    unsigned long long total;  // tiles of all appended requests (the sequence's length)
    unsigned long long apub;   // requests appended to the sequence
    unsigned long long mirrored;  // requests copied into device memory (the mirroring warp's own)
    int mirror_gone;           // the mirroring warp has left (reset before each launch)
};
struct AppendEnt {             // the request appended at position p (entry p % slots)
    long long tag;             // p (an entry is rewritten for p + slots)
    long long first;           // its first tile in the global sequence
    long long req;             // the request
    long long pad_;
};
struct QEnt {                  // a request waiting in the reorder stage
    long long req, nt;
};
struct alignas(128) MirrorState {  // the reorder stage's queues between launches
    long long qh[32], qt[32];
};
struct Held {                  // a warp's claim, kept across launches of the loop
    long long next, end;
};
struct alignas(128) CqLine {
    unsigned long long tail;   // completion-queue positions handed out
};

struct ServeArgs {
    const SlotRec *ring;       // pinned host ring of admitted requests
    Ctrl *ctrl;                // pinned host control words
    int64_t *cq;               // pinned completion queue, one entry per slot: request + 1, or 0
    unsigned long long *cq_tail;  // device: completions so far (positions handed out)
    ClaimLine *claim;
    PubLine *pub;
    AppendEnt *alist;          // per append position modulo slots
    QEnt *gq;                  // per group, `slots` entries: requests waiting to be appended
    MirrorState *mstate;
    long long *sreq;           // per slot: the request last mirrored into it
    unsigned long long *done;  // per slot: tiles finished
    SlotRec *dring;            // per slot: mirrored record
    Held *held;                // per warp of the grid
    int64_t mask, slots;
    int64_t span_min, span_max;
    int64_t backlog_target;    // unclaimed tiles above which requests wait to be appended
    int64_t idle_budget_ns;
};

// The append position of the request holding global tile c (c < total, read
// after the acquire of total), searched by the whole warp.  Positions [apub -
// slots, apub) hold their entries unless the mirroring warp rewrote one for a
// later append, which it does only after the entry's request completed: such
// an entry belongs to a request appended before c's (c's request has not
// completed, so its entry and every later one are intact), so an entry whose
// tag is not its position counts as "starts at or before c".  The predicate
// "starts at or before c" is then true for every position up to c's request
// and false after it.  `lo` satisfies it.  Each pass probes 32 evenly spaced
// positions of [lo, hi) at once and keeps the stretch after the last one that
// satisfies it: two passes for a ring of 1024 slots.  Returns -1 if lo itself
// fails (never expected: the caller retries).
__device__ __forceinline__ long long request_of_tile(const ServeArgs &a, long long lo, long long hi, long long c,
                                                     int lane)
{
    const unsigned FULL = 0xffffffffu;
    while (hi - lo > 1) {
        const long long step = (hi - lo + 31) >> 5;
        const long long p = lo + (long long)lane * step;
        bool starts_before = false;
        if (p < hi) {
            const AppendEnt *st = a.alist + (p & a.mask);
            // first is published with a release after tag: acquiring it orders
            // the tag read after it, so a tag that still matches goes with its
            // own first
            long long f, tg;
            asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(f) : "l"(&st->first) : "memory");
            asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(tg) : "l"(&st->tag) : "memory");
            starts_before = tg != p || f <= c;
        }
        const unsigned m = __ballot_sync(FULL, starts_before);
        if (m == 0) return -1;
        const long long j = 31 - __clz(m);
        lo += j * step;
        hi = min(lo + step, hi);
    }
    return lo;
}

// Announce request r as complete: append r + 1 to the completion queue at the
// next position.  The host reads the queue in position order and clears what
// it read; positions cannot lap an entry the host has not read (every
// completion belongs to an admitted request, and the host admits a request
// only into a slot it retired through the queue, so completions never exceed
// the host's reads by more than the ring's size).
__device__ __forceinline__ void complete_request(const ServeArgs &a, long long r)
{
    __threadfence_system();
    const unsigned long long pos = atomicAdd(a.cq_tail, 1ull);
    st_release_sys(a.cq + (long long)(pos & (unsigned long long)a.mask), r + 1);
}

// Request-loop waits that gave up (a tile search that kept finding nothing),
// on this device; read by dte_device_timeouts.
__device__ unsigned long long g_serve_timeouts;

// CTAs per SM the loop is compiled for (its register budget) and runs by
// default.  The serving mix, 20,000 requests on one box: 72,148 / 114,875 /
// 139,549 / 151,567 requests/s at 1 / 2 / 3 / 4 CTAs per SM (builds for 3
// and 4); a build for 6 (40 registers) reached 145,293 at 6 and one for 8
// (32 registers) 132,919 at 8.
#ifndef DTE_SERVE_CTAS
#define DTE_SERVE_CTAS 4
#endif
constexpr int kServeCtas = DTE_SERVE_CTAS;
#ifndef DTE_SERVE_QUOTA
#define DTE_SERVE_QUOTA 4
#endif
constexpr long long kServeQuota = DTE_SERVE_QUOTA;  // a group's run, in backlog targets

// Requests wait in the mirroring warp's reorder stage in groups that share a
// kernel variant: direction x word class.
constexpr int kGroups = 2 * kNumClasses;
static_assert(kGroups <= 32, "one group per lane of a warp");

__host__ __device__ constexpr int group_of(int kind, int wsel)
{
    return (kind == DTE_BATCH_PACK ? 0 : kNumClasses) + wsel;
}

// The mirroring warp (warp 0 of CTA 0).  It polls the host's publication
// count, copies new records from pinned host memory into device memory, and
// queues each request by group.  It appends queued requests to the global
// tile sequence while the sequence's unclaimed backlog is below the target:
// at moderate load every request is appended as soon as it is mirrored, in
// admission order; once work piles up, the backlog stays near the target and
// the requests behind it are appended group by group, so the warps claiming
// consecutive tiles run the same kernel variant (interleaving variants on
// the same SMs halves the loop's throughput).  It keeps appending the
// current group while that group has requests queued and its quota (the
// target again, in tiles) lasts, then switches to the group whose queued
// request is oldest: no request waits behind more than one quota of every
// other group.
//
// Append position p's entry is rewritten for p + slots only after the
// request appended at p completed (checked before each append: its ring slot
// now holds a later request, or all its tiles are done), so a warp looking up
// a tile of an incomplete request always finds its entry.
__device__ __forceinline__ void serve_mirror(const ServeArgs &a, int lane)
{
    const unsigned FULL = 0xffffffffu;
    int64_t idle_ns = 0;
    unsigned backoff = 128;
    // this warp is the only writer of these counts: it reads them once (past
    // L1) and keeps them in registers; a plain load could return a stale L1
    // copy of a word that the atomics below update in L2
    long long from = (long long)ld_relaxed_gpu(&a.pub->mirrored);
    long long ap = (long long)ld_relaxed_gpu(&a.pub->apub);
    long long tt = (long long)ld_relaxed_gpu(&a.pub->total);
    // lane g < kGroups: group g's queue [qh, qt), kept in device memory when
    // the loop leaves
    long long qh = 0, qt = 0;
    if (lane < kGroups) {
        qh = (long long)ld_relaxed_gpu(reinterpret_cast<const unsigned long long *>(&a.mstate->qh[lane]));
        qt = (long long)ld_relaxed_gpu(reinterpret_cast<const unsigned long long *>(&a.mstate->qt[lane]));
    }
    int cur = -1;
    long long quota = 0;
    for (;;) {
        long long P = 0;
        bool stop = false;
        if (lane == 0) {
            P = ld_acquire_sys(&a.ctrl->published);
            stop = ld_relaxed_sys(&a.ctrl->stop) != 0;
        }
        P = __shfl_sync(FULL, P, 0);
        if (__shfl_sync(FULL, (int)stop, 0)) break;
        const bool arrived = P > from;
        if (arrived) {
            ld_acquire_sys(&a.ctrl->published);  // each lane orders its reads after the publication
            for (long long q0 = from; q0 < P; q0 += 32) {
                const int n = P - q0 < 32 ? (int)(P - q0) : 32;
                for (int j = 0; j < n; j++) {
                    const int64_t *src = reinterpret_cast<const int64_t *>(a.ring + ((q0 + j) & a.mask));
                    int64_t *dst = reinterpret_cast<int64_t *>(a.dring + ((q0 + j) & a.mask));
                    for (int i = lane; i < (int)(sizeof(SlotRec) / 8); i += 32) dst[i] = ld_relaxed_sys(src + i);
                }
                __threadfence();
                __syncwarp();
                // lane j takes request q0 + j
                int gj = -1;
                long long nt = 0;
                if (lane < n) {
                    const long long qq = q0 + lane, slot = qq & a.mask;
                    const SlotRec *rec = a.dring + slot;
                    nt = (long long)ld_relaxed_gpu(reinterpret_cast<const unsigned long long *>(&rec->ntiles));
                    a.done[slot] = 0;
                    a.sreq[slot] = qq;
                    if (nt == 0) {
                        complete_request(a, qq);  // nothing to move: complete at once
                    } else {
                        int kind, wsel;
                        asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(kind) : "l"(&rec->kind) : "memory");
                        asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(wsel) : "l"(&rec->op.wsel) : "memory");
                        gj = group_of(kind, wsel);
                    }
                }
                // queue them in admission order, each by its group's lane
                for (int j = 0; j < n; j++) {
                    const int gjj = __shfl_sync(FULL, gj, j);
                    const long long ntj = __shfl_sync(FULL, nt, j);
                    if (gjj >= 0 && lane == gjj) {
                        a.gq[(long long)gjj * a.slots + (qt & a.mask)] = QEnt{q0 + j, ntj};
                        qt++;
                    }
                }
            }
            from = P;
            __threadfence();
            __syncwarp();
        }
        // append while the unclaimed backlog is short
        long long G = 0;
        if (lane == 0) G = (long long)ld_relaxed_gpu(&a.claim->next);
        long long backlog = tt - __shfl_sync(FULL, G, 0);
        const long long ap0 = ap;
        for (;;) {
            const unsigned ne = __ballot_sync(FULL, lane < kGroups && qt > qh);
            if (!ne || backlog >= a.backlog_target) break;
            if (cur < 0 || !((ne >> cur) & 1u) || quota <= 0) {
                // the group whose queued request is oldest
                long long front = LLONG_MAX;
                if ((ne >> lane) & 1u) front = a.gq[(long long)lane * a.slots + (qh & a.mask)].req;
                long long best = front;
                for (int o = 16; o > 0; o >>= 1) {
                    const long long other = __shfl_xor_sync(FULL, best, o);
                    best = other < best ? other : best;
                }
                cur = __ffs(__ballot_sync(FULL, front == best)) - 1;
                quota = a.backlog_target * kServeQuota;
            }
            // the entry this append rewrites must belong to a completed request
            int ok = 1;
            if (lane == 0 && ap >= a.slots) {
                const long long old = a.alist[ap & a.mask].req;
                const long long os = old & a.mask;
                const long long occ = (long long)ld_relaxed_gpu(reinterpret_cast<const unsigned long long *>(&a.sreq[os]));
                if (occ == old) {
                    const long long dn = (long long)ld_relaxed_gpu(&a.done[os]);
                    const long long ont = (long long)ld_relaxed_gpu(
                        reinterpret_cast<const unsigned long long *>(&a.dring[os].ntiles));
                    ok = dn == ont;
                }
            }
            if (!__shfl_sync(FULL, ok, 0)) break;  // try again at the next poll
            long long r = 0, nt = 0;
            if (lane == cur) {
                const QEnt e = a.gq[(long long)cur * a.slots + (qh & a.mask)];
                r = e.req;
                nt = e.nt;
                qh++;
            }
            r = __shfl_sync(FULL, r, cur);
            nt = __shfl_sync(FULL, nt, cur);
            if (lane == 0) {
                AppendEnt *e = a.alist + (ap & a.mask);
                e->tag = ap;
                e->req = r;
                asm volatile("st.release.gpu.global.s64 [%0], %1;" ::"l"(&e->first), "l"(tt) : "memory");
            }
            tt += nt;
            ap++;
            backlog += nt;
            quota -= nt;
        }
        if (ap > ap0) {
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                // apub before total: a warp that acquires the new total finds
                // every request its tiles belong to
                atomicExch(&a.pub->apub, (unsigned long long)ap);
                __threadfence();
                atomicExch(&a.pub->total, (unsigned long long)tt);
            }
        }
        if (arrived && lane == 0) atomicExch(&a.pub->mirrored, (unsigned long long)from);
        __syncwarp();
        if (arrived || ap > ap0) {
            idle_ns = 0;
            backoff = 128;
            continue;
        }
        // no progress: nothing arrived and nothing could be appended (the
        // backlog is long enough, or an entry's request has not completed)
        const bool queued = __ballot_sync(FULL, lane < kGroups && qt > qh) != 0;
        idle_ns += queued ? 256 : backoff;
        if (idle_ns > a.idle_budget_ns) {
            // bounded: keep the queues for the next launch and leave; the
            // other warps leave once they run out of tiles, and the host
            // relaunches the loop while requests are outstanding (a request
            // can wait on tiles that a warp claimed past the total and carried
            // out of this launch)
            if (lane < kGroups) {
                a.mstate->qh[lane] = qh;
                a.mstate->qt[lane] = qt;
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicExch(&a.pub->mirror_gone, 1);
            break;
        }
        if (queued) {
            __nanosleep(256);
        } else {
            __nanosleep(backoff);
            backoff = backoff < 2048 ? backoff * 2 : 2048;
        }
    }
}

// The mirroring warp (warp 0 of CTA 0) runs serve_mirror and nothing else:
// it appends requests to the global tile sequence and publishes the new
// total.  Every other warp claims ranges [next, next + k)
// of that sequence with one fetch-add (which always succeeds: a
// compare-and-swap claim fails whenever another claim lands between reading
// the counter and swapping it, which at this claim rate is nearly always).  k
// follows the published tiles left unclaimed (guided self-scheduling: about
// half of them spread over all warps) within [span_min, span_max]: a claim
// costs a chain of dependent round trips, so it always takes enough tiles to
// outweigh that, even when hungry warps keep the unclaimed backlog short.  A
// claim may cover the ends of several requests, which are processed in turn,
// and may run past the published total when warps race for the last tiles
// (an over-claim, at most k tiles per warp): the warp keeps those tiles
// and processes them once the requests they belong to are published.  Tiles
// are never handed out twice (fetch-adds give disjoint ranges) and never
// dropped: a warp gives up a range only by finishing it, and a warp that
// leaves while holding one stores it in held[] for the same warp of the next
// launch (the grid size is fixed per loop).
__global__ void __launch_bounds__(kThreads, kServeCtas) serve_kernel(ServeArgs a)
{
    __shared__ BatchOp wop[kWarps];
    __shared__ uint4 scratch[kThreads];  // chunk assembly for the sub-16-byte word classes
    char *scr = reinterpret_cast<char *>(&scratch[threadIdx.x]);
    __shared__ int32_t wkind[kWarps];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const bool mirror = blockIdx.x == 0 && w == 0;
    const long long nwarps = (long long)gridDim.x * kWarps - 1;  // claiming warps
    // Idle warps of a CTA do not all poll the global words: one scout warp
    // per CTA does, and the others sleep on the CTA's epoch in shared memory,
    // which any warp of the CTA bumps when it sees the published total move.
    // (Thousands of warps polling one line with acquire loads saturate its L2
    // slice, and every claim, fence and completion that goes there queues
    // behind the polls.)
    __shared__ unsigned cta_epoch;
    __shared__ long long cta_total;  // the published total the CTA last saw
    __shared__ int cta_leave;        // the scout has left: the CTA's warps leave
    if (threadIdx.x == 0) {
        cta_epoch = 0;
        cta_total = 0;
        cta_leave = 0;
    }
    __syncthreads();
    const bool scout = w == (blockIdx.x == 0 ? 1 : 0);
    volatile unsigned *vepoch = &cta_epoch;
    volatile long long *vtotal = &cta_total;
    volatile int *vleave = &cta_leave;
    int64_t idle_ns = 0;
    unsigned backoff = 128;
    if (mirror) {
        serve_mirror(a, lane);
        return;
    }
    // lane 0's claim [cn, ce) and the request last found
    const int64_t gw = (int64_t)blockIdx.x * kWarps + w;
    long long cn = 0, ce = 0, q = -1, qr = -1, qfirst = 0, qnt = 0;
    if (lane == 0) {
        cn = a.held[gw].next;
        ce = a.held[gw].end;
        a.held[gw] = Held{0, 0};
    }
    int64_t cached = -1;  // request whose record is in wop[w]
    int64_t miss_ns = 0;  // time spent retrying a tile search that found nothing
    Hint h{-1, 0};        // search position in that request's descriptor
    unsigned ep = 0;  // lane 0: the CTA's epoch before its last look at the total
    for (;;) {
        int have = 0;
        if (lane == 0) {
            ep = *vepoch;
            __threadfence_block();
            const long long TT = (long long)ld_acquire_gpu(&a.pub->total);
            if (TT != *vtotal) {  // wake the CTA's sleeping warps
                *vtotal = TT;
                atomicAdd(&cta_epoch, 1u);
            }
            if (cn >= ce) {
                const long long G = (long long)ld_relaxed_gpu(&a.claim->next);
                if (G < TT) {
                    long long k = (TT - G) / (2 * nwarps);
                    k = k < a.span_min ? a.span_min : k > a.span_max ? a.span_max : k;
                    cn = (long long)atomicAdd(&a.claim->next, (unsigned long long)k);
                    ce = cn + k;
                }
            }
            have = cn < ce && cn < TT;
        }
        if (!__shfl_sync(FULL, have, 0)) {
            // nothing published to work on: wait (an over-claim waits for its
            // tiles); leave on stop, when the mirroring warp has left (nothing
            // more is published in this launch), or after the idle budget --
            // keeping any claim for the same warp of the next launch
            if (scout) {
                if (lane == 0) {
                    int gone;
                    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(gone) : "l"(&a.pub->mirror_gone) : "memory");
                    have = gone || ld_relaxed_sys(&a.ctrl->stop) != 0;
                }
                idle_ns += backoff;
                if (__shfl_sync(FULL, have, 0) || idle_ns > a.idle_budget_ns) {
                    if (lane == 0) {
                        if (cn < ce) a.held[gw] = Held{cn, ce};
                        *vleave = 1;
                    }
                    break;
                }
                __nanosleep(backoff);
                const unsigned cap = __shfl_sync(FULL, (int)(cn < ce), 0) ? 512u : 2048u;
                backoff = backoff < cap ? backoff * 2 : cap;
                continue;
            }
            // the other warps sleep until the CTA's epoch moves past the one
            // seen before their look at the total (bounded like the scout)
            int leave = 0;
            if (lane == 0) {
                for (;;) {
                    if (*vleave) {
                        leave = 1;
                        break;
                    }
                    if (*vepoch != ep) break;
                    idle_ns += backoff;
                    if (idle_ns > a.idle_budget_ns) {
                        leave = 1;
                        break;
                    }
                    __nanosleep(backoff);
                    backoff = backoff < 1024u ? backoff * 2 : 1024u;
                }
                if (leave && cn < ce) a.held[gw] = Held{cn, ce};
            }
            if (__shfl_sync(FULL, leave, 0)) break;
            idle_ns = __shfl_sync(FULL, idle_ns, 0);
            continue;
        }
        backoff = 128;
        // the request holding tile cn (lane 0's cached one, else a warp search)
        long long c = __shfl_sync(FULL, cn, 0);
        if (__shfl_sync(FULL, (int)(q < 0 || c < qfirst || c >= qfirst + qnt), 0)) {
            // the total acquired before the claim bounds c; apub was stored
            // before that total, so every request holding tiles below it is
            // among the positions [.., apub)
            long long dp = 0;
            if (lane == 0) dp = (long long)ld_relaxed_gpu(&a.pub->apub);
            dp = __shfl_sync(FULL, dp, 0);
            long long lo = dp - a.slots > 0 ? dp - a.slots : 0;
            const long long qh = __shfl_sync(FULL, q, 0);
            if (qh > lo && qh < dp) lo = qh;  // claims only move forward
            const long long found = request_of_tile(a, lo, dp, c, lane);
            if (lane == 0) {
                q = found;
                if (q >= 0) {
                    const AppendEnt *e = a.alist + (q & a.mask);
                    qfirst = (long long)ld_acquire_gpu(reinterpret_cast<const unsigned long long *>(&e->first));
                    qr = (long long)ld_relaxed_gpu(reinterpret_cast<const unsigned long long *>(&e->req));
                    const long long tg = (long long)ld_relaxed_gpu(reinterpret_cast<const unsigned long long *>(&e->tag));
                    qnt = (long long)ld_relaxed_gpu(
                        reinterpret_cast<const unsigned long long *>(&a.dring[qr & a.mask].ntiles));
                    if (tg != q || c < qfirst || c >= qfirst + qnt) q = -1;  // never expected: search again
                }
            }
            if (__shfl_sync(FULL, (int)(q < 0), 0)) {
                // never expected; retried under a budget of its own (the idle
                // budget's length).  On expiry the warp counts a device
                // timeout (dte_device_timeouts), keeps its claim for the next
                // launch and leaves; the claim's request stays incomplete
                // until then, which the host's bounded wait reports
                miss_ns += 256;
                if (miss_ns > a.idle_budget_ns) {
                    if (lane == 0) {
                        atomicAdd(&g_serve_timeouts, 1ull);
                        a.held[gw] = Held{cn, ce};
                    }
                    break;
                }
                __nanosleep(256);
                continue;
            }
            miss_ns = 0;
        }
        long long r = 0, t0 = 0, m = 0;
        if (lane == 0) {
            r = qr;
            t0 = cn - qfirst;
            m = (ce < qfirst + qnt ? ce : qfirst + qnt) - cn;
        }
        r = __shfl_sync(FULL, r, 0);
        t0 = __shfl_sync(FULL, t0, 0);
        m = __shfl_sync(FULL, m, 0);
        idle_ns = 0;
        __syncwarp();
        if (r != cached) {
            // the request's record, one 8-byte word per lane, read past L1 (a
            // slot is rewritten for each request), after the acquire of total
            constexpr int kWords = (int)(sizeof(BatchOp) / 8) + 1;  // the op, then its kind
            static_assert(kWords <= 32, "record copied one word per lane");
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&a.dring[r & a.mask]);
            if (lane < kWords) {
                const unsigned long long v = ld_relaxed_gpu(src + lane);
                if (lane < kWords - 1) reinterpret_cast<unsigned long long *>(&wop[w])[lane] = v;
                else wkind[w] = (int32_t)v;
            }
            h = Hint{-1, 0};
            cached = r;
        }
        __syncwarp();
        if (wkind[w] == DTE_BATCH_PACK) serve_span_dir<true>(&wop[w], t0, m, lane, scr, h);
        else serve_span_dir<false>(&wop[w], t0, m, lane, scr, h);
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            const long long slot = r & a.mask;
            const unsigned long long old = atomicAdd(a.done + slot, (unsigned long long)m);
            if ((long long)old + m == qnt) complete_request(a, r);
            cn += m;
        }
        __syncwarp();
    }
}

}  // namespace dte

using namespace dte;

struct dte_server_s {
    int device = -1;
    cudaStream_t stream = nullptr;
    int64_t slots = 0, mask = 0, cap = 0;
    int ctas_per_sm = kServeCtas;
    int sms = 1;
    int64_t span = 4;
    int64_t idle_limit = 0;
    SlotRec *ring = nullptr;  // pinned
    Ctrl *ctrl = nullptr;     // pinned
    int64_t *cq = nullptr;    // pinned completion queue, one entry per slot
    int64_t cq_head = 0;      // next completion-queue position to read
    char *dstate = nullptr;   // device: claim and publication lines, per-slot tiles, done counters,
                              // mirrored records and per-warp held claims
    // host bookkeeping
    struct Pending {
        BatchOp op;
        int kind;
        int64_t ntiles, bytes;
        std::shared_ptr<Committed> keep;
    };
    struct Slot {
        int64_t req = -1;
        int64_t bytes = 0;
        bool open = false;  // admitted, completion not yet accounted
        std::shared_ptr<Committed> keep;
    };
    std::deque<Pending> pending;
    std::vector<Slot> slot;
    int64_t next_req = 0;       // next request index to publish
    int64_t next_ticket = 0;    // tickets are handed out in submission order
    int64_t inflight_bytes = 0, inflight = 0;
    bool launched = false;
    int64_t last_query_ns = 0;  // when the runtime was last asked whether the loop runs
};

namespace dte {

// Largest claim a warp takes at once (tiles); the smallest is the loop's
// span_tiles setting.
#ifndef DTE_SERVE_BACKLOG
#define DTE_SERVE_BACKLOG 4
#endif
// Unclaimed tiles, in claims of span_tiles per claiming warp, above which the
// mirroring warp holds requests back in its per-variant queues.
constexpr int64_t kServeBacklog = DTE_SERVE_BACKLOG;
constexpr int64_t kServeSpanMax = 64;
// Largest span_tiles accepted.
constexpr int64_t kServeSpanLimit = 1 << 16;

// Layout of the device state: ClaimLine | PubLine | CqLine | MirrorState | AppendEnt[slots] |
// sreq[slots] | done[slots] | SlotRec[slots] | QEnt[kGroups * slots] | Held[warps].
static size_t dstate_bytes(int64_t slots, int64_t warps)
{
    return sizeof(ClaimLine) + sizeof(PubLine) + sizeof(CqLine) + sizeof(MirrorState) +
           (size_t)slots * (sizeof(AppendEnt) + sizeof(long long) + sizeof(unsigned long long) + sizeof(SlotRec)) +
           (size_t)kGroups * (size_t)slots * sizeof(QEnt) + (size_t)warps * sizeof(Held);
}

static void server_launch(dte_server s)
{
    ServeArgs a;
    char *p = s->dstate;
    a.claim = reinterpret_cast<ClaimLine *>(p);
    p += sizeof(ClaimLine);
    a.pub = reinterpret_cast<PubLine *>(p);
    p += sizeof(PubLine);
    a.cq_tail = &reinterpret_cast<CqLine *>(p)->tail;
    p += sizeof(CqLine);
    a.mstate = reinterpret_cast<MirrorState *>(p);
    p += sizeof(MirrorState);
    a.alist = reinterpret_cast<AppendEnt *>(p);
    p += (size_t)s->slots * sizeof(AppendEnt);
    a.sreq = reinterpret_cast<long long *>(p);
    p += (size_t)s->slots * sizeof(long long);
    a.done = reinterpret_cast<unsigned long long *>(p);
    p += (size_t)s->slots * sizeof(unsigned long long);
    a.dring = reinterpret_cast<SlotRec *>(p);
    p += (size_t)s->slots * sizeof(SlotRec);
    a.gq = reinterpret_cast<QEnt *>(p);
    p += (size_t)kGroups * (size_t)s->slots * sizeof(QEnt);
    a.held = reinterpret_cast<Held *>(p);
    a.ring = s->ring;
    a.ctrl = s->ctrl;
    a.cq = s->cq;
    a.mask = s->mask;
    a.slots = s->slots;
    a.span_min = s->span;
    a.span_max = std::max<int64_t>(s->span, kServeSpanMax);
    a.idle_budget_ns = s->idle_limit * 1000;
    // enough unclaimed tiles for a few claims of the smallest span per warp
    a.backlog_target = kServeBacklog * ((int64_t)s->sms * s->ctas_per_sm * kWarps - 1) * a.span_min;
    __atomic_store_n(&s->ctrl->stop, (int64_t)0, __ATOMIC_RELEASE);
    // stream-ordered after the previous launch has ended
    if (cudaMemsetAsync(&a.pub->mirror_gone, 0, sizeof(int), s->stream) != cudaSuccess) {
        cudaGetLastError();
        s->launched = false;
        return;
    }
    // the grid is the same at every launch: held claims are per warp
    serve_kernel<<<(unsigned)(s->sms * s->ctas_per_sm), kThreads, 0, s->stream>>>(a);
    s->launched = cudaGetLastError() == cudaSuccess;
}

// Account completions, admit queued requests, and make sure the loop runs.
// Completions are read from the queue the device appends to, so a call costs
// the requests completed since the last one, not the requests in flight.
static int server_progress(dte_server s)
{
    for (;;) {
        int64_t *e = s->cq + (s->cq_head & s->mask);
        const int64_t v = __atomic_load_n(e, __ATOMIC_ACQUIRE);
        if (v == 0) break;
        dte_server_s::Slot &sl = s->slot[(size_t)((v - 1) & s->mask)];
        if (sl.open && sl.req == v - 1) {
            sl.open = false;
            sl.keep.reset();
            s->inflight_bytes -= sl.bytes;
            s->inflight--;
        }
        __atomic_store_n(e, (int64_t)0, __ATOMIC_RELAXED);
        s->cq_head++;
    }
    // admissions, in submission order
    while (!s->pending.empty()) {
        dte_server_s::Pending &p = s->pending.front();
        dte_server_s::Slot &sl = s->slot[(size_t)(s->next_req & s->mask)];
        if (sl.open) break;                                               // ring full
        if (s->inflight > 0 && s->inflight_bytes + p.bytes > s->cap) break;  // byte cap
        SlotRec &rec = s->ring[s->next_req & s->mask];
        rec.op = p.op;
        rec.kind = p.kind;
        rec.ntiles = p.ntiles;
        sl.req = s->next_req;
        sl.bytes = p.bytes;
        sl.open = true;
        sl.keep = std::move(p.keep);
        s->inflight_bytes += p.bytes;
        s->inflight++;
        s->next_req++;
        std::atomic_thread_fence(std::memory_order_release);
        __atomic_store_n(&s->ctrl->published, s->next_req, __ATOMIC_RELEASE);
        s->pending.pop_front();
    }
    // (re)start the loop if it left while work is outstanding; whether it is
    // still running is asked of the runtime at most every 20 us (the loop
    // only leaves after idle_exit_us without work)
    if (s->inflight > 0) {
        const int64_t now = std::chrono::duration_cast<std::chrono::nanoseconds>(
                                std::chrono::steady_clock::now().time_since_epoch())
                                .count();
        if (!s->launched || now - s->last_query_ns > 20000) {
            s->last_query_ns = now;
            bool running = s->launched && cudaStreamQuery(s->stream) == cudaErrorNotReady;
            if (!running) {
                cudaGetLastError();
                server_launch(s);
                if (!s->launched) return DTE_ERR_CUDA;
            }
        }
    }
    return DTE_SUCCESS;
}

// Request-loop waits that gave up on the current device (see g_serve_timeouts).
int serve_timeouts(unsigned long long *v)
{
    if (cudaMemcpyFromSymbol(v, g_serve_timeouts, sizeof *v) != cudaSuccess) {
        cudaGetLastError();
        return DTE_ERR_CUDA;
    }
    return DTE_SUCCESS;
}

// The byte cap of a loop created without one: DTE_SERVE_MAX_INFLIGHT_BYTES
// (a positive integer) if set, else 8 GiB.
static int64_t default_cap()
{
    if (const char *v = std::getenv("DTE_SERVE_MAX_INFLIGHT_BYTES")) {
        char *end = nullptr;
        const long long x = std::strtoll(v, &end, 10);
        if (end != v && *end == '\0' && x > 0) return (int64_t)x;
    }
    return (int64_t)8 << 30;
}

static bool ticket_done(dte_server s, int64_t ticket)
{
    if (ticket >= s->next_req) return false;  // still queued on the host
    const dte_server_s::Slot &sl = s->slot[(size_t)(ticket & s->mask)];
    if (sl.req != ticket) return true;        // its slot was reused: it completed
    return !sl.open;
}

}  // namespace dte

extern "C" {

int dte_server_create(const dte_server_config *cfg, dte_server *out)
{
    if (!out) return DTE_ERR_ARG;
    // default smallest claim 4 tiles: the serving mix at 4 CTAs per SM, one
    // box: 142,700 requests/s and p50 / p99 0.59 / 1.44 ms at 80% of that
    // load; with 8 tiles 151,900 requests/s but 1.46 / 2.86 ms
    dte_server_config c{1024, 0, kServeCtas, 4, 50000};
    if (cfg) c = *cfg;
    if (c.max_inflight_bytes == 0) c.max_inflight_bytes = default_cap();
    if (c.ring_slots <= 0 || (c.ring_slots & (c.ring_slots - 1)) || c.ring_slots > (1 << 20)) return DTE_ERR_ARG;
    if (c.max_inflight_bytes <= 0 || c.ctas_per_sm < 1 || c.ctas_per_sm > kServeCtas || c.span_tiles < 1 || c.span_tiles > kServeSpanLimit ||
        c.idle_exit_us < 1)
        return DTE_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DTE_ERR_NODEVICE;
    }
    auto *s = new dte_server_s();
    s->device = dev;
    s->slots = c.ring_slots;
    s->mask = c.ring_slots - 1;
    s->cap = c.max_inflight_bytes;
    s->ctas_per_sm = c.ctas_per_sm;
    s->span = c.span_tiles;
    s->idle_limit = c.idle_exit_us;
    s->slot.resize((size_t)s->slots);
    if (cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s->sms < 1) {
        cudaGetLastError();
        delete s;
        return DTE_ERR_CUDA;
    }
    const int64_t warps = (int64_t)s->sms * s->ctas_per_sm * kWarps;
    bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaHostAlloc(&s->ring, sizeof(SlotRec) * (size_t)s->slots, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s->ctrl, sizeof(Ctrl), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s->cq, sizeof(int64_t) * (size_t)s->slots, cudaHostAllocMapped) == cudaSuccess &&
              cudaMalloc(&s->dstate, dstate_bytes(s->slots, warps)) == cudaSuccess &&
              cudaMemset(s->dstate, 0, dstate_bytes(s->slots, warps)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        dte_server_free(&s);
        return DTE_ERR_NOMEM;
    }
    std::memset(s->ring, 0, sizeof(SlotRec) * (size_t)s->slots);
    std::memset(s->ctrl, 0, sizeof(Ctrl));
    std::memset(s->cq, 0, sizeof(int64_t) * (size_t)s->slots);
    *out = s;
    return DTE_SUCCESS;
}

int dte_server_submit(dte_server s, int kind, const dte_op *op, int64_t *ticket)
{
    DTE_NVTX_RANGE("dte_server_submit");
    try {
        if (!s || !op || !ticket) return DTE_ERR_ARG;
        if (kind != DTE_BATCH_PACK && kind != DTE_BATCH_UNPACK) return DTE_ERR_ARG;
        if (!handle_valid(op->type) || !op->type->committed) return DTE_ERR_TYPE;
        if (op->count < 0) return DTE_ERR_ARG;
        int64_t total;
        if (__builtin_mul_overflow(op->count, op->type->size, &total)) return DTE_ERR_OVERFLOW;
        if (total > 0 && (!op->user || !op->packed)) return DTE_ERR_ARG;
        if (kind == DTE_BATCH_UNPACK && total > 0 &&
            committed_overlaps(*op->type->desc, op->count, op->type->extent()))
            return DTE_ERR_OVERLAP;
        dte_server_s::Pending p;
        std::memset(&p.op, 0, sizeof p.op);
        p.kind = kind;
        p.ntiles = 0;
        p.bytes = 2 * total;
        if (total > 0) {
            const char *dblob;
            int dev;
            if (int rc = device_blob(op->type, &dblob, &dev)) return rc;
            if (dev != s->device) return DTE_ERR_ARG;
            fill_batch_op(p.op, *op->type->desc, op->type->extent(), *op, dblob, op->type->plan);
            p.ntiles = op_tiles(p.op);
            p.keep = op->type->desc;
        }
        *ticket = s->next_ticket++;
        s->pending.push_back(std::move(p));
        return server_progress(s);
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return DTE_ERR_NOMEM;
    }
}

int dte_server_progress(dte_server s, int64_t *inflight, int64_t *queued)
{
    if (!s) return DTE_ERR_ARG;
    int rc = server_progress(s);
    if (inflight) *inflight = s->inflight;
    if (queued) *queued = (int64_t)s->pending.size();
    return rc;
}

int dte_server_test(dte_server s, int64_t ticket, int *done)
{
    if (!s || !done || ticket < 0 || ticket >= s->next_ticket) return DTE_ERR_ARG;
    int rc = server_progress(s);
    *done = ticket_done(s, ticket) ? 1 : 0;
    return rc;
}

int dte_server_wait(dte_server s, int64_t ticket, int64_t timeout_us)
{
    if (!s || ticket < 0 || ticket >= s->next_ticket || timeout_us < 0) return DTE_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        if (int rc = server_progress(s)) return rc;
        if (ticket_done(s, ticket)) return DTE_SUCCESS;
        auto us = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        if (us > timeout_us) return DTE_ERR_TIMEOUT;
    }
}

int dte_server_free(dte_server *sp)
{
    if (!sp || !*sp) return DTE_ERR_ARG;
    dte_server s = *sp;
    int rc = DTE_SUCCESS;
    if (s->ctrl) __atomic_store_n(&s->ctrl->stop, (int64_t)1, __ATOMIC_RELEASE);
    if (s->stream && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = DTE_ERR_CUDA;
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->ring) cudaFreeHost(s->ring);
    if (s->ctrl) cudaFreeHost(s->ctrl);
    if (s->cq) cudaFreeHost(s->cq);
    if (s->dstate) cudaFree(s->dstate);
    delete s;
    *sp = nullptr;
    return rc;
}

}  // extern "C"
