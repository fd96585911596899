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
//   submit -> FIFO; admit while ring       warps walk the published requests
//   slots and the byte cap allow: write    in order and claim tiles with a
//   the record, then publish (release)     fetch-add on the slot's counter,
//                                          tagged with the request number so a
//                                          reused slot is never confused; the
//                                          record is mirrored into device memory
//   progress: read completion words        the last warp of a request writes its
//   (acquire), free capacity, admit more   completion word (release, system scope)
//
// Every device wait is bounded: a warp that finds nothing to do polls with
// __nanosleep and leaves after `idle_limit` empty polls; the host relaunches
// the loop when work arrives after it left.  A host stop flag ends it at once.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
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

constexpr int kTagBits = 36;  // tile counter = request << 36 | tile
constexpr unsigned long long kTileMask = (1ull << kTagBits) - 1;

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
// tiles of a large index table continue the search where it stopped.
template <int W, bool PACK, bool PK16>
__device__ __noinline__ void serve_chunk_span(const BatchOp *b, int64_t t, int64_t k, int lane, char *scr, Hint &h)
{
    const char *blob = b->d.blob;
    const DNode *nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
    for (int64_t tt = t; tt < t + k; tt++)
        warp_step<W, PACK, PK16>(b->op, nodes, blob, tt * kStepOf<W>, b->nchunks, lane, h, scr);
}

template <int W, bool PACK>
__device__ __noinline__ void serve_seg_span(const BatchOp *b, int64_t t, int64_t k, int lane, Hint &h)
{
    const char *blob = b->d.blob;
    const DNode *nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
    for (int64_t tt = t; tt < t + k; tt++)
        seg_round<W, PACK>(b->op, nodes, blob, b->nseg_elem, b->div_nseg, tt * 32, b->nsegs, lane, h);
}

template <bool PACK>
__device__ __forceinline__ void serve_span_dir(const BatchOp *b, int64_t t, int64_t k, int lane, char *scr, Hint &h)
{
    switch (b->wsel) {
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

// Device state of the loop (device memory, zero at creation); the per-slot
// tile counters, completion counters and mirrored records follow it.
struct DevState {
    unsigned long long cur;   // oldest request still being handed out
    unsigned long long dpub;  // requests mirrored into device memory
    int mlock;                // try-lock of the warp mirroring new requests
    int pad_;
};

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

// Warps claim tiles with fetch-adds on the slot counter of the oldest request
// being handed out; a counter holds (request << 36 | next tile), so a warp
// whose view of the oldest request is stale still learns from the counter
// which request its tiles belong to.  Counters are re-tagged only when a
// request is mirrored into its slot, which the host allows only after the
// slot's previous request completed, so no claimed tile is ever lost.  The
// host side of the ring (pinned memory) is touched only by the warp that
// mirrors new requests and by idle warps.
#ifndef DTE_SERVE_CTAS
#define DTE_SERVE_CTAS 2
#endif
constexpr int kServeCtas = DTE_SERVE_CTAS;  // most CTAs per SM the loop is compiled for

__global__ void __launch_bounds__(kThreads, kServeCtas)
    serve_kernel(const SlotRec *ring, int64_t mask, Ctrl *ctrl, DevState *st, unsigned long long *ctr,
                 unsigned long long *done, SlotRec *dring, int64_t *comp, int64_t span, int64_t idle_budget_ns)
{
    __shared__ BatchOp wop[kWarps];
    __shared__ uint4 scratch[kThreads];  // chunk assembly for the sub-16-byte word classes
    char *scr = reinterpret_cast<char *>(&scratch[threadIdx.x]);
    __shared__ int32_t wkind[kWarps];
    __shared__ int64_t wntiles[kWarps];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    int64_t cached = -1;
    Hint h{-1, 0};  // search position in the current request's descriptor
    int64_t idle_ns = 0;
    unsigned backoff = 256;
    for (;;) {
        int action = 0;  // 0 idle, 1 work, 2 leave, 3 retry, 4 mirror
        int64_t r = 0, t = 0, k = 0;
        if (lane == 0) {
            const unsigned long long c = ld_relaxed_gpu(&st->cur);
            const unsigned long long pub = ld_acquire_gpu(&st->dpub);
            if (c >= pub) {
                const int64_t P = ld_acquire_sys(&ctrl->published);
                if ((unsigned long long)P > pub) {
                    action = atomicCAS(&st->mlock, 0, 1) == 0 ? 4 : 3;
                    r = P;
                } else {
                    action = ld_relaxed_sys(&ctrl->stop) ? 2 : 0;
                }
            } else {
                const int64_t slot = (int64_t)(c & (unsigned long long)mask);
                const unsigned long long v = atomicAdd(ctr + slot, (unsigned long long)span);
                __threadfence();
                const int64_t tag = (int64_t)(v >> kTagBits);
                t = (int64_t)(v & kTileMask);
                const int64_t nt = (int64_t)ld_relaxed_gpu(reinterpret_cast<const unsigned long long *>(&dring[slot].ntiles));
                if (t >= nt) {
                    atomicMax(&st->cur, (unsigned long long)(tag + 1));
                    if (t == 0 && nt == 0) {  // empty request: its first claimer completes it
                        __threadfence_system();
                        st_release_sys(comp + slot, tag + 1);
                    }
                    action = 3;
                } else {
                    r = tag;
                    k = min(span, nt - t);
                    action = 1;
                    wntiles[w] = nt;
                }
            }
        }
        action = __shfl_sync(FULL, action, 0);
        if (action == 2) break;
        if (action == 3) continue;
        if (action == 0) {
            idle_ns += backoff;
            if (idle_ns > idle_budget_ns) break;  // bounded: the host relaunches when work arrives
            __nanosleep(backoff);
            backoff = backoff < 8192 ? backoff * 2 : 8192;
            continue;
        }
        idle_ns = 0;
        backoff = 256;
        r = __shfl_sync(FULL, r, 0);
        if (action == 4) {
            // mirror requests [dpub, P) from pinned host memory into device memory
            const int64_t from = (int64_t)ld_relaxed_gpu(&st->dpub);
            ld_acquire_sys(&ctrl->published);  // each lane orders its reads after the publication
            for (int64_t q = from; q < r; q++) {
                const int64_t *src = reinterpret_cast<const int64_t *>(ring + (q & mask));
                int64_t *dst = reinterpret_cast<int64_t *>(dring + (q & mask));
                for (int i = lane; i < (int)(sizeof(SlotRec) / 8); i += 32) dst[i] = ld_relaxed_sys(src + i);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                for (int64_t q = from; q < r; q++) ctr[q & mask] = ((unsigned long long)q) << kTagBits;
                __threadfence();
                atomicExch(&st->dpub, (unsigned long long)r);
                __threadfence();
                atomicExch(&st->mlock, 0);
            }
            __syncwarp();
            continue;
        }
        t = __shfl_sync(FULL, t, 0);
        k = __shfl_sync(FULL, k, 0);
        __syncwarp();  // lane 0's fence after the counter orders the other lanes' reads below
        if (r != cached) {
            // the request's record, one 8-byte word per lane, read past L1 (a
            // slot is rewritten for each request) and after the counter that
            // announced it
            constexpr int kWords = (int)(sizeof(BatchOp) / 8) + 1;  // the op, then its kind
            static_assert(kWords <= 32, "record copied one word per lane");
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&dring[r & mask]);
            if (lane < kWords) {
                const unsigned long long v = ld_relaxed_gpu(src + lane);
                if (lane < kWords - 1) reinterpret_cast<unsigned long long *>(&wop[w])[lane] = v;
                else wkind[w] = (int32_t)v;
            }
        }
        __syncwarp();
        if (r != cached) h = Hint{-1, 0};
        cached = r;
        if (wkind[w] == DTE_BATCH_PACK) serve_span_dir<true>(&wop[w], t, k, lane, scr, h);
        else serve_span_dir<false>(&wop[w], t, k, lane, scr, h);
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            const int64_t slot = r & mask;
            const unsigned long long old = atomicAdd(done + slot, (unsigned long long)k);
            if ((int64_t)old + k == wntiles[w]) {
                done[slot] = 0;
                __threadfence_system();
                st_release_sys(comp + slot, r + 1);
            }
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
    int ctas_per_sm = 2;
    int64_t span = 4;
    int64_t idle_limit = 0;
    SlotRec *ring = nullptr;  // pinned
    Ctrl *ctrl = nullptr;     // pinned
    int64_t *comp = nullptr;  // pinned, one per slot
    char *dstate = nullptr;   // device: DevState, tile counters, done counters, mirrored records
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
    int64_t oldest_open = 0;    // no request below this is still open
    int64_t inflight_bytes = 0, inflight = 0;
    bool launched = false;
};

namespace dte {

static size_t dstate_bytes(int64_t slots)
{
    return sizeof(DevState) + (size_t)slots * (2 * sizeof(unsigned long long) + sizeof(SlotRec));
}

static void server_launch(dte_server s)
{
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    DevState *st = reinterpret_cast<DevState *>(s->dstate);
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(s->dstate + sizeof(DevState));
    unsigned long long *done = ctr + s->slots;
    SlotRec *dring = reinterpret_cast<SlotRec *>(done + s->slots);
    __atomic_store_n(&s->ctrl->stop, (int64_t)0, __ATOMIC_RELEASE);
    serve_kernel<<<(unsigned)(sms * s->ctas_per_sm), kThreads, 0, s->stream>>>(
        s->ring, s->mask, s->ctrl, st, ctr, done, dring, s->comp, s->span, s->idle_limit * 1000);
    s->launched = cudaGetLastError() == cudaSuccess;
}

// Account completions, admit queued requests, and make sure the loop runs.
static int server_progress(dte_server s)
{
    // completions (completion words are written in any order)
    for (int64_t r = s->oldest_open; r < s->next_req; r++) {
        dte_server_s::Slot &sl = s->slot[(size_t)(r & s->mask)];
        if (!sl.open || sl.req != r) continue;
        if (__atomic_load_n(s->comp + (r & s->mask), __ATOMIC_ACQUIRE) == r + 1) {
            sl.open = false;
            sl.keep.reset();
            s->inflight_bytes -= sl.bytes;
            s->inflight--;
        }
    }
    while (s->oldest_open < s->next_req && !s->slot[(size_t)(s->oldest_open & s->mask)].open) s->oldest_open++;
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
    // (re)start the loop if it left while work is outstanding
    if (s->inflight > 0) {
        bool running = s->launched && cudaStreamQuery(s->stream) == cudaErrorNotReady;
        if (!running) {
            cudaGetLastError();
            server_launch(s);
            if (!s->launched) return DTE_ERR_CUDA;
        }
    }
    return DTE_SUCCESS;
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
    dte_server_config c{1024, (int64_t)8 << 30, 2, 4, 50000};
    if (cfg) c = *cfg;
    if (c.ring_slots <= 0 || (c.ring_slots & (c.ring_slots - 1)) || c.ring_slots > (1 << 20)) return DTE_ERR_ARG;
    if (c.max_inflight_bytes <= 0 || c.ctas_per_sm < 1 || c.ctas_per_sm > kServeCtas || c.span_tiles < 1 ||
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
    bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaHostAlloc(&s->ring, sizeof(SlotRec) * (size_t)s->slots, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s->ctrl, sizeof(Ctrl), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&s->comp, sizeof(int64_t) * (size_t)s->slots, cudaHostAllocMapped) == cudaSuccess &&
              cudaMalloc(&s->dstate, dstate_bytes(s->slots)) == cudaSuccess &&
              cudaMemset(s->dstate, 0, dstate_bytes(s->slots)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        dte_server_free(&s);
        return DTE_ERR_NOMEM;
    }
    std::memset(s->ring, 0, sizeof(SlotRec) * (size_t)s->slots);
    std::memset(s->ctrl, 0, sizeof(Ctrl));
    std::memset(s->comp, 0, sizeof(int64_t) * (size_t)s->slots);
    *out = s;
    return DTE_SUCCESS;
}

int dte_server_submit(dte_server s, int kind, const dte_op *op, int64_t *ticket)
{
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
            fill_batch_op(p.op, *op->type->desc, op->type->extent(), *op, dblob);
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
    if (s->comp) cudaFreeHost(s->comp);
    if (s->dstate) cudaFree(s->dstate);
    delete s;
    *sp = nullptr;
    return rc;
}

}  // extern "C"
