// bulk.cuh -- movement of layouts with long runs by the Tensor Memory
// Accelerator's bulk copies (cp.async.bulk, sm_90 and later).
//
// The packed range is cut into 16 KiB tiles.  Each warp of a CTA owns
// kBulkStages shared-memory stages and walks its tiles with kBulkStages - 1
// tiles of loads in flight:
//   pack:   every lane loads the runs of its 512-byte slice of the tile from
//           the user layout into the stage (one bulk copy per run piece, all
//           completing on the stage's mbarrier), then lane 0 writes the whole
//           tile to the packed buffer with one bulk store;
//   unpack: lane 0 loads the tile from the packed buffer with one bulk copy,
//           then every lane stores the run pieces of its slice to the user
//           layout with bulk stores.
// The threads only decode run boundaries and issue copies; the bytes never
// pass through registers.  A stage is refilled only after the bulk stores
// that read it have finished reading (wait_group.read).  Every mbarrier wait
// is bounded by a cycle budget; a wait that gives up is counted in
// g_bulk_timeouts (read by dte_device_timeouts) and the warp drains what it
// issued, with the same bound, before leaving.
#pragma once

#include "move.cuh"

namespace dte {

constexpr int kBulkWarps = 4;                        // warps per CTA, each with its own stages
constexpr int kBulkStages = 3;                       // stages per warp
constexpr int64_t kBulkTile = 16384;                 // packed bytes per stage
constexpr int64_t kBulkSlice = kBulkTile / 32;       // packed bytes per lane of a tile
constexpr int64_t kBulkSmem = (int64_t)kBulkWarps * kBulkStages * kBulkTile;
constexpr int64_t kBulkMinRun = 2048;                // mean run length that selects this path
// The path pays off only when every warp of a one-CTA-per-SM grid has several
// tiles to keep in flight; with one tile per warp, loads and stores serialise
// and the chunk kernels (a whole move in flight at once) are faster.
constexpr int64_t kBulkMinTilesPerWarp = 6;
constexpr long long kBulkWaitCycles = 1ll << 31;     // about one second at 2 GHz
#ifndef DTE_BULK
#define DTE_BULK 1
#endif
constexpr bool kBulk = DTE_BULK != 0;               // build-time switch for the path

__device__ unsigned long long g_bulk_timeouts;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// arrive on the barrier, announcing `bytes` more bulk-copy bytes for this phase
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kBulkWaitCycles) {
            atomicAdd(&g_bulk_timeouts, 1ull);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// all but the newest N bulk groups of this thread have finished reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// every bulk group of this thread has completed (its writes are done)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// One warp's walk over its tiles (gw, gw + nw, ...).  buf: the warp's
// kBulkStages stages; bar0: shared address of its first stage barrier (the
// others follow at 8-byte steps).
template <bool PACK>
__device__ __forceinline__ void bulk_warp(const Op &op, const DNode *nodes, const char *blob, char *buf,
                                          uint32_t bar0, int64_t gw, int64_t nw, int64_t ntiles, int lane)
{
    const int64_t my = gw < ntiles ? (ntiles - 1 - gw) / nw + 1 : 0;
    Hint h{-1, 0};
    uint32_t phase = 0;  // bit s: parity of the next phase of stage s

    auto issue = [&](int64_t i) {
        const int s = (int)(i % kBulkStages);
        const int64_t P0 = (gw + i * nw) * kBulkTile;
        const int64_t tb = op.total - P0 < kBulkTile ? op.total - P0 : kBulkTile;
        const uint32_t bar = bar0 + 8u * (uint32_t)s;
        char *sb = buf + (int64_t)s * kBulkTile;
        if (PACK) {
            const int64_t lo = (int64_t)lane * kBulkSlice < tb ? (int64_t)lane * kBulkSlice : tb;
            const int64_t hi = lo + kBulkSlice < tb ? lo + kBulkSlice : tb;
            mbar_arrive_tx(bar, (uint32_t)(hi - lo));
            for (int64_t q = lo; q < hi;) {
                int64_t dd, rem;
                locate(op, nodes, blob, P0 + q, dd, rem, h);
                const int64_t n = rem < hi - q ? rem : hi - q;
                bulk_load(smem_u32(sb + q), op.user_in + dd, (uint32_t)n, bar);
                q += n;
            }
        } else if (lane == 0) {
            mbar_arrive_tx(bar, (uint32_t)tb);
            bulk_load(smem_u32(sb), op.packed_in + P0, (uint32_t)tb, bar);
        }
    };

    auto drain = [&](int64_t i) {
        const int s = (int)(i % kBulkStages);
        const int64_t P0 = (gw + i * nw) * kBulkTile;
        const int64_t tb = op.total - P0 < kBulkTile ? op.total - P0 : kBulkTile;
        char *sb = buf + (int64_t)s * kBulkTile;
        if (PACK) {
            if (lane == 0) bulk_store(op.packed_out + P0, smem_u32(sb), (uint32_t)tb);
        } else {
            const int64_t lo = (int64_t)lane * kBulkSlice < tb ? (int64_t)lane * kBulkSlice : tb;
            const int64_t hi = lo + kBulkSlice < tb ? lo + kBulkSlice : tb;
            for (int64_t q = lo; q < hi;) {
                int64_t dd, rem;
                locate(op, nodes, blob, P0 + q, dd, rem, h);
                const int64_t n = rem < hi - q ? rem : hi - q;
                bulk_store(op.user_out + dd, smem_u32(sb + q), (uint32_t)n);
                q += n;
            }
        }
        bulk_commit();  // every lane, so the lanes' group counts stay in step
    };

    const int64_t ahead = kBulkStages - 1;
    int64_t issued = 0;
    for (; issued < ahead && issued < my; issued++) issue(issued);
    int64_t i = 0;
    bool ok = true;
    for (; i < my; i++) {
        const int s = (int)(i % kBulkStages);
        ok = mbar_wait(bar0 + 8u * (uint32_t)s, (phase >> s) & 1u);
        phase ^= 1u << s;
        if (!ok) break;
        drain(i);
        if (issued < my) {
            // the stage of tile `issued` was last drained at tile i - 1: its
            // stores must have finished reading it before it is refilled
            bulk_wait_read<1>();
            __syncwarp();
            issue(issued);
            issued++;
        }
    }
    if (!ok) {
        // drain the loads still in flight (bounded), so no copy targets a
        // stage after the warp has left
        for (int64_t j = i + 1; j < issued; j++) {
            const int s = (int)(j % kBulkStages);
            mbar_wait(bar0 + 8u * (uint32_t)s, (phase >> s) & 1u);
            phase ^= 1u << s;
        }
    }
    bulk_wait_all();
}

// buf_off: byte offset of the stages in dynamic shared memory (after the
// staged descriptor, 128-byte aligned).
template <bool PACK>
__global__ void __launch_bounds__(kBulkWarps * 32, 1) bulk_kernel(Desc d, Op op, int64_t ntiles, int32_t buf_off)
{
    extern __shared__ __align__(128) uint4 smem[];
    __shared__ __align__(8) unsigned long long bars[kBulkWarps][kBulkStages];
    const char *blob;
    const DNode *nodes;
    stage_desc(d, smem, blob, nodes);
    allow_dependents();
    prior_grids_wait();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    char *buf = reinterpret_cast<char *>(smem) + buf_off + (int64_t)w * kBulkStages * kBulkTile;
    const uint32_t bar0 = smem_u32(&bars[w][0]);
    if (lane == 0)
        for (int s = 0; s < kBulkStages; s++) mbar_init(bar0 + 8u * (uint32_t)s, PACK ? 32u : 1u);
    mbar_init_fence();
    __syncwarp();
    bulk_warp<PACK>(op, nodes, blob, buf, bar0, (int64_t)blockIdx.x * kBulkWarps + w,
                    (int64_t)gridDim.x * kBulkWarps, ntiles, lane);
}

}  // namespace dte
