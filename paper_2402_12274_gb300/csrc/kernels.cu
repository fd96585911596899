// kernels.cu -- sm_103a pack / unpack / segment-enumeration kernels and the
// stream-enqueue entry points of the GB300 datatype engine.
//
// Paper anchors (arxiv 2402.12274): §5 (operations on a GPU-stream-backed
// context are queued and run in stream order; no host synchronisation,
// §5.3), §5.2 (send/recv of (buf, count, datatype)), §3.1 (iov queries).
//
// Data movement design (pure data movement, no tensor cores):
//  * The packed side is contiguous, so work is split in packed space: each
//    warp owns a contiguous range of 16-byte chunks; lane l of the warp handles
//    chunks l, l+32, l+64, l+96 of every 512 x 4 byte step, so every packed-side
//    access of a warp is one coalesced 512-byte transaction, and four
//    independent 16-byte loads per lane are in flight before the stores.
//  * Each chunk maps back to the user layout through the committed descriptor
//    (desc.h: REG levels by fast invariant division, LIST levels by a search
//    that gallops from the lane's previous position).
//  * W, the copy word, is the largest power of two <= 16 dividing every run
//    length and displacement of the type and both buffer addresses; a word
//    never straddles two runs, so W = 16 moves each chunk with one 16-byte
//    load and one 16-byte store.  Smaller W assembles the chunk from W-byte
//    words, re-walking the descriptor only when a run ends.
//  * Bytes are moved verbatim through integer registers: no value is ever
//    converted, so NaN payloads survive.
//  * Node tables (<= 64 nodes) are staged in shared memory per CTA.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace dte {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kU = 4;                // chunks per lane per step
constexpr int kMaxSmemNodes = 64;

struct MoveArgs {
    const char *blob;       // device descriptor blob
    const char *user_in;    // pack: user buffer (displacement 0)
    char *user_out;         // unpack: user buffer (displacement 0)
    const char *packed_in;  // unpack: packed bytes (already at position)
    char *packed_out;       // pack: packed bytes (already at position)
    int64_t total;          // bytes moved
    int64_t esize;          // element size
    int64_t extent;         // element stride
    FastDiv ediv;           // / esize
    int64_t nchunks;        // ceil(total / 16)
    int64_t per_warp;       // chunks per warp, multiple of 32*kU
    int root;
    int nnodes;
};

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

__device__ __forceinline__ const DNode *stage_nodes(const char *blob, int nnodes, DNode *smem)
{
    const DNode *g = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
    if (nnodes > kMaxSmemNodes) return g;
    const uint4 *s = reinterpret_cast<const uint4 *>(g);
    uint4 *d = reinterpret_cast<uint4 *>(smem);
    int nw = nnodes * (int)(sizeof(DNode) / 16);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) d[i] = s[i];
    __syncthreads();
    return smem;
}

// packed offset P -> user displacement and bytes left in that run
__device__ __forceinline__ void locate(const MoveArgs &a, const DNode *nodes, int64_t P, int64_t &d,
                                       int64_t &rem, Hint &h)
{
    int64_t e = fdiv(P, a.ediv);
    d = e * a.extent;
    decode_bytes(nodes, a.blob, a.root, P - e * a.esize, d, rem, h);
}

template <int W>
__device__ __forceinline__ typename Word<W>::T ldw(const char *p)
{
    return __ldg(reinterpret_cast<const typename Word<W>::T *>(p));
}

template <>
__device__ __forceinline__ uint4 ldw<16>(const char *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

template <int W>
__device__ __forceinline__ void stw(char *p, typename Word<W>::T v)
{
    *reinterpret_cast<typename Word<W>::T *>(p) = v;
}

// gather the nb (<= 16) packed bytes starting at P from the user layout
template <int W>
__device__ __forceinline__ uint4 gather_chunk(const MoveArgs &a, const DNode *nodes, int64_t P, int nb,
                                              Hint &h)
{
    Chunk<W> c;
    if (W == 16) {
        int64_t d, rem;
        locate(a, nodes, P, d, rem, h);
        c.v = ldw<16>(a.user_in + d);
        return c.v;
    }
    c.v = make_uint4(0, 0, 0, 0);
    int64_t d = 0, rem = 0;
#pragma unroll
    for (int s = 0; s < 16 / W; s++) {
        if (s * W < nb) {
            if (rem <= 0) locate(a, nodes, P + s * W, d, rem, h);
            c.w[s] = ldw<W>(a.user_in + d);
            d += W;
            rem -= W;
        }
    }
    return c.v;
}

template <int W>
__device__ __forceinline__ void scatter_chunk(const MoveArgs &a, const DNode *nodes, int64_t P, int nb,
                                              uint4 v, Hint &h)
{
    Chunk<W> c;
    c.v = v;
    if (W == 16) {
        int64_t d, rem;
        locate(a, nodes, P, d, rem, h);
        *reinterpret_cast<uint4 *>(a.user_out + d) = c.v;
        return;
    }
    int64_t d = 0, rem = 0;
#pragma unroll
    for (int s = 0; s < 16 / W; s++) {
        if (s * W < nb) {
            if (rem <= 0) locate(a, nodes, P + s * W, d, rem, h);
            stw<W>(a.user_out + d, c.w[s]);
            d += W;
            rem -= W;
        }
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

template <int W, bool PACK, bool PK16>
__global__ void __launch_bounds__(kThreads) move_kernel(MoveArgs a)
{
    __shared__ DNode snodes[kMaxSmemNodes];
    const DNode *nodes = stage_nodes(a.blob, a.nnodes, snodes);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t c0 = warp * a.per_warp;
    const int64_t c1 = min(c0 + a.per_warp, a.nchunks);
    Hint h{-1, 0};
    for (int64_t base = c0; base < c1; base += 32 * kU) {
        uint4 v[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            int64_t c = base + u * 32 + lane;
            if (c < c1) {
                int64_t P = c * 16;
                int nb = (int)(a.total - P < 16 ? a.total - P : 16);
                if (PACK) v[u] = gather_chunk<W>(a, nodes, P, nb, h);
                else v[u] = load_packed<W, PK16>(a.packed_in + P, nb);
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            int64_t c = base + u * 32 + lane;
            if (c < c1) {
                int64_t P = c * 16;
                int nb = (int)(a.total - P < 16 ? a.total - P : 16);
                if (PACK) store_packed<W, PK16>(a.packed_out + P, v[u], nb);
                else scatter_chunk<W>(a, nodes, P, nb, v[u], h);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// segment enumeration (§3.1 MPIX_Type_iov, device form)
// ---------------------------------------------------------------------------
struct IovArgs {
    const char *blob;
    dte_iov *out;
    int64_t *actual;
    const char *base;
    int64_t first;      // first segment index (over count elements)
    int64_t n;          // segments to write
    int64_t nseg;       // per element
    FastDiv div_nseg;
    int64_t extent;
    int64_t per_warp;
    int root;
    int nnodes;
};

__global__ void __launch_bounds__(kThreads) iov_kernel(IovArgs a)
{
    __shared__ DNode snodes[kMaxSmemNodes];
    const DNode *nodes = stage_nodes(a.blob, a.nnodes, snodes);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t k0 = warp * a.per_warp;
    const int64_t k1 = min(k0 + a.per_warp, a.n);
    Hint h{-1, 0};
    for (int64_t k = k0 + lane; k < k1; k += 32) {
        int64_t s = a.first + k;
        int64_t e = fdiv(s, a.div_nseg);
        int64_t d = e * a.extent, len = 0;
        decode_seg(nodes, a.blob, a.root, s - e * a.nseg, d, len, h);
        dte_iov v;
        v.iov_base = (void *)(a.base + d);
        v.iov_len = len;
        a.out[k] = v;
    }
    if (a.actual && blockIdx.x == 0 && threadIdx.x == 0) *a.actual = a.n;
}

// §3.1 MPIX_Type_iov_len for a batch of budgets
__global__ void __launch_bounds__(kThreads) iov_len_kernel(const char *blob, int root, int64_t nq,
                                                           const int64_t *budget, int64_t *out_len,
                                                           int64_t *out_bytes, int64_t size, int64_t nseg)
{
    const DNode *nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
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
        } else {
            decode_pos(nodes, blob, root, B, k, st);
        }
        out_len[q] = k;
        out_bytes[q] = st;
    }
}

// byte offset -> first segment index and count (first pass of iov_at_bytes)
__global__ void __launch_bounds__(kThreads) at_bytes_first_kernel(const char *blob, int root, int64_t nq,
                                                                  const int64_t *off, int64_t maxlen,
                                                                  int64_t *first, int64_t *actual,
                                                                  int64_t size, int64_t nseg)
{
    const DNode *nodes = reinterpret_cast<const DNode *>(blob + sizeof(BlobHeader));
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t B = off[q];
        if (B < 0 || B >= size) {
            first[q] = -1;
            actual[q] = 0;
            continue;
        }
        int64_t k, st;
        decode_pos(nodes, blob, root, B, k, st);
        first[q] = k;
        actual[q] = min(maxlen, nseg - k);
    }
}

__global__ void __launch_bounds__(kThreads) at_bytes_fill_kernel(const char *blob, int root, int nnodes,
                                                                 int64_t nq, int64_t maxlen,
                                                                 FastDiv div_max, const int64_t *first,
                                                                 const int64_t *actual, dte_iov *out,
                                                                 const char *base)
{
    __shared__ DNode snodes[kMaxSmemNodes];
    const DNode *nodes = stage_nodes(blob, nnodes, snodes);
    Hint h{-1, 0};
    int64_t total = nq * maxlen;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
         it += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = fdiv(it, div_max);
        int64_t i = it - q * maxlen;
        if (i >= actual[q]) continue;
        int64_t d = 0, len = 0;
        decode_seg(nodes, blob, root, first[q] + i, d, len, h);
        dte_iov v;
        v.iov_base = (void *)(base + d);
        v.iov_len = len;
        out[it] = v;
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
struct DevInfo {
    int sms = 0;
};

static DevInfo &dev_info(int dev)
{
    static DevInfo info[64];
    DevInfo &d = info[dev & 63];
    if (d.sms == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        d.sms = v > 0 ? v : 1;
    }
    return d;
}

template <typename K>
static int occupancy(K kernel)
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, kThreads, 0) != cudaSuccess ||
        blocks <= 0) {
        cudaGetLastError();
        blocks = 1;
    }
    return blocks;
}

typedef void (*MoveKernel)(MoveArgs);

template <bool PACK>
static MoveKernel pick_move(int W, bool pk16)
{
    switch (W) {
    case 16: return move_kernel<16, PACK, true>;
    case 8: return pk16 ? move_kernel<8, PACK, true> : move_kernel<8, PACK, false>;
    case 4: return pk16 ? move_kernel<4, PACK, true> : move_kernel<4, PACK, false>;
    case 2: return pk16 ? move_kernel<2, PACK, true> : move_kernel<2, PACK, false>;
    default: return pk16 ? move_kernel<1, PACK, true> : move_kernel<1, PACK, false>;
    }
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

static int launch_move(bool pack, dte_type t, const char *blob, const void *user, void *packed, int64_t count,
                       cudaStream_t stream, int dev)
{
    Committed &c = *t->desc;
    int64_t total = count * c.size;
    if (total == 0) return DTE_SUCCESS;
    int64_t W = std::min<int64_t>(c.align, std::min(p2addr(user), p2addr(packed)));
    if (count > 1) W = std::min(W, p2v(t->extent()));
    bool pk16 = p2addr(packed) >= 16;
    MoveKernel k = pack ? pick_move<true>((int)W, pk16) : pick_move<false>((int)W, pk16);

    static thread_local int occ_cache[64][2][5][2];
    int wi = W == 16 ? 0 : W == 8 ? 1 : W == 4 ? 2 : W == 2 ? 3 : 4;
    int &occ = occ_cache[dev & 63][pack ? 1 : 0][wi][pk16 ? 1 : 0];
    if (occ == 0) occ = occupancy(k);

    MoveArgs a;
    a.blob = blob;
    a.user_in = (const char *)user;
    a.user_out = (char *)user;
    a.packed_in = (const char *)packed;
    a.packed_out = (char *)packed;
    a.total = total;
    a.esize = c.size;
    a.extent = t->extent();
    a.ediv = c.nodes()[c.root].div_size;  // divides by the element size
    a.nchunks = (total + 15) / 16;
    a.root = c.root;
    a.nnodes = c.nnodes;
    const int64_t step = 32 * kU;
    int64_t warps_needed = (a.nchunks + step - 1) / step;
    int64_t max_blocks = (int64_t)dev_info(dev).sms * occ;
    int64_t blocks = std::min<int64_t>((warps_needed + kWarps - 1) / kWarps, max_blocks);
    if (blocks < 1) blocks = 1;
    int64_t per_warp = (a.nchunks + blocks * kWarps - 1) / (blocks * kWarps);
    per_warp = (per_warp + step - 1) / step * step;
    a.per_warp = per_warp;
    blocks = std::min<int64_t>(blocks, (a.nchunks + per_warp * kWarps - 1) / (per_warp * kWarps));
    k<<<(unsigned)blocks, kThreads, 0, stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
    return DTE_SUCCESS;
}

static int prep(dte_type t, const char **blob, int *dev)
{
    if (!handle_valid(t)) return DTE_ERR_TYPE;
    if (!t->committed) return DTE_ERR_TYPE;
    reap_deferred();
    return device_blob(t, blob, dev);
}

}  // namespace dte

using namespace dte;

extern "C" {

int dte_pack_enqueue(const void *inbuf, int64_t incount, dte_type type, void *outbuf, int64_t outsize,
                     int64_t *position, dte_stream_t stream)
{
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
        if (int rc = prep(type, &blob, &dev)) return rc;
        int rc = launch_move(true, type, blob, inbuf, (char *)outbuf + *position, incount,
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
        if (int rc = prep(type, &blob, &dev)) return rc;
        int rc = launch_move(false, type, blob, outbuf, (char *)inbuf + *position, outcount,
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

int dte_type_iov_async(dte_type type, int64_t count, int64_t iov_offset, dte_iov *d_iov, int64_t max_iov_len,
                       int64_t *d_actual_iov_len, const void *base, dte_stream_t stream)
{
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
        if (int rc = prep(type, &blob, &dev)) return rc;
        if (n == 0) {
            if (d_actual_iov_len &&
                cudaMemsetAsync(d_actual_iov_len, 0, sizeof(int64_t), (cudaStream_t)stream) != cudaSuccess)
                return DTE_ERR_CUDA;
            return DTE_SUCCESS;
        }
        IovArgs a;
        a.blob = blob;
        a.out = d_iov;
        a.actual = d_actual_iov_len;
        a.base = (const char *)base;
        a.first = iov_offset;
        a.n = n;
        a.nseg = c.nseg;
        a.div_nseg = c.nodes()[c.root].div_nseg;
        a.extent = type->extent();
        a.root = c.root;
        a.nnodes = c.nnodes;
        int64_t warps_needed = (n + 127) / 128;
        int64_t max_blocks = (int64_t)dev_info(dev).sms * 8;
        int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((warps_needed + kWarps - 1) / kWarps, max_blocks));
        int64_t per_warp = (n + blocks * kWarps - 1) / (blocks * kWarps);
        per_warp = (per_warp + 31) / 32 * 32;
        a.per_warp = per_warp;
        iov_kernel<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(a);
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
    try {
        if (!handle_valid(type)) return DTE_ERR_TYPE;
        if (!type->committed) return DTE_ERR_TYPE;
        if (n < 0 || (n > 0 && (!d_budget || !d_iov_len || !d_iov_bytes))) return DTE_ERR_ARG;
        if (n == 0) return DTE_SUCCESS;
        const char *blob;
        int dev;
        if (int rc = prep(type, &blob, &dev)) return rc;
        Committed &c = *type->desc;
        int64_t blocks = std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)dev_info(dev).sms * 8);
        iov_len_kernel<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(
            blob, c.root, n, d_budget, d_iov_len, d_iov_bytes, c.size, c.nseg);
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
        if (int rc = prep(type, &blob, &dev)) return rc;
        Committed &c = *type->desc;
        int64_t sms = dev_info(dev).sms;
        int64_t b1 = std::min<int64_t>((n + kThreads - 1) / kThreads, sms * 8);
        at_bytes_first_kernel<<<(unsigned)b1, kThreads, 0, (cudaStream_t)stream>>>(
            blob, c.root, n, d_offset, max_iov_len, d_first, d_actual, c.size, c.nseg);
        if (cudaGetLastError() != cudaSuccess) return DTE_ERR_CUDA;
        if (total > 0) {
            FastDiv dm = make_div(max_iov_len);
            int64_t b2 = std::min<int64_t>((total + kThreads - 1) / kThreads, sms * 8);
            at_bytes_fill_kernel<<<(unsigned)b2, kThreads, 0, (cudaStream_t)stream>>>(
                blob, c.root, c.nnodes, n, max_iov_len, dm, d_first, d_actual, d_iov, (const char *)base);
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

}  // extern "C"
