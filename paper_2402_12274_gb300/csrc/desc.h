// desc.h -- the committed datatype descriptor and the routines that walk it.
//
// A committed type is lowered into a small tree of nodes (paper §3: a layout
// that nests, has offsets and may overlap is described in O(1) instead of
// one iovec entry per segment):
//
//   RUN   len bytes, contiguous.
//   REG   `count` copies of a child at a byte `stride` (vector, hvector,
//         contiguous, subarray dimensions, the element level of a pack).
//   LIST  `count` entries; entry b is cnt[b] copies of a child at the child's
//         stride, placed at disp[b] (indexed, hindexed, struct).  Entries
//         carry prefix sums of packed bytes (and of segments, for the iov
//         queries) so any packed byte or segment is found by binary search.
//         A LIST whose entries are all single runs is stored as a run table.
//
// Every node also records how its segments merge: a segment absorbs the
// next typemap entry exactly when that entry starts at the segment's end
// (the merge rule that makes a YZ face Ny*Nz segments, §3).  REG nodes with
// a multi-segment child whose last segment abuts the next copy's first one
// carry NF_MERGE; LIST nodes keep per-entry "merged into the previous entry"
// bits plus the lengths that chains of merges add (tail) or reach back (head).
//
// The same structs and decode routines are compiled for the host (iov
// queries, tests of the commit compiler) and for sm_103a (kernels).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define DTE_HD __host__ __device__ __forceinline__
#else
#define DTE_HD inline
#endif

namespace dte {

enum : int32_t { NK_RUN = 0, NK_REG = 1, NK_LIST = 2 };

enum : int32_t {
    NF_MERGE = 1,       // REG: copy i's last segment merges with copy i+1's first
    NF_RUNS = 2,        // LIST: every entry is one run of pbytes[b+1]-pbytes[b] bytes
    NF_SHARED = 4,      // LIST: one child and one stride for all entries
    NF_XMERGE = 8,      // LIST: some entry's first segment continues the previous one
    NF_PSEGS = 16,      // LIST: explicit segment prefix array present
    NF_EMERGE = 32,     // LIST (shared): NF_MERGE semantics inside every entry
};

// per-entry flag bits of a LIST (a_eflags)
enum : uint8_t { EF_MERGE = 1, EF_MERGED_IN = 2, EF_SINGLE = 4 };

// Division by an invariant positive divisor d, 0 <= n < 2^63 (Granlund &
// Montgomery, "Division by invariant integers using multiplication", PLDI
// 1994, round-up variant with N = 63): l = ceil(log2 d), m = ceil(2^(63+l)/d)
// < 2^64, and floor(n/d) = floor(n*m / 2^(63+l)) = mulhi64(n, m) >> (l-1).
// d == 1 is a pass-through (mode 0).
struct FastDiv {
    uint64_t m;
    uint32_t s;
    uint32_t mode;
};

DTE_HD int64_t fdiv(int64_t n, const FastDiv &d)
{
    if (d.mode == 0) return n;
#if defined(__CUDA_ARCH__)
    uint64_t hi = __umul64hi((uint64_t)n, d.m);
#else
    uint64_t hi = (uint64_t)(((unsigned __int128)(uint64_t)n * d.m) >> 64);
#endif
    return (int64_t)(hi >> d.s);
}

struct alignas(16) DNode {
    int32_t kind;
    int32_t flags;
    int32_t child;          // REG child, or LIST shared child (-1 if none)
    int32_t pad_;
    int64_t base;           // displacement added on entering the node
    int64_t size;           // packed bytes of one copy of this node
    int64_t nseg;           // merged segments of one copy
    int64_t first_len;      // merged length of the first segment
    int64_t last_len;       // merged length of the last segment
    int64_t count;          // REG copies, or LIST entries
    int64_t stride;         // REG stride, or LIST shared stride
    int64_t len;            // RUN length
    FastDiv div_size;       // / size
    FastDiv div_nseg;       // / nseg
    FastDiv div_nsegm1;     // / (nseg - 1)
    // LIST arrays: byte offsets into the blob (0 = absent)
    int64_t a_disp;         // int64[count]  entry displacement
    int64_t a_pbytes;       // int64[count+1] packed-byte prefix
    int64_t a_psegs;        // int64[count+1] segment prefix (NF_PSEGS)
    int64_t a_child;        // int32[count]  per-entry child (no NF_SHARED)
    int64_t a_stride;       // int64[count]  per-entry stride (no NF_SHARED)
    int64_t a_eflags;       // uint8[count]  EF_* bits (absent: all zero)
    int64_t a_tail;         // int64[count]  bytes merged onto the entry's last segment
    int64_t a_head;         // int64[count]  bytes its first segment reaches back
};

static_assert(sizeof(DNode) % 16 == 0, "DNode must stay 16-byte sized");

// Blob header; DNode array follows at offset sizeof(BlobHeader).
struct alignas(16) BlobHeader {
    int32_t root;
    int32_t nnodes;
    int64_t bytes;
};

template <typename T>
DTE_HD const T *arr(const char *blob, int64_t off)
{
    return reinterpret_cast<const T *>(blob + off);
}

// Largest b in [lo, hi) with a[b] <= x, given a[lo] <= x (and a[hi] > x or
// hi the end).
DTE_HD int64_t bsearch_le(const int64_t *a, int64_t lo, int64_t hi, int64_t x)
{
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Cached LIST position for consecutive lookups by one thread.
struct Hint {
    int32_t node;
    int64_t b;
};

DTE_HD int64_t find_le(const int64_t *a, int64_t n, int64_t x, Hint &h, int node)
{
    // Short lists (a struct's members, a record's runs) are searched
    // directly; the hint is kept for the large table on the path, which
    // would otherwise be re-searched from the top after every visit to a
    // short child list.
    if (n <= 32) return bsearch_le(a, 0, n, x);
    if (h.node != node) {
        int64_t b = bsearch_le(a, 0, n, x);
        h.node = node;
        h.b = b;
        return b;
    }
    int64_t g = h.b;
    int64_t lo, hi;
    if (a[g] <= x) {  // gallop forward
        int64_t step = 1;
        lo = g;
        for (;;) {
            hi = lo + step;
            if (hi >= n) { hi = n; break; }
            if (a[hi] > x) break;
            lo = hi;
            step <<= 1;
        }
    } else {          // gallop backward (a[0] == 0 <= x always)
        int64_t step = 1;
        hi = g;
        for (;;) {
            lo = hi - step;
            if (lo <= 0) { lo = 0; break; }
            if (a[lo] <= x) break;
            hi = lo;
            step <<= 1;
        }
    }
    int64_t b = bsearch_le(a, lo, hi, x);
    h.b = b;
    return b;
}

// Segment-prefix of LIST entry b (explicit, or derived when nothing merges).
DTE_HD int64_t list_psegs(const DNode &N, const DNode &C, const char *blob, int64_t b,
                          const int64_t *pb)
{
    if (N.flags & NF_PSEGS) return arr<int64_t>(blob, N.a_psegs)[b];
    if (N.flags & NF_RUNS) return b;
    return fdiv(pb[b], C.div_size) * C.nseg;
}

// ---------------------------------------------------------------------------
// Packed byte -> source displacement.  `P` is a packed offset inside one copy
// of `node` (0 <= P < size).  Adds the displacement of that byte to `disp`
// and returns in `rem` how many bytes of its run follow (>= 1).
// ---------------------------------------------------------------------------
DTE_HD void decode_bytes(const DNode *nodes, const char *blob, int node, int64_t P,
                         int64_t &disp, int64_t &rem, Hint &h)
{
    for (;;) {
        const DNode &N = nodes[node];
        disp += N.base;
        if (N.kind == NK_RUN) {
            disp += P;
            rem = N.len - P;
            return;
        }
        if (N.kind == NK_REG) {
            const DNode &C = nodes[N.child];
            int64_t i = fdiv(P, C.div_size);
            P -= i * C.size;
            disp += i * N.stride;
            node = N.child;
            continue;
        }
        const int64_t *pb = arr<int64_t>(blob, N.a_pbytes);
        int64_t b = find_le(pb, N.count, P, h, node);
        int64_t off = P - pb[b];
        disp += arr<int64_t>(blob, N.a_disp)[b];
        if (N.flags & NF_RUNS) {
            disp += off;
            rem = (pb[b + 1] - pb[b]) - off;
            return;
        }
        int child;
        int64_t stride;
        if (N.flags & NF_SHARED) {
            child = N.child;
            stride = N.stride;
        } else {
            child = arr<int32_t>(blob, N.a_child)[b];
            stride = arr<int64_t>(blob, N.a_stride)[b];
        }
        const DNode &C = nodes[child];
        int64_t j = fdiv(off, C.div_size);
        P = off - j * C.size;
        disp += j * stride;
        node = child;
    }
}

// ---------------------------------------------------------------------------
// Packed byte -> (index of the merged segment containing it, packed offset
// where that segment starts).  0 <= P < size.
// ---------------------------------------------------------------------------
DTE_HD void decode_pos(const DNode *nodes, const char *blob, int node, int64_t P,
                       int64_t &k, int64_t &start)
{
    Hint h{-1, 0};
    k = 0;
    start = 0;
    for (;;) {
        const DNode &N = nodes[node];
        if (N.kind == NK_RUN) return;
        if (N.kind == NK_REG) {
            const DNode &C = nodes[N.child];
            int64_t i = fdiv(P, C.div_size);
            int64_t r = P - i * C.size;
            bool mg = (N.flags & NF_MERGE) != 0;
            if (mg && i > 0 && r < C.first_len) {
                // inside the part of a merged segment that copy i contributes
                k += i * (C.nseg - 1);
                start += i * C.size - C.last_len;
                return;
            }
            k += i * (mg ? C.nseg - 1 : C.nseg);
            start += i * C.size;
            P = r;
            node = N.child;
            continue;
        }
        const int64_t *pb = arr<int64_t>(blob, N.a_pbytes);
        int64_t b = find_le(pb, N.count, P, h, node);
        int64_t off = P - pb[b];
        if (N.flags & NF_RUNS) {
            k += b;
            start += pb[b];
            return;
        }
        int child;
        uint8_t ef = N.a_eflags ? arr<uint8_t>(blob, N.a_eflags)[b] : 0;
        if (N.flags & NF_SHARED) {
            child = N.child;
            if (N.flags & NF_EMERGE) ef |= EF_MERGE;
        } else {
            child = arr<int32_t>(blob, N.a_child)[b];
        }
        const DNode &C = nodes[child];
        int64_t ps = list_psegs(N, C, blob, b, pb);
        int64_t mi = (ef & EF_MERGED_IN) ? 1 : 0;
        if (ef & EF_SINGLE) {  // the whole entry is one run
            if (mi) { k += ps - 1; start += pb[b] - arr<int64_t>(blob, N.a_head)[b]; }
            else { k += ps; start += pb[b]; }
            return;
        }
        int64_t i = fdiv(off, C.div_size);
        int64_t r = off - i * C.size;
        if (mi && i == 0 && r < C.first_len) {
            k += ps - 1;
            start += pb[b] - arr<int64_t>(blob, N.a_head)[b];
            return;
        }
        bool mg = (ef & EF_MERGE) != 0;
        if (mg && i > 0 && r < C.first_len) {
            k += ps - mi + i * (C.nseg - 1);
            start += pb[b] + i * C.size - C.last_len;
            return;
        }
        k += ps - mi + i * (mg ? C.nseg - 1 : C.nseg);
        start += pb[b] + i * C.size;
        P = r;
        node = child;
    }
}

// Index list search of decode_seg: the entry of LIST node N that holds
// segment k of one copy of N (the largest b with segment prefix <= k).
DTE_HD int64_t list_entry_of_seg(const DNode *nodes, const char *blob, const DNode &N, int node, int64_t k,
                                 Hint &h)
{
    if (N.flags & NF_PSEGS) return find_le(arr<int64_t>(blob, N.a_psegs), N.count, k, h, node);
    const DNode &C0 = nodes[N.child];
    return find_le(arr<int64_t>(blob, N.a_pbytes), N.count, fdiv(k, C0.div_nseg) * C0.size, h, node);
}

// ---------------------------------------------------------------------------
// Merged segment index -> (displacement, length, packed offset where the
// segment starts).  0 <= k < nseg.
// ---------------------------------------------------------------------------
DTE_HD void decode_seg(const DNode *nodes, const char *blob, int node, int64_t k,
                       int64_t &disp, int64_t &len, int64_t &pstart, Hint &h)
{
    int64_t ext = 0;
    pstart = 0;
    for (;;) {
        const DNode &N = nodes[node];
        disp += N.base;
        if (N.kind == NK_RUN) {
            len = N.len + ext;
            return;
        }
        if (N.kind == NK_REG) {
            const DNode &C = nodes[N.child];
            int64_t i, j;
            if (N.flags & NF_MERGE) {
                if (k == 0) {
                    i = 0;
                    j = 0;
                } else {
                    i = fdiv(k - 1, C.div_nsegm1);
                    j = k - 1 - i * (C.nseg - 1) + 1;
                }
                if (j == C.nseg - 1 && i < N.count - 1) ext += C.first_len;
            } else {
                i = fdiv(k, C.div_nseg);
                j = k - i * C.nseg;
            }
            disp += i * N.stride;
            pstart += i * C.size;
            k = j;
            node = N.child;
            continue;
        }
        const int64_t *pb = arr<int64_t>(blob, N.a_pbytes);
        int64_t b;
        if (N.flags & NF_RUNS) {
            b = k;
            disp += arr<int64_t>(blob, N.a_disp)[b];
            pstart += pb[b];
            len = (pb[b + 1] - pb[b]) + ext;
            return;
        }
        b = list_entry_of_seg(nodes, blob, N, node, k, h);
        int child;
        int64_t stride;
        uint8_t ef = N.a_eflags ? arr<uint8_t>(blob, N.a_eflags)[b] : 0;
        if (N.flags & NF_SHARED) {
            child = N.child;
            stride = N.stride;
            if (N.flags & NF_EMERGE) ef |= EF_MERGE;
        } else {
            child = arr<int32_t>(blob, N.a_child)[b];
            stride = arr<int64_t>(blob, N.a_stride)[b];
        }
        const DNode &C = nodes[child];
        int64_t ps = list_psegs(N, C, blob, b, pb);
        int64_t local = k - ps + ((ef & EF_MERGED_IN) ? 1 : 0);
        int64_t cnt = fdiv(pb[b + 1] - pb[b], C.div_size);
        disp += arr<int64_t>(blob, N.a_disp)[b];
        pstart += pb[b];
        if (ef & EF_SINGLE) {
            if (N.a_tail) ext += arr<int64_t>(blob, N.a_tail)[b];
            disp += C.base;
            len = cnt * C.size + ext;
            return;
        }
        bool mg = (ef & EF_MERGE) != 0;
        int64_t enseg = mg ? cnt * (C.nseg - 1) + 1 : cnt * C.nseg;
        if (local == enseg - 1 && N.a_tail) ext += arr<int64_t>(blob, N.a_tail)[b];
        int64_t i, j;
        if (mg) {
            if (local == 0) {
                i = 0;
                j = 0;
            } else {
                i = fdiv(local - 1, C.div_nsegm1);
                j = local - 1 - i * (C.nseg - 1) + 1;
            }
            if (j == C.nseg - 1 && i < cnt - 1) ext += C.first_len;
        } else {
            i = fdiv(local, C.div_nseg);
            j = local - i * C.nseg;
        }
        disp += i * stride;
        pstart += i * C.size;
        k = j;
        node = child;
    }
}

DTE_HD void decode_seg(const DNode *nodes, const char *blob, int node, int64_t k,
                       int64_t &disp, int64_t &len, Hint &h)
{
    int64_t pstart;
    decode_seg(nodes, blob, node, k, disp, len, pstart, h);
}

}  // namespace dte
