// typesys.cpp -- type constructors, the commit-time compiler and the host
// segment queries of the GB300 datatype engine.
//
// Paper anchors (arxiv 2402.12274): §3 (a derived datatype describes a
// layout; O(1) description instead of an O(Ny*Nz) segment list), §3.1
// (MPIX_Type_iov_len, MPIX_Type_iov, MPIX_Iov), §3.2 (contiguous + subarray
// example).  Constructors follow the MPI typemap definitions; the layout
// tree they build is normalised on the fly (see desc.h) so that commit only
// has to flatten it into a relocatable blob.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <unordered_map>
#include <unordered_set>

#include "internal.h"

namespace dte {

// ------------------------------------------------------------------------
// checked int64 arithmetic
// ------------------------------------------------------------------------
static int64_t add_ck(int64_t a, int64_t b)
{
    int64_t r;
    if (__builtin_add_overflow(a, b, &r)) throw Error(DTE_ERR_OVERFLOW, "int64 overflow");
    return r;
}
static int64_t sub_ck(int64_t a, int64_t b)
{
    int64_t r;
    if (__builtin_sub_overflow(a, b, &r)) throw Error(DTE_ERR_OVERFLOW, "int64 overflow");
    return r;
}
static int64_t mul_ck(int64_t a, int64_t b)
{
    int64_t r;
    if (__builtin_mul_overflow(a, b, &r)) throw Error(DTE_ERR_OVERFLOW, "int64 overflow");
    return r;
}
static int64_t abs_ck(int64_t a)
{
    if (a == INT64_MIN) throw Error(DTE_ERR_OVERFLOW, "int64 overflow");
    return a < 0 ? -a : a;
}

// largest power of two <= 16 dividing v (16 for v == 0)
static int64_t p2(int64_t v)
{
    if (v == 0) return 16;
    uint64_t u = (uint64_t)v;
    uint64_t low = u & (~u + 1);
    return low >= 16 ? 16 : (int64_t)low;
}

// ------------------------------------------------------------------------
// normal-form builders
// ------------------------------------------------------------------------
NP make_empty()
{
    static const NP e = std::make_shared<Node>();
    return e;
}

NP make_run(int64_t len, int64_t base)
{
    if (len == 0) return make_empty();
    auto n = std::make_shared<Node>();
    n->kind = NK_RUN;
    n->len = len;
    n->base = base;
    n->size = len;
    n->nseg = 1;
    n->first_d = n->last_d = base;
    n->first_len = n->last_len = len;
    n->tlo = base;
    n->thi = add_ck(base, len);
    n->align = std::min(p2(len), p2(base));
    n->maxrun = len;
    n->nonoverlap = true;
    return n;
}

NP shift(const NP &n, int64_t d)
{
    if (d == 0 || n->empty()) return n;
    auto m = std::make_shared<Node>(*n);
    m->base = add_ck(m->base, d);
    m->first_d = add_ck(m->first_d, d);
    m->last_d = add_ck(m->last_d, d);
    m->tlo = add_ck(m->tlo, d);
    m->thi = add_ck(m->thi, d);
    m->align = std::min(m->align, p2(d));
    return m;
}

NP make_reg(int64_t count, int64_t stride, const NP &child)
{
    if (count == 0 || child->empty()) return make_empty();
    if (count == 1) return child;
    const Node &C = *child;
    if (C.nseg == 1 && stride == C.len) return make_run(mul_ck(count, C.len), C.base);
    if (C.kind == NK_REG && C.count > 0) {
        int64_t outer;
        if (!__builtin_mul_overflow(C.count, C.stride, &outer) && outer == stride)
            return shift(make_reg(mul_ck(count, C.count), C.stride, C.child), C.base);
    }
    auto n = std::make_shared<Node>();
    n->kind = NK_REG;
    n->count = count;
    n->stride = stride;
    n->child = child;
    n->size = mul_ck(count, C.size);
    int64_t m = C.nseg;
    int64_t span = mul_ck(count - 1, stride);
    n->merge = m >= 2 && add_ck(C.last_d, C.last_len) == add_ck(stride, C.first_d);
    n->nseg = n->merge ? add_ck(mul_ck(count, m - 1), 1) : mul_ck(count, m);
    n->first_d = C.first_d;
    n->first_len = C.first_len;
    n->last_d = add_ck(span, C.last_d);
    n->last_len = C.last_len;
    n->tlo = add_ck(std::min<int64_t>(0, span), C.tlo);
    n->thi = add_ck(std::max<int64_t>(0, span), C.thi);
    n->align = std::min(C.align, p2(stride));
    n->maxrun = C.maxrun;
    n->nonoverlap = C.nonoverlap && abs_ck(stride) >= sub_ck(C.thi, C.tlo);
    return n;
}

namespace {
struct EA {  // attributes of one LIST entry = cnt copies of kid at stride, at disp
    int64_t size, nseg, first_d, first_len, last_d, last_len, tlo, thi;
    bool merge, single, fold;
};

EA entry_attrs(const Entry &e)
{
    const Node &K = *e.kid;
    EA a{};
    int64_t c = e.cnt, s = e.stride;
    if (K.nseg == 1 && (c == 1 || s == K.len)) {
        a.single = true;
        a.fold = c >= 2;
        a.size = mul_ck(c, K.len);
        a.nseg = 1;
        a.first_d = a.last_d = add_ck(e.disp, K.base);
        a.first_len = a.last_len = a.size;
        a.tlo = a.first_d;
        a.thi = add_ck(a.tlo, a.size);
        return a;
    }
    int64_t m = K.nseg;
    int64_t span = mul_ck(c - 1, s);
    a.merge = m >= 2 && add_ck(K.last_d, K.last_len) == add_ck(s, K.first_d);
    a.size = mul_ck(c, K.size);
    a.nseg = a.merge ? add_ck(mul_ck(c, m - 1), 1) : mul_ck(c, m);
    a.first_d = add_ck(e.disp, K.first_d);
    a.first_len = K.first_len;
    a.last_d = add_ck(add_ck(e.disp, span), K.last_d);
    a.last_len = K.last_len;
    a.tlo = add_ck(add_ck(e.disp, std::min<int64_t>(0, span)), K.tlo);
    a.thi = add_ck(add_ck(e.disp, std::max<int64_t>(0, span)), K.thi);
    return a;
}

// true if the half-open spans [lo[i], hi[i]) are pairwise disjoint
bool spans_disjoint(std::vector<std::pair<int64_t, int64_t>> &sp)
{
    bool sorted = true;
    for (size_t i = 1; i < sp.size(); i++)
        if (sp[i].first < sp[i - 1].first) { sorted = false; break; }
    if (!sorted) std::sort(sp.begin(), sp.end());
    int64_t end = INT64_MIN;
    for (auto &p : sp) {
        if (p.first < end) return false;
        end = std::max(end, p.second);
    }
    return true;
}
}  // namespace

NP make_list(std::vector<Entry> &&in)
{
    std::vector<Entry> ent;
    ent.reserve(in.size());
    for (auto &e : in)
        if (e.cnt > 0 && !e.kid->empty()) ent.push_back(e);
    in.clear();
    in.shrink_to_fit();
    size_t n = ent.size();
    if (n == 0) return make_empty();
    if (n == 1) return shift(make_reg(ent[0].cnt, ent[0].stride, ent[0].kid), ent[0].disp);

    std::vector<EA> ea(n);
    bool all_single = true;
    for (size_t b = 0; b < n; b++) {
        ea[b] = entry_attrs(ent[b]);
        all_single = all_single && ea[b].single;
    }

    if (all_single) {
        // run table; coalesce runs that abut in order
        std::vector<int64_t> st, ln;
        st.reserve(n);
        ln.reserve(n);
        for (size_t b = 0; b < n; b++) {
            if (!st.empty() && st.back() + ln.back() == ea[b].first_d) ln.back() = add_ck(ln.back(), ea[b].size);
            else { st.push_back(ea[b].first_d); ln.push_back(ea[b].size); }
        }
        ea.clear();
        ent.clear();
        size_t r = st.size();
        if (r == 1) return make_run(ln[0], st[0]);
        bool regular = true;
        int64_t step = st[1] - st[0];
        for (size_t b = 1; b < r && regular; b++)
            regular = ln[b] == ln[0] && st[b] - st[b - 1] == step;
        if (regular) return shift(make_reg((int64_t)r, step, make_run(ln[0], 0)), st[0]);
        auto L = std::make_shared<ListData>();
        auto nd = std::make_shared<Node>();
        nd->kind = NK_LIST;
        nd->runs = true;
        nd->count = (int64_t)r;
        L->pbytes.resize(r + 1);
        L->pbytes[0] = 0;
        int64_t lo = st[0], hi = st[0] + ln[0], al = 16;
        std::vector<std::pair<int64_t, int64_t>> sp(r);
        for (size_t b = 0; b < r; b++) {
            L->pbytes[b + 1] = add_ck(L->pbytes[b], ln[b]);
            lo = std::min(lo, st[b]);
            hi = std::max(hi, add_ck(st[b], ln[b]));
            al = std::min(al, std::min(p2(st[b]), p2(ln[b])));
            nd->maxrun = std::max(nd->maxrun, ln[b]);
            sp[b] = {st[b], st[b] + ln[b]};
        }
        nd->size = L->pbytes[r];
        nd->nseg = (int64_t)r;
        nd->first_d = st[0];
        nd->first_len = ln[0];
        nd->last_d = st[r - 1];
        nd->last_len = ln[r - 1];
        nd->tlo = lo;
        nd->thi = hi;
        nd->align = al;
        nd->nonoverlap = spans_disjoint(sp);
        L->disp = std::move(st);
        nd->L = L;
        return nd;
    }

    // general entry list
    bool shared = true, same_cnt = true;
    for (size_t b = 1; b < n; b++) {
        shared = shared && ent[b].kid == ent[0].kid && ent[b].stride == ent[0].stride;
        same_cnt = same_cnt && ent[b].cnt == ent[0].cnt;
    }
    if (shared && same_cnt) {  // indexed with regular displacements: a vector
        int64_t step = ent[1].disp - ent[0].disp;
        bool regular = true;
        for (size_t b = 2; b < n && regular; b++) regular = ent[b].disp - ent[b - 1].disp == step;
        if (regular)
            return shift(make_reg((int64_t)n, step, make_reg(ent[0].cnt, ent[0].stride, ent[0].kid)),
                         ent[0].disp);
    }

    auto L = std::make_shared<ListData>();
    auto nd = std::make_shared<Node>();
    nd->kind = NK_LIST;
    nd->count = (int64_t)n;
    nd->shared = shared;
    std::vector<uint8_t> mi(n, 0);
    bool xmerge = false;
    for (size_t b = 0; b + 1 < n; b++) {
        if (add_ck(ea[b].last_d, ea[b].last_len) == ea[b + 1].first_d) {
            mi[b + 1] = 1;
            xmerge = true;
        }
    }
    nd->xmerge = xmerge;
    if (shared) nd->emerge = ea[0].merge;

    L->pbytes.resize(n + 1);
    std::vector<int64_t> psegs(n + 1);
    L->pbytes[0] = 0;
    psegs[0] = 0;
    std::vector<uint8_t> ef(n, 0);
    bool any_ef = false, any_fold = false;
    for (size_t b = 0; b < n; b++) {
        L->pbytes[b + 1] = add_ck(L->pbytes[b], ea[b].size);
        psegs[b + 1] = add_ck(psegs[b], ea[b].nseg - mi[b]);
        uint8_t f = 0;
        if (!shared && ea[b].merge) f |= EF_MERGE;
        if (mi[b]) f |= EF_MERGED_IN;
        if (ea[b].fold) { f |= EF_SINGLE; any_fold = true; }
        ef[b] = f;
        any_ef = any_ef || f;
    }
    if (xmerge) {
        L->tail.assign(n, 0);
        L->head.assign(n, 0);
        for (size_t b = n - 1; b-- > 0;) {
            if (mi[b + 1])
                L->tail[b] = add_ck(ea[b + 1].first_len, ea[b + 1].nseg == 1 ? L->tail[b + 1] : 0);
        }
        for (size_t b = 1; b < n; b++) {
            if (mi[b])
                L->head[b] = add_ck(ea[b - 1].last_len,
                                    (ea[b - 1].nseg == 1 && mi[b - 1]) ? L->head[b - 1] : 0);
        }
    }
    if (any_ef) L->eflags = ef;
    bool derive = shared && !nd->emerge && !xmerge && !any_fold;
    if (!derive) L->psegs = psegs;

    nd->size = L->pbytes[n];
    nd->nseg = psegs[n];
    nd->first_d = ea[0].first_d;
    nd->first_len = add_ck(ea[0].first_len, (ea[0].nseg == 1 && xmerge) ? L->tail[0] : 0);
    if (mi[n - 1] && ea[n - 1].nseg == 1) {
        nd->last_d = sub_ck(ea[n - 1].first_d, L->head[n - 1]);
        nd->last_len = add_ck(L->head[n - 1], ea[n - 1].size);
    } else {
        nd->last_d = ea[n - 1].last_d;
        nd->last_len = ea[n - 1].last_len;
    }
    int64_t lo = ea[0].tlo, hi = ea[0].thi, al = 16;
    bool nov = true;
    std::vector<std::pair<int64_t, int64_t>> sp(n);
    L->disp.resize(n);
    if (shared) {
        L->kids.push_back(ent[0].kid);
        L->strides.push_back(ent[0].stride);
        al = std::min(ent[0].kid->align, p2(ent[0].stride));
    } else {
        L->kids.resize(n);
        L->strides.resize(n);
    }
    L->cnt.resize(n);
    for (size_t b = 0; b < n; b++) {
        const Entry &e = ent[b];
        L->disp[b] = e.disp;
        L->cnt[b] = e.cnt;
        if (!shared) {
            L->kids[b] = e.kid;
            L->strides[b] = e.stride;
            al = std::min(al, std::min(e.kid->align, p2(e.stride)));
        }
        al = std::min(al, p2(e.disp));
        lo = std::min(lo, ea[b].tlo);
        hi = std::max(hi, ea[b].thi);
        const Node &K = *e.kid;
        nov = nov && K.nonoverlap &&
              (e.cnt == 1 || abs_ck(e.stride) >= sub_ck(K.thi, K.tlo) || ea[b].single);
        nd->maxrun = std::max(nd->maxrun, ea[b].single ? ea[b].size : K.maxrun);
        sp[b] = {ea[b].tlo, ea[b].thi};
    }
    nd->tlo = lo;
    nd->thi = hi;
    nd->align = al;
    nd->nonoverlap = nov && spans_disjoint(sp);
    nd->L = L;
    return nd;
}

// ------------------------------------------------------------------------
// commit: flatten into a blob
// ------------------------------------------------------------------------
FastDiv make_div(int64_t d)
{
    FastDiv f{0, 0, 0};
    if (d <= 1) return f;
    int l = 64 - __builtin_clzll((unsigned long long)(d - 1));  // ceil(log2 d)
    unsigned __int128 num = ((unsigned __int128)1) << (63 + l);
    unsigned __int128 m = (num + (unsigned __int128)(d - 1)) / (unsigned __int128)d;
    f.m = (uint64_t)m;
    f.s = (uint32_t)(l - 1);
    f.mode = 1;
    return f;
}

Committed::~Committed()
{
    bool captured = false;
    for (auto &d : dev) captured = captured || d.captured;
    int cur = -1;
    if (!dev.empty()) cudaGetDevice(&cur);
    for (auto &d : dev) {
        if (!d.ptr || d.captured) continue;
        cudaSetDevice(d.device);
        for (auto &u : d.uses) {
            cudaEventSynchronize((cudaEvent_t)u.second);
            cudaEventDestroy((cudaEvent_t)u.second);
        }
        cudaFree(d.ptr);
    }
    // adjoint inverses are used by the same enqueued work as the descriptor
    if (!captured) {
        for (auto &a : adj) {
            if (!a.dmem) continue;
            cudaSetDevice(a.device);
            cudaFree(a.dmem);
        }
    }
    if (cur >= 0) cudaSetDevice(cur);
}

std::shared_ptr<Committed> commit_node(const NP &root)
{
    std::unordered_map<const Node *, int> idx;
    std::vector<const Node *> order;
    std::vector<const Node *> stack{root.get()};
    // depth-first numbering; root is node 0
    while (!stack.empty()) {
        const Node *n = stack.back();
        stack.pop_back();
        if (idx.count(n)) continue;
        idx[n] = (int)order.size();
        order.push_back(n);
        if (n->kind == NK_REG) stack.push_back(n->child.get());
        if (n->kind == NK_LIST && !n->runs)
            for (auto &k : n->L->kids) stack.push_back(k.get());
    }
    if (order.size() > (1u << 30)) throw Error(DTE_ERR_UNSUPPORTED, "too many nodes");
    auto up16 = [](int64_t x) { return (x + 15) & ~(int64_t)15; };
    int64_t off = up16((int64_t)sizeof(BlobHeader) + (int64_t)order.size() * (int64_t)sizeof(DNode));
    struct Arrays { int64_t disp, pbytes, psegs, child, stride, eflags, tail, head; };
    std::vector<Arrays> A(order.size(), Arrays{0, 0, 0, 0, 0, 0, 0, 0});
    for (size_t i = 0; i < order.size(); i++) {
        const Node *n = order[i];
        if (n->kind != NK_LIST) continue;
        const ListData &L = *n->L;
        int64_t c = n->count;
        auto take = [&](int64_t bytes) { int64_t o = off; off = up16(off + bytes); return o; };
        A[i].disp = take(8 * c);
        A[i].pbytes = take(8 * (c + 1));
        if (!L.psegs.empty()) A[i].psegs = take(8 * (c + 1));
        if (!n->runs && !n->shared) {
            A[i].child = take(4 * c);
            A[i].stride = take(8 * c);
        }
        if (!L.eflags.empty()) A[i].eflags = take(c);
        if (!L.tail.empty()) {
            A[i].tail = take(8 * c);
            A[i].head = take(8 * c);
        }
    }
    auto C = std::make_shared<Committed>();
    C->storage.assign((size_t)(off / 8), 0);
    C->bytes = off;
    C->root = 0;
    C->nnodes = (int)order.size();
    char *blob = reinterpret_cast<char *>(C->storage.data());
    BlobHeader h{};
    h.root = 0;
    h.nnodes = C->nnodes;
    h.bytes = off;
    std::memcpy(blob, &h, sizeof h);
    DNode *dn = reinterpret_cast<DNode *>(blob + sizeof(BlobHeader));
    for (size_t i = 0; i < order.size(); i++) {
        const Node *n = order[i];
        if (n->kind == NK_LIST && n->count > 32) C->big_list = true;
        DNode d;
        std::memset(&d, 0, sizeof d);
        d.kind = n->kind;
        d.child = -1;
        d.base = n->base;
        d.size = n->size;
        d.nseg = n->nseg;
        d.first_len = n->first_len;
        d.last_len = n->last_len;
        d.div_size = make_div(n->size);
        d.div_nseg = make_div(n->nseg);
        d.div_nsegm1 = make_div(n->nseg - 1);
        if (n->kind == NK_RUN) {
            d.len = n->len;
        } else if (n->kind == NK_REG) {
            d.count = n->count;
            d.stride = n->stride;
            d.child = idx.at(n->child.get());
            if (n->merge) d.flags |= NF_MERGE;
        } else {
            const ListData &L = *n->L;
            d.count = n->count;
            if (n->runs) d.flags |= NF_RUNS;
            if (n->shared) {
                d.flags |= NF_SHARED;
                d.child = idx.at(L.kids[0].get());
                d.stride = L.strides[0];
                if (n->emerge) d.flags |= NF_EMERGE;
            }
            if (n->xmerge) d.flags |= NF_XMERGE;
            if (!L.psegs.empty()) d.flags |= NF_PSEGS;
            d.a_disp = A[i].disp;
            d.a_pbytes = A[i].pbytes;
            d.a_psegs = A[i].psegs;
            d.a_child = A[i].child;
            d.a_stride = A[i].stride;
            d.a_eflags = A[i].eflags;
            d.a_tail = A[i].tail;
            d.a_head = A[i].head;
            int64_t c = n->count;
            std::memcpy(blob + d.a_disp, L.disp.data(), 8 * c);
            std::memcpy(blob + d.a_pbytes, L.pbytes.data(), 8 * (c + 1));
            if (d.a_psegs) std::memcpy(blob + d.a_psegs, L.psegs.data(), 8 * (c + 1));
            if (d.a_child) {
                int32_t *ch = reinterpret_cast<int32_t *>(blob + d.a_child);
                for (int64_t b = 0; b < c; b++) ch[b] = idx.at(L.kids[b].get());
                std::memcpy(blob + d.a_stride, L.strides.data(), 8 * c);
            }
            if (d.a_eflags) std::memcpy(blob + d.a_eflags, L.eflags.data(), c);
            if (d.a_tail) {
                std::memcpy(blob + d.a_tail, L.tail.data(), 8 * c);
                std::memcpy(blob + d.a_head, L.head.data(), 8 * c);
            }
        }
        dn[i] = d;
    }
    C->align = root->align;
    C->maxrun = root->maxrun;
    C->nseg = root->nseg;
    C->size = root->size;
    C->nonoverlap = root->nonoverlap;
    C->tlo = root->tlo;
    C->thi = root->thi;
    return C;
}

// Exact overlap test over `count` elements: enumerate every segment and sort.
bool committed_overlaps(Committed &c, int64_t count, int64_t extent)
{
    if (c.size == 0 || count == 0) return false;
    bool elem_disjoint = count == 1 || (extent > 0 && extent >= c.thi - c.tlo) ||
                         (extent < 0 && -extent >= c.thi - c.tlo);
    if (c.nonoverlap && elem_disjoint) return false;
    std::lock_guard<std::mutex> g(c.mu);
    if (c.overlap_exact == 1) return true;
    std::vector<std::pair<int64_t, int64_t>> sp;
    int64_t per = c.nseg;
    int64_t total = mul_ck(per, elem_disjoint ? 1 : count);
    if (total > (int64_t)1 << 31) throw Error(DTE_ERR_UNSUPPORTED, "overlap check too large");
    sp.reserve((size_t)total);
    Hint h{-1, 0};
    const DNode *nd = c.nodes();
    int64_t elems = elem_disjoint ? 1 : count;
    for (int64_t e = 0; e < elems; e++) {
        for (int64_t k = 0; k < per; k++) {
            int64_t d = 0, l = 0;
            decode_seg(nd, c.blob(), c.root, k, d, l, h);
            d += e * extent;
            sp.push_back({d, d + l});
        }
    }
    std::sort(sp.begin(), sp.end());
    int64_t end = INT64_MIN;
    bool hit = false;
    for (auto &p : sp) {
        if (p.first < end) { hit = true; break; }
        end = std::max(end, p.second);
    }
    if (elems == 1) c.overlap_exact = hit ? 1 : 0;
    return hit;
}

// ------------------------------------------------------------------------
// handle registry and deferred device frees
// ------------------------------------------------------------------------
static std::mutex g_mu;
static std::unordered_set<dte_type> *g_live = new std::unordered_set<dte_type>();
static std::vector<std::shared_ptr<Committed>> *g_deferred =
    new std::vector<std::shared_ptr<Committed>>();

bool handle_valid(dte_type t)
{
    if (!t) return false;
    std::lock_guard<std::mutex> g(g_mu);
    return g_live->count(t) != 0;
}

static void register_handle(dte_type t)
{
    std::lock_guard<std::mutex> g(g_mu);
    g_live->insert(t);
}

static bool all_done(Committed &c)
{
    for (auto &d : c.dev) {
        if (d.captured) return false;
        for (auto &u : d.uses)
            if (cudaEventQuery((cudaEvent_t)u.second) == cudaErrorNotReady) return false;
    }
    return true;
}

void reap_deferred()
{
    std::vector<std::shared_ptr<Committed>> done;
    {
        std::lock_guard<std::mutex> g(g_mu);
        auto &v = *g_deferred;
        for (size_t i = 0; i < v.size();) {
            bool ok;
            {
                std::lock_guard<std::mutex> g2(v[i]->mu);
                ok = all_done(*v[i]);
            }
            if (ok) {
                done.push_back(v[i]);
                v[i] = v.back();
                v.pop_back();
            } else {
                i++;
            }
        }
    }
    done.clear();  // destructors free the device copies outside the lock
}

static void release_desc(std::shared_ptr<Committed> &&d)
{
    if (!d) return;
    if (d.use_count() > 1) return;  // another handle (dup) still owns it
    bool pending = false;
    {
        std::lock_guard<std::mutex> g(d->mu);
        pending = !all_done(*d);
    }
    if (pending) {
        std::lock_guard<std::mutex> g(g_mu);
        g_deferred->push_back(std::move(d));
    }
}

static int have_device()
{
    static int cached = -1;
    if (cached < 0) {
        int n = 0;
        cached = (cudaGetDeviceCount(&n) == cudaSuccess && n > 0) ? 1 : 0;
        if (!cached) cudaGetLastError();
    }
    return cached;
}

int device_blob(dte_type t, const char **out, int *device)
{
    if (!have_device()) return DTE_ERR_NODEVICE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DTE_ERR_CUDA;
    Committed &c = *t->desc;
    std::lock_guard<std::mutex> g(c.mu);
    for (auto &d : c.dev) {
        if (d.device == dev) {
            *out = d.ptr;
            *device = dev;
            return DTE_SUCCESS;
        }
    }
    char *p = nullptr;
    if (cudaMalloc(&p, (size_t)c.bytes) != cudaSuccess) {
        cudaGetLastError();
        return DTE_ERR_NOMEM;
    }
    if (cudaMemcpy(p, c.blob(), (size_t)c.bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(p);
        return DTE_ERR_CUDA;
    }
    DevCopy dc;
    dc.device = dev;
    dc.ptr = p;
    c.dev.push_back(dc);
    *out = p;
    *device = dev;
    return DTE_SUCCESS;
}

int device_blob_resident(dte_type t, int dev, const char **out)
{
    Committed &c = *t->desc;
    std::lock_guard<std::mutex> g(c.mu);
    for (auto &d : c.dev) {
        if (d.device == dev) {
            *out = d.ptr;
            return DTE_SUCCESS;
        }
    }
    return DTE_ERR_TYPE;
}

void note_use(dte_type t, int device, void *stream)
{
    Committed &c = *t->desc;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing((cudaStream_t)stream, &cs);
    std::lock_guard<std::mutex> g(c.mu);
    for (auto &d : c.dev) {
        if (d.device != device) continue;
        if (cs != cudaStreamCaptureStatusNone) {
            d.captured = true;
            return;
        }
        for (auto &u : d.uses) {
            if (u.first == stream) {
                cudaEventRecord((cudaEvent_t)u.second, (cudaStream_t)stream);
                return;
            }
        }
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return;
        cudaEventRecord(ev, (cudaStream_t)stream);
        d.uses.push_back({stream, (void *)ev});
        return;
    }
}

}  // namespace dte

// ==========================================================================
// C ABI: constructors, commit/free, attributes, host segment queries
// ==========================================================================
using namespace dte;

#define DTE_TRY try {
#define DTE_CATCH                                              \
    }                                                          \
    catch (const Error &e) { return e.code; }                  \
    catch (const std::bad_alloc &) { return DTE_ERR_NOMEM; }   \
    catch (...) { return DTE_ERR_ARG; }

namespace {

struct Acc {  // lb/ub accumulation over copies (see the MPI typemap rules)
    bool any = false, lbx = false, ubx = false;
    int64_t lb_all = 0, ub_all = 0, lb_x = 0, ub_x = 0, align = 1;

    // copies of `c` at every displacement in [dmin, dmax] that a linear family reaches
    void add(int64_t dmin, int64_t dmax, const dte_type_s *c)
    {
        if (!c->nonempty && !c->lb_x && !c->ub_x) return;
        int64_t lo = add_ck(dmin, c->lb), hi = add_ck(dmax, c->ub);
        if (!any || lo < lb_all) lb_all = lo;
        if (!any || hi > ub_all) ub_all = hi;
        any = true;
        if (c->lb_x) { if (!lbx || lo < lb_x) lb_x = lo; lbx = true; }
        if (c->ub_x) { if (!ubx || hi > ub_x) ub_x = hi; ubx = true; }
        align = std::max(align, c->align);
    }
    // family d0 + j*step for j in [0, n)
    void add_family(int64_t d0, int64_t n, int64_t step, const dte_type_s *c)
    {
        if (n <= 0) return;
        int64_t last = add_ck(d0, mul_ck(n - 1, step));
        add(std::min(d0, last), std::max(d0, last), c);
    }
};

dte_type new_type(const Acc &a, NP node, bool is_struct)
{
    auto *t = new dte_type_s();
    t->node = std::move(node);
    t->size = t->node->size;
    t->nonempty = t->size > 0;
    t->true_lb = t->nonempty ? t->node->tlo : 0;
    t->true_ub = t->nonempty ? t->node->thi : 0;
    t->lb = a.lbx ? a.lb_x : (a.any ? a.lb_all : 0);
    t->ub = a.ubx ? a.ub_x : (a.any ? a.ub_all : 0);
    t->lb_x = a.lbx;
    t->ub_x = a.ubx;
    t->align = a.align;
    if (is_struct && !a.ubx && a.any) {
        int64_t ext = sub_ck(t->ub, t->lb);
        int64_t r = ext % t->align;
        if (r < 0) r += t->align;
        if (r) t->ub = add_ck(t->ub, t->align - r);
    }
    register_handle(t);
    return t;
}

// predefined types live for the whole process (never destroyed at exit)
dte_type_s *g_basic = nullptr;
std::once_flag g_basic_once;
const int64_t kBasicSize[DTE_NBASIC] = {1, 1, 1, 2, 2, 4, 4, 8, 8, 2, 2, 4, 8};

void init_basics()
{
    g_basic = new dte_type_s[DTE_NBASIC];
    for (int i = 0; i < DTE_NBASIC; i++) {
        dte_type_s &b = g_basic[i];
        b.predefined = true;
        b.size = kBasicSize[i];
        b.lb = 0;
        b.ub = b.size;
        b.true_lb = 0;
        b.true_ub = b.size;
        b.align = b.size;
        b.nonempty = true;
        b.node = make_run(b.size, 0);
        b.desc = commit_node(b.node);
        b.committed = true;
        register_handle(&b);
    }
}

int check_old(dte_type t)
{
    std::call_once(g_basic_once, init_basics);
    return handle_valid(t) ? DTE_SUCCESS : DTE_ERR_TYPE;
}

}  // namespace

extern "C" {

const char *dte_error_string(int code)
{
    switch (code) {
    case DTE_SUCCESS: return "success";
    case DTE_ERR_ARG: return "invalid argument";
    case DTE_ERR_TYPE: return "invalid or uncommitted datatype";
    case DTE_ERR_OVERFLOW: return "int64 overflow in a size or displacement";
    case DTE_ERR_TRUNCATE: return "buffer too small for the data";
    case DTE_ERR_OVERLAP: return "unpack target layout writes a byte twice";
    case DTE_ERR_NOMEM: return "out of memory";
    case DTE_ERR_CUDA: return "CUDA runtime error";
    case DTE_ERR_TIMEOUT: return "bounded device wait timed out";
    case DTE_ERR_UNSUPPORTED: return "implementation limit exceeded";
    case DTE_ERR_NODEVICE: return "no CUDA device";
    default: return "unknown error";
    }
}

int dte_type_basic(int which, dte_type *out)
{
    std::call_once(g_basic_once, init_basics);
    if (!out || which < 0 || which >= DTE_NBASIC) return DTE_ERR_ARG;
    *out = &g_basic[which];
    return DTE_SUCCESS;
}

int dte_type_contiguous(int64_t count, dte_type old, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || count < 0) return DTE_ERR_ARG;
    int64_t e = old->extent();
    Acc a;
    a.add_family(0, count, e, old);
    *out = new_type(a, make_reg(count, e, old->node), false);
    return DTE_SUCCESS;
    DTE_CATCH
}

static int vector_common(int64_t count, int64_t bl, int64_t stride_bytes, dte_type old, dte_type *out)
{
    int64_t e = old->extent();
    Acc a;
    if (count > 0 && bl > 0) {
        // copies at i*stride + j*e: extremes sit at the corners of (i, j)
        int64_t c1 = mul_ck(count - 1, stride_bytes), c2 = mul_ck(bl - 1, e);
        int64_t lo = std::min<int64_t>(0, c1) + std::min<int64_t>(0, c2);
        int64_t hi = add_ck(std::max<int64_t>(0, c1), std::max<int64_t>(0, c2));
        a.add(lo, hi, old);
    }
    *out = new_type(a, make_reg(count, stride_bytes, make_reg(bl, e, old->node)), false);
    return DTE_SUCCESS;
}

int dte_type_vector(int64_t count, int64_t bl, int64_t stride, dte_type old, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || count < 0 || bl < 0) return DTE_ERR_ARG;
    return vector_common(count, bl, mul_ck(stride, old->extent()), old, out);
    DTE_CATCH
}

int dte_type_hvector(int64_t count, int64_t bl, int64_t stride_bytes, dte_type old, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || count < 0 || bl < 0) return DTE_ERR_ARG;
    return vector_common(count, bl, stride_bytes, old, out);
    DTE_CATCH
}

static int indexed_common(int64_t count, const int64_t *bl, int64_t blconst, const int64_t *disp,
                          int64_t scale, dte_type old, dte_type *out)
{
    if (count > 0 && (!disp || (!bl && blconst < 0))) return DTE_ERR_ARG;
    int64_t e = old->extent();
    Acc a;
    std::vector<Entry> ent;
    ent.reserve((size_t)count);
    for (int64_t i = 0; i < count; i++) {
        int64_t b = bl ? bl[i] : blconst;
        if (b < 0) return DTE_ERR_ARG;
        int64_t d = mul_ck(disp[i], scale);
        a.add_family(d, b, e, old);
        ent.push_back(Entry{d, b, old->node, e});
    }
    *out = new_type(a, make_list(std::move(ent)), false);
    return DTE_SUCCESS;
}

int dte_type_indexed(int64_t count, const int64_t *bl, const int64_t *disp, dte_type old, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || count < 0 || (count > 0 && !bl)) return DTE_ERR_ARG;
    return indexed_common(count, bl, -1, disp, old->extent(), old, out);
    DTE_CATCH
}

int dte_type_hindexed(int64_t count, const int64_t *bl, const int64_t *disp_bytes, dte_type old,
                      dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || count < 0 || (count > 0 && !bl)) return DTE_ERR_ARG;
    return indexed_common(count, bl, -1, disp_bytes, 1, old, out);
    DTE_CATCH
}

int dte_type_indexed_block(int64_t count, int64_t bl, const int64_t *disp, dte_type old, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || count < 0 || bl < 0) return DTE_ERR_ARG;
    return indexed_common(count, nullptr, bl, disp, old->extent(), old, out);
    DTE_CATCH
}

int dte_type_hindexed_block(int64_t count, int64_t bl, const int64_t *disp_bytes, dte_type old,
                            dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || count < 0 || bl < 0) return DTE_ERR_ARG;
    return indexed_common(count, nullptr, bl, disp_bytes, 1, old, out);
    DTE_CATCH
}

int dte_type_struct(int64_t count, const int64_t *bl, const int64_t *disp_bytes, const dte_type *types,
                    dte_type *out)
{
    DTE_TRY
    std::call_once(g_basic_once, init_basics);
    if (!out || count < 0 || (count > 0 && (!bl || !disp_bytes || !types))) return DTE_ERR_ARG;
    Acc a;
    std::vector<Entry> ent;
    ent.reserve((size_t)count);
    for (int64_t i = 0; i < count; i++) {
        if (!handle_valid(types[i])) return DTE_ERR_TYPE;
        if (bl[i] < 0) return DTE_ERR_ARG;
        int64_t e = types[i]->extent();
        a.add_family(disp_bytes[i], bl[i], e, types[i]);
        ent.push_back(Entry{disp_bytes[i], bl[i], types[i]->node, e});
    }
    *out = new_type(a, make_list(std::move(ent)), true);
    return DTE_SUCCESS;
    DTE_CATCH
}

int dte_type_subarray(int ndims, const int64_t *sizes, const int64_t *subsizes, const int64_t *starts,
                      int order, dte_type old, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || ndims <= 0 || ndims > 32 || !sizes || !subsizes || !starts) return DTE_ERR_ARG;
    if (order != DTE_ORDER_C && order != DTE_ORDER_FORTRAN) return DTE_ERR_ARG;
    for (int d = 0; d < ndims; d++) {
        if (sizes[d] <= 0 || subsizes[d] < 0 || starts[d] < 0) return DTE_ERR_ARG;
        if (add_ck(starts[d], subsizes[d]) > sizes[d]) return DTE_ERR_ARG;
    }
    int64_t e = old->extent();
    // byte stride of each dimension (C: last dimension fastest)
    int64_t stride[32];
    int64_t full = 1;
    if (order == DTE_ORDER_C) {
        for (int d = ndims - 1; d >= 0; d--) { stride[d] = mul_ck(full, e); full = mul_ck(full, sizes[d]); }
    } else {
        for (int d = 0; d < ndims; d++) { stride[d] = mul_ck(full, e); full = mul_ck(full, sizes[d]); }
    }
    // nest from the fastest dimension outwards
    NP node = old->node;
    int64_t base = 0;
    for (int s = 0; s < ndims; s++) {
        int d = order == DTE_ORDER_C ? ndims - 1 - s : s;
        node = make_reg(subsizes[d], stride[d], node);
        base = add_ck(base, mul_ck(starts[d], stride[d]));
    }
    bool empty_sub = false;
    for (int d = 0; d < ndims; d++) empty_sub = empty_sub || subsizes[d] == 0;
    Acc a;
    if (!empty_sub && (old->nonempty || old->lb_x || old->ub_x)) a.align = old->align;
    a.lbx = a.ubx = true;
    a.lb_x = 0;
    a.ub_x = mul_ck(full, e);
    *out = new_type(a, shift(node, base), false);
    return DTE_SUCCESS;
    DTE_CATCH
}

int dte_type_darray(int size, int rank, int ndims, const int64_t *gsizes, const int *distribs, const int64_t *dargs,
                    const int64_t *psizes, int order, dte_type old, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out || ndims <= 0 || ndims > 32 || !gsizes || !distribs || !dargs || !psizes) return DTE_ERR_ARG;
    if (size <= 0 || rank < 0 || rank >= size) return DTE_ERR_ARG;
    if (order != DTE_ORDER_C && order != DTE_ORDER_FORTRAN) return DTE_ERR_ARG;
    int64_t nproc = 1;
    for (int d = 0; d < ndims; d++) {
        if (gsizes[d] <= 0 || psizes[d] <= 0) return DTE_ERR_ARG;
        nproc = mul_ck(nproc, psizes[d]);
    }
    if (nproc != size) return DTE_ERR_ARG;
    int64_t coord[32];
    int64_t r = rank;
    for (int d = ndims - 1; d >= 0; d--) {  // the process grid is row-major
        coord[d] = r % psizes[d];
        r /= psizes[d];
    }
    int64_t e = old->extent();
    int64_t stride[32];
    int64_t full = 1;
    if (order == DTE_ORDER_C) {
        for (int d = ndims - 1; d >= 0; d--) { stride[d] = mul_ck(full, e); full = mul_ck(full, gsizes[d]); }
    } else {
        for (int d = 0; d < ndims; d++) { stride[d] = mul_ck(full, e); full = mul_ck(full, gsizes[d]); }
    }
    // per dimension, the owned index blocks of this process; nest from the
    // fastest dimension outwards
    NP node = old->node;
    bool any = true;
    for (int s = 0; s < ndims; s++) {
        int d = order == DTE_ORDER_C ? ndims - 1 - s : s;
        int64_t g = gsizes[d], p = psizes[d], c = coord[d];
        std::vector<Entry> ent;
        if (distribs[d] == DTE_DISTRIBUTE_NONE) {
            if (p != 1) return DTE_ERR_ARG;
            ent.push_back(Entry{0, g, node, stride[d]});
        } else if (distribs[d] == DTE_DISTRIBUTE_BLOCK) {
            int64_t b = dargs[d] == DTE_DISTRIBUTE_DFLT_DARG ? (g + p - 1) / p : dargs[d];
            if (b <= 0 || mul_ck(b, p) < g) return DTE_ERR_ARG;
            int64_t lo = mul_ck(c, b), hi = std::min(add_ck(lo, b), g);
            if (lo < hi) ent.push_back(Entry{mul_ck(lo, stride[d]), hi - lo, node, stride[d]});
        } else if (distribs[d] == DTE_DISTRIBUTE_CYCLIC) {
            int64_t b = dargs[d] == DTE_DISTRIBUTE_DFLT_DARG ? 1 : dargs[d];
            if (b <= 0) return DTE_ERR_ARG;
            for (int64_t lo = mul_ck(c, b); lo < g; lo = add_ck(lo, mul_ck(p, b)))
                ent.push_back(Entry{mul_ck(lo, stride[d]), std::min(b, g - lo), node, stride[d]});
        } else {
            return DTE_ERR_ARG;
        }
        any = any && !ent.empty();
        node = make_list(std::move(ent));
    }
    Acc a;
    if (any && (old->nonempty || old->lb_x || old->ub_x)) a.align = old->align;
    a.lbx = a.ubx = true;
    a.lb_x = 0;
    a.ub_x = mul_ck(full, e);
    *out = new_type(a, node, false);
    return DTE_SUCCESS;
    DTE_CATCH
}

int dte_type_resized(dte_type old, int64_t lb, int64_t extent, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out) return DTE_ERR_ARG;
    Acc a;
    if (old->nonempty || old->lb_x || old->ub_x) a.align = old->align;
    a.lbx = a.ubx = true;
    a.lb_x = lb;
    a.ub_x = add_ck(lb, extent);
    *out = new_type(a, old->node, false);
    return DTE_SUCCESS;
    DTE_CATCH
}

int dte_type_dup(dte_type old, dte_type *out)
{
    DTE_TRY
    if (int rc = check_old(old)) return rc;
    if (!out) return DTE_ERR_ARG;
    auto *t = new dte_type_s();
    t->size = old->size;
    t->lb = old->lb;
    t->ub = old->ub;
    t->true_lb = old->true_lb;
    t->true_ub = old->true_ub;
    t->align = old->align;
    t->lb_x = old->lb_x;
    t->ub_x = old->ub_x;
    t->nonempty = old->nonempty;
    t->node = old->node;
    t->desc = old->desc;
    t->committed = old->committed;
    t->plan = old->plan;
    register_handle(t);
    *out = t;
    return DTE_SUCCESS;
    DTE_CATCH
}

}  // extern "C"

namespace dte {
// The kernel plan that DTE_PLAN (auto, chunk, chunk_wide, segment or bulk)
// gives every type at commit, or -1 when it is unset or names no plan; read
// once per process.
static int env_plan()
{
    static const int plan = [] {
        const char *v = std::getenv("DTE_PLAN");
        if (!v) return -1;
        static const char *const names[] = {"auto", "chunk", "chunk_wide", "segment", "bulk"};
        for (int i = 0; i < 5; i++)
            if (std::strcmp(v, names[i]) == 0) return i;
        return -1;
    }();
    return plan;
}
}  // namespace dte

extern "C" {

int dte_type_commit(dte_type *type)
{
    DTE_TRY
    if (!type) return DTE_ERR_ARG;
    if (int rc = check_old(*type)) return rc;
    dte_type t = *type;
    reap_deferred();
    if (t->committed) return DTE_SUCCESS;
    t->desc = commit_node(t->node);
    t->committed = true;
    if (t->plan == DTE_PLAN_AUTO && env_plan() > 0) t->plan = env_plan();
    if (have_device()) {
        const char *p;
        int dev;
        int rc = device_blob(t, &p, &dev);
        if (rc) return rc;
    }
    return DTE_SUCCESS;
    DTE_CATCH
}

int dte_type_free(dte_type *type)
{
    DTE_TRY
    if (!type) return DTE_ERR_ARG;
    if (int rc = check_old(*type)) return rc;
    dte_type t = *type;
    if (t->predefined) return DTE_ERR_TYPE;
    {
        std::lock_guard<std::mutex> g(g_mu);
        g_live->erase(t);
    }
    std::shared_ptr<Committed> d = std::move(t->desc);
    delete t;
    release_desc(std::move(d));
    reap_deferred();
    *type = nullptr;
    return DTE_SUCCESS;
    DTE_CATCH
}

int dte_type_size(dte_type t, int64_t *size)
{
    if (int rc = check_old(t)) return rc;
    if (!size) return DTE_ERR_ARG;
    *size = t->size;
    return DTE_SUCCESS;
}

int dte_type_get_extent(dte_type t, int64_t *lb, int64_t *extent)
{
    if (int rc = check_old(t)) return rc;
    if (!lb || !extent) return DTE_ERR_ARG;
    *lb = t->lb;
    *extent = t->ub - t->lb;
    return DTE_SUCCESS;
}

int dte_type_get_true_extent(dte_type t, int64_t *true_lb, int64_t *true_extent)
{
    if (int rc = check_old(t)) return rc;
    if (!true_lb || !true_extent) return DTE_ERR_ARG;
    *true_lb = t->true_lb;
    *true_extent = t->true_ub - t->true_lb;
    return DTE_SUCCESS;
}

int dte_type_num_segments(dte_type t, int64_t *nseg)
{
    if (int rc = check_old(t)) return rc;
    if (!nseg) return DTE_ERR_ARG;
    *nseg = t->node->nseg;
    return DTE_SUCCESS;
}

int dte_type_set_plan(dte_type t, int plan)
{
    if (int rc = check_old(t)) return rc;
    if (t->predefined) return DTE_ERR_TYPE;
    if (plan < DTE_PLAN_AUTO || plan > DTE_PLAN_BULK) return DTE_ERR_ARG;
    t->plan = plan;
    return DTE_SUCCESS;
}

int dte_type_get_plan(dte_type t, int *plan)
{
    if (int rc = check_old(t)) return rc;
    if (!plan) return DTE_ERR_ARG;
    *plan = t->plan;
    return DTE_SUCCESS;
}

int dte_type_descriptor_bytes(dte_type t, int64_t *bytes)
{
    if (int rc = check_old(t)) return rc;
    if (!bytes) return DTE_ERR_ARG;
    if (!t->committed) return DTE_ERR_TYPE;
    *bytes = t->desc->bytes;
    return DTE_SUCCESS;
}

int dte_type_iov_len(dte_type t, int64_t max_iov_bytes, int64_t *iov_len, int64_t *actual_iov_bytes)
{
    DTE_TRY
    if (int rc = check_old(t)) return rc;
    if (!t->committed) return DTE_ERR_TYPE;
    if (!iov_len || !actual_iov_bytes || max_iov_bytes < -1) return DTE_ERR_ARG;
    Committed &c = *t->desc;
    if (max_iov_bytes == -1 || max_iov_bytes >= c.size) {
        *iov_len = c.nseg;
        *actual_iov_bytes = c.size;
        return DTE_SUCCESS;
    }
    int64_t k = 0, start = 0;
    decode_pos(c.nodes(), c.blob(), c.root, max_iov_bytes, k, start);
    *iov_len = k;
    *actual_iov_bytes = start;
    return DTE_SUCCESS;
    DTE_CATCH
}

int dte_type_iov(dte_type t, int64_t iov_offset, dte_iov *iov, int64_t max_iov_len, int64_t *actual_iov_len)
{
    DTE_TRY
    if (int rc = check_old(t)) return rc;
    if (!t->committed) return DTE_ERR_TYPE;
    if (!actual_iov_len || iov_offset < 0 || max_iov_len < 0 || (max_iov_len > 0 && !iov))
        return DTE_ERR_ARG;
    Committed &c = *t->desc;
    int64_t end = iov_offset >= c.nseg ? iov_offset : std::min(c.nseg, iov_offset + std::min(max_iov_len, c.nseg));
    Hint h{-1, 0};
    for (int64_t k = iov_offset; k < end; k++) {
        int64_t d = 0, l = 0;
        decode_seg(c.nodes(), c.blob(), c.root, k, d, l, h);
        iov[k - iov_offset].iov_base = (void *)(intptr_t)d;
        iov[k - iov_offset].iov_len = l;
    }
    *actual_iov_len = end - iov_offset;
    return DTE_SUCCESS;
    DTE_CATCH
}

int dte_pack_size(int64_t incount, dte_type t, int64_t *size)
{
    DTE_TRY
    if (int rc = check_old(t)) return rc;
    if (!size || incount < 0) return DTE_ERR_ARG;
    *size = mul_ck(incount, t->size);
    return DTE_SUCCESS;
    DTE_CATCH
}

}  // extern "C"
