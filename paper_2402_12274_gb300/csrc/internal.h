// internal.h -- host-side objects shared by the type system and the kernels.
#pragma once

#include <atomic>
#include <cstdint>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <vector>

#include "../../include/dte.h"
#include "desc.h"

namespace dte {

// Internal error carrying a DTE_ERR_* code; caught at the C ABI.
struct Error : std::runtime_error {
    int code;
    Error(int c, const char *what) : std::runtime_error(what), code(c) {}
};

// ---------------------------------------------------------------------------
// Normal-form layout tree built by the constructors (immutable, shared).
// ---------------------------------------------------------------------------
struct Node;
using NP = std::shared_ptr<const Node>;

struct ListData {
    std::vector<int64_t> disp;     // entry displacement (RUNS: run start)
    std::vector<int64_t> cnt;      // copies of the child (RUNS: unused)
    std::vector<NP> kids;          // 1 entry when shared
    std::vector<int64_t> strides;  // 1 entry when shared
    std::vector<int64_t> pbytes;   // n+1 packed-byte prefix
    std::vector<int64_t> psegs;    // n+1 segment prefix (empty if derivable)
    std::vector<uint8_t> eflags;   // EF_* per entry (empty if all zero)
    std::vector<int64_t> tail, head;  // only when entries merge across
};

struct Node {
    int kind = NK_RUN;
    int64_t base = 0;
    int64_t size = 0, nseg = 0;
    int64_t first_d = 0, first_len = 0, last_d = 0, last_len = 0;  // incl. base
    int64_t tlo = 0, thi = 0;  // byte bounds of the data, incl. base
    int64_t align = 16;        // power of two <= 16 dividing every offset/length
    int64_t maxrun = 0;        // longest contiguous run a decode can return
    bool nonoverlap = true;    // proven: no byte appears twice
    // RUN
    int64_t len = 0;
    // REG
    int64_t count = 0, stride = 0;
    NP child;
    bool merge = false;
    // LIST
    bool runs = false, shared = false, xmerge = false, emerge = false;
    std::shared_ptr<const ListData> L;

    bool empty() const { return size == 0; }
};

NP make_empty();
NP make_run(int64_t len, int64_t base);
NP make_reg(int64_t count, int64_t stride, const NP &child);
NP shift(const NP &n, int64_t d);
struct Entry {
    int64_t disp;
    int64_t cnt;
    NP kid;
    int64_t stride;
};
NP make_list(std::vector<Entry> &&entries);

// ---------------------------------------------------------------------------
// Committed descriptor: a relocatable blob (header + DNode[] + arrays) kept on
// the host and uploaded once per device.
// ---------------------------------------------------------------------------
struct DevCopy {
    int device = -1;
    char *ptr = nullptr;
    // streams that used the copy, with an event recorded after the last use
    std::vector<std::pair<void *, void *>> uses;  // (cudaStream_t, cudaEvent_t)
    bool captured = false;  // used under stream capture: never freed
};

// Inverse of a float32 pack over `count` elements (for the adjoint of layouts
// that repeat entries): CSR by destination float, sources in packed order.
struct AdjointInverse {
    int device = -1;
    int64_t count = 0;
    int64_t ndest = 0;     // distinct destination floats
    int64_t nsrc = 0;      // packed floats
    char *dmem = nullptr;  // int64 rows[ndest+1], dest[ndest], cols[nsrc]
};

struct Committed {
    std::vector<AdjointInverse> adj;  // cached inverses (device memory)
    std::vector<int64_t> storage;  // 8-byte aligned host blob
    int root = 0;
    int nnodes = 0;
    int64_t bytes = 0;
    int64_t align = 16;            // type alignment class (<= 16)
    int64_t maxrun = 0;            // longest raw run of the descriptor
    bool big_list = false;         // a LIST level of more than 32 entries (searched, not divided)
    int64_t nseg = 0, size = 0;
    bool nonoverlap = true;        // structural proof for one element
    int overlap_exact = -1;        // -1 unknown, 0 no, 1 yes (one element)
    int64_t tlo = 0, thi = 0;
    std::mutex mu;
    std::vector<DevCopy> dev;

    const char *blob() const { return reinterpret_cast<const char *>(storage.data()); }
    const DNode *nodes() const
    {
        return reinterpret_cast<const DNode *>(blob() + sizeof(BlobHeader));
    }
    ~Committed();
};

std::shared_ptr<Committed> commit_node(const NP &root);
FastDiv make_div(int64_t d);
bool committed_overlaps(Committed &c, int64_t count, int64_t extent);

}  // namespace dte

struct dte_type_s {
    uint32_t magic = 0x44544531u;  // 'DTE1'
    std::atomic<int> refs{1};
    bool predefined = false;
    bool committed = false;
    int64_t size = 0, lb = 0, ub = 0, true_lb = 0, true_ub = 0;
    int64_t align = 1;             // natural alignment (max basic alignment)
    bool lb_x = false, ub_x = false, nonempty = false;
    int plan = 0;                  // DTE_PLAN_* (dte_type_set_plan)
    dte::NP node;
    std::shared_ptr<dte::Committed> desc;
    int64_t extent() const { return ub - lb; }
};

namespace dte {
// Handle registry (validity checks at the ABI).
bool handle_valid(dte_type t);
// Device copy of a committed type on the current device; uploads on first use.
int device_blob(dte_type t, const char **out, int *device);
// Device copy on device `dev` if already uploaded (never allocates).
int device_blob_resident(dte_type t, int dev, const char **out);
// Record that work using `t` was enqueued on `stream` (for deferred frees).
void note_use(dte_type t, int device, void *stream);
// Free device copies whose pending work has finished.
void reap_deferred();
// Request-loop waits that gave up on the current device (server.cu).
int serve_timeouts(unsigned long long *v);
}  // namespace dte

#include <nvtx3/nvToolsExt.h>
namespace dte {
// An NVTX range over one ABI call, named after it, for Nsight timelines.
// Without a tool attached, the push and the pop each test one function
// pointer.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace dte
#define DTE_NVTX_RANGE(name) ::dte::NvtxRange dte_nvtx_range_(name)
