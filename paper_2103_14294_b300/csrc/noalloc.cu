// huge_count_noalloc: the persistent COUNT enumeration for callers that must not allocate
// device memory. All scratch the kernel needs (control block, counters, device program, root
// tasks, donation pool and the per-warp level buffers) lives in one file-scope device array of
// fixed size; the caller passes the graph (device CSR) and receives the count on the host.
// The paper has no counterpart to this entry point: it serves callers whose device memory is
// owned elsewhere, and computes what huge_enumerate's COUNT mode computes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

namespace huge {
namespace {

constexpr size_t kScratchBytes = 32ull << 20;  // 32 MiB, held by every GPU that loads the library
constexpr uint32_t kMaxLevelCap = 512;
constexpr uint32_t kPoolSlots = 256, kPoolSlotRows = 32;

// The scratch. In host code this name is only a stand-in for the device object: its device
// address comes from cudaGetSymbolAddress, with that device current.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
std::map<int, unsigned char *> g_addr;  // device ordinal -> device address of g_scratch

// Set-up, once per device: the first call on a device looks up the scratch's device address
// with that device current (which also loads the library's device code there, so that first
// call must come before any stream capture) and caches it. After cudaDeviceReset the module
// would be loaded again at another address and the cached one would be stale: the entry point
// must not be used on a device after it has been reset.
int scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HUGE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_addr.find(dev);
    if (it != g_addr.end()) {
        *out = it->second;
        return HUGE_OK;
    }
    unsigned char *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(HUGE_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
    }
    g_addr[dev] = p;
    *out = p;
    return HUGE_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace huge

using namespace huge;

extern "C" int huge_count_noalloc(const uint32_t *d_offsets, const uint32_t *d_adj, uint32_t n, uint64_t nnz,
                                  uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *order,
                                  const uint32_t *po_pairs, int32_t npo, void *stream, int64_t *out_count) {
    set_error("");
    if (!d_offsets || (!d_adj && nnz) || !out_count) return fail(HUGE_EINVAL, "null argument");
    if (n == 0) return fail(HUGE_EINVAL, "empty graph (n = 0)");
    if (nnz >= 0xffffffffull) return fail(HUGE_EINVAL, "nnz must be below 2^32 - 1");
    QueryG Q;
    std::string err;
    int rc = parse_query(nq, q_edges, mq, &Q, &err);
    if (rc) return fail(rc, err);
    std::vector<std::pair<int, int>> po;
    if (npo < 0) {
        po = symmetry_breaking_po(Q);
    } else {
        if (npo > 0 && !po_pairs) return fail(HUGE_EINVAL, "null partial-order pairs");
        for (int32_t i = 0; i < npo; i++) {
            const uint32_t a = po_pairs[2 * i], b = po_pairs[2 * i + 1];
            if (a >= nq || b >= nq || a == b) return fail(HUGE_EINVAL, "bad partial-order pair");
            po.push_back({(int)a, (int)b});
        }
    }
    uint8_t lt[kMaxK][kMaxK];
    if (!po_closure(Q.k, po, lt)) return fail(HUGE_EINVAL, "the partial order has a cycle (not a DAG)");
    std::vector<int> ord;
    if (order) {
        ord.assign(order, order + nq);
        rc = check_order(Q, ord, &err);
        if (rc) return fail(rc, err);
    } else {
        ord = bfs_order(Q, lt);
    }
    Prog prog = build_chain(Q, ord, lt, false).prog;

    unsigned char *base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    int warps = 0;
    const int grid = persistent_grid(&warps);
    const uint64_t W = (uint64_t)warps;

    // root tasks: equal chunks, about 8 per warp
    const uint64_t want = std::max<uint64_t>(1, 8 * W);
    const uint32_t chunk = (uint32_t)std::max<uint64_t>(1, (n + want - 1) / want);
    std::vector<Task> tasks;
    for (uint64_t a = 0; a < n; a += chunk) tasks.push_back({0, (uint32_t)a, (uint32_t)std::min<uint64_t>(a + chunk, n)});

    // layout of the scratch
    uint64_t unit_words = 0;
    for (int l = 1; l < prog.nsteps; ++l) unit_words += prog.steps[l + 1].w;
    const size_t o_ctl = 0, o_counts = align_up(o_ctl + sizeof(Ctl)), o_lvl = align_up(o_counts + 16),
                 o_stats = align_up(o_lvl + 8 * kMaxSteps), o_tail = align_up(o_stats + 64),
                 o_prog = align_up(o_tail + 64), o_tasks = align_up(o_prog + sizeof(Prog)),
                 o_pool = align_up(o_tasks + sizeof(Task) * tasks.size()),
                 o_prow = align_up(o_pool + sizeof(PoolSlot) * kPoolSlots),
                 o_wbuf = align_up(o_prow + (size_t)kPoolSlots * kPoolSlotRows * kMaxK * 4);
    if (o_wbuf >= kScratchBytes)
        return fail(HUGE_ENOMEM, "graph too large for the static scratch of huge_count_noalloc (" +
                                     std::to_string(kScratchBytes >> 20) + " MiB)");
    uint32_t cap = kMaxLevelCap;
    if (unit_words) {
        const uint64_t avail = kScratchBytes - o_wbuf;
        const uint64_t fit = avail / (W * unit_words * 4);
        if (fit < 32)
            return fail(HUGE_ENOMEM, "query needs " + std::to_string(W * unit_words * 4 * 32 + o_wbuf) +
                                         " bytes of scratch for 32 rows per level per warp; the static scratch of "
                                         "huge_count_noalloc holds " + std::to_string(kScratchBytes) + " bytes");
        cap = (uint32_t)std::min<uint64_t>(kMaxLevelCap, fit / 32 * 32);
    } else {
        cap = 32;
    }
    uint32_t o = 0;
    for (int l = 0; l < kMaxSteps; ++l) prog.lvl_off[l] = 0;
    for (int l = 1; l < prog.nsteps; ++l) {
        prog.lvl_off[l] = o;
        o += cap * prog.steps[l + 1].w;
    }
    prog.region_words = o;
    prog.cap = cap;
    prog.merge_ratio = 8;

    cudaStream_t s = (cudaStream_t)stream;
    Ctl h_ctl;
    memset(&h_ctl, 0, sizeof(h_ctl));
    cudaError_t e;
    // everything that must start at zero is cleared on every call: the array keeps the
    // previous call's contents
    if ((e = cudaMemcpyAsync(base + o_ctl, &h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemsetAsync(base + o_counts, 0, o_prog - o_counts, s)) ||
        (e = cudaMemcpyAsync(base + o_prog, &prog, sizeof(Prog), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(base + o_tasks, tasks.data(), sizeof(Task) * tasks.size(), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemsetAsync(base + o_pool, 0, sizeof(PoolSlot) * kPoolSlots, s))) {
        cudaGetLastError();
        return fail(HUGE_ECUDA, std::string("preparing the static scratch: ") + cudaGetErrorString(e));
    }
    KParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.off = d_offsets;
    kp.adj = d_adj;
    kp.n = n;
    kp.progs = (const Prog *)(base + o_prog);
    kp.tasks = (const Task *)(base + o_tasks);
    kp.ntasks = (uint32_t)tasks.size();
    kp.ctl = (Ctl *)(base + o_ctl);
    kp.counts = (unsigned long long *)(base + o_counts);
    kp.lvl_rows = (unsigned long long *)(base + o_lvl);
    kp.stats = (unsigned long long *)(base + o_stats);
    kp.wbuf = (uint32_t *)(base + o_wbuf);
    kp.wstride = (uint64_t)cap * unit_words;
    kp.pool = (PoolSlot *)(base + o_pool);
    kp.pool_rows = (uint32_t *)(base + o_prow);
    kp.nslots = kPoolSlots;
    kp.slot_rows = std::min(kPoolSlotRows, cap);
    kp.sink = nullptr;
    kp.sink_cap = 0;
    kp.sink_tail = (unsigned long long *)(base + o_tail);
    kp.sink_width = (uint32_t)Q.k;
    kp.steal = 1;
    kp.idle_ns = 30ull * 1000 * 1000 * 1000;
    kp.limit_ns = 600ull * 1000 * 1000 * 1000;
    // the caller's adjacency array is not padded: vector loads only when none can pass its end
    kp.vec_ok = ((((uintptr_t)d_adj & 15) == 0) && nnz % 4 == 0) ? 1u : 0u;
    e = launch_persistent(kp, HUGE_COUNT, false, grid, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HUGE_ECUDA, std::string("launching the enumeration kernel: ") + cudaGetErrorString(e));
    }
    unsigned long long h_counts[2] = {0, 0};
    cudaMemcpyAsync(h_counts, base + o_counts, 16, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&h_ctl, base + o_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(HUGE_ECUDA, std::string("enumeration kernel: ") + cudaGetErrorString(e));
    if (h_ctl.error) return fail(HUGE_ETIMEOUT, "the enumeration kernel reached its time limit");
    if (h_counts[1] != 0 || h_counts[0] > (unsigned long long)INT64_MAX)
        return fail(HUGE_EOVERFLOW, "exact count does not fit in int64");
    *out_count = (int64_t)h_counts[0];
    return HUGE_OK;
}
