// Host driver of the persistent enumerator: memory bound -> per-level capacity, device
// buffers, root tasks, one launch, read-back of exact counts and per-level logs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace huge {

namespace {
constexpr uint32_t kDefaultCap = 512;      // rows per level per warp when mem_bound allows
constexpr uint32_t kMaxSlotRows = 256;     // rows per donation slot
constexpr unsigned long long kLimitNs = 600ull * 1000 * 1000 * 1000;  // default kernel time limit

int cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();
    return fail(HUGE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace

void make_tasks(const DevGraph &G, uint32_t q, uint32_t r0, uint32_t r1, uint32_t chunk_roots,
                const float *weights, size_t target, std::vector<Task> *tasks) {
    if (r1 > G.n) r1 = G.n;
    if (r0 >= r1) return;
    if (chunk_roots) {
        for (uint64_t a = r0; a < r1; a += chunk_roots)
            tasks->push_back({q, (uint32_t)a, (uint32_t)std::min<uint64_t>(a + chunk_roots, r1)});
        return;
    }
    // weight(r) = 1 + deg(r), or the caller's estimate; split into ~target equal-weight chunks
    double total = 0;
    if (weights) {
        for (uint32_t r = r0; r < r1; r++) total += 1.0 + std::max(0.0f, weights[r]);
    } else {
        total = (double)(r1 - r0) + (double)(G.h_off[r1] - G.h_off[r0]);
    }
    if (target < 1) target = 1;
    const double per = total / (double)target;
    double accw = 0;
    uint32_t start = r0;
    for (uint32_t r = r0; r < r1; r++) {
        accw += weights ? 1.0 + std::max(0.0f, weights[r]) : 1.0 + (double)(G.h_off[r + 1] - G.h_off[r]);
        if (accw >= per || r + 1 == r1) {
            tasks->push_back({q, start, r + 1});
            start = r + 1;
            accw = 0;
        }
    }
}

int run_chains(DevGraph &G, std::vector<Prog> progs, const std::vector<Task> &tasks_in, int mode,
               const RunCfg &cfg, uint32_t *sink, uint64_t sink_cap, uint32_t sink_width,
               uint64_t *sink_total, cudaStream_t s, RunResult *out) {
    // a labelled root takes only its label's ids: clip every task to its query's root range
    std::vector<Task> clipped;
    const std::vector<Task> *tp = &tasks_in;
    bool clip = false;
    for (const Prog &p : progs) clip = clip || p.root_lo > 0 || p.root_hi < G.n;
    if (clip) {
        for (const Task &t : tasks_in) {
            const Prog &p = progs[t.query];
            const uint32_t a = std::max(t.r0, p.root_lo), b = std::min(t.r1, p.root_hi);
            if (a < b) clipped.push_back({t.query, a, b});
        }
        if (clipped.empty()) {  // no root carries the label: nothing to run
            const size_t nq = progs.size();
            out->counts.assign(nq, 0);
            out->lvl_rows.assign(kMaxSteps * nq, 0);
            if (sink_total) *sink_total = 0;
            return HUGE_OK;
        }
        tp = &clipped;
    }
    const std::vector<Task> &tasks = *tp;
    const uint64_t mem_bound = cfg.mem_bound;
    const bool stats = cfg.stats, steal = cfg.steal;
    const uint32_t limit_ms = cfg.limit_ms;
    const int W = G.warps, grid = G.grid;
    const size_t nq = progs.size();
    // per query: words per "row of capacity" of its levels, the requested rows per level, the
    // intersection variant; a warp's region holds the largest query's levels
    std::vector<uint64_t> unit(nq, 0);
    std::vector<uint32_t> want(nq);
    uint64_t unit_max = 0, need_words = 0;
    uint32_t want_min = 0xffffffffu;
    for (size_t q = 0; q < nq; q++) {
        const Prog &p = progs[q];
        for (int l = 1; l < p.nsteps; ++l) unit[q] += p.steps[l + 1].w;
        uint32_t c = (cfg.caps.size() == nq && cfg.caps[q]) ? cfg.caps[q] : (cfg.cap ? cfg.cap : kDefaultCap);
        want[q] = std::max<uint32_t>(32, c / 32 * 32);
        progs[q].merge_ratio = cfg.merges.size() == nq ? cfg.merges[q] : cfg.merge_ratio;
        if (unit[q]) {
            unit_max = std::max(unit_max, unit[q]);
            need_words = std::max<uint64_t>(need_words, want[q] * unit[q]);
            want_min = std::min(want_min, want[q]);
        }
    }
    const uint32_t nslots = (uint32_t)std::min(1024, std::max(32, W));
    uint32_t slot_rows = unit_max ? std::min(kMaxSlotRows, want_min) : kMaxSlotRows;
    uint64_t wstride = 0;
    if (unit_max > 0) {
        const uint64_t pool_bytes = (uint64_t)nslots * (sizeof(PoolSlot) + (uint64_t)slot_rows * kMaxK * 4);
        const uint64_t min_words = 32 * unit_max;
        const uint64_t min_bytes = (uint64_t)W * min_words * 4 + pool_bytes;
        if (mem_bound < min_bytes)
            return fail(HUGE_ENOMEM, "mem_bound " + std::to_string(mem_bound) + " B is below the minimum " +
                                         std::to_string(min_bytes) + " B (one 32-row batch per level for each of " +
                                         std::to_string(W) + " warps)");
        wstride = std::min<uint64_t>(need_words, (mem_bound - pool_bytes) / (4ull * W));
        wstride = std::max(wstride, min_words);
    }
    uint32_t cap = 32;
    for (size_t q = 0; q < nq; q++) {
        Prog &p = progs[q];
        p.cap = unit[q] ? (uint32_t)std::min<uint64_t>(want[q], wstride / unit[q] / 32 * 32) : 32u;
        if (unit[q]) slot_rows = std::min(slot_rows, p.cap);
        cap = std::max(cap, p.cap);
        uint32_t o = 0;
        for (int l = 0; l < kMaxSteps; ++l) p.lvl_off[l] = 0;
        for (int l = 1; l < p.nsteps; ++l) {
            p.lvl_off[l] = o;
            o += p.cap * p.steps[l + 1].w;
        }
        p.region_words = o;
    }
    Workspace &ws = G.ws;
    Prog *d_progs = (Prog *)ws.get(0, sizeof(Prog) * nq);
    Task *d_tasks = (Task *)ws.get(1, sizeof(Task) * std::max<size_t>(tasks.size(), 1));
    Ctl *d_ctl = (Ctl *)ws.get(2, sizeof(Ctl));
    unsigned long long *d_counts = (unsigned long long *)ws.get(3, 16 * nq);
    unsigned long long *d_lvl = (unsigned long long *)ws.get(4, 8 * kMaxSteps * nq);
    unsigned long long *d_stats = (unsigned long long *)ws.get(5, 64);
    uint32_t *d_wbuf = (uint32_t *)ws.get(6, std::max<uint64_t>(16, (uint64_t)W * wstride * 4));
    PoolSlot *d_pool = (PoolSlot *)ws.get(7, sizeof(PoolSlot) * nslots);
    uint32_t *d_prow = (uint32_t *)ws.get(8, (uint64_t)nslots * slot_rows * kMaxK * 4);
    unsigned long long *d_tail = (unsigned long long *)ws.get(9, 64);
    if (!d_progs || !d_tasks || !d_ctl || !d_counts || !d_lvl || !d_stats || !d_wbuf || !d_pool ||
        !d_prow || !d_tail)
        return fail(HUGE_ENOMEM, "device allocation for enumeration buffers failed");
    Ctl h_ctl;
    memset(&h_ctl, 0, sizeof(h_ctl));
    h_ctl.active = 0;  // each warp registers itself when it starts
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_progs, progs.data(), sizeof(Prog) * nq, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(Task) * tasks.size(), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_ctl, &h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemsetAsync(d_counts, 0, 16 * nq, s)) ||
        (e = cudaMemsetAsync(d_lvl, 0, 8 * kMaxSteps * nq, s)) || (e = cudaMemsetAsync(d_stats, 0, 64, s)) ||
        (e = cudaMemsetAsync(d_pool, 0, sizeof(PoolSlot) * nslots, s)) ||
        (e = cudaMemsetAsync(d_tail, 0, 64, s)))
        return cuda_fail(e, "preparing the enumeration");
    KParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.off = G.d_off;
    kp.adj = G.d_adj;
    kp.n = G.n;
    kp.progs = d_progs;
    kp.tasks = d_tasks;
    kp.ntasks = (uint32_t)tasks.size();
    kp.ctl = d_ctl;
    kp.counts = d_counts;
    kp.lvl_rows = d_lvl;
    kp.stats = d_stats;
    kp.wbuf = d_wbuf;
    kp.wstride = wstride;
    kp.pool = d_pool;
    kp.pool_rows = d_prow;
    kp.nslots = nslots;
    kp.slot_rows = slot_rows;
    kp.sink = sink;
    kp.sink_cap = sink ? sink_cap : 0;
    kp.sink_tail = d_tail;
    kp.sink_width = sink_width;
    kp.steal = steal ? 1u : 0u;
    // idle warps keep polling for donations until the launch's own time limit: a long launch
    // keeps all its stealers for its tail (they leave as soon as no warp is active)
    kp.limit_ns = limit_ms ? (unsigned long long)limit_ms * 1000000ull : kLimitNs;
    kp.idle_ns = kp.limit_ns;
    kp.vec_ok = (((uintptr_t)G.d_adj & 15) == 0) ? 1u : 0u;  // graph_load pads adj to 4 entries
    kp.dir_base = G.directed ? G.n : 0u;
    if (G.hub_count) {
        kp.hub_row = G.d_hub_row;
        kp.hub_bits = G.d_hub_bits;
        kp.hub_wpr = G.hub_wpr;
        // the rank index reads 32-byte blocks of a row: only with 32-byte aligned rows
        if (((uintptr_t)G.d_hub_bits & 31) == 0) {
            kp.hub_rank = G.d_hub_rank;
            kp.hub_nblk = G.hub_nblk;
        }
    }
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);
    e = launch_persistent(kp, mode, stats, grid, s);
    cudaEventRecord(ev1, s);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        return cuda_fail(e, "launching the enumeration kernel");
    }
    std::vector<unsigned long long> h_counts(2 * nq), h_lvl(kMaxSteps * nq);
    unsigned long long h_stats[8] = {0}, h_tail = 0;
    cudaMemcpyAsync(h_counts.data(), d_counts, 16 * nq, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h_lvl.data(), d_lvl, 8 * kMaxSteps * nq, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h_stats, d_stats, 64, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&h_ctl, d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&h_tail, d_tail, 8, cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    float ms = 0;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (e != cudaSuccess) return cuda_fail(e, "enumeration kernel");
    if (h_ctl.error)
        return fail(HUGE_ETIMEOUT,
                    "the enumeration kernel reached its time limit (error flags " + std::to_string(h_ctl.error) +
                        "; active " + std::to_string(h_ctl.active) + ", hungry " + std::to_string(h_ctl.hungry) +
                        ", pool_ready " + std::to_string(h_ctl.pool_ready) + ", tasks taken " +
                        std::to_string(std::min<unsigned long long>(h_ctl.task_next, tasks.size())) + "/" +
                        std::to_string(tasks.size()) + ", donations " + std::to_string(h_ctl.donations) +
                        ", steals " + std::to_string(h_ctl.steals) + ", exits done/idle/limit " +
                        std::to_string(h_ctl.exits_done) + "/" + std::to_string(h_ctl.exits_idle) + "/" +
                        std::to_string(h_ctl.exits_limit) + ")");
    out->counts.assign(nq, 0);
    out->lvl_rows.assign(kMaxSteps * nq, 0);
    for (size_t q = 0; q < nq; q++) {
        out->counts[q] = ((unsigned __int128)h_counts[2 * q + 1] << 64) | h_counts[2 * q];
        for (int l = 0; l < kMaxSteps; l++) out->lvl_rows[q * kMaxSteps + l] = h_lvl[q * kMaxSteps + l];
    }
    out->intersections = h_stats[0];
    out->list_bytes = h_stats[1];
    out->donations = h_ctl.donations;
    out->device_ms = ms;
    out->cap = cap;
    out->peak_bytes = (uint64_t)W * wstride * 4 + (uint64_t)nslots * (sizeof(PoolSlot) + (uint64_t)slot_rows * kMaxK * 4);
    out->launches = 1;
    out->donations = h_ctl.donations;
    out->steals = h_ctl.steals;
    out->idle_exits = h_ctl.exits_idle;
    if (sink_total) *sink_total = h_tail;
    return HUGE_OK;
}

}  // namespace huge
