// Internal types shared by the host planner and the device kernels of the enumerator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/huge.h"

namespace huge {

constexpr int kMaxK = HUGE_MAX_QUERY_VERTICES;  // query vertices
constexpr int kMaxSteps = 16;                   // operator levels (EXTEND + verify-only)
constexpr int kMaxExt = kMaxK - 1;              // lists intersected by one EXTEND
constexpr int kWarpsPerBlock = 8;
constexpr int kBlockThreads = kWarpsPerBlock * 32;

enum StepKind : uint8_t { kExtend = 0, kVerify = 1 };

// One operator of an EXTEND chain. Rows entering it have `w` bound positions.
//  EXTEND(Ext) (Sec. 4.2): new vertex u in the intersection of N(f[ext[j]]) for j < n_ext,
//    restricted to f[lo[j]] < u (j < n_lo) and u < f[hi[j]] (j < n_hi) — the symmetry-breaking
//    partial order — and u != f[inj[j]] (j < n_inj) for the positions not already excluded by
//    adjacency or by a strict bound. The row grows to w + 1 positions.
//  VERIFY (Sec. 5.2, verify-only EXTEND): keeps the row iff f[ext[j]] is adjacent to
//    f[ext2[j]] for all j < n_ext. The row keeps its w positions.
//  A labelled query vertex adds constant id bounds clo <= u < chi: the data graph's ids are
//    grouped by label, so one label is one id range (0 / 0xffffffff when unlabelled).
//  Directed graphs: bit j of `dirs` selects the in-list of f[ext[j]] instead of its out-list
//    (a query arc into the bound vertex); VERIFY checks the arc f[ext[j]] -> f[ext2[j]], or the
//    reverse arc when the bit is set.
struct alignas(16) StepDesc {
    uint8_t kind;
    uint8_t w;
    uint8_t n_ext, n_lo, n_hi, n_inj;
    uint8_t dirs, pad;
    uint8_t ext[kMaxK];
    uint8_t ext2[kMaxK];
    uint8_t lo[kMaxK];
    uint8_t hi[kMaxK];
    uint8_t inj[kMaxK];
    uint32_t clo, chi;
};

constexpr uint32_t kAnyLabel = 0xffffffffu;

// The device program of one EXTEND chain. Level 0 holds roots (width 1); operator t
// (1 <= t <= nsteps) turns level t-1 rows into level t rows; the last operator feeds the sink.
struct Prog {
    int32_t nsteps;
    int32_t width_out;               // width of the final rows (= query vertices)
    uint32_t lvl_off[kMaxSteps];     // word offset of level l's buffer in a warp's region
    uint32_t region_words;           // words of one warp's region
    uint8_t col_of_pos[kMaxK];       // LIST: output column (query vertex) of each position
    // optional partition filter on final rows (PUSH-JOIN passes): keep a row iff
    // hash(f[key_pos[0..n_key)]) % part_mod == part_id
    uint8_t n_key, pad0[3];
    uint8_t key_pos[4];
    uint32_t part_mod, part_id;
    uint32_t cap;                    // rows per level per warp of this query (filled at launch)
    uint32_t merge_ratio;            // last operator: merge-path rows when 2nd list <= ratio x 1st
    uint32_t root_lo, root_hi;       // ids the root (position 0) may take: its label's range
    StepDesc steps[kMaxSteps];       // steps[1..nsteps]
};

struct Task {           // a chunk of roots of one query
    uint32_t query;
    uint32_t r0, r1;
};

// Pool slot for work donated to idle warps (Sec. 5.3 work stealing, done by the victim).
struct PoolSlot {
    int32_t state;      // 0 empty, 1 being written, 2 ready, 3 being read
    int32_t level;
    uint32_t query;
    uint32_t nrows;     // rows (level >= 1) ...
    uint32_t r0, r1;    // ... or a root range (level 0)
    uint32_t pad[2];
};

struct Ctl {            // device control block of one persistent launch
    unsigned long long task_next;
    int32_t active;
    int32_t hungry;
    int32_t pool_ready;
    int32_t error;             // bit 0: a warp hit the kernel time limit
    unsigned long long donations;
    unsigned long long steals;
    unsigned long long exits_done, exits_idle, exits_limit;
    int32_t overflow;          // LIST: the sink is full, the launch is abandoned
    int32_t pad1;
};

struct KParams {
    const uint32_t *off;       // CSR offsets (one entry per list + 1), device
    const uint32_t *adj;       // adjacency, device
    uint32_t n;
    uint32_t dir_base;         // directed graphs: list id of v's in-list = v + dir_base (n); else 0
    const Prog *progs;         // per query
    const Task *tasks;
    uint32_t ntasks;
    Ctl *ctl;
    unsigned long long *counts;      // per query: [lo, hi] 128-bit accumulators
    unsigned long long *lvl_rows;    // per query: kMaxSteps counters
    unsigned long long *stats;       // [0] intersections, [1] list bytes
    uint32_t *wbuf;                  // per-warp level buffers
    uint64_t wstride;                // words per warp region (each query's levels fit in it)
    PoolSlot *pool;
    uint32_t *pool_rows;             // nslots * slot_rows * kMaxK words
    uint32_t nslots, slot_rows;
    uint32_t *sink;                  // LIST rows
    uint64_t sink_cap;               // rows
    unsigned long long *sink_tail;
    uint32_t sink_width;
    uint32_t steal;                  // 0 disables donation
    unsigned long long idle_ns;      // idle warps give up stealing after this long
    unsigned long long limit_ns;     // every warp stops (error bit 0) after this long
    // adjacency bitmaps of the high-degree vertices (degree bucket "hub"): hub_row[v] is the
    // bitmap row of v or kNoHub; row r holds bit x of N(v) at word r * hub_wpr + x / 32
    const uint32_t *hub_row;
    const uint32_t *hub_bits;
    uint64_t hub_wpr;                // words per bitmap row (a multiple of 8: rows are 32-byte aligned)
    // rank index of the bitmaps (or null): hub_rank[r * hub_nblk + b] = set bits of row r below
    // bit 256 b, so |N(v) ∩ [0, k)| takes one index load and one 32-byte block
    const uint32_t *hub_rank;
    uint64_t hub_nblk;
    // adj is 16-byte aligned and readable up to the next multiple of 4 entries past nnz, so
    // 16-byte vector loads from 16-byte boundaries stay inside it (else: 4-byte loads only)
    uint32_t vec_ok;
};

constexpr uint32_t kNoHub = 0xffffffffu;

// Grow-only device buffers reused across calls (one set per loaded graph).
struct Workspace {
    void *ptr[16] = {nullptr};
    size_t bytes[16] = {0};
    size_t peak = 0;
    // Returns a device buffer of at least `n` bytes for role `slot`, or nullptr on failure.
    void *get(int slot, size_t n);
    void release();
};

// Device copy of a loaded graph (library-owned).
struct DevGraph {
    uint32_t n = 0;
    uint64_t nnz = 0;              // adjacency entries stored (directed: out-lists + in-lists)
    bool directed = false;         // lists 0..n-1 are out-lists, n..2n-1 in-lists (list v + n)
    uint32_t nlists = 0;           // n, or 2n when directed
    uint64_t narcs = 0;            // directed: arcs (= nnz / 2)
    uint32_t max_deg = 0;
    uint32_t *d_off = nullptr;
    uint32_t *d_adj = nullptr;
    std::vector<uint32_t> h_off;   // offsets after relabelling (host copy; nnz < 2^32)
    std::vector<uint32_t> new_of_old;
    int device = 0;
    int grid = 0, warps = 0;       // persistent launch shape on this device
    Workspace ws;
    std::vector<float> gstats;     // graph statistics used as estimator features
    // out-of-core residency (huge_graph_set_residency): adj in managed memory, the highest-id
    // lists (the hubs under degree ordering) kept in HBM, the rest in host memory
    bool adj_managed = false;
    uint64_t adj_hbm_bytes = 0;
    // vertex labels: label L owns the ids [lstart[L], lstart[L + 1]) (empty when unlabelled)
    std::vector<uint32_t> lstart;
    // hub bitmaps (KParams::hub_row / hub_bits); none when hub_count == 0
    uint32_t *d_hub_row = nullptr;
    uint32_t *d_hub_bits = nullptr;
    uint32_t *d_hub_rank = nullptr;
    uint32_t hub_count = 0, hub_min_deg = 0;
    uint64_t hub_wpr = 0, hub_nblk = 0, hub_bytes = 0;
};

// (Re)builds the adjacency bitmaps of every vertex of degree >= min_deg, highest degree first,
// while their total size stays within max_bytes (min_deg 0 or max_bytes 0: none). graph.cu.
int build_hub_bitmaps(DevGraph &G, uint32_t min_deg, uint64_t max_bytes);
void free_hub_bitmaps(DevGraph &G);
// Moves adj to managed memory with the last `hbm_bytes` (whole 2 MiB pages) preferred in HBM and
// the rest preferred in host memory and mapped for the device (graph.cu).
int set_residency(DevGraph &G, uint64_t hbm_bytes);
// Default hub bitmap policy: a row costs n/8 bytes, a list 4 d bytes; keep rows of vertices
// whose bitmap is at most 32 x their list (d >= n / 1024), at least degree 256, within 4 GiB.
uint32_t default_hub_min_degree(uint32_t n);
constexpr uint64_t kDefaultHubBytes = 4ull << 30;

// Plan of one EXTEND chain over a (sub-)query given in its own vertex ids 0..k-1.
struct Chain {
    int k = 0;
    std::vector<int> order;        // matching order (query vertex at each position)
    Prog prog;                     // device program (lvl_off filled at launch)
    double est_cost = 0;
};

// Result of one engine run (one persistent launch or a sequence of them).
struct RunResult {
    std::vector<unsigned __int128> counts;        // per query
    std::vector<unsigned long long> lvl_rows;     // per query x kMaxSteps
    unsigned long long intersections = 0, list_bytes = 0, donations = 0, steals = 0, idle_exits = 0;
    double device_ms = 0;
    uint32_t cap = 0;
    uint64_t peak_bytes = 0;
    uint32_t launches = 0;
};

// Runs EXTEND chains over root tasks (engine.cu). Progs are host copies; `cap` 0 derives the
// per-level capacity from mem_bound. LIST mode writes into sink/sink_cap (rows of width
// sink_width) and returns the total produced in *sink_total (may exceed sink_cap).
struct RunCfg {
    uint64_t mem_bound = 1ull << 30;
    uint32_t cap = 0;             // rows per level per warp (0: default, clamped by mem_bound)
    bool stats = false;           // count algorithmic bytes
    bool steal = true;            // work donation between warps
    uint32_t limit_ms = 0;        // kernel time limit (0: default)
    uint32_t merge_ratio = 8;     // intersection variant of the last operator (0: binary search)
    // per-query settings (batched launches); empty = cap / merge_ratio for every query
    std::vector<uint32_t> caps, merges;
};
int run_chains(DevGraph &G, std::vector<Prog> progs, const std::vector<Task> &tasks, int mode,
               const RunCfg &cfg, uint32_t *sink, uint64_t sink_cap, uint32_t sink_width,
               uint64_t *sink_total, cudaStream_t s, RunResult *out);
// Root tasks covering [r0, r1) of query q, split into chunks balanced by `weight(r)` =
// 1 + degree(r) (or the given weights), with about `target` chunks.
void make_tasks(const DevGraph &G, uint32_t q, uint32_t r0, uint32_t r1, uint32_t chunk_roots,
                const float *weights, size_t target, std::vector<Task> *tasks);

// Launch the persistent enumerator (enumerate.cu).
cudaError_t launch_persistent(const KParams &kp, int mode, bool stats, int grid, cudaStream_t s);
int persistent_grid(int *warps);   // resident blocks for the persistent kernel, warps total

// Join kernels (join.cu).
struct JoinSpec {
    int nl, nr;                 // widths of left / right rows (query-vertex order of each side)
    int nkey;                   // key columns
    int lkey[4], rkey[4];       // key column in left / right rows
    int nonkey_l[kMaxK], n_nonkey_l;
    int nonkey_r[kMaxK], n_nonkey_r;
    // cross partial-order pairs: left column < right column, or right < left
    int n_lr, lr_l[16], lr_r[16];   // f_l[lr_l] < f_r[lr_r]
    int n_rl, rl_r[16], rl_l[16];   // f_r[rl_r] < f_l[rl_l]
    int k;                      // output width (query vertices)
    int out_col_l[kMaxK];       // output column of each left column
    int out_col_r[kMaxK];       // output column of each right column (-1 for key columns)
};
// Table and group buffers come from workspace slot 13 (grow-only). limit_ms 0 = 600 s.
int join_count_or_list(const JoinSpec &js, const uint32_t *d_left, uint64_t nleft,
                       const uint32_t *d_right, uint64_t nright, int mode, uint32_t *sink,
                       uint64_t sink_cap, unsigned long long *d_tail, Workspace &ws, uint32_t limit_ms,
                       cudaStream_t s, unsigned __int128 *count, std::string *err);

// Device memory (alloc.cu): the caller's allocator hook if set, else cudaMalloc / cudaFree.
cudaError_t dev_malloc_raw(void **p, size_t n);
template <class T>
cudaError_t dev_malloc(T **p, size_t n) {
    void *v = nullptr;
    const cudaError_t e = dev_malloc_raw(&v, n);
    *p = (T *)v;
    return e;
}
void dev_free(void *p);

// Error helpers (api.cpp).
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

}  // namespace huge
