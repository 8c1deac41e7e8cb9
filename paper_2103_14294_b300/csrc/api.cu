// extern "C" entry points of huge.h: argument checks, planning, and the host drivers around
// the persistent enumerator (COUNT, chunked LIST with drain, PUSH-JOIN, batch, autotune).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "plan.h"

namespace huge {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int graph_load(const uint64_t *offsets, const uint32_t *adj, uint32_t n, uint64_t nnz, uint32_t flags,
               const uint32_t *labels, uint32_t nlabels, DevGraph **out);
void graph_free(DevGraph *G);
int mlp_predict(const huge_mlp_t *m, const float *x, int rows, float *y, std::string *err);

namespace {

constexpr uint64_t kEstimateMemBound = 1ull << 30;
constexpr uint32_t kSampleRoots = 2048;
constexpr uint32_t kEstimateLimitMs = 2000;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int count_to_i64(unsigned __int128 c, int64_t *out) {
    if (c > (unsigned __int128)INT64_MAX) return fail(HUGE_EOVERFLOW, "exact count does not fit in int64");
    *out = (int64_t)c;
    return HUGE_OK;
}

// The label ranges a plan's chains use: its graph's, else those an offline plan was given.
const std::vector<uint32_t> *plan_labels(const huge_plan_t *P) {
    if (P->G) return &P->G->lstart;
    return P->offline_lstart.empty() ? nullptr : &P->offline_lstart;
}

// s stratified roots of [base, base + n), one per stratum (all of them when n <= s).
std::vector<Task> sample_tasks(uint32_t base, uint32_t n, uint32_t s, uint64_t seed) {
    std::vector<Task> t;
    if (n <= s) {
        for (uint32_t r = 0; r < n; r++) t.push_back({0, base + r, base + r + 1});
        return t;
    }
    uint64_t x = seed;
    for (uint32_t i = 0; i < s; i++) {
        x += 0x9e3779b97f4a7c15ULL;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        const double u = (double)(z >> 11) / 9007199254740992.0;
        uint32_t r = (uint32_t)(((double)i + u) * (double)n / (double)s);
        if (r >= n) r = n - 1;
        t.push_back({0, base + r, base + r + 1});
    }
    return t;
}

// |R(q[mask])| by exact enumeration from a stratified root sample, scaled by n / s.
int sample_card(DevGraph &G, const QueryG &Q, const uint8_t lt[kMaxK][kMaxK], uint32_t mask, cudaStream_t s,
                double *out) {
    uint8_t slt[kMaxK][kMaxK];
    int loc[kMaxK], glob[kMaxK];
    QueryG S = sub_query(Q, mask, lt, slt, loc, glob);
    const bool labelled = S.lab[0] != kAnyLabel || S.lab[1] != kAnyLabel;
    if (S.k == 2 && !labelled && !G.directed) {  // a single edge: exact
        *out = (slt[0][1] || slt[1][0]) ? (double)G.nnz / 2.0 : (double)G.nnz;
        return HUGE_OK;
    }
    Chain c = build_chain(S, bfs_order(S, slt), slt, false, &G.lstart);
    // roots sampled inside the root's label range, scaled by that range's size
    const uint32_t rlo = std::min(c.prog.root_lo, G.n), rhi = std::min(c.prog.root_hi, G.n);
    if (rhi <= rlo) {
        *out = 0;
        return HUGE_OK;
    }
    std::vector<Task> tasks = sample_tasks(rlo, rhi - rlo, kSampleRoots, 0x5eed0000ull + mask);
    RunResult rr;
    RunCfg rc0;
    rc0.mem_bound = kEstimateMemBound;
    rc0.limit_ms = kEstimateLimitMs;
    int rc = run_chains(G, {c.prog}, tasks, HUGE_COUNT, rc0, nullptr, 0, 0, nullptr, s, &rr);
    if (rc == HUGE_ETIMEOUT) {  // a sub-query too large to sample in time: treat as enormous
        set_error("");
        *out = 1e18;
        return HUGE_OK;
    }
    if (rc) return rc;
    *out = (double)rr.counts[0] * (double)(rhi - rlo) / (double)tasks.size();
    return HUGE_OK;
}

void fill_join(huge_plan_t *P, const DpResult &dp) {
    const QueryG &Q = P->Q;
    uint32_t L = dp.jl, R = dp.jr;
    if (dp.cards.size() > std::max(L, R) && dp.cards[R] >= 0 && dp.cards[L] >= 0 && dp.cards[R] < dp.cards[L])
        std::swap(L, R);  // build the hash table on the smaller side
    const uint32_t K = L & R;
    uint8_t slt[kMaxK][kMaxK];
    int lloc[kMaxK], rloc[kMaxK], lglob[kMaxK], rglob[kMaxK];
    QueryG SL = sub_query(Q, L, P->lt, slt, lloc, lglob);
    std::vector<int> og = recover_order(Q, P->lt, dp, L), ol;
    for (int v : og) ol.push_back(lloc[v]);
    P->left = build_chain(SL, ol, slt, false, plan_labels(P));
    QueryG SR = sub_query(Q, R, P->lt, slt, rloc, rglob);
    og = recover_order(Q, P->lt, dp, R);
    std::vector<int> orr;
    for (int v : og) orr.push_back(rloc[v]);
    P->right = build_chain(SR, orr, slt, false, plan_labels(P));
    P->lmask = L;
    P->rmask = R;
    memcpy(P->l_global, lglob, sizeof(lglob));
    memcpy(P->r_global, rglob, sizeof(rglob));
    JoinSpec &js = P->js;
    memset(&js, 0, sizeof(js));
    js.nl = SL.k;
    js.nr = SR.k;
    js.k = Q.k;
    for (int v = 0; v < Q.k; v++) {
        if (K >> v & 1) {
            js.lkey[js.nkey] = lloc[v];
            js.rkey[js.nkey] = rloc[v];
            // positions of the key in each side's matching order (partition passes)
            for (int p = 0; p < SL.k; p++)
                if (P->left.order[p] == lloc[v]) P->left.prog.key_pos[js.nkey] = (uint8_t)p;
            for (int p = 0; p < SR.k; p++)
                if (P->right.order[p] == rloc[v]) P->right.prog.key_pos[js.nkey] = (uint8_t)p;
            js.nkey++;
        }
    }
    P->left.prog.n_key = P->right.prog.n_key = (uint8_t)js.nkey;
    for (int v = 0; v < Q.k; v++) {
        if ((L & ~K) >> v & 1) js.nonkey_l[js.n_nonkey_l++] = lloc[v];
        if ((R & ~K) >> v & 1) js.nonkey_r[js.n_nonkey_r++] = rloc[v];
    }
    for (int a = 0; a < Q.k; a++)
        for (int b = 0; b < Q.k; b++) {
            if (!((L & ~K) >> a & 1) || !((R & ~K) >> b & 1)) continue;
            if (P->lt[a][b]) {
                js.lr_l[js.n_lr] = lloc[a];
                js.lr_r[js.n_lr] = rloc[b];
                js.n_lr++;
            }
            if (P->lt[b][a]) {
                js.rl_r[js.n_rl] = rloc[b];
                js.rl_l[js.n_rl] = lloc[a];
                js.n_rl++;
            }
        }
    for (int c = 0; c < SL.k; c++) js.out_col_l[c] = lglob[c];
    for (int c = 0; c < SR.k; c++) js.out_col_r[c] = (K >> rglob[c] & 1) ? -1 : rglob[c];
}

struct EnumCfg {
    RunCfg run;
    size_t target;
    uint32_t chunk;
    const float *weights;
};

void add_run(RunResult *agg, const RunResult &r, size_t nq) {
    if (agg->counts.empty()) {
        agg->counts.assign(nq, 0);
        agg->lvl_rows.assign(nq * kMaxSteps, 0);
    }
    for (size_t q = 0; q < nq && q < r.counts.size(); q++) agg->counts[q] += r.counts[q];
    for (size_t i = 0; i < r.lvl_rows.size() && i < agg->lvl_rows.size(); i++) agg->lvl_rows[i] += r.lvl_rows[i];
    agg->intersections += r.intersections;
    agg->list_bytes += r.list_bytes;
    agg->donations += r.donations;
    agg->device_ms += r.device_ms;
    agg->cap = r.cap;
    agg->peak_bytes = std::max(agg->peak_bytes, r.peak_bytes);
    agg->launches += r.launches;
}

// LIST for an EXTEND chain: a piece of work (a root range, or a slice of an explicit root list)
// is tried whole and halved when its matches do not fit in the free part of the sink; a full
// sink is drained through the caller's callback first.
int list_chain(DevGraph &G, const Prog &prog, int k, uint32_t r0, uint32_t r1, const std::vector<Task> *fixed,
               const EnumCfg &cfg, const huge_sink_t *sink, cudaStream_t s, unsigned __int128 *count,
               RunResult *agg) {
    uint64_t used = 0;
    *count = 0;
    // stack of [lo, hi): root ids (range mode) or indices into *fixed (list mode)
    std::vector<std::pair<uint64_t, uint64_t>> stack;
    if (fixed)
        stack.push_back({0, fixed->size()});
    else
        stack.push_back({r0, r1});
    while (!stack.empty()) {
        const std::pair<uint64_t, uint64_t> rg = stack.back();
        stack.pop_back();
        if (rg.first >= rg.second) continue;
        std::vector<Task> tasks;
        if (fixed)
            tasks.assign(fixed->begin() + rg.first, fixed->begin() + rg.second);
        else
            make_tasks(G, 0, (uint32_t)rg.first, (uint32_t)rg.second, cfg.chunk, cfg.weights, cfg.target, &tasks);
        if (tasks.empty()) continue;
        RunResult rr;
        uint64_t produced = 0;
        const uint64_t room = sink->capacity_rows - used;
        int rc = run_chains(G, {prog}, tasks, HUGE_LIST, cfg.run, sink->rows + used * (uint64_t)k, room,
                            (uint32_t)k, &produced, s, &rr);
        if (rc) return rc;
        if (produced <= room) {
            used += produced;
            *count += produced;
            add_run(agg, rr, 1);
            continue;
        }
        // overflow: the rows of this attempt are discarded
        if (!sink->drain)
            return fail(HUGE_ERANGE, "LIST output exceeds the sink capacity of " + std::to_string(sink->capacity_rows) +
                                         " rows and no drain callback was given");
        if (used > 0) {  // drain, then retry the same piece with the whole sink
            sink->drain(sink->ctx, sink->rows, used);
            used = 0;
            stack.push_back(rg);
            continue;
        }
        if (rg.second - rg.first <= 1)
            return fail(HUGE_ERANGE, "the matches of a single root exceed the sink capacity");
        const uint64_t mid = rg.first + (rg.second - rg.first) / 2;
        stack.push_back({mid, rg.second});
        stack.push_back({rg.first, mid});
    }
    if (used > 0 && sink->drain) sink->drain(sink->ctx, sink->rows, used);
    return HUGE_OK;
}

// PUSH-JOIN plan: enumerate both sides (LIST) into bounded buffers, join on the key. If a side
// does not fit, both sides are re-enumerated in P passes, each keeping one hash bucket of the
// key (the shuffle by join key of Sec. 4.2, done as a partition of the key space).
int join_enumerate(huge_plan_t *P, int mode, const EnumCfg &cfg, const huge_sink_t *sink, cudaStream_t s,
                   unsigned __int128 *count, RunResult *agg, int64_t side_rows[2]) {
    DevGraph &G = *P->G;
    const JoinSpec &js = P->js;
    const uint64_t quarter = std::max<uint64_t>(cfg.run.mem_bound / 4, 1 << 20);
    uint64_t capL = quarter / (4ull * js.nl), capR = quarter / (4ull * js.nr);
    capL = std::min<uint64_t>(capL, quarter / 48);
    if (capL < 1024 || capR < 1024) return fail(HUGE_ENOMEM, "mem_bound too small for a PUSH-JOIN plan");
    uint32_t *dL = (uint32_t *)G.ws.get(10, capL * 4ull * js.nl);
    uint32_t *dR = (uint32_t *)G.ws.get(11, capR * 4ull * js.nr);
    unsigned long long *dtail = (unsigned long long *)G.ws.get(12, 64);
    if (!dL || !dR || !dtail) return fail(HUGE_ENOMEM, "device allocation for join buffers failed");
    RunCfg side = cfg.run;
    side.mem_bound = quarter;
    uint32_t passes = 1;
    uint64_t used = 0;
    for (int attempt = 0; attempt < 12; attempt++) {
        bool restart = false;
        unsigned __int128 total = 0;
        used = 0;
        side_rows[0] = side_rows[1] = 0;
        RunResult part;
        for (uint32_t p = 0; p < passes && !restart; p++) {
            Prog lp = P->left.prog, rp = P->right.prog;
            lp.part_mod = rp.part_mod = passes;
            lp.part_id = rp.part_id = p;
            std::vector<Task> tl, tr;
            make_tasks(G, 0, 0, G.n, cfg.chunk, nullptr, cfg.target, &tl);
            tr = tl;
            uint64_t nL = 0, nR = 0;
            RunResult r1, r2;
            int rc = run_chains(G, {lp}, tl, HUGE_LIST, side, dL, capL, (uint32_t)js.nl, &nL, s, &r1);
            if (rc) return rc;
            if (nL > capL) {
                passes = (uint32_t)std::min<uint64_t>(1u << 20, (uint64_t)std::ceil((double)passes * nL / capL * 1.3));
                restart = true;
                break;
            }
            rc = run_chains(G, {rp}, tr, HUGE_LIST, side, dR, capR, (uint32_t)js.nr, &nR, s, &r2);
            if (rc) return rc;
            if (nR > capR) {
                passes = (uint32_t)std::min<uint64_t>(1u << 20, (uint64_t)std::ceil((double)passes * nR / capR * 1.3));
                restart = true;
                break;
            }
            add_run(&part, r1, 1);
            add_run(&part, r2, 1);
            side_rows[0] += (int64_t)nL;
            side_rows[1] += (int64_t)nR;
            // the left side (the smaller estimate, chosen by the planner) builds the hash table
            const JoinSpec &j = js;
            const uint32_t *bL = dL, *bR = dR;
            const uint64_t n1 = nL, n2 = nR;
            unsigned __int128 c = 0;
            std::string err;
            if (mode == HUGE_LIST) {
                for (int tries = 0;; tries++) {
                    cudaMemsetAsync(dtail, 0, 8, s);
                    const uint64_t room = sink->capacity_rows - used;
                    rc = join_count_or_list(j, bL, n1, bR, n2, HUGE_LIST, sink->rows + used * (uint64_t)js.k, room,
                                            dtail, G.ws, cfg.run.limit_ms, s, &c, &err);
                    if (rc) return fail(rc, err);
                    if ((uint64_t)c <= room) {
                        used += (uint64_t)c;
                        break;
                    }
                    if (!sink->drain)
                        return fail(HUGE_ERANGE, "LIST output of the join exceeds the sink and no drain callback was given");
                    if (used == 0) {  // one pass alone does not fit: use more passes
                        passes *= 2;
                        restart = true;
                        break;
                    }
                    sink->drain(sink->ctx, sink->rows, used);
                    used = 0;
                }
                if (restart) break;
            } else {
                rc = join_count_or_list(j, bL, n1, bR, n2, HUGE_COUNT, nullptr, 0, dtail, G.ws, cfg.run.limit_ms, s,
                                        &c, &err);
                if (rc) return fail(rc, err);
            }
            total += c;
        }
        if (restart) continue;
        *count = total;
        add_run(agg, part, 1);
        agg->launches += 3 * passes;
        if (mode == HUGE_LIST && used > 0 && sink->drain) sink->drain(sink->ctx, sink->rows, used);
        return HUGE_OK;
    }
    return fail(HUGE_ENOMEM, "PUSH-JOIN did not fit in mem_bound even with many partition passes");
}
}  // namespace
}  // namespace huge

using namespace huge;

extern "C" {

const char *huge_last_error(void) { return g_err.c_str(); }

int huge_graph_load(const uint64_t *offsets, const uint32_t *adj, uint32_t n, uint64_t nnz, uint32_t flags,
                    huge_graph_t **out) {
    return huge_graph_load_labeled(offsets, adj, n, nnz, nullptr, 0, flags, out);
}

int huge_graph_load_labeled(const uint64_t *offsets, const uint32_t *adj, uint32_t n, uint64_t nnz,
                            const uint32_t *labels, uint32_t nlabels, uint32_t flags, huge_graph_t **out) {
    g_err.clear();
    if (!out) return fail(HUGE_EINVAL, "null output pointer");
    DevGraph *G = nullptr;
    int rc = graph_load(offsets, adj, n, nnz, flags, labels, nlabels, &G);
    if (rc) return rc;
    huge_graph_t *h = new huge_graph_t();
    h->G = G;
    *out = h;
    return HUGE_OK;
}

int huge_graph_label_ranges(const huge_graph_t *g, uint32_t *nlabels, uint32_t *lstart) {
    if (!g || !g->G) return fail(HUGE_EINVAL, "null graph");
    const std::vector<uint32_t> &ls = g->G->lstart;
    const uint32_t L = ls.empty() ? 0u : (uint32_t)ls.size() - 1;
    if (nlabels) *nlabels = L;
    if (lstart && L) memcpy(lstart, ls.data(), sizeof(uint32_t) * ls.size());
    return HUGE_OK;
}

int huge_graph_free(huge_graph_t *g) {
    if (!g) return HUGE_OK;
    graph_free(g->G);
    delete g;
    return HUGE_OK;
}

int huge_graph_info(const huge_graph_t *g, uint32_t *n, uint64_t *nnz, uint32_t *max_degree) {
    if (!g || !g->G) return fail(HUGE_EINVAL, "null graph");
    if (n) *n = g->G->n;
    if (nnz) *nnz = g->G->nnz;
    if (max_degree) *max_degree = g->G->max_deg;
    return HUGE_OK;
}

int huge_graph_new_ids(const huge_graph_t *g, uint32_t *new_of_old) {
    if (!g || !g->G || !new_of_old) return fail(HUGE_EINVAL, "null argument");
    memcpy(new_of_old, g->G->new_of_old.data(), sizeof(uint32_t) * g->G->n);
    return HUGE_OK;
}

int huge_graph_set_hub_bitmaps(huge_graph_t *g, uint32_t min_degree, uint64_t max_bytes) {
    g_err.clear();
    if (!g || !g->G) return fail(HUGE_EINVAL, "null graph");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->G->device);
    if (min_degree == UINT32_MAX) min_degree = default_hub_min_degree(g->G->n);
    const int rc = build_hub_bitmaps(*g->G, min_degree, max_bytes);
    cudaSetDevice(cur);
    return rc;
}

int huge_graph_set_residency(huge_graph_t *g, uint64_t hbm_bytes, uint64_t *resident_bytes) {
    g_err.clear();
    if (!g || !g->G) return fail(HUGE_EINVAL, "null graph");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->G->device);
    const int rc = set_residency(*g->G, hbm_bytes);
    cudaSetDevice(cur);
    if (rc == HUGE_OK && resident_bytes) *resident_bytes = g->G->adj_hbm_bytes;
    return rc;
}

int huge_graph_hub_info(const huge_graph_t *g, uint32_t *count, uint32_t *min_degree, uint64_t *bytes) {
    if (!g || !g->G) return fail(HUGE_EINVAL, "null graph");
    if (count) *count = g->G->hub_count;
    if (min_degree) *min_degree = g->G->hub_min_deg;
    if (bytes) *bytes = g->G->hub_bytes;
    return HUGE_OK;
}

}  // extern "C"

namespace {

// The partial order of a plan: the given pairs (a, b) meaning f(a) < f(b), or with npo < 0 the
// automatic symmetry-breaking order of Q.
int parse_partial_order(const QueryG &Q, const uint32_t *po_pairs, int32_t npo, std::vector<std::pair<int, int>> *po) {
    po->clear();
    if (npo < 0) {
        *po = symmetry_breaking_po(Q);
        return HUGE_OK;
    }
    if (npo > 0 && !po_pairs) return fail(HUGE_EINVAL, "null partial-order pairs");
    for (int32_t i = 0; i < npo; i++) {
        const uint32_t a = po_pairs[2 * i], b = po_pairs[2 * i + 1];
        if (a >= (uint32_t)Q.k || b >= (uint32_t)Q.k || a == b) return fail(HUGE_EINVAL, "bad partial-order pair");
        po->push_back({(int)a, (int)b});
    }
    return HUGE_OK;
}

// The plan Alg. 1 chose (dp): a PUSH-JOIN at the top when it is cheaper (or forced), else the
// EXTEND chain of the best matching order; fills P's device programs and estimated cost.
int finish_plan(huge_plan_t *P, DpResult &dp, uint32_t flags, bool tree_verify) {
    const uint32_t full = (1u << P->Q.k) - 1;
    const bool use_join = dp.join_cost >= 0 && (dp.extend_cost < 0 || dp.join_cost < dp.extend_cost);
    if ((flags & HUGE_PLAN_FORCE_JOIN) && dp.join_cost < 0)
        return fail(HUGE_EINVAL, "the query has no valid PUSH-JOIN split (key must be an independent set of "
                                 "at most 4 vertices and cover every crossing edge)");
    if (use_join) {
        P->join = true;
        fill_join(P, dp);
        P->est_cost = dp.join_cost;
    } else {
        P->chain = build_chain(P->Q, recover_order(P->Q, P->lt, dp, full), P->lt, tree_verify, plan_labels(P));
        P->est_cost = dp.extend_cost;
    }
    return HUGE_OK;
}

int build_plan(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *order,
               const uint32_t *po_pairs, int32_t npo, uint32_t flags, const huge_mlp_t *model, huge_plan_t **out,
               const uint32_t *q_labels = nullptr) {
    g_err.clear();
    const double t0 = now_s();
    if (!g || !g->G || !out) return fail(HUGE_EINVAL, "null graph or output pointer");
    QueryG Q;
    std::string err;
    int rc = parse_query(nq, q_edges, mq, &Q, &err, g->G->directed);
    if (rc) return fail(rc, err);
    if (q_labels) {
        if (g->G->lstart.empty()) return fail(HUGE_EINVAL, "query labels need a graph loaded with labels");
        for (uint32_t v = 0; v < nq; v++) Q.lab[v] = q_labels[v];
    }
    std::vector<std::pair<int, int>> po;
    rc = parse_partial_order(Q, po_pairs, npo, &po);
    if (rc) return rc;
    huge_plan_t *P = new huge_plan_t();
    P->G = g->G;
    P->Q = Q;
    P->po = po;
    if (!po_closure(Q.k, po, P->lt)) {
        delete P;
        return fail(HUGE_EINVAL, "the partial order has a cycle (not a DAG)");
    }
    const bool tree_verify = flags & HUGE_PLAN_TREE_VERIFY;
    if (order) {
        std::vector<int> ord(order, order + nq);
        rc = check_order(Q, ord, &err);
        if (rc) {
            delete P;
            return fail(rc, err);
        }
        P->chain = build_chain(Q, ord, P->lt, tree_verify, plan_labels(P));
        P->how = "given";
    } else {
        const bool learned = flags & HUGE_PLAN_LEARNED;
        if (learned && !model) {
            delete P;
            return fail(HUGE_EINVAL, "HUGE_PLAN_LEARNED needs a model (huge_plan_ex)");
        }
        const uint32_t full = (1u << Q.k) - 1;
        std::vector<double> card(full + 1, -1.0);
        double est_s = 0;
        int est_rc = 0;
        std::string est_err;
        if (learned) {  // one batched inference over every connected sub-query
            const double te = now_s();
            std::vector<uint32_t> masks;
            for (uint32_t m = 1; m <= full; m++)
                if (__builtin_popcount(m) >= 2) masks.push_back(m);
            std::vector<float> X(masks.size() * 64), Y(masks.size());
            for (size_t i = 0; i < masks.size(); i++) subquery_features(Q, P->lt, masks[i], P->G->gstats, &X[i * 64]);
            est_rc = mlp_predict(model, X.data(), (int)masks.size(), Y.data(), &est_err);
            for (size_t i = 0; i < masks.size(); i++) {
                const uint32_t m = masks[i];
                if (__builtin_popcount(m) == 2) {  // a single query edge: |R| is known exactly
                    const int a = __builtin_ctz(m), b = 31 - __builtin_clz(m);
                    card[m] = P->G->directed ? (double)P->G->narcs
                              : (P->lt[a][b] || P->lt[b][a]) ? (double)P->G->nnz / 2.0 : (double)P->G->nnz;
                } else {  // clamp: log(1 + |R|) <= 60 keeps every cost finite
                    card[m] = std::expm1((double)std::min(60.0f, std::max(0.0f, Y[i])));
                }
            }
            est_s += now_s() - te;
        }
        auto cardf = [&](uint32_t m) -> double {
            if (card[m] >= 0) return card[m];
            if (est_rc) return 0.0;
            const double te = now_s();
            double v = 0;
            est_rc = sample_card(*P->G, Q, P->lt, m, 0, &v);
            est_s += now_s() - te;
            card[m] = v;
            return v;
        };
        const bool allow_ext = !(flags & HUGE_PLAN_FORCE_JOIN);
        const bool allow_join = !(flags & (HUGE_PLAN_EXTEND_ONLY | HUGE_PLAN_TREE_VERIFY));
        DpResult dp = optimise(Q, P->lt, cardf, (double)P->G->nnz / 2.0, allow_ext, allow_join);
        if (est_rc) {
            delete P;
            return est_err.empty() ? est_rc : fail(est_rc, est_err);
        }
        P->est_s = est_s;
        dp.cards = card;
        rc = finish_plan(P, dp, flags, tree_verify);
        if (rc) {
            delete P;
            return rc;
        }
        P->how = learned ? "learned" : "plain";
    }
    P->plan_s = now_s() - t0;
    *out = P;
    return HUGE_OK;
}

void fill_stats(huge_stats_t *st, const RunResult &rr, int64_t roots, int nsteps, unsigned __int128 count, int W) {
    if (!st) return;
    memset(st, 0, sizeof(*st));
    st->level_rows[0] = roots;
    for (int l = 1; l < nsteps && l < 16 && l < (int)rr.lvl_rows.size(); l++)
        st->level_rows[l] = (int64_t)rr.lvl_rows[l];
    if (nsteps < 16) st->level_rows[nsteps] = (int64_t)std::min<unsigned __int128>(count, INT64_MAX);
    st->nlevels = std::min(nsteps + 1, 16);
    st->intersections = rr.intersections;
    st->list_bytes = rr.list_bytes;
    st->peak_bytes = rr.peak_bytes;
    st->device_ms = rr.device_ms;
    st->level_cap = rr.cap;
    st->warps = (uint32_t)W;
    st->launches = rr.launches;
}

int enumerate_impl(const huge_plan_t *Pc, int mode, uint64_t mem_bound, const huge_sink_t *sink, void *stream,
                   const huge_enum_opts_t *o, int64_t *out_count, huge_stats_t *st) {
    g_err.clear();
    if (!Pc || !Pc->G || !out_count) return fail(HUGE_EINVAL, "null plan or output pointer");
    huge_plan_t *P = const_cast<huge_plan_t *>(Pc);
    if (mode != HUGE_COUNT && mode != HUGE_LIST) return fail(HUGE_EINVAL, "mode must be HUGE_COUNT or HUGE_LIST");
    if (mode == HUGE_LIST && (!sink || !sink->rows || sink->capacity_rows == 0))
        return fail(HUGE_EINVAL, "HUGE_LIST needs a sink with device rows and a non-zero capacity");
    huge_enum_opts_t opt;
    memset(&opt, 0, sizeof(opt));
    if (o) opt = *o;
    if (opt.per_root) return fail(HUGE_EINVAL, "per_root is reserved and must be NULL");
    DevGraph &G = *P->G;
    cudaStream_t s = (cudaStream_t)stream;
    EnumCfg cfg;
    cfg.run.mem_bound = mem_bound;
    cfg.run.cap = opt.level_cap ? opt.level_cap : P->tuned_cap;
    cfg.run.stats = opt.flags & HUGE_EF_STATS;
    cfg.run.steal = !(opt.flags & HUGE_EF_NO_STEAL);
    cfg.run.limit_ms = opt.time_limit_ms;
    cfg.run.merge_ratio = opt.variant == 1 ? 0u : opt.variant >= 2 ? opt.variant : P->tuned_merge;
    cfg.chunk = opt.chunk_roots ? opt.chunk_roots : P->tuned_chunk;
    cfg.weights = opt.root_weights;
    cfg.target = (size_t)G.warps * 8;
    uint32_t r0 = opt.root_begin, r1 = opt.root_end ? std::min(opt.root_end, G.n) : G.n;
    std::vector<Task> fixed;
    int64_t nroots = 0;
    if (opt.roots) {
        for (uint64_t i = 0; i < opt.nroots; i++) {
            if (opt.roots[i] >= G.n) return fail(HUGE_EINVAL, "root id out of range");
            fixed.push_back({0, opt.roots[i], opt.roots[i] + 1});
        }
        nroots = (int64_t)opt.nroots;
    } else {
        nroots = r1 > r0 ? (int64_t)(r1 - r0) : 0;
    }
    RunResult agg;
    unsigned __int128 count = 0;
    int rc;
    if (P->join) {
        if (opt.roots || opt.root_begin || opt.root_end)
            return fail(HUGE_EINVAL, "root restrictions are not supported for PUSH-JOIN plans");
        int64_t side_rows[2] = {0, 0};
        rc = join_enumerate(P, mode, cfg, sink, s, &count, &agg, side_rows);
        if (rc) return rc;
        rc = count_to_i64(count, out_count);
        if (rc) return rc;
        if (st) {
            fill_stats(st, agg, G.n, 0, count, G.warps);
            st->level_rows[0] = side_rows[0];
            st->level_rows[1] = side_rows[1];
            st->level_rows[2] = *out_count;
            st->nlevels = 3;
        }
        return HUGE_OK;
    }
    const Prog &prog = P->chain.prog;
    if (mode == HUGE_COUNT) {
        std::vector<Task> tasks;
        if (opt.roots)
            tasks = fixed;
        else
            make_tasks(G, 0, r0, r1, cfg.chunk, cfg.weights, cfg.target, &tasks);
        if (tasks.empty()) {
            *out_count = 0;
            fill_stats(st, agg, 0, prog.nsteps, 0, G.warps);
            return HUGE_OK;
        }
        rc = run_chains(G, {prog}, tasks, HUGE_COUNT, cfg.run, nullptr, 0, 0, nullptr, s, &agg);
        if (rc) return rc;
        count = agg.counts[0];
    } else {
        rc = list_chain(G, prog, P->Q.k, r0, r1, opt.roots ? &fixed : nullptr, cfg, sink, s, &count, &agg);
        if (rc) return rc;
    }
    rc = count_to_i64(count, out_count);
    if (rc) return rc;
    fill_stats(st, agg, nroots, prog.nsteps, count, G.warps);
    return HUGE_OK;
}

// JSON description of a plan (the form huge_plan_describe returns).
std::string describe_plan(const huge_plan_t *p) {
    std::string d = "{\"how\":\"" + p->how + "\",\"k\":" + std::to_string(p->Q.k) + ",\"po\":[";
    for (size_t i = 0; i < p->po.size(); i++)
        d += (i ? "," : "") + std::string("[") + std::to_string(p->po[i].first) + "," +
             std::to_string(p->po[i].second) + "]";
    d += "]";
    if (p->Q.directed) d += ",\"directed\":true";
    bool labelled = false;
    for (int v = 0; v < p->Q.k; v++) labelled = labelled || p->Q.lab[v] != kAnyLabel;
    if (labelled) {
        d += ",\"labels\":[";
        for (int v = 0; v < p->Q.k; v++)
            d += (v ? "," : "") + (p->Q.lab[v] == kAnyLabel ? std::string("null") : std::to_string(p->Q.lab[v]));
        d += "]";
    }
    const double ec = std::isfinite(p->est_cost) ? std::min(p->est_cost, 1e300) : -1.0;
    d += ",\"est_cost\":" + std::to_string(ec);
    if (p->join) {
        d += ",\"op\":\"PUSH-JOIN\",\"left_vertices\":[";
        for (int c = 0; c < p->js.nl; c++) d += (c ? "," : "") + std::to_string(p->l_global[c]);
        d += "],\"right_vertices\":[";
        for (int c = 0; c < p->js.nr; c++) d += (c ? "," : "") + std::to_string(p->r_global[c]);
        d += "],\"left\":" + describe_chain(p->left) + ",\"right\":" + describe_chain(p->right) + "}";
    } else {
        d += ",\"op\":\"EXTEND-CHAIN\",\"chain\":" + describe_chain(p->chain) + "}";
    }
    return d;
}

int copy_out(const std::string &d, char *buf, size_t len) {
    const size_t n = std::min(len - 1, d.size());
    memcpy(buf, d.data(), n);
    buf[n] = 0;
    return HUGE_OK;
}

// The PUSH-JOIN spec as JSON: key and non-key columns of each side (in that side's own
// vertex numbering), the cross-side partial-order pairs and the output columns.
std::string describe_join_spec(const JoinSpec &js) {
    auto arr = [](const int *a, int n) {
        std::string r = "[";
        for (int i = 0; i < n; i++) r += (i ? "," : "") + std::to_string(a[i]);
        return r + "]";
    };
    return "{\"lkey\":" + arr(js.lkey, js.nkey) + ",\"rkey\":" + arr(js.rkey, js.nkey) +
           ",\"nonkey_l\":" + arr(js.nonkey_l, js.n_nonkey_l) + ",\"nonkey_r\":" + arr(js.nonkey_r, js.n_nonkey_r) +
           ",\"lr_l\":" + arr(js.lr_l, js.n_lr) + ",\"lr_r\":" + arr(js.lr_r, js.n_lr) +
           ",\"rl_r\":" + arr(js.rl_r, js.n_rl) + ",\"rl_l\":" + arr(js.rl_l, js.n_rl) +
           ",\"out_col_l\":" + arr(js.out_col_l, js.nl) + ",\"out_col_r\":" + arr(js.out_col_r, js.nr) + "}";
}

}  // namespace

extern "C" {

int huge_plan(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *order,
              const uint32_t *po_pairs, int32_t npo, uint32_t flags, huge_plan_t **out) {
    return build_plan(g, nq, q_edges, mq, order, po_pairs, npo, flags, nullptr, out);
}

int huge_plan_ex(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *order,
                 const uint32_t *po_pairs, int32_t npo, uint32_t flags, const huge_mlp_t *model, huge_plan_t **out) {
    return build_plan(g, nq, q_edges, mq, order, po_pairs, npo, flags, model, out);
}

int huge_plan_labeled(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq,
                      const uint32_t *q_labels, const uint32_t *order, const uint32_t *po_pairs, int32_t npo,
                      uint32_t flags, const huge_mlp_t *model, huge_plan_t **out) {
    return build_plan(g, nq, q_edges, mq, order, po_pairs, npo, flags, model, out, q_labels);
}

int huge_plan_offline(uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *order,
                      const uint32_t *po_pairs, int32_t npo, uint32_t flags, const double *card, double edges_g,
                      char *buf, size_t len) {
    return huge_plan_offline_labeled(nq, q_edges, mq, nullptr, nullptr, 0, order, po_pairs, npo, flags, card,
                                     edges_g, buf, len);
}

int huge_plan_offline_labeled(uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *q_labels,
                              const uint32_t *lstart, uint32_t nlabels, const uint32_t *order,
                              const uint32_t *po_pairs, int32_t npo, uint32_t flags, const double *card,
                              double edges_g, char *buf, size_t len) {
    g_err.clear();
    if (q_labels && (!lstart || nlabels == 0)) return fail(HUGE_EINVAL, "query labels need the label ranges");
    if (!buf || len == 0) return fail(HUGE_EINVAL, "null output buffer");
    if (flags & HUGE_PLAN_LEARNED) return fail(HUGE_EINVAL, "huge_plan_offline takes the cardinalities as given");
    if (!order && !card) return fail(HUGE_EINVAL, "without an order the optimiser needs the cardinalities");
    QueryG Q;
    std::string err;
    int rc = parse_query(nq, q_edges, mq, &Q, &err, (flags & HUGE_PLAN_DIRECTED) != 0);
    if (rc) return fail(rc, err);
    if (q_labels) {  // before the partial order: an automatic one breaks only label-preserving symmetry
        for (uint32_t v = 0; v < nq; v++) Q.lab[v] = q_labels[v];
        for (uint32_t L = 0; L < nlabels; L++)
            if (lstart[L] > lstart[L + 1]) return fail(HUGE_EINVAL, "label ranges must not decrease");
    }
    std::vector<std::pair<int, int>> po;
    rc = parse_partial_order(Q, po_pairs, npo, &po);
    if (rc) return rc;
    huge_plan_t P;
    P.Q = Q;
    P.po = po;
    if (q_labels) P.offline_lstart.assign(lstart, lstart + nlabels + 1);
    if (!po_closure(Q.k, po, P.lt)) return fail(HUGE_EINVAL, "the partial order has a cycle (not a DAG)");
    const bool tree_verify = flags & HUGE_PLAN_TREE_VERIFY;
    if (order) {
        std::vector<int> ord(order, order + nq);
        rc = check_order(Q, ord, &err);
        if (rc) return fail(rc, err);
        P.chain = build_chain(Q, ord, P.lt, tree_verify, plan_labels(&P));
        P.how = "given";
    } else {
        const bool allow_ext = !(flags & HUGE_PLAN_FORCE_JOIN);
        const bool allow_join = !(flags & (HUGE_PLAN_EXTEND_ONLY | HUGE_PLAN_TREE_VERIFY));
        DpResult dp = optimise(Q, P.lt, [&](uint32_t m) { return card[m]; }, edges_g, allow_ext, allow_join);
        rc = finish_plan(&P, dp, flags, tree_verify);
        if (rc) return rc;
        P.how = "offline";
    }
    std::string d = describe_plan(&P);
    if (P.join) d = d.substr(0, d.size() - 1) + ",\"join_spec\":" + describe_join_spec(P.js) + "}";
    if (d.size() + 1 > len) return fail(HUGE_ERANGE, "description longer than the buffer");
    return copy_out(d, buf, len);
}

int huge_plan_free(huge_plan_t *p) {
    delete p;
    return HUGE_OK;
}

int huge_plan_describe(const huge_plan_t *p, char *buf, size_t len) {
    if (!p || !buf || len == 0) return fail(HUGE_EINVAL, "null argument");
    return copy_out(describe_plan(p), buf, len);
}

int huge_plan_timing(const huge_plan_t *p, double *plan_s, double *estimate_s) {
    if (!p) return fail(HUGE_EINVAL, "null plan");
    if (plan_s) *plan_s = p->plan_s;
    if (estimate_s) *estimate_s = p->est_s;
    return HUGE_OK;
}

int huge_enumerate(const huge_plan_t *p, int mode, uint64_t mem_bound_bytes, const huge_sink_t *sink, void *stream,
                   int64_t *out_count) {
    return enumerate_impl(p, mode, mem_bound_bytes, sink, stream, nullptr, out_count, nullptr);
}

int huge_enumerate_ex(const huge_plan_t *p, int mode, uint64_t mem_bound_bytes, const huge_sink_t *sink, void *stream,
                      const huge_enum_opts_t *opts, int64_t *out_count, huge_stats_t *stats) {
    return enumerate_impl(p, mode, mem_bound_bytes, sink, stream, opts, out_count, stats);
}

int huge_enumerate_batch(const huge_plan_t *const *plans, uint32_t nplans, uint64_t mem_bound_bytes, void *stream,
                         int64_t *out_counts, huge_stats_t *stats) {
    return huge_enumerate_batch_ex(plans, nplans, mem_bound_bytes, stream, nullptr, out_counts, nullptr, stats);
}

int huge_enumerate_batch_ex(const huge_plan_t *const *plans, uint32_t nplans, uint64_t mem_bound_bytes, void *stream,
                            const huge_enum_opts_t *opts, int64_t *out_counts, int64_t *level_rows,
                            huge_stats_t *stats) {
    g_err.clear();
    if (!plans || !out_counts || nplans == 0) return fail(HUGE_EINVAL, "null argument or empty batch");
    DevGraph *G = plans[0] ? plans[0]->G : nullptr;
    if (!G) return fail(HUGE_EINVAL, "null plan");
    std::vector<Prog> progs;
    RunCfg rcfg;
    rcfg.mem_bound = mem_bound_bytes;
    // tasks of every query with an estimate of their work: the roots' weight 1 + degree times
    // the query's estimated cost per unit of root weight (Alg. 1's cost when the plan has one)
    struct WTask {
        Task t;
        double work;
    };
    std::vector<WTask> wt;
    uint64_t nroots_all = 0;
    const double total_weight = (double)G->n + (double)G->h_off[G->n];
    for (uint32_t q = 0; q < nplans; q++) {
        const huge_plan_t *P = plans[q];
        if (!P || P->G != G) return fail(HUGE_EINVAL, "every plan of a batch must be on the same graph");
        if (P->join) return fail(HUGE_EINVAL, "batched enumeration takes EXTEND-chain plans only");
        huge_enum_opts_t o;
        memset(&o, 0, sizeof(o));
        if (opts) o = opts[q];
        if (o.per_root) return fail(HUGE_EINVAL, "per_root is reserved and must be NULL");
        progs.push_back(P->chain.prog);
        rcfg.caps.push_back(o.level_cap ? o.level_cap : P->tuned_cap);
        rcfg.merges.push_back(o.variant == 1 ? 0u : o.variant >= 2 ? o.variant : P->tuned_merge);
        if (o.flags & HUGE_EF_STATS) rcfg.stats = true;
        if (o.flags & HUGE_EF_NO_STEAL) rcfg.steal = false;
        rcfg.limit_ms = std::max(rcfg.limit_ms, o.time_limit_ms);
        const double per_weight = P->est_cost > 0 && std::isfinite(P->est_cost) ? P->est_cost / total_weight : 1.0;
        auto weight = [&](uint32_t a, uint32_t b) { return (double)(b - a) + (double)(G->h_off[b] - G->h_off[a]); };
        std::vector<Task> tq;
        if (o.roots) {
            for (uint64_t i = 0; i < o.nroots; i++) {
                if (o.roots[i] >= G->n) return fail(HUGE_EINVAL, "root id out of range");
                tq.push_back({q, o.roots[i], o.roots[i] + 1});
            }
            nroots_all += o.nroots;
        } else {
            const uint32_t r0 = o.root_begin, r1 = o.root_end ? std::min(o.root_end, G->n) : G->n;
            const uint32_t chunk = o.chunk_roots ? o.chunk_roots : P->tuned_chunk;
            // the same chunking as a plain launch of this query: a heavy query keeps fine chunks
            make_tasks(*G, q, r0, r1, chunk, o.root_weights, (size_t)G->warps * 8, &tq);
            nroots_all += r1 > r0 ? r1 - r0 : 0;
        }
        for (const Task &t : tq) wt.push_back({t, weight(t.r0, t.r1) * per_weight});
    }
    // heaviest first across all queries (longest-processing-time order): the light tasks of
    // every query fill the tail of the launch instead of one query's tail idling the GPU
    std::stable_sort(wt.begin(), wt.end(), [](const WTask &a, const WTask &b) { return a.work > b.work; });
    std::vector<Task> tasks;
    tasks.reserve(wt.size());
    for (const WTask &w : wt) tasks.push_back(w.t);
    RunResult rr;
    std::vector<int64_t> res(nplans, 0);
    if (!tasks.empty()) {
        int rc = run_chains(*G, progs, tasks, HUGE_COUNT, rcfg, nullptr, 0, 0, nullptr, (cudaStream_t)stream, &rr);
        if (rc) return rc;
        for (uint32_t q = 0; q < nplans; q++) {
            rc = count_to_i64(rr.counts[q], &res[q]);
            if (rc) return rc;
        }
    }
    memcpy(out_counts, res.data(), sizeof(int64_t) * nplans);
    if (level_rows) {  // per plan: rows after each operator, the last one's = the count
        for (uint32_t q = 0; q < nplans; q++) {
            for (int l = 0; l < kMaxSteps; l++)
                level_rows[(size_t)q * kMaxSteps + l] =
                    tasks.empty() ? 0 : (int64_t)rr.lvl_rows[(size_t)q * kMaxSteps + l];
            const int ns = progs[q].nsteps;
            if (ns > 0 && ns < kMaxSteps) level_rows[(size_t)q * kMaxSteps + ns] = res[q];
        }
    }
    if (stats) {
        fill_stats(stats, rr, (int64_t)nroots_all, 0, 0, G->warps);
        stats->nlevels = 0;
    }
    return HUGE_OK;
}

int huge_autotune(huge_plan_t *const *plans, uint32_t nplans, uint64_t mem_bound_bytes, double budget_ms, void *stream,
                  uint32_t *level_cap, uint32_t *chunk_roots) {
    g_err.clear();
    if (!plans || nplans == 0) return fail(HUGE_EINVAL, "null argument or empty plan list");
    // candidate settings: rows per level per warp (BFS width), root chunking, and the
    // intersection variant of the last operator (0 = binary search only, r = merge-path ratio)
    const uint32_t caps[] = {128, 512, 2048};
    const uint32_t chunks[] = {0, 16};
    const uint32_t merges[] = {0, 4, 16};
    double best = -1, spent = 0;
    uint32_t best_cap = 0, best_chunk = 0, best_merge = 8;
    std::vector<uint32_t> save_cap(nplans), save_chunk(nplans), save_merge(nplans);
    for (uint32_t i = 0; i < nplans; i++) {
        save_cap[i] = plans[i]->tuned_cap;
        save_chunk[i] = plans[i]->tuned_chunk;
        save_merge[i] = plans[i]->tuned_merge;
    }
    auto restore = [&]() {
        for (uint32_t i = 0; i < nplans; i++) {
            plans[i]->tuned_cap = save_cap[i];
            plans[i]->tuned_chunk = save_chunk[i];
            plans[i]->tuned_merge = save_merge[i];
        }
    };
    for (uint32_t mg : merges)
        for (uint32_t c : caps)
            for (uint32_t ch : chunks) {
                if (best >= 0 && spent > budget_ms) break;
                for (uint32_t i = 0; i < nplans; i++) {
                    plans[i]->tuned_cap = c;
                    plans[i]->tuned_chunk = ch;
                    plans[i]->tuned_merge = mg;
                }
                huge_stats_t st;
                int rc;
                if (nplans == 1) {
                    int64_t cnt = 0;
                    rc = enumerate_impl(plans[0], HUGE_COUNT, mem_bound_bytes, nullptr, stream, nullptr, &cnt, &st);
                } else {
                    std::vector<int64_t> cnt(nplans);
                    rc = huge_enumerate_batch(plans, nplans, mem_bound_bytes, stream, cnt.data(), &st);
                }
                if (rc == HUGE_ENOMEM) continue;
                if (rc) {
                    restore();
                    return rc;
                }
                spent += st.device_ms;
                if (best < 0 || st.device_ms < best) {
                    best = st.device_ms;
                    best_cap = st.level_cap;
                    best_chunk = ch;
                    best_merge = mg;
                }
            }
    if (best < 0) {
        restore();
        return fail(HUGE_ENOMEM, "no autotuner candidate fits mem_bound");
    }
    for (uint32_t i = 0; i < nplans; i++) {
        plans[i]->tuned_cap = best_cap;
        plans[i]->tuned_chunk = best_chunk;
        plans[i]->tuned_merge = best_merge;
    }
    // the degree bucket of the bit-probe variant: the graph's hub threshold at half and twice
    // its current value (the bitmaps are rebuilt for each candidate; the fastest stays)
    DevGraph &G = *plans[0]->G;
    if (G.hub_count && spent <= budget_ms) {
        const uint32_t d0 = G.hub_min_deg;
        const uint64_t bytes0 = kDefaultHubBytes;
        uint32_t best_deg = d0;
        for (uint32_t d : {std::max(2u, d0 / 2), d0 * 2}) {
            if (spent > budget_ms) break;
            if (build_hub_bitmaps(G, d, bytes0) != HUGE_OK) {
                set_error("");
                continue;
            }
            huge_stats_t st;
            int rc;
            if (nplans == 1) {
                int64_t cnt = 0;
                rc = enumerate_impl(plans[0], HUGE_COUNT, mem_bound_bytes, nullptr, stream, nullptr, &cnt, &st);
            } else {
                std::vector<int64_t> cnt(nplans);
                rc = huge_enumerate_batch(plans, nplans, mem_bound_bytes, stream, cnt.data(), &st);
            }
            if (rc) {
                set_error("");
                continue;
            }
            spent += st.device_ms;
            if (st.device_ms < best) {
                best = st.device_ms;
                best_deg = d;
            }
        }
        if (G.hub_min_deg != best_deg || G.hub_count == 0) {
            const int rc = build_hub_bitmaps(G, best_deg, bytes0);
            if (rc) return rc;
        }
    }
    if (level_cap) *level_cap = best_cap;
    if (chunk_roots) *chunk_roots = best_chunk;
    return HUGE_OK;
}

int huge_plan_features(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq,
                       const uint32_t *po_pairs, int32_t npo, uint32_t mask, float *out) {
    g_err.clear();
    if (!g || !g->G || !out) return fail(HUGE_EINVAL, "null argument");
    QueryG Q;
    std::string err;
    int rc = parse_query(nq, q_edges, mq, &Q, &err, g->G->directed);
    if (rc) return fail(rc, err);
    std::vector<std::pair<int, int>> po;
    rc = parse_partial_order(Q, po_pairs, npo, &po);
    if (rc) return rc;
    uint8_t lt[kMaxK][kMaxK];
    if (!po_closure(Q.k, po, lt)) return fail(HUGE_EINVAL, "the partial order has a cycle (not a DAG)");
    if (mask == 0 || mask >= (1u << Q.k)) return fail(HUGE_EINVAL, "mask must be a non-empty vertex set");
    subquery_features(Q, lt, mask, g->G->gstats, out);
    return HUGE_OK;
}

}  // extern "C"
