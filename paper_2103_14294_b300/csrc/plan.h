// Host planner interfaces (plan.cpp, api.cu).
#pragma once

#include <array>
#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace huge {

struct QueryG {
    int k;
    uint8_t a[kMaxK][kMaxK];     // underlying undirected adjacency
    uint32_t lab[kMaxK];         // query vertex labels (kAnyLabel: any data vertex)
    bool directed;               // arcs: arc[u][v] = 1 for a query arc u -> v
    uint8_t arc[kMaxK][kMaxK];
};

struct DpResult {
    std::vector<double> cost_of, cards;
    std::vector<int> last_of;
    double extend_cost = -1, join_cost = -1;
    uint32_t jl = 0, jr = 0;
};

// directed: the pairs are arcs (a -> b); a pair and its reverse may both be given
int parse_query(uint32_t nq, const uint32_t *q_edges, uint32_t mq, QueryG *Q, std::string *err,
                bool directed = false);
std::vector<std::array<int, kMaxK>> automorphisms(const QueryG &Q);
std::vector<std::pair<int, int>> symmetry_breaking_po(const QueryG &Q);
bool po_closure(int k, const std::vector<std::pair<int, int>> &po, uint8_t lt[kMaxK][kMaxK]);
int check_order(const QueryG &Q, const std::vector<int> &order, std::string *err);
// lstart: the data graph's label ranges (label L = ids [lstart[L], lstart[L+1])), or null /
// empty for an unlabelled graph; labelled query vertices get their label's id range.
Chain build_chain(const QueryG &Q, const std::vector<int> &order, const uint8_t lt[kMaxK][kMaxK],
                  bool tree_verify, const std::vector<uint32_t> *lstart = nullptr);
// [lo, hi) ids of a query vertex with label `lab` (the whole id space for kAnyLabel or an
// unlabelled graph, an empty range for a label the graph does not have).
void label_range(const std::vector<uint32_t> *lstart, uint32_t lab, uint32_t *lo, uint32_t *hi);
DpResult optimise(const QueryG &Q, const uint8_t lt[kMaxK][kMaxK],
                  const std::function<double(uint32_t)> &card, double edges_g, bool allow_extend_top,
                  bool allow_join_top);
std::vector<int> recover_order(const QueryG &Q, const uint8_t lt[kMaxK][kMaxK], const DpResult &r,
                               uint32_t m);
QueryG sub_query(const QueryG &Q, uint32_t mask, const uint8_t lt[kMaxK][kMaxK],
                 uint8_t sub_lt[kMaxK][kMaxK], int *local_of, int *global_of);
std::vector<int> bfs_order(const QueryG &Q, const uint8_t lt[kMaxK][kMaxK]);
std::string describe_chain(const Chain &c);

// Features of a sub-query (mask) of Q for the learned cardinality estimator (64 floats).
void subquery_features(const QueryG &Q, const uint8_t lt[kMaxK][kMaxK], uint32_t mask,
                       const std::vector<float> &gstats, float *out64);

}  // namespace huge

// Opaque plan object of the C ABI.
struct huge_plan {
    huge::DevGraph *G = nullptr;
    huge::QueryG Q;
    uint8_t lt[huge::kMaxK][huge::kMaxK];
    std::vector<std::pair<int, int>> po;
    bool join = false;
    huge::Chain chain;             // EXTEND-chain plan (join == false)
    huge::Chain left, right;       // PUSH-JOIN sides (join == true)
    uint32_t lmask = 0, rmask = 0;
    int l_global[huge::kMaxK], r_global[huge::kMaxK];
    huge::JoinSpec js;
    double est_cost = 0;
    double plan_s = 0, est_s = 0;
    uint32_t tuned_cap = 0, tuned_chunk = 0, tuned_merge = 8;
    std::string how;               // "given", "plain", "learned", ...
    std::vector<uint32_t> offline_lstart;  // label ranges of an offline plan (no graph)
};

struct huge_graph {
    huge::DevGraph *G = nullptr;
};
