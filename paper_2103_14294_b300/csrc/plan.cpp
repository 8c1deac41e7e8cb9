// Query analysis and planning (host).
//  * automorphisms and the symmetry-breaking partial order (Sec. 2; the paper cites Grochow &
//    Kellis): fix the smallest vertex with a non-trivial orbit below the rest of its orbit,
//    keep only automorphisms that fix it, repeat;
//  * Alg. 1 (OptimalExecutionPlan): dynamic programming over connected sub-queries with the
//    cost sum of |R(q')| plus the communication term of each join, and Eq. 3 deciding between
//    the pulling EXTEND (complete star join) and the pushing hash join (PUSH-JOIN);
//  * Alg. 2 (ExecutionPlanTranslation): an EXTEND chain becomes a device program of steps,
//    each with its extend index Ext (Sec. 4.2) and the partial-order bounds it must obey.
#include "plan.h"
#include <array>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <sstream>

namespace huge {

constexpr double kDownPenalty = 0.25;   // extension bounded only from above
constexpr double kUpperPenalty = 0.05;  // extension with an upper bound besides a lower one

int parse_query(uint32_t nq, const uint32_t *q_edges, uint32_t mq, QueryG *Q, std::string *err, bool directed) {
    if (nq < 2 || nq > (uint32_t)kMaxK) {
        *err = "query must have 2.." + std::to_string(kMaxK) + " vertices";
        return HUGE_EINVAL;
    }
    if (mq && !q_edges) {
        *err = "null query edge list";
        return HUGE_EINVAL;
    }
    memset(Q, 0, sizeof(*Q));
    Q->k = (int)nq;
    Q->directed = directed;
    for (int v = 0; v < kMaxK; v++) Q->lab[v] = kAnyLabel;
    for (uint32_t i = 0; i < mq; i++) {
        const uint32_t a = q_edges[2 * i], b = q_edges[2 * i + 1];
        if (a >= nq || b >= nq || a == b) {
            *err = "bad query edge (" + std::to_string(a) + "," + std::to_string(b) + ")";
            return HUGE_EINVAL;
        }
        if (directed) Q->arc[a][b] = 1;
        Q->a[a][b] = Q->a[b][a] = 1;
    }
    // connectivity
    uint32_t seen = 1, frontier = 1;
    while (frontier) {
        uint32_t next = 0;
        for (int v = 0; v < Q->k; v++)
            if (frontier >> v & 1)
                for (int u = 0; u < Q->k; u++)
                    if (Q->a[v][u] && !(seen >> u & 1)) next |= 1u << u;
        seen |= next;
        frontier = next;
    }
    if (seen != (1u << nq) - 1) {
        *err = "query graph is not connected";
        return HUGE_EINVAL;
    }
    if (directed)  // one intersected list per incident arc: at most kMaxExt per vertex
        for (int v = 0; v < Q->k; v++) {
            int arcs = 0;
            for (int u = 0; u < Q->k; u++) arcs += Q->arc[v][u] + Q->arc[u][v];
            if (arcs > kMaxExt) {
                *err = "a query vertex has more than " + std::to_string(kMaxExt) + " incident arcs";
                return HUGE_EINVAL;
            }
        }
    return HUGE_OK;
}

std::vector<std::array<int, kMaxK>> automorphisms(const QueryG &Q) {
    std::vector<std::array<int, kMaxK>> out;
    std::array<int, kMaxK> p;
    for (int i = 0; i < kMaxK; i++) p[i] = i;
    do {
        bool ok = true;
        for (int u = 0; u < Q.k && ok; u++) ok = Q.lab[p[u]] == Q.lab[u];  // label-preserving
        for (int u = 0; u < Q.k && ok; u++)
            for (int v = u + 1; v < Q.k && ok; v++)
                if (Q.a[u][v] != Q.a[p[u]][p[v]]) ok = false;
        for (int u = 0; u < Q.k && ok && Q.directed; u++)  // arc-preserving
            for (int v = 0; v < Q.k && ok; v++)
                if (Q.arc[u][v] != Q.arc[p[u]][p[v]]) ok = false;
        if (ok) out.push_back(p);
    } while (std::next_permutation(p.begin(), p.begin() + Q.k));
    return out;
}

std::vector<std::pair<int, int>> symmetry_breaking_po(const QueryG &Q) {
    auto group = automorphisms(Q);
    std::vector<std::pair<int, int>> po;
    while (group.size() > 1) {
        int v = -1;
        for (int x = 0; x < Q.k && v < 0; x++)
            for (auto &g : group)
                if (g[x] != x) {
                    v = x;
                    break;
                }
        uint32_t orbit = 0;
        for (auto &g : group) orbit |= 1u << g[v];
        for (int u = 0; u < Q.k; u++)
            if ((orbit >> u & 1) && u != v) po.push_back({v, u});
        std::vector<std::array<int, kMaxK>> stab;
        for (auto &g : group)
            if (g[v] == v) stab.push_back(g);
        group.swap(stab);
    }
    return po;
}

bool po_closure(int k, const std::vector<std::pair<int, int>> &po, uint8_t lt[kMaxK][kMaxK]) {
    memset(lt, 0, kMaxK * kMaxK);
    for (auto &pr : po) lt[pr.first][pr.second] = 1;
    for (int m = 0; m < k; m++)
        for (int a = 0; a < k; a++)
            if (lt[a][m])
                for (int b = 0; b < k; b++)
                    if (lt[m][b]) lt[a][b] = 1;
    for (int a = 0; a < k; a++)
        if (lt[a][a]) return false;
    return true;
}

static bool connected_mask(const QueryG &Q, uint32_t mask) {
    if (!mask) return false;
    const uint32_t start = mask & (~mask + 1);
    uint32_t seen = start, frontier = start;
    while (frontier) {
        uint32_t next = 0;
        for (int v = 0; v < Q.k; v++)
            if (frontier >> v & 1)
                for (int u = 0; u < Q.k; u++)
                    if ((mask >> u & 1) && Q.a[v][u] && !(seen >> u & 1)) next |= 1u << u;
        seen |= next;
        frontier = next;
    }
    return seen == mask;
}

int check_order(const QueryG &Q, const std::vector<int> &order, std::string *err) {
    if ((int)order.size() != Q.k) {
        *err = "order must list every query vertex once";
        return HUGE_EINVAL;
    }
    uint32_t seen = 0;
    for (int j = 0; j < Q.k; j++) {
        const int v = order[j];
        if (v < 0 || v >= Q.k || (seen >> v & 1)) {
            *err = "order must be a permutation of the query vertices";
            return HUGE_EINVAL;
        }
        if (j > 0) {
            bool adj = false;
            for (int t = 0; t < j; t++) adj = adj || Q.a[v][order[t]];
            if (!adj) {
                *err = "every prefix of the matching order must be connected (position " + std::to_string(j) + ")";
                return HUGE_EINVAL;
            }
        }
        seen |= 1u << v;
    }
    return HUGE_OK;
}

// Alg. 2 for an EXTEND chain: position j binds order[j]; EXTEND(Ext) intersects the lists of
// the earlier-bound query neighbours (complete star join, Def. 3.1), the partial order becomes
// strict lower/upper bounds, and injectivity (Alg. 4) is checked only where neither adjacency
// nor a strict bound already excludes equality. With tree_verify, each EXTEND uses only the
// spanning-tree parent and the remaining edges are checked by a verify-only EXTEND (Sec. 5.2).
void label_range(const std::vector<uint32_t> *lstart, uint32_t lab, uint32_t *lo, uint32_t *hi) {
    *lo = 0;
    *hi = 0xffffffffu;
    if (lab == kAnyLabel || !lstart || lstart->size() < 2) return;
    if ((size_t)lab + 1 >= lstart->size()) {  // a label no data vertex carries
        *lo = *hi = 0;
        return;
    }
    *lo = (*lstart)[lab];
    *hi = (*lstart)[lab + 1];
}

Chain build_chain(const QueryG &Q, const std::vector<int> &order, const uint8_t lt[kMaxK][kMaxK],
                  bool tree_verify, const std::vector<uint32_t> *lstart) {
    Chain c;
    c.k = Q.k;
    c.order = order;
    Prog &P = c.prog;
    memset(&P, 0, sizeof(P));
    P.width_out = Q.k;
    for (int j = 0; j < Q.k; j++) P.col_of_pos[j] = (uint8_t)order[j];
    label_range(lstart, Q.lab[order[0]], &P.root_lo, &P.root_hi);
    int t = 0;
    for (int j = 1; j < Q.k; j++) {
        const int v = order[j];
        StepDesc &s = P.steps[++t];
        s.kind = kExtend;
        s.w = (uint8_t)j;
        label_range(lstart, Q.lab[v], &s.clo, &s.chi);
        uint32_t excl = 0;
        int parent = -1;
        for (int p = 0; p < j; p++)
            if (Q.a[v][order[p]]) {
                if (tree_verify && parent >= 0) continue;
                if (parent < 0) parent = p;
                excl |= 1u << p;
                if (!Q.directed) {
                    s.ext[s.n_ext++] = (uint8_t)p;
                    continue;
                }
                // arc order[p] -> v: v in the out-list of f(p); arc v -> order[p]: its in-list
                for (int d = 0; d < 2; d++) {
                    const bool has = d ? Q.arc[v][order[p]] : Q.arc[order[p]][v];
                    if (!has || s.n_ext >= kMaxExt) continue;
                    if (d) s.dirs |= (uint8_t)(1u << s.n_ext);
                    s.ext[s.n_ext++] = (uint8_t)p;
                }
            }
        for (int p = 0; p < j; p++) {
            if (lt[order[p]][v]) {
                s.lo[s.n_lo++] = (uint8_t)p;
                excl |= 1u << p;
            } else if (lt[v][order[p]]) {
                s.hi[s.n_hi++] = (uint8_t)p;
                excl |= 1u << p;
            }
        }
        for (int p = 0; p < j; p++)
            if (!(excl >> p & 1)) s.inj[s.n_inj++] = (uint8_t)p;
        if (tree_verify) {
            StepDesc vs;
            memset(&vs, 0, sizeof(vs));
            vs.chi = 0xffffffffu;
            vs.kind = kVerify;
            vs.w = (uint8_t)(j + 1);
            for (int p = 0; p < j; p++)
                if (Q.a[v][order[p]] && p != parent) {
                    for (int d = 0; d < (Q.directed ? 2 : 1); d++) {
                        if (Q.directed && !(d ? Q.arc[v][order[p]] : Q.arc[order[p]][v])) continue;
                        if (vs.n_ext >= kMaxExt) continue;
                        if (d) vs.dirs |= (uint8_t)(1u << vs.n_ext);
                        vs.ext[vs.n_ext] = (uint8_t)p;
                        vs.ext2[vs.n_ext] = (uint8_t)j;
                        vs.n_ext++;
                    }
                }
            if (vs.n_ext) P.steps[++t] = vs;
        }
    }
    P.nsteps = t;
    P.part_mod = 1;
    return c;
}

// ------------------------------------------------------------------------------------------
// Alg. 1 over connected induced sub-queries (bitmasks of query vertices).
// ------------------------------------------------------------------------------------------
DpResult optimise(const QueryG &Q, const uint8_t lt[kMaxK][kMaxK], const std::function<double(uint32_t)> &card,
                  double edges_g, bool allow_extend_top, bool allow_join_top) {
    const uint32_t full = (1u << Q.k) - 1;
    std::vector<double> cost(full + 1, -1.0);
    std::vector<int> last(full + 1, -1);
    std::vector<double> cards(full + 1, -1.0);
    auto C = [&](uint32_t m) {
        if (cards[m] < 0) cards[m] = std::max(0.0, card(m));
        return cards[m];
    };
    for (uint32_t m = 1; m <= full; m++) {
        const int pc = __builtin_popcount(m);
        if (pc < 2 || !connected_mask(Q, m)) continue;
        if (pc == 2) {  // an edge: a join unit scanned directly
            cost[m] = C(m);
            continue;
        }
        if (m == full && !allow_extend_top) continue;
        for (int v = 0; v < Q.k; v++) {
            if (!(m >> v & 1)) continue;
            const uint32_t l = m & ~(1u << v);
            if (cost[l] < 0) continue;
            // complete star join (v; N(v) in l): pulling wco join = EXTEND; the star itself is
            // never materialised, the pull term is k|E_G| with k = 1 machine
            double c = cost[l] + C(m) + edges_g;
            // Alg. 1 charges |R(q')| only, so plans that differ in the direction of their
            // partial-order bounds tie (every order of a clique does). On degree-ordered ids an
            // extension bounded only from above scans the long lower neighbourhoods of hubs;
            // it is charged kDownPenalty x |R(q')| extra. An extension bounded from both sides
            // keeps a range between an early (small) and a late vertex, where an upward-only
            // order restricts to above its latest (largest) vertex: it is charged
            // kUpperPenalty x |R(q')| (measured: the upward 4-clique order runs 25% faster).
            // Both only decide ties.
            bool lo = false, hi = false;
            for (int u = 0; u < Q.k; u++)
                if (l >> u & 1) {
                    lo = lo || lt[u][v];
                    hi = hi || lt[v][u];
                }
            if (hi) c += (lo ? kUpperPenalty : kDownPenalty) * C(m);
            if (cost[m] < 0 || c < cost[m]) {
                cost[m] = c;
                last[m] = v;
            }
        }
    }
    DpResult r;
    r.extend_cost = cost[full];
    // PUSH-JOIN at the top: q = q_l JOIN q_r on K = V_l & V_r (hash join, pushing: Eq. 3 case 3)
    r.join_cost = -1;
    if (allow_join_top && Q.k >= 4) {
        for (uint32_t L = 1; L < full; L++) {
            if (cost[L] < 0) continue;
            for (uint32_t R = L; R < full; R++) {  // R >= L avoids mirrored pairs
                if ((L | R) != full || cost[R] < 0) continue;
                const uint32_t K = L & R;
                if (!K || L == K || R == K || __builtin_popcount(K) > 4) continue;
                bool ok = true;
                for (int a = 0; a < Q.k && ok; a++)
                    for (int b = 0; b < Q.k && ok; b++) {
                        if (!Q.a[a][b]) continue;
                        if ((K >> a & 1) && (K >> b & 1)) ok = false;               // key edges
                        if ((L & ~K) >> a & 1 && (R & ~K) >> b & 1) ok = false;    // uncovered
                    }
                if (!ok) continue;
                const double c = cost[L] + cost[R] + C(full) + C(L) + C(R);
                if (r.join_cost < 0 || c < r.join_cost) {
                    r.join_cost = c;
                    r.jl = L;
                    r.jr = R;
                }
            }
        }
    }
    r.cost_of = cost;
    r.last_of = last;
    r.cards = cards;
    return r;
}

std::vector<int> recover_order(const QueryG &Q, const uint8_t lt[kMaxK][kMaxK], const DpResult &r, uint32_t m) {
    (void)Q;
    std::vector<int> order;
    uint32_t cur = m;
    while (__builtin_popcount(cur) > 2) {
        const int v = r.last_of[cur];
        order.push_back(v);
        cur &= ~(1u << v);
    }
    int a = __builtin_ctz(cur), b = 31 - __builtin_clz(cur);
    if (lt[b][a]) std::swap(a, b);
    order.push_back(b);
    order.push_back(a);
    std::reverse(order.begin(), order.end());
    return order;
}

// Sub-query induced by `mask`, its vertices renumbered by increasing original id.
QueryG sub_query(const QueryG &Q, uint32_t mask, const uint8_t lt[kMaxK][kMaxK], uint8_t sub_lt[kMaxK][kMaxK],
                 int *local_of, int *global_of) {
    QueryG S;
    memset(&S, 0, sizeof(S));
    S.directed = Q.directed;
    for (int v = 0; v < kMaxK; v++) S.lab[v] = kAnyLabel;
    int k = 0;
    for (int v = 0; v < Q.k; v++)
        if (mask >> v & 1) {
            local_of[v] = k;
            global_of[k] = v;
            S.lab[k] = Q.lab[v];
            k++;
        } else {
            local_of[v] = -1;
        }
    S.k = k;
    memset(sub_lt, 0, kMaxK * kMaxK);
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) {
            S.a[a][b] = Q.a[global_of[a]][global_of[b]];
            S.arc[a][b] = Q.arc[global_of[a]][global_of[b]];
            sub_lt[a][b] = lt[global_of[a]][global_of[b]];
        }
    return S;
}

std::vector<int> bfs_order(const QueryG &Q, const uint8_t lt[kMaxK][kMaxK]) {
    // root: a vertex that the partial order keeps smallest where possible (fewest "greater than")
    int root = 0, best = 1 << 30;
    for (int v = 0; v < Q.k; v++) {
        int above = 0;
        for (int u = 0; u < Q.k; u++) above += lt[u][v];
        if (above < best) {
            best = above;
            root = v;
        }
    }
    std::vector<int> order = {root};
    uint32_t seen = 1u << root;
    while ((int)order.size() < Q.k) {
        // most connections to the already-ordered prefix first (densest EXTEND), then a
        // vertex bounded from below by the prefix (upward extension on degree-ordered ids)
        int bv = -1, bc = -1;
        for (int v = 0; v < Q.k; v++) {
            if (seen >> v & 1) continue;
            int c = 0, lo = 0;
            for (int u : order) {
                c += Q.a[v][u];
                lo |= lt[u][v];
            }
            if (c == 0) continue;
            c = 2 * c + lo;
            if (c > bc) {
                bc = c;
                bv = v;
            }
        }
        order.push_back(bv);
        seen |= 1u << bv;
    }
    return order;
}

std::string describe_chain(const Chain &c) {
    std::ostringstream os;
    os << "{\"order\":[";
    for (size_t i = 0; i < c.order.size(); i++) os << (i ? "," : "") << c.order[i];
    os << "]";
    if (c.prog.root_lo > 0 || c.prog.root_hi != 0xffffffffu)  // a labelled root: its id range
        os << ",\"root\":[" << c.prog.root_lo << "," << c.prog.root_hi << "]";
    os << ",\"steps\":[";
    for (int t = 1; t <= c.prog.nsteps; t++) {
        const StepDesc &s = c.prog.steps[t];
        os << (t > 1 ? "," : "") << "{\"op\":\"" << (s.kind == kExtend ? "EXTEND" : "VERIFY") << "\",\"w\":" << (int)s.w
           << ",\"ext\":[";
        for (int j = 0; j < s.n_ext; j++) os << (j ? "," : "") << (int)s.ext[j];
        os << "]";
        if (s.dirs) {  // directed: 1 = the in-list of that position's vertex
            os << ",\"dirs\":[";
            for (int j = 0; j < s.n_ext; j++) os << (j ? "," : "") << ((s.dirs >> j) & 1);
            os << "]";
        }
        if (s.kind == kVerify) {
            os << ",\"with\":[";
            for (int j = 0; j < s.n_ext; j++) os << (j ? "," : "") << (int)s.ext2[j];
            os << "]";
        }
        os << ",\"lo\":[";
        for (int j = 0; j < s.n_lo; j++) os << (j ? "," : "") << (int)s.lo[j];
        os << "],\"hi\":[";
        for (int j = 0; j < s.n_hi; j++) os << (j ? "," : "") << (int)s.hi[j];
        os << "],\"inj\":[";
        for (int j = 0; j < s.n_inj; j++) os << (j ? "," : "") << (int)s.inj[j];
        os << "]";
        if (s.kind == kExtend && (s.clo > 0 || s.chi != 0xffffffffu))  // a label's id range
            os << ",\"ids\":[" << s.clo << "," << s.chi << "]";
        os << "}";
    }
    os << "]}";
    return os.str();
}

}  // namespace huge

namespace huge {

// 64 features of the sub-query q[mask] (with the partial-order pairs inside it) on graph G:
// graph statistics (10), sub-query size and shape counts, sorted degree sequence, and
// partial-order structure. Invariant under renaming of the query vertices.
void subquery_features(const QueryG &Q, const uint8_t lt[kMaxK][kMaxK], uint32_t mask,
                       const std::vector<float> &gstats, float *x) {
    for (int i = 0; i < 64; i++) x[i] = 0.f;
    for (size_t i = 0; i < gstats.size() && i < 10; i++) x[i] = gstats[i];
    int vs[kMaxK], k = 0;
    for (int v = 0; v < Q.k; v++)
        if (mask >> v & 1) vs[k++] = v;
    int deg[kMaxK] = {0}, m = 0, npo = 0, tri = 0, wedge = 0, c4 = 0;
    int below[kMaxK] = {0}, above[kMaxK] = {0};
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++) {
            if (Q.a[vs[i]][vs[j]]) deg[i]++;
            if (lt[vs[i]][vs[j]]) {
                npo++;
                above[i]++;
                below[j]++;
            }
        }
    for (int i = 0; i < k; i++) m += deg[i];
    m /= 2;
    for (int i = 0; i < k; i++) {
        wedge += deg[i] * (deg[i] - 1) / 2;
        for (int j = i + 1; j < k; j++)
            for (int l = j + 1; l < k; l++)
                if (Q.a[vs[i]][vs[j]] && Q.a[vs[j]][vs[l]] && Q.a[vs[i]][vs[l]]) tri++;
    }
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++) {
            int common = 0;
            for (int l = 0; l < k; l++)
                if (l != i && l != j && Q.a[vs[i]][vs[l]] && Q.a[vs[j]][vs[l]]) common++;
            c4 += common * (common - 1) / 2;
        }
    c4 /= 2;
    int sd[kMaxK];
    for (int i = 0; i < k; i++) sd[i] = deg[i];
    std::sort(sd, sd + k, [](int a, int b) { return a > b; });
    float *f = x + 10;
    f[0] = (float)k;
    f[1] = (float)m;
    f[2] = (float)npo;
    f[3] = (float)tri;
    f[4] = (float)wedge;
    f[5] = (float)c4;
    f[6] = (m == k * (k - 1) / 2) ? 1.f : 0.f;  // clique
    f[7] = (m == k - 1) ? 1.f : 0.f;            // tree
    f[8] = (m == k && sd[0] == 2) ? 1.f : 0.f;  // cycle
    for (int i = 0; i < kMaxK; i++) f[9 + i] = i < k ? (float)sd[i] : 0.f;
    int nmin = 0, nmax = 0, chain = 0;
    for (int i = 0; i < k; i++) {
        if (below[i] == 0 && above[i] > 0) nmin++;
        if (above[i] == 0 && below[i] > 0) nmax++;
        chain = std::max(chain, below[i]);
    }
    f[17] = (float)nmin;
    f[18] = (float)nmax;
    f[19] = (float)chain;
    // size x graph interaction terms (log-scale growth per extension step)
    const float logd = gstats.size() > 2 ? gstats[2] : 0.f, logmax = gstats.size() > 3 ? gstats[3] : 0.f;
    const float m2 = gstats.size() > 8 ? gstats[8] : 0.f;
    f[20] = (float)k * logd;
    f[21] = (float)(k - 1) * logmax;
    f[22] = (float)m * logd;
    f[23] = (float)(m - (k - 1)) * logd;  // closing edges
    f[24] = (float)npo * 0.6931f;         // log 2 per symmetry-breaking pair
    f[25] = (float)tri * logd;
    f[26] = (float)wedge * m2;
    f[27] = (gstats.size() > 1 ? gstats[0] : 0.f) + (float)(k - 1) * logd - (float)(m - (k - 1)) * (gstats.size() > 0 ? gstats[0] : 0.f) * 0.5f;
    for (int i = 0; i < k; i++) f[28 + i] = (float)(above[i] - below[i]);
    x[63] = 1.f;  // bias feature
}

}  // namespace huge
