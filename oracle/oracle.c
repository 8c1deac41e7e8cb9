/*
 * CPU ORACLE for subgraph enumeration — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load this file's
 * library. The product path never calls it. It shares no code with the CUDA path.
 *
 * What it computes is the plain definition of a match (Sec. 2, "Subgraph Enumeration"):
 * a map f from the query vertices to data vertices that is injective and sends every query
 * edge to a data edge (non-induced matching), restricted by the symmetry-breaking partial
 * order (Sec. 2, symmetry breaking: f(a) < f(b) for every constrained pair a < b, with "<" on
 * data vertex ids).
 *
 * Method: nested-loop backtracking in a fixed matching order v_0..v_{k-1} whose every prefix
 * is connected. Position 0 runs over the root vertices; position j runs over the adjacency
 * list of ONE earlier-bound query neighbour of v_j and then checks, one candidate at a time,
 * (i) adjacency to every other earlier-bound neighbour by binary search, (ii) that the vertex
 * is not already used, (iii) every partial-order pair whose two ends are now bound. No
 * intersection kernels, no range restriction, no last-level counting shortcut.
 *
 * A separate brute force tries every k-tuple of distinct vertices (tiny graphs only).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OMAXK 16

#define OANY_LABEL 0xffffffffu

typedef struct {
    const uint64_t *off;
    const uint32_t *adj;
    const uint32_t *dlab;  /* data vertex labels (n), or NULL: unlabelled */
    const uint32_t *qlab;  /* query vertex labels (k; OANY_LABEL = any), or NULL */
    const uint64_t *ioff;  /* directed graphs: in-lists (CSR of the reversed arcs) */
    const uint32_t *iadj;
    int directed;          /* arcs: qarc[a][b] = query arc a -> b; off/adj hold out-lists */
    uint8_t qarc[OMAXK][OMAXK];
    int k;
    uint8_t qadj[OMAXK][OMAXK];
    int order[OMAXK];
    int parent[OMAXK];   /* query vertex whose list is scanned for position j */
    int npo;
    int po[2 * 64];
} oracle_q;

static int has_edge(const oracle_q *Q, uint32_t a, uint32_t b) {
    uint64_t lo = Q->off[a], hi = Q->off[a + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        uint32_t x = Q->adj[mid];
        if (x == b) return 1;
        if (x < b) lo = mid + 1; else hi = mid;
    }
    return 0;
}

/* Does data vertex w carry the label query vertex v asks for (labelled queries, Sec. 2)? */
static int label_ok(const oracle_q *Q, int v, uint32_t w) {
    if (!Q->qlab || !Q->dlab || Q->qlab[v] == OANY_LABEL) return 1;
    return Q->dlab[w] == Q->qlab[v];
}

/* Is the assignment of query vertex v := w consistent with everything bound so far? */
static int consistent(const oracle_q *Q, const uint32_t *f, const uint8_t *bound, int v, uint32_t w) {
    if (!label_ok(Q, v, w)) return 0;
    for (int u = 0; u < Q->k; u++) {
        if (!bound[u]) continue;
        if (f[u] == w) return 0;                                   /* injective */
        if (Q->directed) {                                         /* query arc -> data arc */
            if (Q->qarc[u][v] && !has_edge(Q, f[u], w)) return 0;
            if (Q->qarc[v][u] && !has_edge(Q, w, f[u])) return 0;
        } else if (Q->qadj[v][u] && !has_edge(Q, f[u], w)) return 0;  /* query edge -> data edge */
    }
    for (int i = 0; i < Q->npo; i++) {                              /* f(a) < f(b) */
        int a = Q->po[2 * i], b = Q->po[2 * i + 1];
        if (a == v && bound[b] && !(w < f[b])) return 0;
        if (b == v && bound[a] && !(f[a] < w)) return 0;
    }
    return 1;
}

typedef struct {
    int64_t count;
    uint32_t *rows;      /* optional listing, query-vertex order */
    uint64_t cap;
} oracle_sink;

static void extend(const oracle_q *Q, int j, uint32_t *f, uint8_t *bound, oracle_sink *S) {
    if (j == Q->k) {
        if (S->rows && (uint64_t)S->count < S->cap)
            memcpy(S->rows + (uint64_t)S->count * Q->k, f, sizeof(uint32_t) * Q->k);
        S->count++;
        return;
    }
    int v = Q->order[j];
    int p = Q->parent[j];
    uint32_t up = f[p];
    /* scan the parent's out-list (arc p -> v, or any undirected edge), else its in-list */
    const int in = Q->directed && !Q->qarc[p][v];
    const uint64_t *lo = in ? Q->ioff : Q->off;
    const uint32_t *la = in ? Q->iadj : Q->adj;
    for (uint64_t e = lo[up]; e < lo[up + 1]; e++) {
        uint32_t w = la[e];
        if (!consistent(Q, f, bound, v, w)) continue;
        f[v] = w;
        bound[v] = 1;
        extend(Q, j + 1, f, bound, S);
        bound[v] = 0;
    }
}

static int setup(oracle_q *Q, const uint64_t *off, const uint32_t *adj, int k, const uint8_t *qadj,
                 const int *order, int npo, const int *po) {
    if (k < 1 || k > OMAXK || npo < 0 || npo > 64) return -1;
    memset(Q, 0, sizeof(*Q));
    Q->off = off; Q->adj = adj; Q->k = k; Q->npo = npo;
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) Q->qadj[a][b] = qadj[a * k + b] ? 1 : 0;
    uint8_t seen[OMAXK] = {0};
    for (int j = 0; j < k; j++) {
        int v = order[j];
        if (v < 0 || v >= k || seen[v]) return -1;
        seen[v] = 1;
        Q->order[j] = v;
        Q->parent[j] = -1;
        for (int t = 0; t < j && Q->parent[j] < 0; t++)
            if (Q->qadj[v][order[t]]) Q->parent[j] = order[t];
        if (j > 0 && Q->parent[j] < 0) return -2;  /* prefix not connected */
    }
    for (int i = 0; i < 2 * npo; i++) {
        if (po[i] < 0 || po[i] >= k) return -1;
        Q->po[i] = po[i];
    }
    return 0;
}

/*
 * Counts matches whose position-0 vertex (order[0]) lies in [root_lo, root_hi). If per_root is
 * not NULL, per_root[r - root_lo] receives the count for root r. Uses `threads` OpenMP threads
 * (dynamic schedule over roots). Returns the total, or a negative value on bad arguments.
 */
int64_t oracle_count(uint32_t n, const uint64_t *off, const uint32_t *adj, int k, const uint8_t *qadj,
                     const int *order, int npo, const int *po, uint32_t root_lo, uint32_t root_hi,
                     int64_t *per_root, int threads) {
    oracle_q Q;
    int rc = setup(&Q, off, adj, k, qadj, order, npo, po);
    if (rc) return rc;
    if (root_hi > n) root_hi = n;
    if (root_lo >= root_hi) return 0;
    int64_t total = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t r = root_lo; r < (int64_t)root_hi; r++) {
        uint32_t f[OMAXK];
        uint8_t bound[OMAXK] = {0};
        oracle_sink S = {0, NULL, 0};
        f[Q.order[0]] = (uint32_t)r;
        bound[Q.order[0]] = 1;
        if (label_ok(&Q, Q.order[0], (uint32_t)r)) extend(&Q, 1, f, bound, &S);
        if (per_root) per_root[r - root_lo] = S.count;
        total += S.count;
    }
    return total;
}

/* Counts matches rooted at each vertex of an explicit root list (per_root[i] for roots[i]). */
int64_t oracle_count_roots(uint32_t n, const uint64_t *off, const uint32_t *adj, int k,
                           const uint8_t *qadj, const int *order, int npo, const int *po,
                           const uint32_t *roots, uint64_t nroots, int64_t *per_root, int threads) {
    oracle_q Q;
    int rc = setup(&Q, off, adj, k, qadj, order, npo, po);
    if (rc) return rc;
    int64_t total = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (int64_t i = 0; i < (int64_t)nroots; i++) {
        uint32_t f[OMAXK];
        uint8_t bound[OMAXK] = {0};
        oracle_sink S = {0, NULL, 0};
        int64_t c = 0;
        if (roots[i] < n && label_ok(&Q, Q.order[0], roots[i])) {
            f[Q.order[0]] = roots[i];
            bound[Q.order[0]] = 1;
            extend(&Q, 1, f, bound, &S);
            c = S.count;
        }
        if (per_root) per_root[i] = c;
        total += c;
    }
    return total;
}

/*
 * Lists every match (single thread) into rows[cap][k], column v = f(v) (query-vertex order).
 * Returns the total number of matches (rows beyond cap are counted, not written).
 */
int64_t oracle_list(uint32_t n, const uint64_t *off, const uint32_t *adj, int k, const uint8_t *qadj,
                    const int *order, int npo, const int *po, uint32_t *rows, uint64_t cap) {
    oracle_q Q;
    int rc = setup(&Q, off, adj, k, qadj, order, npo, po);
    if (rc) return rc;
    oracle_sink S = {0, rows, cap};
    for (uint32_t r = 0; r < n; r++) {
        uint32_t f[OMAXK];
        uint8_t bound[OMAXK] = {0};
        f[Q.order[0]] = r;
        bound[Q.order[0]] = 1;
        if (label_ok(&Q, Q.order[0], r)) extend(&Q, 1, f, bound, &S);
    }
    return S.count;
}

/*
 * Labelled queries (Sec. 2: the method extends to labelled graphs): the same plain backtracking
 * with one more condition per assignment, label(f(v)) = qlab[v] (qlab[v] = OANY_LABEL matches
 * any label). dlab: n data labels; qlab: k query labels. Counts the roots in [root_lo, root_hi)
 * into per_root when given.
 */
int64_t oracle_count_labeled(uint32_t n, const uint64_t *off, const uint32_t *adj, const uint32_t *dlab, int k,
                             const uint8_t *qadj, const uint32_t *qlab, const int *order, int npo, const int *po,
                             uint32_t root_lo, uint32_t root_hi, int64_t *per_root, int threads) {
    oracle_q Q;
    int rc = setup(&Q, off, adj, k, qadj, order, npo, po);
    if (rc) return rc;
    Q.dlab = dlab;
    Q.qlab = qlab;
    if (root_hi > n) root_hi = n;
    if (root_lo >= root_hi) return 0;
    int64_t total = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t r = root_lo; r < (int64_t)root_hi; r++) {
        uint32_t f[OMAXK];
        uint8_t bound[OMAXK] = {0};
        oracle_sink S = {0, NULL, 0};
        f[Q.order[0]] = (uint32_t)r;
        bound[Q.order[0]] = 1;
        if (label_ok(&Q, Q.order[0], (uint32_t)r)) extend(&Q, 1, f, bound, &S);
        if (per_root) per_root[r - root_lo] = S.count;
        total += S.count;
    }
    return total;
}

/* Brute force over all k-tuples of distinct vertices with the label condition (tiny graphs). */
int64_t oracle_brute_labeled(uint32_t n, const uint64_t *off, const uint32_t *adj, const uint32_t *dlab, int k,
                             const uint8_t *qadj, const uint32_t *qlab, int npo, const int *po) {
    if (k < 1 || k > 8) return -1;
    uint64_t total = 1;
    for (int i = 0; i < k; i++) total *= n;
    oracle_q Q;
    memset(&Q, 0, sizeof(Q));
    Q.off = off; Q.adj = adj; Q.k = k;
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) Q.qadj[a][b] = qadj[a * k + b] ? 1 : 0;
    int64_t count = 0;
    uint32_t t[8];
    for (uint64_t code = 0; code < total; code++) {
        uint64_t c = code;
        for (int i = 0; i < k; i++) { t[i] = (uint32_t)(c % n); c /= n; }
        int ok = 1;
        for (int a = 0; a < k && ok; a++)
            if (qlab[a] != OANY_LABEL && dlab[t[a]] != qlab[a]) ok = 0;
        for (int a = 0; a < k && ok; a++)
            for (int b = a + 1; b < k && ok; b++)
                if (t[a] == t[b]) ok = 0;
        for (int a = 0; a < k && ok; a++)
            for (int b = a + 1; b < k && ok; b++)
                if (Q.qadj[a][b] && !has_edge(&Q, t[a], t[b])) ok = 0;
        for (int i = 0; i < npo && ok; i++)
            if (!(t[po[2 * i]] < t[po[2 * i + 1]])) ok = 0;
        count += ok;
    }
    return count;
}

/*
 * Brute force: every k-tuple (t_0..t_{k-1}) of distinct vertices with t_v = f(v) is tested
 * against every query edge and every partial-order pair. Intended for n <= 16, k <= 5.
 */
int64_t oracle_brute(uint32_t n, const uint64_t *off, const uint32_t *adj, int k, const uint8_t *qadj,
                     int npo, const int *po) {
    if (k < 1 || k > 8) return -1;
    oracle_q Q;
    int order[OMAXK];
    for (int i = 0; i < k; i++) order[i] = i;
    /* setup() requires a connected order only for the backtracker; fill fields directly */
    memset(&Q, 0, sizeof(Q));
    Q.off = off; Q.adj = adj; Q.k = k; Q.npo = npo;
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) Q.qadj[a][b] = qadj[a * k + b] ? 1 : 0;
    for (int i = 0; i < 2 * npo; i++) Q.po[i] = po[i];
    (void)order;
    uint64_t total = 1;
    for (int i = 0; i < k; i++) total *= n;
    int64_t count = 0;
    uint32_t t[8];
    for (uint64_t code = 0; code < total; code++) {
        uint64_t c = code;
        for (int i = 0; i < k; i++) { t[i] = (uint32_t)(c % n); c /= n; }
        int ok = 1;
        for (int a = 0; a < k && ok; a++)
            for (int b = a + 1; b < k && ok; b++)
                if (t[a] == t[b]) ok = 0;
        for (int a = 0; a < k && ok; a++)
            for (int b = a + 1; b < k && ok; b++)
                if (Q.qadj[a][b] && !has_edge(&Q, t[a], t[b])) ok = 0;
        for (int i = 0; i < npo && ok; i++)
            if (!(t[po[2 * i]] < t[po[2 * i + 1]])) ok = 0;
        count += ok;
    }
    return count;
}

/*
 * Closed walks of the adjacency matrix A, for the trace identities that pin whole-graph counts
 * without any enumeration: tr(A^3) = 6 #triangles and
 * tr(A^4) = 8 #4-cycles + 2m + 4 sum_v C(d(v), 2) (a closed 4-walk either runs round a 4-cycle,
 * or goes back and forth on one edge, or visits two distinct edges at one vertex).
 *
 * Method: (A^2)[u][w] is the number of common neighbours c(u, w). For every u, count the
 * 2-walks u - v - w into cnt[w] (every v in N(u), every w in N(v)); then
 * tr(A^4) = sum_u sum_w c(u, w)^2 and tr(A^3) = sum_u sum_{w in N(u)} c(u, w).
 * out[0] = tr(A^3), out[1] = tr(A^4). Returns 0, or -1 if a per-thread array cannot be had.
 */
int oracle_walk_traces(uint32_t n, const uint64_t *off, const uint32_t *adj, int threads, uint64_t *out) {
    uint64_t t3 = 0, t4 = 0;
    int bad = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel reduction(+ : t3, t4) reduction(| : bad)
    {
        uint32_t *cnt = (uint32_t *)calloc(n ? n : 1, sizeof(uint32_t));
        uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
        if (!cnt || !touched) {
            bad = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t u = 0; u < (int64_t)n; u++) {
                uint64_t nt = 0;
                for (uint64_t e = off[u]; e < off[u + 1]; e++) {
                    uint32_t v = adj[e];
                    for (uint64_t f = off[v]; f < off[v + 1]; f++) {
                        uint32_t w = adj[f];
                        if (cnt[w]++ == 0) touched[nt++] = w;
                    }
                }
                for (uint64_t e = off[u]; e < off[u + 1]; e++) t3 += cnt[adj[e]];
                for (uint64_t i = 0; i < nt; i++) {
                    uint64_t c = cnt[touched[i]];
                    t4 += c * c;
                    cnt[touched[i]] = 0;
                }
            }
        }
        free(cnt);
        free(touched);
    }
    if (bad) return -1;
    out[0] = t3;
    out[1] = t4;
    return 0;
}

/*
 * Number of k-vertex cliques (complete subgraphs K_k), k >= 1, by the textbook orientation
 * method (Chiba and Nishizeki, 1985): direct every edge from the endpoint that is smaller in
 * the total order (degree, id) to the larger one; every clique then has exactly one vertex
 * from which all its other vertices are out-neighbours, and is counted once from there by
 * growing candidate sets S := S ∩ N+(w) one vertex at a time. No partial order, no matching
 * order and no code of the backtracker are involved. Returns the count, or -1 on bad
 * arguments / allocation failure.
 */
static int rank_less(const uint64_t *off, uint32_t a, uint32_t b) {
    uint64_t da = off[a + 1] - off[a], db = off[b + 1] - off[b];
    return da < db || (da == db && a < b);
}

static int64_t clique_rec(const uint64_t *ooff, const uint32_t *oadj, const uint32_t *S, uint64_t ns, int left,
                          uint32_t *buf, uint64_t bufcap) {
    if (left == 0) return (int64_t)ns;
    int64_t total = 0;
    uint32_t *next = buf;
    for (uint64_t i = 0; i < ns; i++) {
        uint32_t w = S[i];
        /* S' = S ∩ N+(w) by a merge of two id-sorted lists */
        uint64_t a = 0, b = ooff[w], be = ooff[w + 1], nn = 0;
        while (a < ns && b < be) {
            if (S[a] < oadj[b]) a++;
            else if (S[a] > oadj[b]) b++;
            else { next[nn++] = S[a]; a++; b++; }
        }
        if (left == 1) total += (int64_t)nn;
        else if (nn) total += clique_rec(ooff, oadj, next, nn, left - 1, buf + nn, bufcap - nn);
    }
    return total;
}

int64_t oracle_clique_count(uint32_t n, const uint64_t *off, const uint32_t *adj, int k, int threads) {
    if (k < 1 || k > OMAXK) return -1;
    if (k == 1) return (int64_t)n;
    uint64_t nnz = off[n];
    uint64_t *ooff = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint32_t *oadj = (uint32_t *)malloc(sizeof(uint32_t) * (nnz / 2 + 1));
    if (!ooff || !oadj) { free(ooff); free(oadj); return -1; }
    for (uint32_t u = 0; u < n; u++) {
        uint64_t c = 0;
        for (uint64_t e = off[u]; e < off[u + 1]; e++) c += rank_less(off, u, adj[e]);
        ooff[u + 1] = ooff[u] + c;
    }
    uint64_t maxout = 0;
    for (uint32_t u = 0; u < n; u++) {
        uint64_t p = ooff[u];
        for (uint64_t e = off[u]; e < off[u + 1]; e++)
            if (rank_less(off, u, adj[e])) oadj[p++] = adj[e];  /* stays id-sorted */
        if (ooff[u + 1] - ooff[u] > maxout) maxout = ooff[u + 1] - ooff[u];
    }
    int64_t total = 0;
    int bad = 0;
    const uint64_t bufcap = maxout * (uint64_t)k + 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel reduction(+ : total) reduction(| : bad)
    {
        uint32_t *buf = (uint32_t *)malloc(sizeof(uint32_t) * bufcap);
        if (!buf) {
            bad = 1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t u = 0; u < (int64_t)n; u++)
                total += clique_rec(ooff, oadj, oadj + ooff[u], ooff[u + 1] - ooff[u], k - 2, buf, bufcap);
        }
        free(buf);
    }
    free(ooff);
    free(oadj);
    return bad ? -1 : total;
}

/*
 * Directed queries on directed graphs (Sec. 2: the method carries over to directed graphs): a
 * match maps every query arc a -> b to a data arc f(a) -> f(b). off/adj: out-lists, ioff/iadj:
 * in-lists of the same graph; qarc: k x k, qarc[a*k+b] = 1 for a query arc a -> b. The
 * matching order must be connected in the underlying undirected query. dlab / qlab (both
 * NULL, or n data and k query labels, OANY_LABEL = any) add the label condition of labelled
 * matches, which carries over to directed graphs in the same way.
 */
int64_t oracle_count_directed(uint32_t n, const uint64_t *off, const uint32_t *adj, const uint64_t *ioff,
                              const uint32_t *iadj, const uint32_t *dlab, int k, const uint8_t *qarc,
                              const uint32_t *qlab, const int *order, int npo, const int *po, uint32_t root_lo,
                              uint32_t root_hi, int64_t *per_root, int threads) {
    uint8_t und[OMAXK * OMAXK];
    if (k < 1 || k > OMAXK) return -1;
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) und[a * k + b] = (qarc[a * k + b] || qarc[b * k + a]) ? 1 : 0;
    oracle_q Q;
    int rc = setup(&Q, off, adj, k, und, order, npo, po);
    if (rc) return rc;
    Q.directed = 1;
    Q.ioff = ioff;
    Q.iadj = iadj;
    Q.dlab = dlab;
    Q.qlab = qlab;
    for (int a = 0; a < k; a++)
        for (int b = 0; b < k; b++) Q.qarc[a][b] = qarc[a * k + b] ? 1 : 0;
    if (root_hi > n) root_hi = n;
    if (root_lo >= root_hi) return 0;
    int64_t total = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t r = root_lo; r < (int64_t)root_hi; r++) {
        uint32_t f[OMAXK];
        uint8_t bound[OMAXK] = {0};
        oracle_sink S = {0, NULL, 0};
        f[Q.order[0]] = (uint32_t)r;
        bound[Q.order[0]] = 1;
        if (label_ok(&Q, Q.order[0], (uint32_t)r)) extend(&Q, 1, f, bound, &S);
        if (per_root) per_root[r - root_lo] = S.count;
        total += S.count;
    }
    return total;
}

/* Directed brute force over all k-tuples of distinct vertices (tiny graphs); dlab / qlab as in
 * oracle_count_directed. */
int64_t oracle_brute_directed(uint32_t n, const uint64_t *off, const uint32_t *adj, const uint32_t *dlab, int k,
                              const uint8_t *qarc, const uint32_t *qlab, int npo, const int *po) {
    if (k < 1 || k > 8) return -1;
    uint64_t total = 1;
    for (int i = 0; i < k; i++) total *= n;
    oracle_q Q;
    memset(&Q, 0, sizeof(Q));
    Q.off = off; Q.adj = adj; Q.k = k;
    Q.dlab = dlab; Q.qlab = qlab;
    int64_t count = 0;
    uint32_t t[8];
    for (uint64_t code = 0; code < total; code++) {
        uint64_t c = code;
        for (int i = 0; i < k; i++) { t[i] = (uint32_t)(c % n); c /= n; }
        int ok = 1;
        for (int a = 0; a < k && ok; a++)
            for (int b = a + 1; b < k && ok; b++)
                if (t[a] == t[b]) ok = 0;
        for (int a = 0; a < k && ok; a++)
            if (!label_ok(&Q, a, t[a])) ok = 0;
        for (int a = 0; a < k && ok; a++)
            for (int b = 0; b < k && ok; b++)
                if (qarc[a * k + b] && !has_edge(&Q, t[a], t[b])) ok = 0;
        for (int i = 0; i < npo && ok; i++)
            if (!(t[po[2 * i]] < t[po[2 * i + 1]])) ok = 0;
        count += ok;
    }
    return count;
}
