/*
 * Seeded synthetic inputs: data graphs as simple undirected CSR, and query graphs.
 *
 * This module holds no arithmetic of the enumeration method. It only draws random graphs and
 * turns an edge multiset into a simple, symmetric CSR with sorted adjacency (no self-loops, no
 * duplicates): the input format the method takes. Both the CUDA path's tests and the CPU oracle
 * read their inputs from here; neither side links anything else in common.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through SplitMix64 (Steele,
 * Lea & Flood, 2014). Bulk generators split the sample stream into fixed chunks of CHUNK
 * samples; chunk c is seeded with SplitMix64(seed, c), so the output does not depend on the
 * number of threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CHUNK (1u << 16)

static inline uint64_t sm64(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } rng_t;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

static void rng_seed(rng_t *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (0xd1b54a32d192ed03ULL * (stream + 1));
    for (int i = 0; i < 4; i++) r->s[i] = sm64(&x);
}

/* Uniform integer in [0, n) by Lemire's multiply-shift with rejection (unbiased). */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
    uint64_t x = rng_next(r);
    unsigned __int128 m = (unsigned __int128)x * n;
    uint64_t l = (uint64_t)m;
    if (l < n) {
        uint64_t t = (0 - n) % n;
        while (l < t) {
            x = rng_next(r);
            m = (unsigned __int128)x * n;
            l = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

/* ------------------------------------------------------------------------------------------ */
/* CSR assembly: directed entry list -> sorted, deduplicated, symmetric CSR.                   */
/* ------------------------------------------------------------------------------------------ */

/*
 * Builds the CSR of the undirected simple graph whose edges are {src[i], dst[i]} (i < ne).
 * Self-loops are dropped, both directions are inserted, and duplicates are removed.
 * Two stable counting-sort passes (by destination, then by source) give sorted lists.
 * Outputs are malloc'ed: *offsets (n+1 entries), *adj (offsets[n] entries).
 */
static int csr_build(uint32_t n, uint64_t ne, const uint32_t *src, const uint32_t *dst, int symmetric,
                     uint64_t **offsets_out, uint32_t **adj_out);

static int csr_from_edges(uint32_t n, uint64_t ne, const uint32_t *src, const uint32_t *dst,
                          uint64_t **offsets_out, uint32_t **adj_out) {
    return csr_build(n, ne, src, dst, 1, offsets_out, adj_out);
}

/* As csr_from_edges, but for a directed graph: arc src[i] -> dst[i] only (out-lists). */
static int csr_from_arcs(uint32_t n, uint64_t ne, const uint32_t *src, const uint32_t *dst,
                         uint64_t **offsets_out, uint32_t **adj_out) {
    return csr_build(n, ne, src, dst, 0, offsets_out, adj_out);
}

static int csr_build(uint32_t n, uint64_t ne, const uint32_t *src, const uint32_t *dst, int symmetric,
                     uint64_t **offsets_out, uint32_t **adj_out) {
    uint64_t nd = 0;
    for (uint64_t i = 0; i < ne; i++) nd += (src[i] != dst[i]) ? (symmetric ? 2 : 1) : 0;
    uint32_t *a = (uint32_t *)malloc(sizeof(uint32_t) * (nd ? nd : 1));
    uint32_t *b = (uint32_t *)malloc(sizeof(uint32_t) * (nd ? nd : 1));
    uint32_t *a2 = (uint32_t *)malloc(sizeof(uint32_t) * (nd ? nd : 1));
    uint32_t *b2 = (uint32_t *)malloc(sizeof(uint32_t) * (nd ? nd : 1));
    uint64_t *cnt = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!a || !b || !a2 || !b2 || !cnt) return -1;
    uint64_t k = 0;
    for (uint64_t i = 0; i < ne; i++) {
        if (src[i] == dst[i]) continue;
        a[k] = src[i]; b[k] = dst[i]; k++;
        if (symmetric) { a[k] = dst[i]; b[k] = src[i]; k++; }
    }
    /* pass 1: stable counting sort by destination (b) */
    for (uint64_t i = 0; i < nd; i++) cnt[b[i] + 1]++;
    for (uint32_t v = 0; v < n; v++) cnt[v + 1] += cnt[v];
    for (uint64_t i = 0; i < nd; i++) {
        uint64_t p = cnt[b[i]]++;
        a2[p] = a[i]; b2[p] = b[i];
    }
    /* pass 2: stable counting sort by source (a2) -> lists sorted by destination */
    memset(cnt, 0, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t i = 0; i < nd; i++) cnt[a2[i] + 1]++;
    for (uint32_t v = 0; v < n; v++) cnt[v + 1] += cnt[v];
    for (uint64_t i = 0; i < nd; i++) {
        uint64_t p = cnt[a2[i]]++;
        a[p] = a2[i]; b[p] = b2[i];
    }
    free(a2); free(b2);
    /* dedup: entries are sorted by (a, b) */
    uint64_t *off = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t w = 0;
    for (uint64_t i = 0; i < nd; i++) {
        if (i > 0 && a[i] == a[i - 1] && b[i] == b[i - 1]) continue;
        b[w] = b[i];
        off[a[i] + 1]++;
        w++;
    }
    for (uint32_t v = 0; v < n; v++) off[v + 1] += off[v];
    free(a); free(cnt);
    uint32_t *adj = (uint32_t *)realloc(b, sizeof(uint32_t) * (w ? w : 1));
    *offsets_out = off;
    *adj_out = adj;
    return 0;
}

void gen_free(void *p) { free(p); }

/* ------------------------------------------------------------------------------------------ */
/* Generators. Each returns 0 on success and malloc'ed CSR arrays (free with gen_free).         */
/* ------------------------------------------------------------------------------------------ */

/* Erdos-Renyi G(n, m): m distinct unordered pairs {u, v}, u != v, drawn uniformly. */
int gen_er(uint32_t n, uint64_t m, uint64_t seed, uint64_t **offsets, uint32_t **adj) {
    if (n < 2) return -1;
    uint64_t maxm = (uint64_t)n * (n - 1) / 2;
    if (m > maxm) return -1;
    uint64_t cap = 1;
    while (cap < 2 * m + 16) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    memset(set, 0xff, sizeof(uint64_t) * cap);
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    rng_t r;
    rng_seed(&r, seed, 0);
    uint64_t got = 0;
    while (got < m) {
        uint32_t u = (uint32_t)rng_below(&r, n), v = (uint32_t)rng_below(&r, n);
        if (u == v) continue;
        uint32_t lo = u < v ? u : v, hi = u < v ? v : u;
        uint64_t key = ((uint64_t)lo << 32) | hi;
        uint64_t h = (key * 0x9e3779b97f4a7c15ULL) & (cap - 1);
        int dup = 0;
        while (set[h] != ~0ULL) {
            if (set[h] == key) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        set[h] = key;
        src[got] = lo; dst[got] = hi; got++;
    }
    free(set);
    int rc = csr_from_edges(n, m, src, dst, offsets, adj);
    free(src); free(dst);
    return rc;
}

/* Erdos-Renyi G(n, p) for tiny graphs: each pair independently with probability p_num/p_den. */
int gen_gnp(uint32_t n, uint32_t p_num, uint32_t p_den, uint64_t seed, uint64_t **offsets,
            uint32_t **adj) {
    uint64_t maxm = (uint64_t)n * (n ? n - 1 : 0) / 2;
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (maxm ? maxm : 1));
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * (maxm ? maxm : 1));
    rng_t r;
    rng_seed(&r, seed, 0);
    uint64_t k = 0;
    for (uint32_t u = 0; u < n; u++)
        for (uint32_t v = u + 1; v < n; v++)
            if (rng_below(&r, p_den) < p_num) { src[k] = u; dst[k] = v; k++; }
    int rc = csr_from_edges(n, k, src, dst, offsets, adj);
    free(src); free(dst);
    return rc;
}

/* Complete graph K_n. */
int gen_complete(uint32_t n, uint64_t **offsets, uint32_t **adj) {
    uint64_t m = (uint64_t)n * (n ? n - 1 : 0) / 2;
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint64_t k = 0;
    for (uint32_t u = 0; u < n; u++)
        for (uint32_t v = u + 1; v < n; v++) { src[k] = u; dst[k] = v; k++; }
    int rc = csr_from_edges(n, k, src, dst, offsets, adj);
    free(src); free(dst);
    return rc;
}

/* Complete bipartite K_{a,b}: parts {0..a-1} and {a..a+b-1}. */
int gen_complete_bipartite(uint32_t a, uint32_t b, uint64_t **offsets, uint32_t **adj) {
    uint64_t m = (uint64_t)a * b;
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint64_t k = 0;
    for (uint32_t u = 0; u < a; u++)
        for (uint32_t v = 0; v < b; v++) { src[k] = u; dst[k] = a + v; k++; }
    int rc = csr_from_edges(a + b, k, src, dst, offsets, adj);
    free(src); free(dst);
    return rc;
}

/*
 * R-MAT (Chakrabarti, Zhan & Faloutsos, 2004) without noise: (ef << scale) directed samples,
 * each descending `scale` levels of the adjacency matrix, choosing the quadrant (a, b, c, d)
 * with probabilities (pa, pb, pc, 1 - pa - pb - pc). Probabilities are given as 53-bit fixed
 * point thresholds so the draw is exact integer arithmetic. Self-loops are dropped, then the
 * graph is symmetrised and deduplicated. No vertex permutation is applied.
 */
int gen_rmat(uint32_t scale, uint32_t ef, double pa, double pb, double pc, uint64_t seed,
             uint64_t **offsets, uint32_t **adj) {
    if (scale < 1 || scale > 31) return -1;
    uint32_t n = 1u << scale;
    uint64_t ne = (uint64_t)ef << scale;
    const double two53 = 9007199254740992.0;
    uint64_t ta = (uint64_t)(pa * two53);
    uint64_t tb = ta + (uint64_t)(pb * two53);
    uint64_t tc = tb + (uint64_t)(pc * two53);
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * ne);
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * ne);
    if (!src || !dst) return -1;
    uint64_t nchunks = (ne + CHUNK - 1) / CHUNK;
#pragma omp parallel for schedule(dynamic, 4)
    for (uint64_t c = 0; c < nchunks; c++) {
        rng_t r;
        rng_seed(&r, seed, c);
        uint64_t e0 = c * CHUNK, e1 = e0 + CHUNK < ne ? e0 + CHUNK : ne;
        for (uint64_t e = e0; e < e1; e++) {
            uint32_t u = 0, v = 0;
            for (uint32_t l = 0; l < scale; l++) {
                uint32_t bit = 1u << (scale - 1 - l);
                uint64_t x = rng_next(&r) >> 11;
                if (x < ta) {
                } else if (x < tb) {
                    v |= bit;
                } else if (x < tc) {
                    u |= bit;
                } else {
                    u |= bit; v |= bit;
                }
            }
            src[e] = u; dst[e] = v;
        }
    }
    int rc = csr_from_edges(n, ne, src, dst, offsets, adj);
    free(src); free(dst);
    return rc;
}

/*
 * Directed R-MAT: the same (ef << scale) samples as gen_rmat, kept as arcs u -> v (self-loops
 * dropped, repeated arcs merged, no symmetrisation). CSR of out-lists.
 */
int gen_rmat_directed(uint32_t scale, uint32_t ef, double pa, double pb, double pc, uint64_t seed,
                      uint64_t **offsets, uint32_t **adj) {
    if (scale < 1 || scale > 31) return -1;
    uint32_t n = 1u << scale;
    uint64_t ne = (uint64_t)ef << scale;
    const double two53 = 9007199254740992.0;
    uint64_t ta = (uint64_t)(pa * two53);
    uint64_t tb = ta + (uint64_t)(pb * two53);
    uint64_t tc = tb + (uint64_t)(pc * two53);
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * ne);
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * ne);
    if (!src || !dst) return -1;
    uint64_t nchunks = (ne + CHUNK - 1) / CHUNK;
#pragma omp parallel for schedule(dynamic, 4)
    for (uint64_t c = 0; c < nchunks; c++) {
        rng_t r;
        rng_seed(&r, seed, c);
        uint64_t e0 = c * CHUNK, e1 = e0 + CHUNK < ne ? e0 + CHUNK : ne;
        for (uint64_t e = e0; e < e1; e++) {
            uint32_t u = 0, v = 0;
            for (uint32_t l = 0; l < scale; l++) {
                uint32_t bit = 1u << (scale - 1 - l);
                uint64_t x = rng_next(&r) >> 11;
                if (x < ta) {
                } else if (x < tb) {
                    v |= bit;
                } else if (x < tc) {
                    u |= bit;
                } else {
                    u |= bit; v |= bit;
                }
            }
            src[e] = u; dst[e] = v;
        }
    }
    int rc = csr_from_arcs(n, ne, src, dst, offsets, adj);
    free(src); free(dst);
    return rc;
}

/* Directed G(n, p): every ordered pair (u, v), u != v, is an arc with probability p_num/p_den. */
int gen_gnp_directed(uint32_t n, uint32_t p_num, uint32_t p_den, uint64_t seed, uint64_t **offsets,
                     uint32_t **adj) {
    if (p_den == 0 || p_num > p_den) return -1;
    uint64_t cap = (uint64_t)n * n;
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (cap ? cap : 1));
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * (cap ? cap : 1));
    if (!src || !dst) return -1;
    rng_t r;
    rng_seed(&r, seed, 0);
    uint64_t k = 0;
    for (uint32_t u = 0; u < n; u++)
        for (uint32_t v = 0; v < n; v++) {
            if (u == v) continue;
            if (rng_below(&r, p_den) < p_num) { src[k] = u; dst[k] = v; k++; }
        }
    int rc = csr_from_arcs(n, k, src, dst, offsets, adj);
    free(src); free(dst);
    return rc;
}

/*
 * Chung-Lu power-law graph: weights w_i = C (i + i0)^(-1/(gamma-1)), i < n, with i0 and C
 * chosen so that w_0 = max_w and sum_i w_i = 2 m (sum approximated by its integral, then C is
 * fixed exactly from the discrete sum). Endpoint pairs are drawn independently with
 * probability proportional to w (inverse CDF over an integer cumulative table); self-loops
 * and repeats are rejected until m distinct edges exist (first m in draw order).
 */
int gen_chung_lu(uint32_t n, uint64_t m, double gamma, double max_w, uint64_t seed,
                 uint64_t **offsets, uint32_t **adj) {
    if (n < 2 || gamma <= 1.0) return -1;
    double alpha = 1.0 / (gamma - 1.0);
    double target = 2.0 * (double)m;
    /* F(i0) = integral_{i0-0.5}^{n+i0-0.5} x^-alpha dx * max_w * i0^alpha ; solve F = target */
    double lo = 1e-3, hi = (double)n * 1e3;
    for (int it = 0; it < 200; it++) {
        double i0 = sqrt(lo * hi);
        double x0 = i0 - 0.5 > 1e-9 ? i0 - 0.5 : 1e-9, x1 = (double)n + i0 - 0.5;
        double integ = (pow(x1, 1.0 - alpha) - pow(x0, 1.0 - alpha)) / (1.0 - alpha);
        double f = integ * max_w * pow(i0, alpha);
        if (f < target) lo = i0; else hi = i0;
    }
    double i0 = sqrt(lo * hi);
    double *w = (double *)malloc(sizeof(double) * n);
    double s = 0.0;
    for (uint32_t i = 0; i < n; i++) { w[i] = pow((double)i + i0, -alpha); s += w[i]; }
    /* integer cumulative table scaled to 2^52 total */
    uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    const double scale52 = 4503599627370496.0;
    double acc = 0.0;
    cum[0] = 0;
    for (uint32_t i = 0; i < n; i++) {
        acc += w[i];
        cum[i + 1] = (uint64_t)(acc / s * scale52);
    }
    cum[n] = (uint64_t)scale52;
    free(w);
    uint64_t total = cum[n];
    uint64_t cap = 1;
    while (cap < 2 * m + 16) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    memset(set, 0xff, sizeof(uint64_t) * cap);
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *bu = (uint32_t *)malloc(sizeof(uint32_t) * CHUNK * 16);
    uint32_t *bv = (uint32_t *)malloc(sizeof(uint32_t) * CHUNK * 16);
    uint64_t got = 0, chunk = 0;
    while (got < m) {
        /* draw 16 chunks in parallel, then insert sequentially in draw order */
#pragma omp parallel for schedule(static)
        for (int cc = 0; cc < 16; cc++) {
            rng_t r;
            rng_seed(&r, seed, chunk + (uint64_t)cc);
            for (uint32_t e = 0; e < CHUNK; e++) {
                uint32_t ends[2];
                for (int t = 0; t < 2; t++) {
                    uint64_t x = rng_below(&r, total);
                    uint32_t l = 0, h = n; /* find i with cum[i] <= x < cum[i+1] */
                    while (h - l > 1) {
                        uint32_t mid = l + (h - l) / 2;
                        if (cum[mid] <= x) l = mid; else h = mid;
                    }
                    ends[t] = l;
                }
                bu[(size_t)cc * CHUNK + e] = ends[0];
                bv[(size_t)cc * CHUNK + e] = ends[1];
            }
        }
        chunk += 16;
        for (size_t e = 0; e < (size_t)CHUNK * 16 && got < m; e++) {
            uint32_t u = bu[e], v = bv[e];
            if (u == v) continue;
            uint32_t a = u < v ? u : v, b = u < v ? v : u;
            uint64_t key = ((uint64_t)a << 32) | b;
            uint64_t h = (key * 0x9e3779b97f4a7c15ULL) & (cap - 1);
            int dup = 0;
            while (set[h] != ~0ULL) {
                if (set[h] == key) { dup = 1; break; }
                h = (h + 1) & (cap - 1);
            }
            if (dup) continue;
            set[h] = key;
            src[got] = a; dst[got] = b; got++;
        }
    }
    free(set); free(cum); free(bu); free(bv);
    int rc = csr_from_edges(n, m, src, dst, offsets, adj);
    free(src); free(dst);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Query graphs                                                                                */
/* ------------------------------------------------------------------------------------------ */

/*
 * Random connected query on k vertices: a uniformly random labelled spanning tree drawn by
 * attaching vertex i (i = 1..k-1) to a uniform earlier vertex of a random permutation, then
 * every remaining pair added independently with probability p_num/p_den. Writes 2*mq vertex
 * ids into edges (capacity 2*k*(k-1)/2) and returns mq.
 */
int gen_random_query(uint32_t k, uint32_t p_num, uint32_t p_den, uint64_t seed, uint32_t *edges) {
    if (k < 2 || k > 16) return -1;
    rng_t r;
    rng_seed(&r, seed, 0);
    uint32_t perm[16];
    for (uint32_t i = 0; i < k; i++) perm[i] = i;
    for (uint32_t i = k - 1; i > 0; i--) {
        uint32_t j = (uint32_t)rng_below(&r, i + 1);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    uint8_t a[16][16];
    memset(a, 0, sizeof(a));
    for (uint32_t i = 1; i < k; i++) {
        uint32_t j = (uint32_t)rng_below(&r, i);
        a[perm[i]][perm[j]] = a[perm[j]][perm[i]] = 1;
    }
    for (uint32_t u = 0; u < k; u++)
        for (uint32_t v = u + 1; v < k; v++)
            if (!a[u][v] && rng_below(&r, p_den) < p_num) a[u][v] = a[v][u] = 1;
    int mq = 0;
    for (uint32_t u = 0; u < k; u++)
        for (uint32_t v = u + 1; v < k; v++)
            if (a[u][v]) { edges[2 * mq] = u; edges[2 * mq + 1] = v; mq++; }
    return mq;
}

/* Uniform draws for callers that need seeded integers (e.g. root samples): out[i] in [0, n). */
void gen_uniform(uint64_t count, uint64_t n, uint64_t seed, uint64_t *out) {
    rng_t r;
    rng_seed(&r, seed, 0);
    for (uint64_t i = 0; i < count; i++) out[i] = rng_below(&r, n);
}
