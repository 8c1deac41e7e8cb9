// Data graph loading: validation, degree relabelling (Sec. 2 total order), device upload.
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace huge {

void *Workspace::get(int slot, size_t n) {
    if (n == 0) n = 16;
    if (bytes[slot] >= n) return ptr[slot];
    if (ptr[slot]) dev_free(ptr[slot]);
    ptr[slot] = nullptr;
    bytes[slot] = 0;
    size_t want = n + n / 8;  // some headroom to avoid re-allocating on small growth
    if (dev_malloc(&ptr[slot], want) != cudaSuccess) {
        cudaGetLastError();
        if (dev_malloc(&ptr[slot], n) != cudaSuccess) {
            cudaGetLastError();
            ptr[slot] = nullptr;
            return nullptr;
        }
        want = n;
    }
    bytes[slot] = want;
    size_t tot = 0;
    for (int i = 0; i < 16; i++) tot += bytes[i];
    peak = std::max(peak, tot);
    return ptr[slot];
}

void Workspace::release() {
    for (int i = 0; i < 16; i++) {
        if (ptr[i]) dev_free(ptr[i]);
        ptr[i] = nullptr;
        bytes[i] = 0;
    }
}

// One block per hub: set bit x of the hub's row for every neighbour x.
__global__ void hub_bits_kernel(const uint32_t *__restrict__ off, const uint32_t *__restrict__ adj,
                                const uint32_t *__restrict__ hubs, uint32_t nh, uint64_t wpr, uint32_t *bits) {
    for (uint32_t h = blockIdx.x; h < nh; h += gridDim.x) {
        const uint32_t v = hubs[h];
        uint32_t *row = bits + (uint64_t)h * wpr;
        for (uint32_t e = off[v] + threadIdx.x; e < off[v + 1]; e += blockDim.x) {
            const uint32_t x = adj[e];
            atomicOr(row + (x >> 5), 1u << (x & 31));
        }
    }
}

// One block per hub row: rank[b] = set bits of the row in words [0, 8 b), for every 8-word
// (256-bit) block b of the row. Each thread sums a contiguous run of blocks, then the block
// scans the per-thread sums.
__global__ void hub_rank_kernel(const uint32_t *__restrict__ bits, uint32_t nh, uint64_t wpr, uint64_t nblk,
                                uint32_t *rank) {
    __shared__ uint32_t part[256];
    const uint32_t t = threadIdx.x;
    const uint64_t per = (nblk + 255) / 256;
    for (uint32_t h = blockIdx.x; h < nh; h += gridDim.x) {
        const uint32_t *row = bits + (uint64_t)h * wpr;
        uint32_t *rk = rank + (uint64_t)h * nblk;
        const uint64_t b0 = per * t < nblk ? per * t : nblk;
        const uint64_t b1 = b0 + per < nblk ? b0 + per : nblk;
        uint32_t sum = 0;
        for (uint64_t w = b0 * 8; w < b1 * 8; w++) sum += __popc(row[w]);
        part[t] = sum;
        __syncthreads();
        if (t == 0) {  // exclusive scan of 256 partial sums
            uint32_t acc = 0;
            for (int i = 0; i < 256; i++) {
                const uint32_t x = part[i];
                part[i] = acc;
                acc += x;
            }
        }
        __syncthreads();
        uint32_t acc = part[t];
        for (uint64_t b = b0; b < b1; b++) {
            rk[b] = acc;
            for (int i = 0; i < 8; i++) acc += __popc(row[b * 8 + i]);
        }
        __syncthreads();
    }
}

uint32_t default_hub_min_degree(uint32_t n) { return std::max<uint32_t>(256u, (n + 1023u) / 1024u); }

void free_hub_bitmaps(DevGraph &G) {
    if (G.d_hub_row) dev_free(G.d_hub_row);
    if (G.d_hub_bits) dev_free(G.d_hub_bits);
    if (G.d_hub_rank) dev_free(G.d_hub_rank);
    G.d_hub_row = G.d_hub_bits = G.d_hub_rank = nullptr;
    G.hub_count = 0;
    G.hub_min_deg = 0;
    G.hub_bytes = 0;
}

int build_hub_bitmaps(DevGraph &G, uint32_t min_deg, uint64_t max_bytes) {
    free_hub_bitmaps(G);
    G.hub_wpr = ((uint64_t)G.n + 255) / 256 * 8;  // whole 256-bit blocks: rows stay 32-byte aligned
    G.hub_nblk = G.hub_wpr / 8;
    const uint64_t row_bytes = G.hub_wpr * 4 + G.hub_nblk * 4;  // bitmap + rank index
    if (min_deg == 0 || max_bytes < row_bytes) return HUGE_OK;
    std::vector<uint32_t> cand;  // lists (a directed graph's in-list of v is list n + v)
    for (uint32_t v = 0; v < G.nlists; v++)
        if (G.h_off[v + 1] - G.h_off[v] >= min_deg) cand.push_back(v);
    std::stable_sort(cand.begin(), cand.end(), [&](uint32_t a, uint32_t b) {
        return G.h_off[a + 1] - G.h_off[a] > G.h_off[b + 1] - G.h_off[b];
    });
    const uint64_t keep = std::min<uint64_t>(cand.size(), max_bytes / row_bytes);
    cand.resize(keep);
    if (cand.empty()) return HUGE_OK;
    std::vector<uint32_t> row(G.nlists, kNoHub);
    for (uint32_t h = 0; h < cand.size(); h++) row[cand[h]] = h;
    uint32_t *d_hubs = nullptr;
    const uint64_t bits_bytes = G.hub_wpr * 4 * cand.size();
    const uint64_t rank_bytes = G.hub_nblk * 4 * cand.size();
    cudaError_t e = dev_malloc(&G.d_hub_row, sizeof(uint32_t) * (size_t)G.nlists);
    if (e == cudaSuccess) e = dev_malloc(&G.d_hub_bits, bits_bytes);
    if (e == cudaSuccess) e = dev_malloc(&G.d_hub_rank, rank_bytes);
    if (e == cudaSuccess) e = dev_malloc(&d_hubs, sizeof(uint32_t) * cand.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (d_hubs) dev_free(d_hubs);
        free_hub_bitmaps(G);
        return fail(HUGE_ENOMEM, "device allocation for the hub bitmaps failed");
    }
    if ((e = cudaMemcpy(G.d_hub_row, row.data(), sizeof(uint32_t) * (size_t)G.nlists, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_hubs, cand.data(), sizeof(uint32_t) * cand.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(G.d_hub_bits, 0, bits_bytes))) {
        dev_free(d_hubs);
        free_hub_bitmaps(G);
        return fail(HUGE_ECUDA, std::string("preparing the hub bitmaps: ") + cudaGetErrorString(e));
    }
    hub_bits_kernel<<<(unsigned)std::min<size_t>(cand.size(), 4096), 256>>>(G.d_off, G.d_adj, d_hubs,
                                                                            (uint32_t)cand.size(), G.hub_wpr,
                                                                            G.d_hub_bits);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        hub_rank_kernel<<<(unsigned)std::min<size_t>(cand.size(), 4096), 256>>>(G.d_hub_bits, (uint32_t)cand.size(),
                                                                                G.hub_wpr, G.hub_nblk, G.d_hub_rank);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    dev_free(d_hubs);
    if (e != cudaSuccess) {
        free_hub_bitmaps(G);
        return fail(HUGE_ECUDA, std::string("building the hub bitmaps: ") + cudaGetErrorString(e));
    }
    G.hub_count = (uint32_t)cand.size();
    G.hub_min_deg = min_deg;
    G.hub_bytes = bits_bytes + rank_bytes + sizeof(uint32_t) * (uint64_t)G.nlists;
    return HUGE_OK;
}

int set_residency(DevGraph &G, uint64_t hbm_bytes) {
    const uint64_t words = (G.nnz + 3) / 4 * 4 + 4;  // the padded adjacency of graph_load
    const uint64_t bytes = words * 4;
    cudaError_t e;
    if (!G.adj_managed) {
        uint32_t *m = nullptr;
        if ((e = cudaMallocManaged(&m, bytes)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HUGE_ENOMEM, std::string("managed allocation for the adjacency: ") + cudaGetErrorString(e));
        }
        if ((e = cudaMemcpy(m, G.d_adj, bytes, cudaMemcpyDefault)) != cudaSuccess) {
            cudaFree(m);
            return fail(HUGE_ECUDA, std::string("copying the adjacency to managed memory: ") + cudaGetErrorString(e));
        }
        dev_free(G.d_adj);
        G.d_adj = m;
        G.adj_managed = true;
    }
    constexpr uint64_t kPage = 2ull << 20;
    const uint64_t keep = std::min(bytes, hbm_bytes);
    // [0, split) in host memory: whole pages, so the HBM part never exceeds the budget
    const uint64_t split = std::min(bytes, (bytes - keep + kPage - 1) / kPage * kPage);
    cudaMemLocation host, dev;
    host.type = cudaMemLocationTypeHost;
    host.id = 0;
    dev.type = cudaMemLocationTypeDevice;
    dev.id = G.device;
    char *base = reinterpret_cast<char *>(G.d_adj);
    e = cudaSuccess;
    if (split > 0) {
        if (e == cudaSuccess) e = cudaMemAdvise(base, split, cudaMemAdviseSetPreferredLocation, host);
        if (e == cudaSuccess) e = cudaMemAdvise(base, split, cudaMemAdviseSetAccessedBy, dev);
        if (e == cudaSuccess) e = cudaMemPrefetchAsync(base, split, host, 0, 0);
    }
    if (split < bytes) {
        if (e == cudaSuccess) e = cudaMemAdvise(base + split, bytes - split, cudaMemAdviseSetPreferredLocation, dev);
        if (e == cudaSuccess) e = cudaMemPrefetchAsync(base + split, bytes - split, dev, 0, 0);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HUGE_ECUDA, std::string("placing the adjacency: ") + cudaGetErrorString(e));
    }
    G.adj_hbm_bytes = bytes - split;
    return HUGE_OK;
}

// Checks the CSR contract of huge_graph_load. Returns "" or a description of the first fault.
static std::string validate_csr(const uint64_t *off, const uint32_t *adj, uint32_t n, uint64_t nnz, bool symmetric) {
    if (off[0] != 0) return "offsets[0] must be 0";
    if (off[n] != nnz) return "offsets[n] must equal nnz";
    for (uint32_t v = 0; v < n; v++)
        if (off[v + 1] < off[v]) return "offsets must be non-decreasing (vertex " + std::to_string(v) + ")";
    // Symmetry: every upper entry u of N(v) (u > v) must have its mirror v in N(u). Mirrors of
    // distinct upper entries are distinct lower entries (lists hold no repeats), so when the
    // upper and lower entries are equally many, the mirrors are all the lower entries and the
    // graph is symmetric; only the upper half needs a search.
    int bad = 0;
    uint32_t bad_v = 0;
    std::string why;
    uint64_t upper = 0, lower = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : upper, lower)
    for (int64_t vv = 0; vv < (int64_t)n; vv++) {
        if (bad) continue;
        const uint32_t v = (uint32_t)vv;
        for (uint64_t e = off[v]; e < off[v + 1]; e++) {
            const uint32_t u = adj[e];
            const char *msg = nullptr;
            if (u >= n) msg = "neighbour id >= n";
            else if (u == v) msg = "self-loop";
            else if (e > off[v] && adj[e - 1] >= u) msg = "adjacency list not strictly increasing";
            else if (symmetric && u < v) lower++;
            else if (symmetric) {
                upper++;
                const uint32_t *b = adj + off[u], *t = adj + off[u + 1];
                if (!std::binary_search(b, t, v)) msg = "graph is not symmetric";
            }
            if (msg) {
#pragma omp critical
                {
                    if (!bad) {
                        bad = 1;
                        bad_v = v;
                        why = msg;
                    }
                }
                break;
            }
        }
    }
    if (bad) return why + " (vertex " + std::to_string(bad_v) + ")";
    if (symmetric && upper != lower) return "graph is not symmetric (an entry u -> v with u > v has no mirror)";
    return "";
}

int graph_load(const uint64_t *offsets, const uint32_t *adj, uint32_t n, uint64_t nnz,
               uint32_t flags, const uint32_t *labels, uint32_t nlabels, DevGraph **out) {
    if (!offsets || (!adj && nnz) || !out) return fail(HUGE_EINVAL, "null argument");
    if (labels) {
        if (nlabels == 0 || nlabels > (1u << 24)) return fail(HUGE_EINVAL, "nlabels must be in 1..2^24");
        for (uint32_t v = 0; v < n; v++)
            if (labels[v] >= nlabels) return fail(HUGE_EINVAL, "vertex label >= nlabels (vertex " + std::to_string(v) + ")");
    }
    if (n == 0) return fail(HUGE_EINVAL, "empty graph (n = 0)");
    if (n == 0xffffffffu) return fail(HUGE_EINVAL, "n must be below 2^32 - 1");
    if (nnz >= 0xffffffffull) return fail(HUGE_EINVAL, "nnz must be below 2^32 - 1");
    const bool directed = flags & HUGE_DIRECTED;
    if (directed && 2 * nnz >= 0xffffffffull) return fail(HUGE_EINVAL, "a directed graph needs 2 nnz below 2^32 - 1");
    if (!(flags & HUGE_TRUST_SORTED)) {
        std::string why = validate_csr(offsets, adj, n, nnz, !directed);
        if (!why.empty()) return fail(HUGE_EINVAL, "malformed CSR: " + why);
    }
    DevGraph *G = new DevGraph();
    G->n = n;
    G->nnz = directed ? 2 * nnz : nnz;
    G->directed = directed;
    G->nlists = directed ? 2 * n : n;
    G->narcs = directed ? nnz : 0;
    cudaGetDevice(&G->device);
    G->new_of_old.resize(n);
    G->h_off.resize((size_t)n + 1);
    std::vector<uint32_t> new_adj;
    const uint32_t *dev_src_adj = adj;
    // degree for the relabelling: out + in degree of a directed graph
    std::vector<uint32_t> indeg;
    if (directed) {
        indeg.assign(n, 0);
        for (uint64_t e = 0; e < nnz; e++) indeg[adj[e]]++;
    }
    auto total_degree = [&](uint32_t v) -> uint64_t {
        return (offsets[v + 1] - offsets[v]) + (directed ? indeg[v] : 0);
    };
    if ((flags & HUGE_RELABEL_BY_DEGREE) || labels || directed) {
        // new ids in (label, degree, id) order: a stable counting sort by degree (when
        // relabelling by degree), then a stable counting sort by label (labelled graphs); each
        // label's vertices then hold one contiguous id range
        std::vector<uint32_t> old_of_new(n), tmp(n);
        for (uint32_t v = 0; v < n; v++) old_of_new[v] = v;
        auto counting_pass = [&](auto key, uint64_t nkeys) {
            std::vector<uint64_t> cnt(nkeys + 1, 0);
            for (uint32_t i = 0; i < n; i++) cnt[key(old_of_new[i]) + 1]++;
            for (uint64_t k = 0; k < nkeys; k++) cnt[k + 1] += cnt[k];
            for (uint32_t i = 0; i < n; i++) tmp[cnt[key(old_of_new[i])]++] = old_of_new[i];
            old_of_new.swap(tmp);
        };
        if (flags & HUGE_RELABEL_BY_DEGREE) {
            uint64_t maxd = 0;
            for (uint32_t v = 0; v < n; v++) maxd = std::max(maxd, total_degree(v));
            counting_pass(total_degree, maxd + 1);
        }
        if (labels) {
            counting_pass([&](uint32_t v) { return (uint64_t)labels[v]; }, nlabels);
            G->lstart.assign((size_t)nlabels + 1, 0);
            for (uint32_t v = 0; v < n; v++) G->lstart[labels[v] + 1]++;
            for (uint32_t L = 0; L < nlabels; L++) G->lstart[L + 1] += G->lstart[L];
        }
        for (uint32_t r = 0; r < n; r++) G->new_of_old[old_of_new[r]] = r;
        G->h_off[0] = 0;
        for (uint32_t r = 0; r < n; r++) {
            const uint32_t u = old_of_new[r];
            G->h_off[r + 1] = G->h_off[r] + (uint32_t)(offsets[u + 1] - offsets[u]);
        }
        new_adj.resize((directed ? 2 * nnz : nnz) + 1);
        const std::vector<uint32_t> &nol = G->new_of_old;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t rr = 0; rr < (int64_t)n; rr++) {
            const uint32_t r = (uint32_t)rr, u = old_of_new[r];
            uint32_t *dst = new_adj.data() + G->h_off[r];
            const uint64_t d = offsets[u + 1] - offsets[u];
            for (uint64_t i = 0; i < d; i++) dst[i] = nol[adj[offsets[u] + i]];
            std::sort(dst, dst + d);
        }
        if (directed) {
            // in-lists (the reversed arcs) after the out-lists: list n + v is v's in-list;
            // sources are visited in increasing new id, so every in-list comes out sorted
            G->h_off.resize(2 * (size_t)n + 1);
            std::vector<uint32_t> fill(n, 0);
            for (uint64_t e = 0; e < nnz; e++) fill[new_adj[e]]++;
            G->h_off[n] = (uint32_t)nnz;
            for (uint32_t v = 0; v < n; v++) G->h_off[n + v + 1] = G->h_off[n + v] + fill[v];
            for (uint32_t v = 0; v < n; v++) fill[v] = G->h_off[n + v];
            for (uint32_t r = 0; r < n; r++)
                for (uint32_t e = G->h_off[r]; e < G->h_off[r + 1]; e++) new_adj[fill[new_adj[e]]++] = r;
        }
        dev_src_adj = new_adj.data();
    } else {
        for (uint32_t v = 0; v < n; v++) G->new_of_old[v] = v;
        for (uint32_t v = 0; v <= n; v++) G->h_off[v] = (uint32_t)offsets[v];
    }
    nnz = G->nnz;  // entries stored (directed: out-lists and in-lists)
    uint32_t maxd = 0;
    for (uint32_t v = 0; v < G->nlists; v++) maxd = std::max(maxd, G->h_off[v + 1] - G->h_off[v]);
    G->max_deg = maxd;

    cudaError_t e1 = dev_malloc(&G->d_off, sizeof(uint32_t) * ((size_t)G->nlists + 1));
    // adj padded to the next multiple of 4 entries plus 4 (zeros), for 16-byte vector loads
    const uint64_t adj_alloc = (nnz + 3) / 4 * 4 + 4;
    cudaError_t e2 = dev_malloc(&G->d_adj, sizeof(uint32_t) * adj_alloc);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        if (G->d_off) dev_free(G->d_off);
        if (G->d_adj) dev_free(G->d_adj);
        delete G;
        return fail(HUGE_ENOMEM, "device allocation for the graph failed");
    }
    cudaError_t e3 = cudaMemcpy(G->d_off, G->h_off.data(), sizeof(uint32_t) * ((size_t)G->nlists + 1),
                                cudaMemcpyHostToDevice);
    cudaError_t e4 = nnz ? cudaMemcpy(G->d_adj, dev_src_adj, sizeof(uint32_t) * nnz, cudaMemcpyHostToDevice)
                         : cudaSuccess;
    if (e4 == cudaSuccess) e4 = cudaMemset(G->d_adj + nnz, 0, sizeof(uint32_t) * (adj_alloc - nnz));
    if (e3 != cudaSuccess || e4 != cudaSuccess) {
        std::string msg = cudaGetErrorString(e3 != cudaSuccess ? e3 : e4);
        dev_free(G->d_off);
        dev_free(G->d_adj);
        delete G;
        return fail(HUGE_ECUDA, "copying the graph to the device failed: " + msg);
    }
    G->grid = persistent_grid(&G->warps);
    {
        const int hrc = build_hub_bitmaps(*G, default_hub_min_degree(n), kDefaultHubBytes);
        if (hrc != HUGE_OK) {
            dev_free(G->d_off);
            dev_free(G->d_adj);
            delete G;
            return hrc;
        }
    }

    // graph statistics for the learned estimator: log-scaled size and degree moments/quantiles
    {
        std::vector<uint32_t> deg(n);
        double s1 = 0, s2 = 0, s3 = 0;
        for (uint32_t v = 0; v < n; v++) {
            deg[v] = G->h_off[v + 1] - G->h_off[v];
            const double d = deg[v];
            s1 += d;
            s2 += d * d;
            s3 += d * d * d;
        }
        std::vector<uint32_t> sorted = deg;
        std::sort(sorted.begin(), sorted.end());
        auto q = [&](double p) { return (double)sorted[std::min<size_t>(n - 1, (size_t)(p * (n - 1)))]; };
        G->gstats = {(float)std::log2(1.0 + n), (float)std::log2(1.0 + nnz / 2.0),
                     (float)std::log2(1.0 + s1 / n), (float)std::log2(1.0 + maxd),
                     (float)std::log2(1.0 + q(0.5)), (float)std::log2(1.0 + q(0.9)),
                     (float)std::log2(1.0 + q(0.99)), (float)std::log2(1.0 + q(0.999)),
                     (float)std::log2(1.0 + s2 / n), (float)(std::log2(1.0 + s3 / n) / 2.0)};
    }
    *out = G;
    return HUGE_OK;
}

void graph_free(DevGraph *G) {
    if (!G) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(G->device);
    G->ws.release();
    free_hub_bitmaps(*G);
    if (G->d_off) dev_free(G->d_off);
    if (G->d_adj) dev_free(G->d_adj);
    cudaSetDevice(cur);
    delete G;
}

}  // namespace huge
