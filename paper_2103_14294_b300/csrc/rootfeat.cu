// Per-root features for a learned model of per-root work: the plan's sub-query features of the
// whole query (graph statistics and query shape, the estimator's inputs) plus statistics of the
// root's neighbourhood computed on the device, one warp per root.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "plan.h"

namespace huge {
namespace {

constexpr int kRootFeat0 = 46;  // first feature slot the query features leave free

// out[i * 8 + t]: deg(r), |N(r) ∩ (r, n)|, sum / max of deg(u) over N(r), sum of deg(u) over
// N(r) ∩ (r, n), sum of |N(u) ∩ (r, n)| over N(r) ∩ (r, n) (two-hop upward work), r / n
__global__ void root_stats_kernel(const uint32_t *__restrict__ off, const uint32_t *__restrict__ adj, uint32_t n,
                                  const uint32_t *__restrict__ roots, uint64_t nroots, float *out) {
    const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31;
    if (w >= nroots) return;
    const uint32_t r = roots[w];
    const uint32_t b = off[r], e = off[r + 1];
    double sdeg = 0, sup_deg = 0, up2 = 0;
    uint32_t mdeg = 0, nup = 0;
    for (uint32_t i = b + lane; i < e; i += 32) {
        const uint32_t u = adj[i];
        const uint32_t du = off[u + 1] - off[u];
        sdeg += du;
        mdeg = max(mdeg, du);
        if (u > r) {
            nup++;
            sup_deg += du;
            // |N(u) ∩ (r, n)|: the tail of u's sorted list above r
            uint32_t lo = off[u], hi = off[u + 1];
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (adj[mid] <= r) lo = mid + 1;
                else hi = mid;
            }
            up2 += off[u + 1] - lo;
        }
    }
    for (int s = 16; s >= 1; s >>= 1) {
        sdeg += __shfl_xor_sync(0xffffffffu, sdeg, s);
        sup_deg += __shfl_xor_sync(0xffffffffu, sup_deg, s);
        up2 += __shfl_xor_sync(0xffffffffu, up2, s);
        mdeg = max(mdeg, __shfl_xor_sync(0xffffffffu, mdeg, s));
        nup += __shfl_xor_sync(0xffffffffu, nup, s);
    }
    if (lane == 0) {
        float *o = out + w * 8;
        o[0] = (float)(e - b);
        o[1] = (float)nup;
        o[2] = (float)sdeg;
        o[3] = (float)mdeg;
        o[4] = (float)sup_deg;
        o[5] = (float)up2;
        o[6] = (float)r / (float)n;
        o[7] = 0.f;
    }
}

}  // namespace
}  // namespace huge

using namespace huge;

extern "C" int huge_root_features(const huge_plan_t *p, const uint32_t *roots, uint64_t nroots, float *out) {
    set_error("");
    if (!p || !p->G || (!roots && nroots) || (!out && nroots)) return fail(HUGE_EINVAL, "null argument");
    DevGraph &G = *p->G;
    if (G.directed) return fail(HUGE_EINVAL, "root features are defined for undirected graphs");
    for (uint64_t i = 0; i < nroots; i++)
        if (roots[i] >= G.n) return fail(HUGE_EINVAL, "root id out of range");
    if (nroots == 0) return HUGE_OK;
    float q[64];
    subquery_features(p->Q, p->lt, (1u << p->Q.k) - 1, G.gstats, q);
    uint32_t *d_roots = (uint32_t *)G.ws.get(14, nroots * 4);
    float *d_out = (float *)G.ws.get(15, nroots * 8 * sizeof(float));
    if (!d_roots || !d_out) return fail(HUGE_ENOMEM, "device allocation for root features failed");
    cudaError_t e = cudaMemcpy(d_roots, roots, nroots * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const uint64_t threads = nroots * 32;
        root_stats_kernel<<<(unsigned)((threads + 255) / 256), 256>>>(G.d_off, G.d_adj, G.n, d_roots, nroots, d_out);
        e = cudaGetLastError();
    }
    std::vector<float> st(nroots * 8);
    if (e == cudaSuccess) e = cudaMemcpy(st.data(), d_out, st.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HUGE_ECUDA, std::string("root features: ") + cudaGetErrorString(e));
    }
    const float k = (float)p->Q.k;
    for (uint64_t i = 0; i < nroots; i++) {
        float *o = out + i * 64;
        memcpy(o, q, sizeof(q));
        const float *s = &st[i * 8];
        float *f = o + kRootFeat0;
        for (int t = 0; t < 6; t++) f[t] = std::log1p(s[t]);
        f[6] = s[6];
        f[7] = (k - 1.f) * std::log1p(s[1]);  // growth if each step kept the upward degree
        f[8] = std::log1p(s[5]) + (k - 3.f) * std::log1p(s[1]) * 0.5f;
        f[9] = f[0] * f[0];
        f[10] = f[1] * f[1];
    }
    return HUGE_OK;
}
