// PUSH-JOIN (Sec. 4.2-4.3): hash join of two partial-match sets R(q_l), R(q_r) on the join key
// V_l & V_r. On one GPU the shuffle by join key becomes a device hash table: the left rows are
// grouped by key (open addressing on the packed key, one contiguous group per key), and every
// right row is matched against its key group. A joined pair is a match of q iff the non-key
// vertices of the two sides are distinct and the partial-order pairs that span the two sides
// hold (the local join of Sec. 4.3 compares all rows of a key group: a nested loop per key).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "internal.h"

namespace huge {

#define JFULL 0xffffffffu
constexpr unsigned long long kEmptyKey = ~0ull;

struct JoinDev {
    JoinSpec js;
    const uint32_t *L;
    const uint32_t *R;
    unsigned long long nleft, nright;
    unsigned long long *keys;  // H
    uint32_t *cnt;             // H
    uint32_t *start;           // H
    uint32_t *fill;            // H
    uint32_t *slot_of;         // nleft
    uint32_t *perm;            // nleft
    unsigned long long H;
    unsigned long long *total; // group allocator, then [1..2] 128-bit count
    uint32_t *sink;
    unsigned long long sink_cap;
    unsigned long long *tail;
    unsigned long long limit_ns;  // the probe gives up (total[3] = 1) after this long
};

__device__ __forceinline__ unsigned long long hash64(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

template <int N>
__device__ __forceinline__ uint32_t jsel(const uint32_t (&f)[N], int idx) {
    uint32_t v = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) v = (p == idx) ? f[p] : v;
    return v;
}

// Key of a row: exact packing for one or two key vertices, else a 64-bit mix (groups may then
// hold several keys; the probe compares the full key).
__device__ __forceinline__ unsigned long long row_key(const uint32_t (&f)[kMaxK], const int *cols, int nkey) {
    if (nkey == 1) return (unsigned long long)jsel(f, cols[0]);
    if (nkey == 2) return ((unsigned long long)jsel(f, cols[0]) << 32) | jsel(f, cols[1]);
    unsigned long long h = 0x9e3779b97f4a7c15ULL;
    for (int i = 0; i < nkey; i++) h = hash64(h ^ (unsigned long long)jsel(f, cols[i]) * 0x100000001b3ULL);
    return h == kEmptyKey ? h - 1 : h;
}

__global__ void join_build_insert(JoinDev d) {
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= d.nleft) return;
    uint32_t f[kMaxK];
#pragma unroll
    for (int p = 0; p < kMaxK; ++p) f[p] = (p < d.js.nl) ? d.L[i * d.js.nl + p] : 0u;
    const unsigned long long key = row_key(f, d.js.lkey, d.js.nkey);
    unsigned long long h = hash64(key) & (d.H - 1);
    for (unsigned long long probe = 0; probe < d.H; probe++) {
        const unsigned long long prev = atomicCAS(d.keys + h, kEmptyKey, key);
        if (prev == kEmptyKey || prev == key) {
            d.slot_of[i] = (uint32_t)h;
            atomicAdd(d.cnt + h, 1u);
            return;
        }
        h = (h + 1) & (d.H - 1);
    }
}

// One contiguous range per non-empty slot (group order is arbitrary).
__global__ void join_alloc_groups(JoinDev d) {
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t c = (i < d.H) ? d.cnt[i] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const uint32_t t = __shfl_up_sync(JFULL, incl, s);
        if ((int)lane >= s) incl += t;
    }
    unsigned long long base = 0;
    if (lane == 31 && incl) base = atomicAdd(d.total, (unsigned long long)incl);
    base = __shfl_sync(JFULL, base, 31);
    if (i < d.H) d.start[i] = (uint32_t)(base + incl - c);
}

__global__ void join_scatter(JoinDev d) {
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= d.nleft) return;
    const uint32_t s = d.slot_of[i];
    const uint32_t pos = d.start[s] + atomicAdd(d.fill + s, 1u);
    d.perm[pos] = (uint32_t)i;
}

// Largest lane i with pre_i <= g (pre non-decreasing over lanes, pre_0 = 0). 64-bit: a key
// group may hold up to 2^32 - 1 left rows, so a batch's 32 groups can exceed 2^32 candidates.
__device__ __forceinline__ int jfind_owner(unsigned long long pre, unsigned long long g) {
    int own = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const unsigned long long pc = __shfl_sync(JFULL, pre, own + s);
        if (pc <= g) own += s;
    }
    return own;
}

__device__ __forceinline__ unsigned long long jtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return __shfl_sync(JFULL, t, 0);
}

template <int MODE>
__global__ void __launch_bounds__(256) join_probe(JoinDev d) {
    const uint32_t lane = threadIdx.x & 31;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    const JoinSpec &js = d.js;
    unsigned long long acc = 0;
    const unsigned long long t_start = jtimer();
    uint32_t iters = 0;
    for (unsigned long long b = warp * 32; b < d.nright; b += nwarps * 32) {
        const unsigned long long r = b + lane;
        const bool valid = r < d.nright;
        uint32_t fr[kMaxK];
#pragma unroll
        for (int p = 0; p < kMaxK; ++p) fr[p] = (valid && p < js.nr) ? d.R[r * js.nr + p] : 0u;
        uint32_t gstart = 0, glen = 0;
        if (valid) {
            const unsigned long long key = row_key(fr, js.rkey, js.nkey);
            unsigned long long h = hash64(key) & (d.H - 1);
            for (unsigned long long probe = 0; probe < d.H; probe++) {
                const unsigned long long k = d.keys[h];
                if (k == key) {
                    gstart = d.start[h];
                    glen = d.cnt[h];
                    break;
                }
                if (k == kEmptyKey) break;
                h = (h + 1) & (d.H - 1);
            }
        }
        unsigned long long incl = glen;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const unsigned long long t = __shfl_up_sync(JFULL, incl, s);
            if ((int)lane >= s) incl += t;
        }
        const unsigned long long pre = incl - glen;
        const unsigned long long T = __shfl_sync(JFULL, incl, 31);
        for (unsigned long long base = 0; base < T; base += 32) {
            if ((++iters & 1023u) == 0 && jtimer() - t_start > d.limit_ns) {  // bounded run time
                if (lane == 0) atomicExch(d.total + 3, 1ull);
                return;
            }
            const unsigned long long g = base + lane;
            const int own = jfind_owner(pre, g);
            bool ok = g < T;
            const uint32_t gi = __shfl_sync(JFULL, gstart, own) + (uint32_t)(g - __shfl_sync(JFULL, pre, own));
            uint32_t fo[kMaxK], fl[kMaxK];
#pragma unroll
            for (int p = 0; p < kMaxK; ++p) fo[p] = __shfl_sync(JFULL, fr[p], own);
#pragma unroll
            for (int p = 0; p < kMaxK; ++p) fl[p] = 0;
            if (ok) {
                const unsigned long long li = d.perm[gi];
#pragma unroll
                for (int p = 0; p < kMaxK; ++p)
                    if (p < js.nl) fl[p] = d.L[li * js.nl + p];
            }
            if (ok && js.nkey > 2)
                for (int kk = 0; kk < js.nkey; kk++) ok = ok && jsel(fl, js.lkey[kk]) == jsel(fo, js.rkey[kk]);
            for (int a = 0; a < js.n_nonkey_l && ok; a++) {
                const uint32_t x = jsel(fl, js.nonkey_l[a]);
                for (int c = 0; c < js.n_nonkey_r; c++) ok = ok && x != jsel(fo, js.nonkey_r[c]);
            }
            for (int t = 0; t < js.n_lr && ok; t++) ok = jsel(fl, js.lr_l[t]) < jsel(fo, js.lr_r[t]);
            for (int t = 0; t < js.n_rl && ok; t++) ok = jsel(fo, js.rl_r[t]) < jsel(fl, js.rl_l[t]);
            const unsigned m = __ballot_sync(JFULL, ok);
            const uint32_t nm = __popc(m);
            acc += nm;
            if (MODE == HUGE_LIST && nm) {
                unsigned long long slot0 = 0;
                if (lane == 0) slot0 = atomicAdd(d.tail, (unsigned long long)nm);
                slot0 = __shfl_sync(JFULL, slot0, 0);
                const uint32_t rank = __popc(m & ((1u << lane) - 1u));
                if (ok && slot0 + rank < d.sink_cap) {
                    uint32_t *dst = d.sink + (slot0 + rank) * js.k;
                    for (int c = 0; c < js.nl; c++) dst[js.out_col_l[c]] = jsel(fl, c);
                    for (int c = 0; c < js.nr; c++)
                        if (js.out_col_r[c] >= 0) dst[js.out_col_r[c]] = jsel(fo, c);
                }
            }
        }
    }
    if (lane == 0 && acc) {
        const unsigned long long old = atomicAdd(d.total + 1, acc);
        if (old + acc < old) atomicAdd(d.total + 2, 1ull);
    }
}

int join_count_or_list(const JoinSpec &js, const uint32_t *d_left, uint64_t nleft, const uint32_t *d_right,
                       uint64_t nright, int mode, uint32_t *sink, uint64_t sink_cap,
                       unsigned long long *d_tail, Workspace &ws, uint32_t limit_ms, cudaStream_t s,
                       unsigned __int128 *count, std::string *err) {
    *count = 0;
    if (nleft == 0 || nright == 0) return HUGE_OK;
    if (nleft >= 0xffffffffull) {
        *err = "join side too large";
        return HUGE_ENOMEM;
    }
    unsigned long long H = 1;
    while (H < 2 * nleft) H <<= 1;
    JoinDev d;
    memset(&d, 0, sizeof(d));
    d.js = js;
    d.L = d_left;
    d.R = d_right;
    d.nleft = nleft;
    d.nright = nright;
    d.H = H;
    const size_t bytes = H * (8 + 4 + 4 + 4) + nleft * 8 + 64;
    void *buf = ws.get(13, bytes);  // grow-only: reused by every partition pass and call
    if (!buf) {
        *err = "device allocation for the join table failed";
        return HUGE_ENOMEM;
    }
    cudaError_t e;
    char *p = (char *)buf;
    d.keys = (unsigned long long *)p;
    p += H * 8;
    d.total = (unsigned long long *)p;
    p += 64;
    d.cnt = (uint32_t *)p;
    p += H * 4;
    d.start = (uint32_t *)p;
    p += H * 4;
    d.fill = (uint32_t *)p;
    p += H * 4;
    d.slot_of = (uint32_t *)p;
    p += nleft * 4;
    d.perm = (uint32_t *)p;
    d.sink = sink;
    d.sink_cap = sink ? sink_cap : 0;
    d.tail = d_tail;
    d.limit_ns = (limit_ms ? (unsigned long long)limit_ms : 600000ull) * 1000000ull;
    cudaMemsetAsync(d.keys, 0xff, H * 8, s);
    cudaMemsetAsync(d.total, 0, 64, s);
    cudaMemsetAsync(d.cnt, 0, H * 4, s);
    cudaMemsetAsync(d.fill, 0, H * 4, s);
    const unsigned bt = 256;
    join_build_insert<<<(unsigned)((nleft + bt - 1) / bt), bt, 0, s>>>(d);
    join_alloc_groups<<<(unsigned)((H + bt - 1) / bt), bt, 0, s>>>(d);
    join_scatter<<<(unsigned)((nleft + bt - 1) / bt), bt, 0, s>>>(d);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long batches = (nright + 31) / 32;
    unsigned grid = (unsigned)std::min<unsigned long long>((batches + 7) / 8, (unsigned long long)sms * 8);
    if (grid < 1) grid = 1;
    if (mode == HUGE_LIST)
        join_probe<HUGE_LIST><<<grid, 256, 0, s>>>(d);
    else
        join_probe<HUGE_COUNT><<<grid, 256, 0, s>>>(d);
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(h, d.total, 32, cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *err = std::string("join kernels: ") + cudaGetErrorString(e);
        return HUGE_ECUDA;
    }
    if (h[3]) {
        *err = "the join probe reached its time limit";
        return HUGE_ETIMEOUT;
    }
    *count = ((unsigned __int128)h[2] << 64) | h[1];
    return HUGE_OK;
}

}  // namespace huge
