// Persistent PULL-EXTEND enumerator for sm_103a.
//
// One launch runs a whole EXTEND chain (Sec. 4.2 dataflow SCAN -> EXTEND ... -> SINK) for one
// or many queries. Every warp is a worker that runs the DFS/BFS-adaptive schedule of Alg. 5
// on its own bounded buffers:
//  * level l holds rows of partial matches (l = 0: a range of root ids); each level has a
//    fixed capacity `cap` rows per warp (the fixed-capacity output queue Q_O of Sec. 5.2);
//  * the warp always works on the deepest level that still has input (backtracking to the
//    precursor when a level runs dry), and keeps consuming input rows of that level while
//    the next level has room for another 32-candidate batch (it yields when Q_O is full);
//  * a row whose candidates do not fit is split: the warp records the position inside the
//    row's driver list and resumes there, so one row never needs D_G rows of space.
// An EXTEND batch (Alg. 4 intersect stage, Eq. 2) takes up to 32 input rows, one per lane.
// Each lane range-restricts its row's lists to the partial-order bounds by binary search,
// picks the shortest restricted list as the driver, and the warp flattens all drivers into
// one candidate space that it walks 32 candidates at a time (warp-level load balance over
// uneven rows). Each candidate is checked against the other lists by binary search and
// against the bound vertices (injectivity, Alg. 4); survivors are compacted with a ballot
// and appended to the next level, counted (COUNT sink) or written (LIST sink).
// Work stealing (Sec. 5.3): once the root queue is empty, idle warps announce themselves and
// busy warps donate half of their shallowest pending level into a pool of slots; nobody ever
// waits on another warp, and idle warps stop polling after a time limit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace huge {

#define FULLMASK 0xffffffffu

#ifndef HUGE_LONG_ROW
#define HUGE_LONG_ROW 64
#endif
#ifndef HUGE_LONG_VEC
#define HUGE_LONG_VEC 2
#endif
#ifndef HUGE_MIN_BLOCKS
#define HUGE_MIN_BLOCKS 4
#endif
constexpr uint32_t kLongRow = HUGE_LONG_ROW;  // last COUNT operator: rows with this many candidates run alone
constexpr int kLongVec = HUGE_LONG_VEC;        // 16-byte driver loads per lane per step of such a row

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The same timer value in every lane (decisions taken on it must be warp-uniform).
__device__ __forceinline__ unsigned long long wtimer() {
    unsigned long long t = 0;
    if ((threadIdx.x & 31) == 0) t = gtimer();
    return __shfl_sync(0xffffffffu, t, 0);
}

__device__ __forceinline__ uint32_t lower_bound_dev(const uint32_t *__restrict__ a, uint32_t lo,
                                                    uint32_t hi, uint32_t key) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Is key in the sorted range a[lo, hi)?
__device__ __forceinline__ bool contains_dev(const uint32_t *__restrict__ a, uint32_t lo, uint32_t hi,
                                             uint32_t key) {
    if (lo >= hi) return false;
    uint32_t n = hi - lo, base = lo;
    while (n > 1) {
        const uint32_t h = n >> 1;
        base = (__ldg(a + base + h) <= key) ? base + h : base;
        n -= h;
    }
    return __ldg(a + base) == key;
}

template <int N>
__device__ __forceinline__ uint32_t sel(const uint32_t (&f)[N], int idx) {
    uint32_t v = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) v = (p == idx) ? f[p] : v;
    return v;
}

// Largest lane i with pre_i <= g, for pre non-decreasing over lanes and pre_0 = 0.
__device__ __forceinline__ int find_owner(uint32_t pre, uint32_t g) {
    int own = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t pc = __shfl_sync(FULLMASK, pre, own + s);
        if (pc <= g) own += s;
    }
    return own;
}

__device__ __forceinline__ void add_u128(unsigned long long *lohi, unsigned long long x) {
    const unsigned long long old = atomicAdd(lohi, x);
    if (old + x < old) atomicAdd(lohi + 1, 1ull);
}

__device__ __forceinline__ uint32_t mix_key(uint32_t h, uint32_t x) {
    h ^= x * 0x9e3779b1u;
    h = (h ^ (h >> 15)) * 0x85ebca6bu;
    return h ^ (h >> 13);
}

// Per-warp mutable state; level-l fields live in lane l (lane-distributed).
struct WState {
    uint32_t cnt, cur, res;   // rows in level (lane l), consumed rows, resume offset in row `cur`
    unsigned long long prod;  // rows produced into level (lane l), for the per-level log
};

// Per-warp shared-memory tile of the current batch: field[x][lane] describes the row held by
// `lane` (list ranges after the partial-order restriction, row values, values to exclude).
// A lane reads the owner's entry of a candidate as field[x][own]: broadcast or conflict-free.
struct RowTile {
    uint32_t b[kMaxExt][32];
    uint32_t e[kMaxExt][32];
    uint32_t h[kMaxExt][32];   // hub bitmap row of the list's vertex, or kNoHub
    uint32_t inj[kMaxExt][32];
    uint32_t f[kMaxK][32];
};

// Is v in N(x), x a hub with bitmap row hr? One probe of the n-bit row.
__device__ __forceinline__ bool hub_bit(const KParams &kp, uint32_t hr, uint32_t v) {
    return (__ldg(kp.hub_bits + (uint64_t)hr * kp.hub_wpr + (v >> 5)) >> (v & 31)) & 1u;
}

// |N(v) ∩ [0, k)| for a hub v with bitmap row hr, k < n: the rank index gives the set bits below
// k's 256-bit block, one 32-byte load gives the block's words below k.
__device__ __forceinline__ uint32_t hub_rank_lt(const KParams &kp, uint32_t hr, uint32_t k) {
    const uint32_t blk = k >> 8;
    const uint32_t *__restrict__ row = kp.hub_bits + (uint64_t)hr * kp.hub_wpr;
    uint32_t r = __ldg(kp.hub_rank + (uint64_t)hr * kp.hub_nblk + blk);
    const uint4 *p = reinterpret_cast<const uint4 *>(row + (uint64_t)blk * 8);
    const uint4 a = __ldg(p), b = __ldg(p + 1);
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const uint32_t wi = (k >> 5) & 7u, below = (1u << (k & 31)) - 1u;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) r += __popc(i < wi ? w[i] : (i == wi ? (w[i] & below) : 0u));
    return r;
}

// Is candidate v in list j of the row held by lane `own`? The candidate already lies inside the
// partial-order range every list of the row is restricted to, so a hub's whole-list bitmap
// answers for the restricted list; other lists are binary-searched in their restricted range.
__device__ __forceinline__ bool in_list(const KParams &kp, const RowTile &rt, int j, int own, uint32_t v) {
    const uint32_t hr = rt.h[j][own];
    return hr != kNoHub ? hub_bit(kp, hr, v) : contains_dev(kp.adj, rt.b[j][own], rt.e[j][own], v);
}

// Last operator: count the survivors (COUNT sink) or write them as rows in query-vertex order
// (LIST sink). `own` is the lane holding the row that candidate v extends. In a PUSH-JOIN
// partition pass only rows whose key hashes to the pass's bucket are kept.
template <int MODE>
__device__ __forceinline__ void emit_last(const KParams &kp, const Prog *__restrict__ pg, int w, bool ok,
                                          uint32_t v, int own, const RowTile &rt, unsigned long long &acc) {
    const uint32_t lane = threadIdx.x & 31;
    if (MODE == HUGE_COUNT && pg->part_mod <= 1) {
        acc += __popc(__ballot_sync(FULLMASK, ok));
        return;
    }
    if (pg->part_mod > 1) {
        uint32_t h = 0x12345u;
        for (int kk = 0; kk < pg->n_key; ++kk) {
            const int pos = pg->key_pos[kk];
            h = mix_key(h, pos < w ? rt.f[pos][own] : v);
        }
        ok = ok && (h % pg->part_mod == pg->part_id);
    }
    const unsigned m = __ballot_sync(FULLMASK, ok);
    const uint32_t nm = __popc(m);
    acc += nm;
    if (MODE == HUGE_COUNT || nm == 0) return;
    const uint32_t rank = __popc(m & ((1u << lane) - 1u));
    unsigned long long slot0 = 0;
    if (lane == 0) {
        slot0 = atomicAdd(kp.sink_tail, (unsigned long long)nm);
        if (slot0 + nm > kp.sink_cap) atomicExch(&kp.ctl->overflow, 1);  // the host retries smaller
    }
    slot0 = __shfl_sync(FULLMASK, slot0, 0);
    if (ok) {
        const unsigned long long r = slot0 + rank;
        if (r < kp.sink_cap) {
            uint32_t *dst = kp.sink + r * kp.sink_width;
            for (int p = 0; p < w; ++p) dst[pg->col_of_pos[p]] = rt.f[p][own];
            dst[pg->col_of_pos[w]] = v;
        }
    }
}

// One step of a long row whose other lists are NP hub bitmaps: kLongVec 16-byte driver loads
// per lane (positions from the 16-byte boundary a0), each candidate probed in every bitmap
// with a funnel shift (the shift count is taken mod 32). FULL: every position of the step lies
// inside the row [db, a1), so no masking. Returns this lane's matches.
template <int NP, bool FULL>
__device__ __forceinline__ uint32_t hub_probe_step(const uint4 *__restrict__ src, uint32_t i0, uint32_t lane,
                                                   uint32_t a0, uint32_t db, uint32_t a1,
                                                   const uint32_t *__restrict__ bmA,
                                                   const uint32_t *__restrict__ bmB) {
    uint32_t v[4 * kLongVec];
#pragma unroll
    for (int u = 0; u < kLongVec; ++u) {
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        if (FULL || a0 + i0 + 128u * u + 4u * lane < a1) q = __ldg(src + ((i0 + 128u * u) >> 2) + lane);
        v[4 * u + 0] = q.x;
        v[4 * u + 1] = q.y;
        v[4 * u + 2] = q.z;
        v[4 * u + 3] = q.w;
    }
    uint32_t hits = 0;
#pragma unroll
    for (int u = 0; u < 4 * kLongVec; ++u) {
        const uint32_t wa = __ldg(bmA + (v[u] >> 5));
        uint32_t bit = __funnelshift_r(wa, wa, v[u]);
        if (NP == 2) {
            const uint32_t wb = __ldg(bmB + (v[u] >> 5));
            bit &= __funnelshift_r(wb, wb, v[u]);
        }
        if (!FULL) {
            const uint32_t e = a0 + i0 + 128u * (u / 4) + 4u * lane + (u % 4);
            bit &= (e >= db && e < a1) ? 1u : 0u;
        }
        hits += bit & 1u;
    }
    return hits;
}

// ---------------------------------------------------------------------------------------
// EXTEND batch: up to 32 rows of level l -> level l + 1 (or the sink when `last`).
// ---------------------------------------------------------------------------------------
template <int MODE, bool STATS>
__device__ __forceinline__ void extend_batch(const KParams &kp, const Prog *__restrict__ pg,
                                             const StepDesc &st, int l, bool last, uint32_t *region,
                                             WState &ws, RowTile &rt, unsigned long long &acc,
                                             unsigned long long &inter, unsigned long long &bytes,
                                             unsigned long long t_start, bool &abort) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t cnt_l = __shfl_sync(FULLMASK, ws.cnt, l);
    const uint32_t cur_l = __shfl_sync(FULLMASK, ws.cur, l);
    const uint32_t res_l = __shfl_sync(FULLMASK, ws.res, l);
    const uint32_t R = min(32u, cnt_l - cur_l);
    const int w = st.w;
    const int n_ext = st.n_ext, n_inj = st.n_inj;
    const bool has_row = lane < R;

    // ---- set-up: one row per lane ----
    uint32_t len = 0, drv_b = 0, slen = 0xffffffffu, sec_b = 0, sec_e = 0;
    uint32_t drv_h = kNoHub, sec_h = kNoHub;
    int drv = 0, sec = 0;
    unsigned long long rbytes = 0;  // algorithmic bytes of this lane's row: its restricted lists
    {
        uint32_t f[kMaxK];
#pragma unroll
        for (int p = 0; p < kMaxK; ++p) f[p] = 0;
        if (has_row) {
            const uint32_t row = cur_l + lane;
            if (l == 0) {
                f[0] = row;
            } else {
                const uint32_t *src = region + pg->lvl_off[l] + (uint64_t)row * w;
#pragma unroll
                for (int p = 0; p < kMaxK; ++p)
                    if (p < w) f[p] = src[p];
            }
        }
#pragma unroll
        for (int p = 0; p < kMaxK; ++p)
            if (p < w) rt.f[p][lane] = f[p];
        // partial-order bounds and the label's id range: candidates u with lo_key <= u < hi_key
        uint32_t lo_key = st.clo, hi_key = st.chi;
#pragma unroll
        for (int j = 0; j < kMaxK; ++j) {
            if (j < st.n_lo) lo_key = max(lo_key, sel(f, st.lo[j]) + 1u);
            if (j < st.n_hi) hi_key = min(hi_key, sel(f, st.hi[j]));
        }
        len = 0xffffffffu;
#pragma unroll
        for (int j = 0; j < kMaxExt; ++j) {
            if (j < n_ext) {
                uint32_t bb = 0, ee = 0, hr = kNoHub;
                if (has_row) {
                    // the list of f[ext[j]]: its out-list, or its in-list (list id + n) by the arc
                    const uint32_t x = sel(f, st.ext[j]) + (((st.dirs >> j) & 1u) ? kp.dir_base : 0u);
                    bb = __ldg(kp.off + x);
                    ee = __ldg(kp.off + x + 1);
                    if (kp.hub_row) hr = __ldg(kp.hub_row + x);
                    if (hr != kNoHub && kp.hub_rank) {  // a hub's bounds from its rank index
                        const uint32_t b0 = bb;
                        if (lo_key) bb = lo_key >= kp.n ? ee : b0 + hub_rank_lt(kp, hr, lo_key);
                        if (hi_key != 0xffffffffu) ee = max(bb, hi_key >= kp.n ? ee : b0 + hub_rank_lt(kp, hr, hi_key));
                    } else {
                        if (lo_key) bb = lower_bound_dev(kp.adj, bb, ee, lo_key);
                        if (hi_key != 0xffffffffu) ee = lower_bound_dev(kp.adj, bb, ee, hi_key);
                    }
                }
                rt.b[j][lane] = bb;
                rt.e[j][lane] = ee;
                rt.h[j][lane] = hr;
                if (STATS) rbytes += 4ull * (ee - bb);
                const uint32_t lj = ee - bb;
                if (lj < len) {  // shortest list drives, second shortest is the merge partner
                    slen = len;
                    sec = drv;
                    sec_b = drv_b;
                    sec_e = drv_b + len;
                    sec_h = drv_h;
                    len = lj;
                    drv = j;
                    drv_b = bb;
                    drv_h = hr;
                } else if (lj < slen) {
                    slen = lj;
                    sec = j;
                    sec_b = bb;
                    sec_e = ee;
                    sec_h = hr;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kMaxExt; ++q)
            if (q < n_inj) rt.inj[q][lane] = sel(f, st.inj[q]);
        if (!has_row || len == 0xffffffffu) len = 0;
        if (STATS && has_row) rbytes += 4ull * (unsigned)w;
    }
    if (lane == 0 && has_row) {  // resume inside the first row
        drv_b += res_l;
        len -= res_l;
    }
    __syncwarp();

    // ---- merge-path rows (last operator) ----
    // When the two shortest restricted lists have comparable lengths and the second is not a
    // hub's (whose bitmap answers in one probe), the warp intersects them cooperatively, 32 + 32
    // elements per step (coalesced windows, a 5-step shuffle search per element) instead of one
    // binary search per candidate. Skewed rows stay on the probe path below.
    if (last && pg->merge_ratio && n_ext >= 2) {
        const bool use_merge = has_row && len >= 16u && sec_h == kNoHub &&
                               (unsigned long long)slen <= (unsigned long long)pg->merge_ratio * len;
        unsigned mm = __ballot_sync(FULLMASK, use_merge);
        const uint32_t mlen = len;
        if (use_merge) len = 0;
        while (mm) {
            const int r = __ffs(mm) - 1;
            mm &= mm - 1;
            uint32_t ia = __shfl_sync(FULLMASK, drv_b, r);
            const uint32_t a1 = ia + __shfl_sync(FULLMASK, mlen, r);
            uint32_t ib = __shfl_sync(FULLMASK, sec_b, r);
            const uint32_t b1 = __shfl_sync(FULLMASK, sec_e, r);
            const int od = __shfl_sync(FULLMASK, drv, r), os = __shfl_sync(FULLMASK, sec, r);
            uint32_t steps = 0;
            while (ia < a1 && ib < b1) {
                if ((++steps & 1023u) == 0 && wtimer() - t_start > kp.limit_ns) {
                    abort = true;
                    return;
                }
                const uint32_t x = (ia + lane < a1) ? __ldg(kp.adj + ia + lane) : 0xffffffffu;
                const uint32_t y = (ib + lane < b1) ? __ldg(kp.adj + ib + lane) : 0xffffffffu;
                int jj = 0;  // largest lane with y <= x (y ascends over lanes)
#pragma unroll
                for (int sft = 16; sft >= 1; sft >>= 1) {
                    const uint32_t yy = __shfl_sync(FULLMASK, y, jj + sft);
                    if (yy <= x) jj += sft;
                }
                const uint32_t yj = __shfl_sync(FULLMASK, y, jj);  // every lane takes part
                bool ok = (x != 0xffffffffu) && (yj == x);
                for (int j = 0; j < n_ext; ++j)
                    if (ok && j != od && j != os) ok = in_list(kp, rt, j, r, x);
                for (int q = 0; q < n_inj; ++q) ok = ok && (x != rt.inj[q][r]);
                emit_last<MODE>(kp, pg, w, ok, x, r, rt, acc);
                const uint32_t amax = __shfl_sync(FULLMASK, x, 31), bmax = __shfl_sync(FULLMASK, y, 31);
                if (amax <= bmax) {  // every x of the window is resolved
                    ia += 32;
                    ib += __popc(__ballot_sync(FULLMASK, y <= amax));
                } else {             // every y of the window is resolved
                    ia += __popc(__ballot_sync(FULLMASK, x <= bmax));
                    ib += 32;
                }
            }
        }
    }

    // ---- long rows of the last operator in COUNT mode: one row at a time, vectorised ----
    // A row with many candidates is walked by the whole warp. The driver list is read with
    // 16-byte loads from the 16-byte boundary at or below its start (kLongVec vectors = 4 x
    // kLongVec candidates per lane per step; positions outside the row are masked), so one step
    // issues kLongVec coalesced loads and 4 x kLongVec independent probes per lane. The row's
    // driver start, its other lists' hub rows or ranges and its excluded values are
    // warp-uniform; matches are counted per lane and reduced once per row.
    if (MODE == HUGE_COUNT && last && pg->part_mod <= 1 && kp.vec_ok) {
        unsigned lm = __ballot_sync(FULLMASK, has_row && len >= kLongRow);
        while (lm) {
            const int r = __ffs(lm) - 1;
            lm &= lm - 1;
            const uint32_t L = __shfl_sync(FULLMASK, len, r);
            const uint32_t db = __shfl_sync(FULLMASK, drv_b, r);
            const int od = __shfl_sync(FULLMASK, drv, r);
            if ((int)lane == r) len = 0;  // consumed here, not by the flattened path below
            const uint32_t a0 = db & ~3u, a1 = db + L;  // aligned start, end (exclusive)
            const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(kp.adj + a0);
            uint32_t cnt = 0, steps = 0;
            // hub-only rows (every other list has a bitmap, nothing to exclude): bit probes only
            int np = 0;
            const uint32_t *bmA = nullptr, *bmB = nullptr;
            bool hub_only = n_inj == 0;
            for (int j = 0; j < n_ext; ++j) {
                if (j == od) continue;
                const uint32_t hr = rt.h[j][r];
                if (hr == kNoHub) hub_only = false;
                else if (np == 0) bmA = kp.hub_bits + (uint64_t)hr * kp.hub_wpr;
                else bmB = kp.hub_bits + (uint64_t)hr * kp.hub_wpr;
                ++np;
            }
            if (hub_only && np == 0) {  // no list to probe, nothing to exclude: every candidate counts
                acc += L;
                continue;
            }
            if (hub_only && np <= 2) {
                for (uint32_t i0 = 0; a0 + i0 < a1; i0 += 128u * kLongVec) {
                    if ((++steps & 255u) == 0 && wtimer() - t_start > kp.limit_ns) {
                        abort = true;
                        return;
                    }
                    const bool full = a0 + i0 >= db && a0 + i0 + 128u * kLongVec <= a1;  // warp-uniform
                    if (full) {
                        if (np == 1) cnt += hub_probe_step<1, true>(src, i0, lane, a0, db, a1, bmA, bmA);
                        else cnt += hub_probe_step<2, true>(src, i0, lane, a0, db, a1, bmA, bmB);
                    } else {
                        if (np == 1) cnt += hub_probe_step<1, false>(src, i0, lane, a0, db, a1, bmA, bmA);
                        else cnt += hub_probe_step<2, false>(src, i0, lane, a0, db, a1, bmA, bmB);
                    }
                }
                acc += __reduce_add_sync(FULLMASK, cnt);
                continue;
            }
            for (uint32_t i0 = 0; a0 + i0 < a1; i0 += 128u * kLongVec) {
                if ((++steps & 255u) == 0 && wtimer() - t_start > kp.limit_ns) {
                    abort = true;
                    return;
                }
                uint32_t v[4 * kLongVec];
                bool ok[4 * kLongVec];
#pragma unroll
                for (int u = 0; u < kLongVec; ++u) {
                    const uint32_t e0 = a0 + i0 + 128u * u + 4u * lane;  // first position of this vector
                    uint4 q = make_uint4(0u, 0u, 0u, 0u);
                    if (e0 < a1) q = __ldg(src + ((i0 + 128u * u) >> 2) + lane);
                    v[4 * u + 0] = q.x;
                    v[4 * u + 1] = q.y;
                    v[4 * u + 2] = q.z;
                    v[4 * u + 3] = q.w;
#pragma unroll
                    for (int c = 0; c < 4; ++c) ok[4 * u + c] = (e0 + c >= db) && (e0 + c < a1);
                }
                for (int j = 0; j < n_ext; ++j) {
                    if (j == od) continue;
                    const uint32_t hr = rt.h[j][r];
                    if (hr != kNoHub) {
                        const uint32_t *__restrict__ bm = kp.hub_bits + (uint64_t)hr * kp.hub_wpr;
#pragma unroll
                        for (int u = 0; u < 4 * kLongVec; ++u)
                            ok[u] = ok[u] & ((__ldg(bm + (v[u] >> 5)) >> (v[u] & 31)) & 1u);
                    } else {
                        const uint32_t bb = rt.b[j][r], ee = rt.e[j][r];
#pragma unroll
                        for (int u = 0; u < 4 * kLongVec; ++u) ok[u] = ok[u] && contains_dev(kp.adj, bb, ee, v[u]);
                    }
                }
                for (int q = 0; q < n_inj; ++q) {
                    const uint32_t x = rt.inj[q][r];
#pragma unroll
                    for (int u = 0; u < 4 * kLongVec; ++u) ok[u] = ok[u] && v[u] != x;
                }
#pragma unroll
                for (int u = 0; u < 4 * kLongVec; ++u) cnt += ok[u] ? 1u : 0u;
            }
            acc += __reduce_add_sync(FULLMASK, cnt);
        }
    }

    // ---- probe path over the flattened candidates of all remaining rows ----
    uint32_t incl = len;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const uint32_t t = __shfl_up_sync(FULLMASK, incl, s);
        if ((int)lane >= s) incl += t;
    }
    const uint32_t pre = incl - len;
    const uint32_t T = __shfl_sync(FULLMASK, incl, 31);
    const int wo = w + 1;
    uint32_t *out = last ? nullptr : region + pg->lvl_off[l + 1];

    // o: the row holding candidate `base` (warp-uniform), o_end: its end in the flattened space
    int o = 0;
    uint32_t o_end = __shfl_sync(FULLMASK, incl, 0);
    for (uint32_t base = 0; base < T; base += 32) {
        if ((base & 32767u) == 32767u - 31u && wtimer() - t_start > kp.limit_ns) {  // every 1024 chunks
            abort = true;
            return;
        }
        while (o_end <= base) {  // base < T = incl[31], so this stops at a row o <= 31
            ++o;
            o_end = __shfl_sync(FULLMASK, incl, o);
        }
        if (!last) {
            const uint32_t cnt_n = __shfl_sync(FULLMASK, ws.cnt, l + 1);
            if (cnt_n + 32u > pg->cap) {  // Q_O full: yield, remember where to resume
                const uint32_t pre_o = __shfl_sync(FULLMASK, pre, o);
                const uint32_t nres = base - pre_o + (o == 0 ? res_l : 0u);
                if ((int)lane == l) {
                    ws.cur = cur_l + o;
                    ws.res = nres;
                }
                inter += o;
                if (STATS && (int)lane < o) bytes += rbytes;
                __syncwarp();
                return;
            }
        }
        const uint32_t g = base + lane;
        const bool valid = g < T;
        // a window inside one row (the common case for long lists) needs no owner search
        const int own = (o_end >= min(base + 32u, T)) ? o : find_owner(pre, g);
        const uint32_t off_in = g - __shfl_sync(FULLMASK, pre, own);
        const uint32_t db = __shfl_sync(FULLMASK, drv_b, own);
        const int od = __shfl_sync(FULLMASK, drv, own);
        const uint32_t v = valid ? __ldg(kp.adj + db + off_in) : 0u;
        bool ok = valid;
        for (int j = 0; j < n_ext; ++j)
            if (ok && j != od) ok = in_list(kp, rt, j, own, v);
        for (int q = 0; q < n_inj; ++q) ok = ok && (v != rt.inj[q][own]);
        if (last) {
            emit_last<MODE>(kp, pg, w, ok, v, own, rt, acc);
            continue;
        }
        const unsigned m = __ballot_sync(FULLMASK, ok);
        const uint32_t nm = __popc(m);
        const uint32_t rank = __popc(m & ((1u << lane) - 1u));
        const uint32_t cnt_n = __shfl_sync(FULLMASK, ws.cnt, l + 1);
        if (ok) {
            uint32_t *dst = out + (uint64_t)(cnt_n + rank) * wo;
            for (int p = 0; p < w; ++p) dst[p] = rt.f[p][own];
            dst[w] = v;
        }
        if ((int)lane == l + 1) {
            ws.cnt += nm;
            ws.prod += nm;
        }
        if (STATS && lane == 0) bytes += 4ull * wo * nm;
    }
    if ((int)lane == l) {
        ws.cur = cur_l + R;
        ws.res = 0;
    }
    inter += R;
    if (STATS && has_row) bytes += rbytes;
    __syncwarp();
}

// ---------------------------------------------------------------------------------------
// Verify-only EXTEND batch (Sec. 5.2): keep a row iff the listed pairs are data edges.
// ---------------------------------------------------------------------------------------
template <int MODE, bool STATS>
__device__ __forceinline__ void verify_batch(const KParams &kp, const Prog *__restrict__ pg,
                                             const StepDesc &st, int l, bool last, uint32_t *region,
                                             WState &ws, unsigned long long &acc,
                                             unsigned long long &inter, unsigned long long &bytes) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t cnt_l = __shfl_sync(FULLMASK, ws.cnt, l);
    const uint32_t cur_l = __shfl_sync(FULLMASK, ws.cur, l);
    const uint32_t R = min(32u, cnt_l - cur_l);
    const int w = st.w;
    bool ok = lane < R;
    uint32_t f[kMaxK];
#pragma unroll
    for (int p = 0; p < kMaxK; ++p) f[p] = 0;
    if (ok) {
        const uint32_t *src = region + pg->lvl_off[l] + (uint64_t)(cur_l + lane) * w;
#pragma unroll
        for (int p = 0; p < kMaxK; ++p)
            if (p < w) f[p] = src[p];
    }
#pragma unroll
    for (int j = 0; j < kMaxK; ++j) {
        if (j < st.n_ext && ok) {
            // the pair is an edge iff y is in x's list; for a directed graph the arc x -> y
            // (x's out-list, y's in-list) or, with the direction bit, y -> x
            const bool rev = (st.dirs >> j) & 1u;
            const uint32_t x = sel(f, st.ext[j]), y = sel(f, st.ext2[j]);
            const uint32_t lx = x + (rev ? kp.dir_base : 0u), ly = y + (rev ? 0u : kp.dir_base);
            const uint32_t bb = __ldg(kp.off + lx), ee = __ldg(kp.off + lx + 1);
            if (STATS) bytes += 4ull * (ee - bb);
            const uint32_t hx = kp.hub_row ? __ldg(kp.hub_row + lx) : kNoHub;
            const uint32_t hy = kp.hub_row ? __ldg(kp.hub_row + ly) : kNoHub;
            if (hx != kNoHub) ok = hub_bit(kp, hx, y);       // y in x's list
            else if (hy != kNoHub) ok = hub_bit(kp, hy, x);  // x in y's list of the other direction
            else ok = contains_dev(kp.adj, bb, ee, y);
        }
    }
    const unsigned m = __ballot_sync(FULLMASK, ok);
    const uint32_t nm = __popc(m);
    const uint32_t rank = __popc(m & ((1u << lane) - 1u));
    if (!last) {
        const uint32_t cnt_n = __shfl_sync(FULLMASK, ws.cnt, l + 1);
        if (ok) {
            uint32_t *dst = region + pg->lvl_off[l + 1] + (uint64_t)(cnt_n + rank) * w;
#pragma unroll
            for (int p = 0; p < kMaxK; ++p)
                if (p < w) dst[p] = f[p];
        }
        if ((int)lane == l + 1) {
            ws.cnt += nm;
            ws.prod += nm;
        }
    } else if (MODE == HUGE_COUNT) {
        acc += nm;
    } else {
        unsigned long long slot0 = 0;
        if (lane == 0 && nm) slot0 = atomicAdd(kp.sink_tail, (unsigned long long)nm);
        slot0 = __shfl_sync(FULLMASK, slot0, 0);
        if (ok) {
            const unsigned long long r = slot0 + rank;
            if (r < kp.sink_cap) {
                uint32_t *dst = kp.sink + r * kp.sink_width;
#pragma unroll
                for (int p = 0; p < kMaxK; ++p)
                    if (p < w) dst[pg->col_of_pos[p]] = f[p];
            }
        }
        acc += nm;
    }
    if ((int)lane == l) ws.cur = cur_l + R;
    inter += R;
    __syncwarp();
}

// ---------------------------------------------------------------------------------------
// Task queue, donation pool and termination.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void flush_query(const KParams &kp, int q, int nsteps, WState &ws,
                                            unsigned long long &acc) {
    const uint32_t lane = threadIdx.x & 31;
    if (q >= 0) {
        if (lane == 0 && acc) add_u128(kp.counts + 2 * q, acc);
        if ((int)lane < nsteps && ws.prod) atomicAdd(kp.lvl_rows + (size_t)q * kMaxSteps + lane, ws.prod);
    }
    acc = 0;
    ws.prod = 0;
}

// Finds a slot in state `from` and moves it to `to` (lane-parallel scan). Returns -1 if none.
__device__ __forceinline__ int claim_slot(const KParams &kp, int from, int to, uint32_t start) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t base = 0; base < kp.nslots; base += 32) {
        const uint32_t i = base + lane;
        const uint32_t idx = (start + i) % kp.nslots;
        int s = -1;
        if (i < kp.nslots) s = *((volatile int32_t *)&kp.pool[idx].state);
        unsigned m = __ballot_sync(FULLMASK, s == from);
        while (m) {
            const int src = __ffs(m) - 1;
            const uint32_t sidx = __shfl_sync(FULLMASK, idx, src);
            int won = 0;
            if (lane == 0) won = (atomicCAS(&kp.pool[sidx].state, from, to) == from);
            won = __shfl_sync(FULLMASK, won, 0);
            if (won) return (int)sidx;
            m &= m - 1;
        }
    }
    return -1;
}

__device__ __forceinline__ void maybe_donate(const KParams &kp, const Prog *__restrict__ pg, int q,
                                             int nsteps, uint32_t *region, WState &ws,
                                             uint32_t gwarp) {
    const uint32_t lane = threadIdx.x & 31;
    int hungry = 0, ready = 0;
    if (lane == 0) {
        hungry = *((volatile int32_t *)&kp.ctl->hungry);
        ready = *((volatile int32_t *)&kp.ctl->pool_ready);
    }
    hungry = __shfl_sync(FULLMASK, hungry, 0);
    ready = __shfl_sync(FULLMASK, ready, 0);
    if (hungry <= ready) return;
    // rows strictly after the row at the cursor may be given away
    const uint32_t avail = ((int)lane < nsteps && ws.cur < ws.cnt) ? ws.cnt - ws.cur - 1u : 0u;
    const unsigned cand = __ballot_sync(FULLMASK, avail >= 2u);
    if (!cand) return;
    const int l = __ffs(cand) - 1;
    const uint32_t avail_l = __shfl_sync(FULLMASK, avail, l);
    uint32_t h = avail_l / 2u;
    if (l > 0) h = min(h, kp.slot_rows);
    if (h == 0) return;
    const int slot = claim_slot(kp, 0, 1, gwarp * 2654435761u);
    if (slot < 0) return;
    const uint32_t cnt_l = __shfl_sync(FULLMASK, ws.cnt, l);
    PoolSlot *ps = kp.pool + slot;
    if (l == 0) {
        if (lane == 0) {
            ps->r0 = cnt_l - h;
            ps->r1 = cnt_l;
            ps->nrows = 0;
        }
    } else {
        const int w = pg->steps[l + 1].w;
        const uint32_t *src = region + pg->lvl_off[l] + (uint64_t)(cnt_l - h) * w;
        uint32_t *dst = kp.pool_rows + (uint64_t)slot * kp.slot_rows * kMaxK;
        const uint32_t words = h * (uint32_t)w;
        for (uint32_t i = lane; i < words; i += 32) dst[i] = src[i];
        if (lane == 0) ps->nrows = h;
    }
    if (lane == 0) {
        ps->level = l;
        ps->query = (uint32_t)q;
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        atomicExch(&ps->state, 2);
        atomicAdd(&kp.ctl->pool_ready, 1);
        atomicAdd(&kp.ctl->donations, 1ull);
    }
    if ((int)lane == l) ws.cnt = cnt_l - h;
    __syncwarp();
}

// Gets the next unit of work: a root task, else (after the queue is empty) a donated slot.
// Returns false when all work is done (or this warp gave up waiting for donations).
__device__ __forceinline__ bool acquire(const KParams &kp, int &q, const Prog *&pg, int &nsteps,
                                        uint32_t *region, WState &ws, unsigned long long &acc,
                                        uint32_t gwarp, unsigned long long t_start) {
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(&kp.ctl->task_next, 1ull);
    t = __shfl_sync(FULLMASK, t, 0);
    if (t < kp.ntasks) {
        const Task tk = kp.tasks[t];
        if ((int)tk.query != q) {
            flush_query(kp, q, nsteps, ws, acc);
            q = (int)tk.query;
            pg = kp.progs + q;
            nsteps = pg->nsteps;
        }
        ws.cnt = ws.cur = ws.res = 0;
        if (lane == 0) {
            ws.cur = tk.r0;
            ws.cnt = tk.r1;
        }
        return true;
    }
    if (!kp.steal) {
        if (lane == 0) {
            atomicSub(&kp.ctl->active, 1);
            atomicAdd(&kp.ctl->exits_done, 1ull);
        }
        return false;
    }
    if (lane == 0) {
        atomicSub(&kp.ctl->active, 1);
        atomicAdd(&kp.ctl->hungry, 1);
    }
    const unsigned long long t0 = wtimer();
    while (true) {
        int ready = 0;
        if (lane == 0) ready = *((volatile int32_t *)&kp.ctl->pool_ready);
        ready = __shfl_sync(FULLMASK, ready, 0);
        if (ready > 0) {
            if (lane == 0) atomicAdd(&kp.ctl->active, 1);
            __threadfence();
            const int slot = claim_slot(kp, 2, 3, gwarp * 40503u);
            if (slot >= 0) {
                if (lane == 0) atomicSub(&kp.ctl->pool_ready, 1);
                __threadfence();
                PoolSlot *ps = kp.pool + slot;
                const int l = __ldcg(&ps->level);
                const uint32_t qq = __ldcg(&ps->query);
                if ((int)qq != q) {
                    flush_query(kp, q, nsteps, ws, acc);
                    q = (int)qq;
                    pg = kp.progs + q;
                    nsteps = pg->nsteps;
                }
                ws.cnt = ws.cur = ws.res = 0;
                if (l == 0) {
                    const uint32_t r0 = __ldcg(&ps->r0), r1 = __ldcg(&ps->r1);
                    if (lane == 0) {
                        ws.cur = r0;
                        ws.cnt = r1;
                    }
                } else {
                    const uint32_t nrows = __ldcg(&ps->nrows);
                    const int w = pg->steps[l + 1].w;
                    const uint32_t *src = kp.pool_rows + (uint64_t)slot * kp.slot_rows * kMaxK;
                    uint32_t *dst = region + pg->lvl_off[l];
                    const uint32_t words = nrows * (uint32_t)w;
                    for (uint32_t i = lane; i < words; i += 32) dst[i] = __ldcg(src + i);
                    if ((int)lane == l) ws.cnt = nrows;
                }
                __threadfence();
                __syncwarp();
                if (lane == 0) {
                    atomicExch(&ps->state, 0);
                    atomicSub(&kp.ctl->hungry, 1);
                    atomicAdd(&kp.ctl->steals, 1ull);
                }
                return true;
            }
            if (lane == 0) atomicSub(&kp.ctl->active, 1);
        }
        int act = 0;
        if (lane == 0) {
            act = *((volatile int32_t *)&kp.ctl->active);
            ready = *((volatile int32_t *)&kp.ctl->pool_ready);
        }
        act = __shfl_sync(FULLMASK, act, 0);
        ready = __shfl_sync(FULLMASK, ready, 0);
        const unsigned long long now = wtimer();
        int ov = 0;
        if (lane == 0) ov = *((volatile int32_t *)&kp.ctl->overflow);
        ov = __shfl_sync(FULLMASK, ov, 0);
        const bool done = (act == 0 && ready == 0) || ov;
        const bool gave_up = !done && now - t0 > kp.idle_ns && ready == 0;
        const bool limit = now - t_start > kp.limit_ns;
        if (done || gave_up || limit) {
            if (lane == 0) {
                atomicSub(&kp.ctl->hungry, 1);
                atomicAdd(done ? &kp.ctl->exits_done : gave_up ? &kp.ctl->exits_idle : &kp.ctl->exits_limit, 1ull);
                if (limit && !done && !gave_up) atomicOr(&kp.ctl->error, 1);
            }
            return false;
        }
        __nanosleep(2000);
    }
}

template <int MODE, bool STATS>
__global__ void __launch_bounds__(kBlockThreads, HUGE_MIN_BLOCKS) persistent_kernel(const KParams kp) {
    __shared__ RowTile tiles[kWarpsPerBlock];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t *region = kp.wbuf + (uint64_t)gwarp * kp.wstride;
    WState ws;
    ws.cnt = ws.cur = ws.res = 0;
    ws.prod = 0;
    unsigned long long acc = 0, inter = 0, bytes = 0;
    int q = -1, nsteps = 0;
    const Prog *pg = nullptr;
    uint32_t since = 0, iter = 0;
    const unsigned long long t_start = wtimer();
    if (lane == 0) atomicAdd(&kp.ctl->active, 1);  // counted from start; see acquire()
    while (true) {
        const unsigned pend = __ballot_sync(FULLMASK, (int)lane < nsteps && ws.cur < ws.cnt);
        if (pend == 0) {
            if (!acquire(kp, q, pg, nsteps, region, ws, acc, gwarp, t_start)) break;
            continue;
        }
        if (MODE == HUGE_LIST && (iter & 15u) == 0) {  // sink overflowed: abandon this launch
            int ov = 0;
            if (lane == 0) ov = *((volatile int32_t *)&kp.ctl->overflow);
            if (__shfl_sync(FULLMASK, ov, 0)) {
                if (lane == 0) atomicSub(&kp.ctl->active, 1);
                break;
            }
        }
        if ((++iter & 63u) == 0 && wtimer() - t_start > kp.limit_ns) {  // bounded run time
            if (lane == 0) {
                atomicOr(&kp.ctl->error, 1);
                atomicAdd(&kp.ctl->exits_limit, 1ull);
            }
            break;
        }
        const int l = 31 - __clz(pend);
        if ((int)lane == l + 1) {  // deepest pending level is l, so level l+1 is drained
            ws.cnt = 0;
            ws.cur = 0;
            ws.res = 0;
        }
        const StepDesc st = pg->steps[l + 1];
        const bool last = (l + 1 == nsteps);
        bool abort = false;
        if (st.kind == kExtend)
            extend_batch<MODE, STATS>(kp, pg, st, l, last, region, ws, tiles[threadIdx.x >> 5], acc, inter, bytes,
                                      t_start, abort);
        else
            verify_batch<MODE, STATS>(kp, pg, st, l, last, region, ws, acc, inter, bytes);
        if (abort) {  // the time limit passed inside a batch (abort is warp-uniform)
            if (lane == 0) {
                atomicOr(&kp.ctl->error, 1);
                atomicAdd(&kp.ctl->exits_limit, 1ull);
            }
            break;
        }
        if (acc > (1ull << 62)) {
            if (lane == 0) add_u128(kp.counts + 2 * q, acc);
            acc = 0;
        }
        if (kp.steal && ++since >= 4) {
            since = 0;
            maybe_donate(kp, pg, q, nsteps, region, ws, gwarp);
        }
    }
    flush_query(kp, q, nsteps, ws, acc);
    if (STATS) {
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) bytes += __shfl_xor_sync(FULLMASK, bytes, s);
    }
    if (lane == 0) {
        atomicAdd(kp.stats + 0, inter);
        if (STATS) atomicAdd(kp.stats + 1, bytes);
    }
}

int persistent_grid(int *warps) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel<HUGE_COUNT, false>,
                                                  kBlockThreads, 0);
    int per_sm2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, persistent_kernel<HUGE_LIST, true>,
                                                  kBlockThreads, 0);
    if (per_sm2 < per_sm) per_sm = per_sm2;
    if (per_sm < 1) per_sm = 1;
    const int grid = sms * per_sm;
    if (warps) *warps = grid * kWarpsPerBlock;
    return grid;
}

cudaError_t launch_persistent(const KParams &kp, int mode, bool stats, int grid, cudaStream_t s) {
    if (mode == HUGE_COUNT) {
        if (stats)
            persistent_kernel<HUGE_COUNT, true><<<grid, kBlockThreads, 0, s>>>(kp);
        else
            persistent_kernel<HUGE_COUNT, false><<<grid, kBlockThreads, 0, s>>>(kp);
    } else {
        if (stats)
            persistent_kernel<HUGE_LIST, true><<<grid, kBlockThreads, 0, s>>>(kp);
        else
            persistent_kernel<HUGE_LIST, false><<<grid, kBlockThreads, 0, s>>>(kp);
    }
    return cudaGetLastError();
}

}  // namespace huge
