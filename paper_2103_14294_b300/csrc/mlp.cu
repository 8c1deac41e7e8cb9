// Learned cardinality estimator: a 64 -> 128 -> 128 -> 1 ReLU perceptron predicting
// log(1 + |R(q')|) for a sub-query q', the quantity Alg. 1 needs for each sub-query (its
// cardinality term and the join costs). Weights are fp32 masters used in bf16; the dense layers run on the 5th
// generation tensor cores: operands staged in shared memory (no-swizzle K-major core-matrix
// layout), tcgen05.mma issued by one thread with the fp32 accumulators in tensor memory,
// completion tracked through an mbarrier (bounded waits), results read back with tcgen05.ld.
// One CTA of 128 threads handles a tile of 128 rows: forward (two MMAs) and, for training,
// backward (three more MMAs: dH1 = dZ2 W2, dW2 = dZ2^T H1, dW1 = dZ1^T X); weight gradients are
// reduced across tiles with atomics and applied by an Adam step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace huge {
namespace mlpk {

constexpr int kIn = 64, kHid = 128, kTile = 128;
constexpr int kW1 = kHid * kIn, kB1 = kHid, kW2 = kHid * kHid, kB2 = kHid, kW3 = kHid, kB3 = 1;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kW1, kOffW2 = kOffB1 + kB1, kOffB2 = kOffW2 + kW2,
              kOffW3 = kOffB2 + kB2, kOffB3 = kOffW3 + kW3, kParams = kOffB3 + kB3;

// shared-memory operand buffers (bytes)
constexpr uint32_t kSzW1 = kHid * kIn * 2;    // [128 out][64 in]
constexpr uint32_t kSzW2 = kHid * kHid * 2;   // [128 out][128 in]
constexpr uint32_t kSzX = kTile * kIn * 2;    // [128 rows][64 in]
constexpr uint32_t kSzXT = kIn * kTile * 2;   // [64 in][128 rows]
constexpr uint32_t kSzH = kTile * kHid * 2;   // [128][128]
constexpr uint32_t kOW1 = 0, kOW2 = kOW1 + kSzW1, kOW2T = kOW2 + kSzW2, kOX = kOW2T + kSzW2, kOXT = kOX + kSzX,
                   kOH = kOXT + kSzXT, kOHT = kOH + kSzH, kODT = kOHT + kSzH, kOBar = kODT + kSzH,
                   kSmem = kOBar + 64;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColD1 = 0, kColD2 = 128, kColDW2 = 256, kColDW1 = 384;
constexpr int kWaitIters = 1 << 22;

struct Args {
    const __nv_bfloat16 *w1b, *w2b, *w2tb;  // [out][in], [out][in], [in][out]
    const float *params;                    // fp32 masters (biases, w3, b3)
    const float *mu, *sd;                   // input standardisation
    const float *x;                         // [rows][64]
    const float *t;                         // [rows] targets (training)
    float *y;                               // [rows] outputs (may be null)
    float *grad;                            // [kParams] (training)
    float *loss;                            // [1]
    int *err;                               // [1] bounded-wait failures
    uint32_t rows;
    float inv_total;                        // 1 / rows of the whole batch
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a K-major operand with K columns, no swizzle:
// 8 x 16-byte core matrices; K-adjacent core matrices 128 B apart (LBO), row groups SBO apart
__device__ __forceinline__ uint32_t kmaj(uint32_t r, uint32_t k, uint32_t K) {
    return (r >> 3) * (K / 8) * 128u + (k >> 3) * 128u + (r & 7) * 16u + (k & 7) * 2u;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; base offset 0; no swizzle
    return d;
}

// kind::f16 instruction descriptor: D fp32, A and B bf16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
    for (int i = 0; i < kWaitIters; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive fp32 columns of this thread's TMEM lane (row)
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// 8 consecutive K-values of row r as one 16-byte store into a K-major operand
__device__ __forceinline__ void st8(unsigned char *base, uint32_t r, uint32_t k0, uint32_t K, const float *v) {
    uint4 q;
    q.x = (uint32_t)bf16_bits(v[0]) | ((uint32_t)bf16_bits(v[1]) << 16);
    q.y = (uint32_t)bf16_bits(v[2]) | ((uint32_t)bf16_bits(v[3]) << 16);
    q.z = (uint32_t)bf16_bits(v[4]) | ((uint32_t)bf16_bits(v[5]) << 16);
    q.w = (uint32_t)bf16_bits(v[6]) | ((uint32_t)bf16_bits(v[7]) << 16);
    *reinterpret_cast<uint4 *>(base + kmaj(r, k0, K)) = q;
}

__device__ __forceinline__ void st1(unsigned char *base, uint32_t r, uint32_t k, uint32_t K, float v) {
    *reinterpret_cast<uint16_t *>(base + kmaj(r, k, K)) = bf16_bits(v);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// copies a [R][K] bf16 global matrix (row-major) into a K-major shared operand
__device__ __forceinline__ void load_operand(unsigned char *dst, const __nv_bfloat16 *src, uint32_t R, uint32_t K) {
    const uint32_t chunks = R * K / 8;
    for (uint32_t c = threadIdx.x; c < chunks; c += blockDim.x) {
        const uint32_t r = c / (K / 8), k0 = (c % (K / 8)) * 8;
        *reinterpret_cast<uint4 *>(dst + kmaj(r, k0, K)) = *reinterpret_cast<const uint4 *>(src + (size_t)r * K + k0);
    }
}

template <bool TRAIN>
__global__ void __launch_bounds__(128, 1) mlp_tile_kernel(const Args a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint32_t tmem_slot;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t row = blockIdx.x * kTile + tid;  // this thread's row (= its TMEM lane)
    const bool valid = row < a.rows;
    const uint32_t bar = smem_u32(sm + kOBar);
    bool ok = true;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operands: weights and this tile's standardised inputs
    load_operand(sm + kOW1, a.w1b, kHid, kIn);
    load_operand(sm + kOW2, a.w2b, kHid, kHid);
    if (TRAIN) load_operand(sm + kOW2T, a.w2tb, kHid, kHid);
    {
        float xs[kIn];
#pragma unroll
        for (int k = 0; k < kIn; ++k) xs[k] = valid ? (a.x[(size_t)row * kIn + k] - a.mu[k]) / a.sd[k] : 0.f;
#pragma unroll
        for (int k0 = 0; k0 < kIn; k0 += 8) st8(sm + kOX, tid, k0, kIn, xs + k0);
        if (TRAIN) {
#pragma unroll
            for (int k = 0; k < kIn; ++k) st1(sm + kOXT, k, tid, kTile, xs[k]);  // X^T: [64][128 rows]
        }
    }
    fence_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = tmem_slot;
    const uint32_t tlane = tbase + ((warp * 32u) << 16);
    uint32_t phase = 0;

    // ---- layer 1: D1 = X W1^T (M 128, N 128, K 64) ----
    if (tid == 0) {
        for (uint32_t kk = 0; kk < kIn / 16; ++kk)
            mma(tbase + kColD1, sdesc(smem_u32(sm + kOX) + kk * 256, 128, (kIn / 8) * 128),
                sdesc(smem_u32(sm + kOW1) + kk * 256, 128, (kIn / 8) * 128), idesc_bf16(128), kk > 0);
        commit(bar);
    }
    ok = __syncthreads_and(wait_bar(bar, phase));  // CTA-uniform: warp reductions below need it
    phase ^= 1;
    fence_after();
    uint32_t relu1[4] = {0, 0, 0, 0};  // ReLU masks of z1 (128 bits)
    if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            ld32(tlane + kColD1 + c0, v);
            uint32_t m = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                v[i] += a.params[kOffB1 + c0 + i];
                if (v[i] > 0.f) m |= 1u << i;
                v[i] = fmaxf(v[i], 0.f);
            }
            relu1[c0 / 32] = m;
#pragma unroll
            for (int i = 0; i < 32; i += 8) st8(sm + kOH, tid, c0 + i, kHid, v + i);  // H1 [rows][128]
            if (TRAIN) {
#pragma unroll
                for (int i = 0; i < 32; ++i) st1(sm + kOHT, c0 + i, tid, kTile, v[i]);  // H1^T [128][rows]
            }
        }
    }
    fence_async();
    fence_before();
    __syncthreads();
    fence_after();

    // ---- layer 2: D2 = H1 W2^T (K 128) ----
    if (tid == 0 && ok) {
        for (uint32_t kk = 0; kk < kHid / 16; ++kk)
            mma(tbase + kColD2, sdesc(smem_u32(sm + kOH) + kk * 256, 128, (kHid / 8) * 128),
                sdesc(smem_u32(sm + kOW2) + kk * 256, 128, (kHid / 8) * 128), idesc_bf16(128), kk > 0);
        commit(bar);
    }
    ok = __syncthreads_and(ok && wait_bar(bar, phase));
    phase ^= 1;
    fence_after();

    // ---- head: y = relu(z2) . w3 + b3; training: loss, dy, dz2 ----
    float y = a.params[kOffB3];
    float dy = 0.f;
    if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            ld32(tlane + kColD2 + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) y += fmaxf(v[i] + a.params[kOffB2 + c0 + i], 0.f) * a.params[kOffW3 + c0 + i];
        }
    }
    if (!TRAIN) {
        if (valid && a.y) a.y[row] = y;
    } else {
        const float diff = valid ? y - a.t[row] : 0.f;
        dy = diff * a.inv_total;
        const float l = warp_sum(0.5f * diff * diff * a.inv_total);
        const float sdy = warp_sum(dy);
        if (lane == 0) {
            atomicAdd(a.loss, l);
            atomicAdd(a.grad + kOffB3, sdy);
        }
        // dz2 = dy w3 [z2 > 0]; reduce db2 and dw3 over the tile's rows
        if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < kHid; c0 += 32) {
                float v[32];
                ld32(tlane + kColD2 + c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float z2 = v[i] + a.params[kOffB2 + c0 + i];
                    const float h2 = fmaxf(z2, 0.f);
                    const float dz = z2 > 0.f ? dy * a.params[kOffW3 + c0 + i] : 0.f;
                    const float sw3 = warp_sum(h2 * dy), sb2 = warp_sum(dz);
                    if (lane == 0) {
                        atomicAdd(a.grad + kOffW3 + c0 + i, sw3);
                        atomicAdd(a.grad + kOffB2 + c0 + i, sb2);
                    }
                    v[i] = dz;
                }
                // dZ2 as A of dH1 = dZ2 W2 (reuses the H1 buffer: layer 2 is complete)
#pragma unroll
                for (int i = 0; i < 32; i += 8) st8(sm + kOH, tid, c0 + i, kHid, v + i);
#pragma unroll
                for (int i = 0; i < 32; ++i) st1(sm + kODT, c0 + i, tid, kTile, v[i]);  // dZ2^T [128][rows]
            }
        }
        fence_async();
        fence_before();
        __syncthreads();
        fence_after();
        // dH1 = dZ2 W2 ; dW2 = dZ2^T H1
        if (tid == 0 && ok) {
            for (uint32_t kk = 0; kk < kHid / 16; ++kk)
                mma(tbase + kColD1, sdesc(smem_u32(sm + kOH) + kk * 256, 128, (kHid / 8) * 128),
                    sdesc(smem_u32(sm + kOW2T) + kk * 256, 128, (kHid / 8) * 128), idesc_bf16(128), kk > 0);
            for (uint32_t kk = 0; kk < kTile / 16; ++kk)
                mma(tbase + kColDW2, sdesc(smem_u32(sm + kODT) + kk * 256, 128, (kTile / 8) * 128),
                    sdesc(smem_u32(sm + kOHT) + kk * 256, 128, (kTile / 8) * 128), idesc_bf16(128), kk > 0);
            commit(bar);
        }
        ok = __syncthreads_and(ok && wait_bar(bar, phase));
        phase ^= 1;
        fence_after();
        if (ok) {
            // dz1 = dh1 [z1 > 0] -> dZ1^T (A of dW1, reuses the dZ2 A buffer: dH1 is complete)
#pragma unroll 1
            for (int c0 = 0; c0 < kHid; c0 += 32) {
                float v[32];
                ld32(tlane + kColD1 + c0, v);
                const uint32_t m = relu1[c0 / 32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float dz = (m >> i & 1u) ? v[i] : 0.f;
                    const float sb1 = warp_sum(dz);
                    if (lane == 0) atomicAdd(a.grad + kOffB1 + c0 + i, sb1);
                    st1(sm + kOH, c0 + i, tid, kTile, dz);  // dZ1^T [128][rows]
                }
            }
            // dW2 rows: this thread holds dW2[out = tid][0..127]
#pragma unroll 1
            for (int c0 = 0; c0 < kHid; c0 += 32) {
                float v[32];
                ld32(tlane + kColDW2 + c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) atomicAdd(a.grad + kOffW2 + tid * kHid + c0 + i, v[i]);
            }
        }
        fence_async();
        fence_before();
        __syncthreads();
        fence_after();
        // dW1 = dZ1^T X  (M 128 hidden, N 64 inputs, K 128 rows)
        if (tid == 0 && ok) {
            for (uint32_t kk = 0; kk < kTile / 16; ++kk)
                mma(tbase + kColDW1, sdesc(smem_u32(sm + kOH) + kk * 256, 128, (kTile / 8) * 128),
                    sdesc(smem_u32(sm + kOXT) + kk * 256, 128, (kTile / 8) * 128), idesc_bf16(64), kk > 0);
            commit(bar);
        }
        ok = __syncthreads_and(ok && wait_bar(bar, phase));
        phase ^= 1;
        fence_after();
        if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < kIn; c0 += 32) {
                float v[32];
                ld32(tlane + kColDW1 + c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) atomicAdd(a.grad + kOffW1 + tid * kIn + c0 + i, v[i]);
            }
        }
    }
    if (!ok && tid == 0) atomicAdd(a.err, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
}

// fp32 masters -> bf16 operand copies: W1 [out][in], W2 [out][in], W2^T [in][out]
__global__ void mlp_cast_kernel(const float *p, __nv_bfloat16 *w1b, __nv_bfloat16 *w2b, __nv_bfloat16 *w2tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kW1) w1b[i] = __float2bfloat16_rn(p[kOffW1 + i]);
    if (i < kW2) {
        const int o = i / kHid, in = i % kHid;
        const __nv_bfloat16 v = __float2bfloat16_rn(p[kOffW2 + i]);
        w2b[i] = v;
        w2tb[in * kHid + o] = v;
    }
}

// Adam (Kingma & Ba) on the fp32 masters; clears the gradient
__global__ void mlp_adam_kernel(float *p, float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                                float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
}

}  // namespace mlpk
}  // namespace huge

using namespace huge;
using namespace huge::mlpk;

struct huge_mlp {
    int device = 0;
    float *d_params = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
    __nv_bfloat16 *d_w1b = nullptr, *d_w2b = nullptr, *d_w2tb = nullptr;
    float *d_mu = nullptr, *d_sd = nullptr, *d_loss = nullptr;
    int *d_err = nullptr;
    float *d_x = nullptr, *d_y = nullptr;  // staging for host-array predictions
    uint32_t buf_rows = 0;
    uint64_t steps = 0;
};

namespace huge {
namespace {

int mlp_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return HUGE_OK;
    cudaGetLastError();
    return fail(HUGE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int mlp_smem_attr() {
    static int done = 0;
    if (done) return HUGE_OK;
    cudaError_t e1 = cudaFuncSetAttribute(mlp_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    cudaError_t e2 = cudaFuncSetAttribute(mlp_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return mlp_cuda(e1 != cudaSuccess ? e1 : e2, "shared memory attribute");
    done = 1;
    return HUGE_OK;
}

int mlp_cast(huge_mlp_t *M, cudaStream_t s) {
    mlp_cast_kernel<<<(kW2 + 255) / 256, 256, 0, s>>>(M->d_params, M->d_w1b, M->d_w2b, M->d_w2tb);
    return mlp_cuda(cudaGetLastError(), "casting weights");
}

Args make_args(const huge_mlp_t *M, const float *x, const float *t, float *y, uint32_t rows, uint32_t total) {
    Args a;
    memset(&a, 0, sizeof(a));
    a.w1b = M->d_w1b;
    a.w2b = M->d_w2b;
    a.w2tb = M->d_w2tb;
    a.params = M->d_params;
    a.mu = M->d_mu;
    a.sd = M->d_sd;
    a.x = x;
    a.t = t;
    a.y = y;
    a.grad = M->d_grad;
    a.loss = M->d_loss;
    a.err = M->d_err;
    a.rows = rows;
    a.inv_total = 1.f / (float)std::max<uint32_t>(total, 1);
    return a;
}

int check_err(huge_mlp_t *M, cudaStream_t s) {
    int h = 0;
    cudaMemcpyAsync(&h, M->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    int rc = mlp_cuda(cudaStreamSynchronize(s), "MLP kernels");
    if (rc) return rc;
    if (h) {
        cudaMemsetAsync(M->d_err, 0, sizeof(int), s);
        return fail(HUGE_ETIMEOUT, "a tensor-core completion wait of the MLP gave up");
    }
    return HUGE_OK;
}

}  // namespace

// Predictions for host feature rows (used by the planner).
int mlp_predict(const huge_mlp_t *Mc, const float *x, int rows, float *y, std::string *err) {
    huge_mlp_t *M = const_cast<huge_mlp_t *>(Mc);
    if (!M) {
        *err = "null model";
        return HUGE_EINVAL;
    }
    if (rows <= 0) return HUGE_OK;
    int rc = mlp_smem_attr();
    if (rc) return rc;
    if ((uint32_t)rows > M->buf_rows) {
        if (M->d_x) dev_free(M->d_x);
        if (M->d_y) dev_free(M->d_y);
        M->d_x = M->d_y = nullptr;
        if (dev_malloc(&M->d_x, sizeof(float) * kIn * rows) != cudaSuccess ||
            dev_malloc(&M->d_y, sizeof(float) * rows) != cudaSuccess) {
            cudaGetLastError();
            M->buf_rows = 0;
            *err = "device allocation for MLP inputs failed";
            return HUGE_ENOMEM;
        }
        M->buf_rows = (uint32_t)rows;
    }
    cudaMemcpy(M->d_x, x, sizeof(float) * kIn * rows, cudaMemcpyHostToDevice);
    Args a = make_args(M, M->d_x, nullptr, M->d_y, (uint32_t)rows, (uint32_t)rows);
    mlp_tile_kernel<false><<<(rows + kTile - 1) / kTile, kTile, kSmem, 0>>>(a);
    rc = mlp_cuda(cudaGetLastError(), "MLP forward launch");
    if (rc) {
        *err = huge_last_error();
        return rc;
    }
    rc = check_err(M, 0);
    if (rc) {
        *err = huge_last_error();
        return rc;
    }
    cudaMemcpy(y, M->d_y, sizeof(float) * rows, cudaMemcpyDeviceToHost);
    return HUGE_OK;
}

}  // namespace huge

extern "C" {

int huge_mlp_create(uint64_t seed, huge_mlp_t **out) {
    set_error("");
    if (!out) return fail(HUGE_EINVAL, "null output pointer");
    huge_mlp_t *M = new huge_mlp_t();
    cudaGetDevice(&M->device);
    bool okm = dev_malloc(&M->d_params, 4 * kParams) == cudaSuccess && dev_malloc(&M->d_m, 4 * kParams) == cudaSuccess &&
               dev_malloc(&M->d_v, 4 * kParams) == cudaSuccess && dev_malloc(&M->d_grad, 4 * kParams) == cudaSuccess &&
               dev_malloc(&M->d_w1b, 2 * kW1) == cudaSuccess && dev_malloc(&M->d_w2b, 2 * kW2) == cudaSuccess &&
               dev_malloc(&M->d_w2tb, 2 * kW2) == cudaSuccess && dev_malloc(&M->d_mu, 4 * kIn) == cudaSuccess &&
               dev_malloc(&M->d_sd, 4 * kIn) == cudaSuccess && dev_malloc(&M->d_loss, 4) == cudaSuccess &&
               dev_malloc(&M->d_err, 4) == cudaSuccess;
    if (!okm) {
        cudaGetLastError();
        huge_mlp_free(M);
        return fail(HUGE_ENOMEM, "device allocation for the MLP failed");
    }
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a SplitMix64 stream
    std::vector<float> p(kParams);
    uint64_t x = seed;
    auto next = [&]() {
        uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        return (double)(z >> 11) / 9007199254740992.0;
    };
    for (int i = 0; i < kParams; i++) {
        const double fan = i < kOffW2 ? kIn : kHid;
        p[i] = (float)((2.0 * next() - 1.0) / std::sqrt(fan));
    }
    std::vector<float> mu(kIn, 0.f), sd(kIn, 1.f);
    cudaMemcpy(M->d_params, p.data(), 4 * kParams, cudaMemcpyHostToDevice);
    cudaMemset(M->d_m, 0, 4 * kParams);
    cudaMemset(M->d_v, 0, 4 * kParams);
    cudaMemset(M->d_grad, 0, 4 * kParams);
    cudaMemset(M->d_err, 0, 4);
    cudaMemcpy(M->d_mu, mu.data(), 4 * kIn, cudaMemcpyHostToDevice);
    cudaMemcpy(M->d_sd, sd.data(), 4 * kIn, cudaMemcpyHostToDevice);
    int rc = mlp_cast(M, 0);
    if (!rc) rc = mlp_cuda(cudaDeviceSynchronize(), "initialising the MLP");
    if (rc) {
        huge_mlp_free(M);
        return rc;
    }
    *out = M;
    return HUGE_OK;
}

int huge_mlp_free(huge_mlp_t *M) {
    if (!M) return HUGE_OK;
    void *ps[] = {M->d_params, M->d_m, M->d_v, M->d_grad, M->d_w1b, M->d_w2b, M->d_w2tb,
                  M->d_mu, M->d_sd, M->d_loss, M->d_err, M->d_x, M->d_y};
    for (void *p : ps)
        if (p) dev_free(p);
    delete M;
    return HUGE_OK;
}

uint32_t huge_mlp_num_params(void) { return (uint32_t)kParams; }

int huge_mlp_set_params(huge_mlp_t *M, const float *params, const float *mu, const float *sd) {
    set_error("");
    if (!M) return fail(HUGE_EINVAL, "null model");
    if (params) cudaMemcpy(M->d_params, params, 4 * kParams, cudaMemcpyHostToDevice);
    if (mu) cudaMemcpy(M->d_mu, mu, 4 * kIn, cudaMemcpyHostToDevice);
    if (sd) cudaMemcpy(M->d_sd, sd, 4 * kIn, cudaMemcpyHostToDevice);
    cudaMemset(M->d_m, 0, 4 * kParams);
    cudaMemset(M->d_v, 0, 4 * kParams);
    M->steps = 0;
    int rc = mlp_cast(M, 0);
    if (rc) return rc;
    return mlp_cuda(cudaDeviceSynchronize(), "setting MLP parameters");
}

int huge_mlp_get_params(const huge_mlp_t *M, float *params, float *mu, float *sd) {
    set_error("");
    if (!M) return fail(HUGE_EINVAL, "null model");
    if (params) cudaMemcpy(params, M->d_params, 4 * kParams, cudaMemcpyDeviceToHost);
    if (mu) cudaMemcpy(mu, M->d_mu, 4 * kIn, cudaMemcpyDeviceToHost);
    if (sd) cudaMemcpy(sd, M->d_sd, 4 * kIn, cudaMemcpyDeviceToHost);
    return mlp_cuda(cudaDeviceSynchronize(), "reading MLP parameters");
}

int huge_mlp_forward(const huge_mlp_t *Mc, const float *x, uint32_t rows, float *y, void *stream) {
    set_error("");
    huge_mlp_t *M = const_cast<huge_mlp_t *>(Mc);
    if (!M || (!x && rows) || (!y && rows)) return fail(HUGE_EINVAL, "null argument");
    if (rows == 0) return HUGE_OK;
    int rc = mlp_smem_attr();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    Args a = make_args(M, x, nullptr, y, rows, rows);
    mlp_tile_kernel<false><<<(rows + kTile - 1) / kTile, kTile, kSmem, s>>>(a);
    rc = mlp_cuda(cudaGetLastError(), "MLP forward launch");
    if (rc) return rc;
    return check_err(M, s);
}

int huge_mlp_loss_grad(const huge_mlp_t *Mc, const float *x, const float *t, uint32_t rows, float *grad, float *loss,
                       void *stream) {
    set_error("");
    huge_mlp_t *M = const_cast<huge_mlp_t *>(Mc);
    if (!M || !x || !t || !grad || !loss || rows == 0) return fail(HUGE_EINVAL, "null argument or no rows");
    int rc = mlp_smem_attr();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(M->d_grad, 0, 4 * kParams, s);
    cudaMemsetAsync(M->d_loss, 0, 4, s);
    Args a = make_args(M, x, t, nullptr, rows, rows);
    mlp_tile_kernel<true><<<(rows + kTile - 1) / kTile, kTile, kSmem, s>>>(a);
    rc = mlp_cuda(cudaGetLastError(), "MLP gradient launch");
    if (rc) return rc;
    cudaMemcpyAsync(grad, M->d_grad, 4 * kParams, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(loss, M->d_loss, 4, cudaMemcpyDeviceToHost, s);
    rc = check_err(M, s);
    cudaMemsetAsync(M->d_grad, 0, 4 * kParams, s);
    return rc;
}

int huge_mlp_train(huge_mlp_t *M, const float *x, const float *t, uint32_t rows, uint32_t epochs,
                   uint32_t batch_rows, float lr, float *final_loss, void *stream) {
    set_error("");
    if (!M || !x || !t || rows == 0 || epochs == 0) return fail(HUGE_EINVAL, "null argument or empty training set");
    int rc = mlp_smem_attr();
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (batch_rows == 0 || batch_rows > rows) batch_rows = rows;
    batch_rows = std::max<uint32_t>(kTile, batch_rows / kTile * kTile);
    cudaMemsetAsync(M->d_grad, 0, 4 * kParams, s);
    float last = 0.f;
    for (uint32_t ep = 0; ep < epochs; ep++) {
        cudaMemsetAsync(M->d_loss, 0, 4, s);
        for (uint32_t b0 = 0; b0 < rows; b0 += batch_rows) {
            const uint32_t nb = std::min(batch_rows, rows - b0);
            Args a = make_args(M, x + (size_t)b0 * kIn, t + b0, nullptr, nb, nb);
            mlp_tile_kernel<true><<<(nb + kTile - 1) / kTile, kTile, kSmem, s>>>(a);
            M->steps++;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, (float)M->steps), c2 = 1.f - std::pow(b2, (float)M->steps);
            mlp_adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(M->d_params, M->d_grad, M->d_m, M->d_v, lr, b1, b2,
                                                                  1e-8f, c1, c2);
            rc = mlp_cast(M, s);
            if (rc) return rc;
        }
        if (ep + 1 == epochs) {
            float l = 0.f;
            cudaMemcpyAsync(&l, M->d_loss, 4, cudaMemcpyDeviceToHost, s);
            rc = check_err(M, s);
            if (rc) return rc;
            last = l * (float)batch_rows / (float)rows;  // mean over batches of per-batch mean losses
        }
    }
    if (final_loss) *final_loss = last;
    return HUGE_OK;
}

}  // extern "C"
