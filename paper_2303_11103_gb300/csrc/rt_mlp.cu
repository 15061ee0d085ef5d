// rt_mlp.cu -- learned path-gain surrogate (not in the paper; it cites
// neural path-loss prediction as related work, Sec. I): Fourier features of
// (tx, rx) -> n_hidden ReLU layers -> (path logit, path gain in dB).
//
// Dense layers are tcgen05 GEMMs: BF16 operands staged in shared memory by
// TMA (128-byte swizzle, 4-stage mbarrier pipeline), FP32 accumulators in
// TMEM, one thread issuing MMAs, the four warps reading TMEM in the
// epilogue (bias, ReLU, BF16 or FP32 store). Features, the 2-wide head, the
// loss, transposes, column sums and Adam run on CUDA cores.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "rt_internal.h"
#include "rt_tc.cuh"

namespace {

constexpr int GM = 128, GK = 64, GSTAGES = 4;

// sin and cos of 2 pi a for a in [-0.5, 0.5] (the reduced Fourier phase):
// the hardware approximation, absolute error about 4e-7 on [-pi, pi], far
// below the BF16 rounding the features then get.
__device__ __forceinline__ void feature_sincos(float a, float* s, float* c) {
    __sincosf(6.283185307179586f * a, s, c);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
}

// C[M x N] = act(A[M x K] B[N x K]^T + bias), A and B BF16 row-major (K
// contiguous), C FP32 or BF16 row-major with leading dimension ldc.
template <int BN>
__global__ void __launch_bounds__(128, 1) k_gemm(const __grid_constant__ CUtensorMap ta,
                                                  const __grid_constant__ CUtensorMap tb, int M, int N, int K,
                                                  const float* __restrict__ bias, int relu, int out_bf16,
                                                  void* __restrict__ C, int ldc, unsigned* err) {
    extern __shared__ uint8_t dyn[];
    __shared__ __align__(8) uint64_t bar_full[GSTAGES], bar_empty[GSTAGES], bar_done;
    __shared__ uint32_t tmem_slot;
    constexpr uint32_t A_BYTES = GM * GK * 2, B_BYTES = BN * GK * 2, ST_BYTES = A_BYTES + B_BYTES;
    constexpr uint32_t TCOLS = BN;  // 64, 128 or 256 FP32 columns
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * BN;
    const int nk = (K + GK - 1) / GK;
    if (warp == 0) {
        tmem_alloc(su32(&tmem_slot), TCOLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < GSTAGES; s++) {
            mbar_init(su32(&bar_full[s]), 1);
            mbar_init(su32(&bar_empty[s]), 1);
        }
        mbar_init(su32(&bar_done), 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kb = 0; kb < nk; kb++) {
            const int s = kb % GSTAGES;
            if (kb >= GSTAGES && !mbar_wait(su32(&bar_empty[s]), ((kb / GSTAGES) - 1) & 1, err)) break;
            const uint32_t sa = su32(base + s * ST_BYTES), sb = sa + A_BYTES;
            mbar_expect_tx(su32(&bar_full[s]), ST_BYTES);
            tma_load_2d(sa, &ta, kb * GK, m0, su32(&bar_full[s]));
            tma_load_2d(sb, &tb, kb * GK, n0, su32(&bar_full[s]));
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(GM, BN);
        for (int kb = 0; kb < nk; kb++) {
            const int s = kb % GSTAGES;
            if (!mbar_wait(su32(&bar_full[s]), (kb / GSTAGES) & 1, err)) break;
            tc_fence_after();
            const uint32_t sa = su32(base + s * ST_BYTES), sb = sa + A_BYTES;
#pragma unroll
            for (int k = 0; k < GK / 16; k++)
                mma_bf16(tmem, desc_sw128(sa + k * 32), desc_sw128(sb + k * 32), idesc, (kb | k) != 0 ? 1u : 0u);
            mma_commit(su32(&bar_empty[s]));
        }
        mma_commit(su32(&bar_done));
    }
    __syncwarp();
    const bool done = mbar_wait(su32(&bar_done), 0, err);
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    if (done) {
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            tmem_wait_ld();
            const int col = n0 + c0;
            if (row >= M || col >= N) continue;
            float v[32];
#pragma unroll
            for (int j = 0; j < 32; j++) {
                float x = __uint_as_float(r[j]);
                if (bias && col + j < N) x += bias[col + j];
                if (relu) x = fmaxf(x, 0.0f);
                v[j] = x;
            }
            if (col + 32 <= N) {
                if (out_bf16) {
                    uint4* p = reinterpret_cast<uint4*>((__nv_bfloat16*)C + (size_t)row * ldc + col);
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        p[q] = make_uint4(pack_bf16(v[8 * q], v[8 * q + 1]), pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                                          pack_bf16(v[8 * q + 4], v[8 * q + 5]), pack_bf16(v[8 * q + 6], v[8 * q + 7]));
                } else {
                    float4* p = reinterpret_cast<float4*>((float*)C + (size_t)row * ldc + col);
#pragma unroll
                    for (int q = 0; q < 8; q++) p[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            } else {
                for (int j = 0; j < 32 && col + j < N; j++) {
                    if (out_bf16)
                        ((__nv_bfloat16*)C)[(size_t)row * ldc + col + j] = __float2bfloat16_rn(v[j]);
                    else
                        ((float*)C)[(size_t)row * ldc + col + j] = v[j];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

// ------------------------------------------------------------ CUDA-core parts
// features: x [B x 6] (tx xyz, rx xyz) -> [sin(2 pi Bx'), cos(2 pi Bx')] (BF16 [B x 2F]),
// x' = 2 (x - lo) / (hi - lo) - 1 per coordinate.
__global__ void k_features(const float* __restrict__ x, int64_t n, const float* __restrict__ Bf, int F,
                           const float* __restrict__ lo, const float* __restrict__ hi,
                           __nv_bfloat16* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (i >= n) return;
    float xn[6];
    for (int k = 0; k < 6; k++) xn[k] = 2.0f * (x[6 * i + k] - lo[k]) / (hi[k] - lo[k]) - 1.0f;
    for (int j = threadIdx.x; j < F; j += blockDim.x) {
        float a = 0.0f;
        for (int k = 0; k < 6; k++) a = fmaf(Bf[6 * j + k], xn[k], a);
        a -= rintf(a);  // integer periods drop out of sin/cos(2 pi a)
        float s, c;
        feature_sincos(a, &s, &c);
        out[(size_t)i * 2 * F + j] = __float2bfloat16_rn(s);
        out[(size_t)i * 2 * F + F + j] = __float2bfloat16_rn(c);
    }
}

// head: y[b][o] = sum_j H[b][j] W[o][j] + bias[o], o in {0, 1}; one warp per row
__global__ void k_head(const __nv_bfloat16* __restrict__ H, int64_t n, int W, const float* __restrict__ Wh,
                       const float* __restrict__ bh, float* __restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    float a0 = 0.0f, a1 = 0.0f;
    for (int j = lane; j < W; j += 32) {
        float h = __bfloat162float(H[(size_t)i * W + j]);
        a0 = fmaf(h, Wh[j], a0);
        a1 = fmaf(h, Wh[W + j], a1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if (lane == 0) {
        y[2 * i] = a0 + bh[0];
        y[2 * i + 1] = a1 + bh[1];
    }
}

// Free-space gain 20 log10(lambda / (4 pi d)) in dB of the query x [6]
// (d = |rx - tx|, at least 1 m); 0 when lam == 0 (no baseline).
__device__ __forceinline__ float fspl_db(const float* __restrict__ x, float lam) {
    if (lam <= 0.0f) return 0.0f;
    float dx = x[3] - x[0], dy = x[4] - x[1], dz = x[5] - x[2];
    float d = fmaxf(sqrtf(dx * dx + dy * dy + dz * dz), 1.0f);
    return 20.0f * log10f(lam / (4.0f * RT_PI_F * d));
}

// outputs in user units: (path logit, gain dB = y1 * scale + offset + baseline)
__global__ void k_head_out(const float* __restrict__ y, const float* __restrict__ x, int64_t n, float scale,
                           float offset, float lam, float* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[2 * i] = y[2 * i];
    out[2 * i + 1] = y[2 * i + 1] * scale + offset + fspl_db(x + 6 * i, lam);
}

// loss = mean_b [BCE(logit, has) + has * (y1 - t)^2], t = (gain_db - offset) / scale;
// dy = d loss / d y
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ tgt, const float* __restrict__ x, int n,
                       float scale, float offset, float lam, float* __restrict__ dy, float* __restrict__ loss) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < n) {
        float z = y[2 * i], has = tgt[2 * i], t = (tgt[2 * i + 1] - offset - fspl_db(x + 6 * i, lam)) / scale;
        float p = 1.0f / (1.0f + __expf(-z));
        // BCE with logits, stable form: max(z,0) - z has + log(1 + e^-|z|)
        l = fmaxf(z, 0.0f) - z * has + log1pf(__expf(-fabsf(z)));
        float e = y[2 * i + 1] - t;
        l += has * e * e;
        dy[2 * i] = (p - has) / n;
        dy[2 * i + 1] = 2.0f * has * e / n;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / n);
}

// head backward: gWh[o][j] += sum_b dy[b][o] H[b][j] (block per 32 columns),
// gbh[o] += sum_b dy[b][o]
__global__ void k_head_wgrad(const __nv_bfloat16* __restrict__ H, const float* __restrict__ dy, int n, int W,
                             float* __restrict__ gWh, float* __restrict__ gbh) {
    __shared__ float s0[8][33], s1[8][33];
    int j = blockIdx.x * 32 + threadIdx.x;   // blockDim (32, 8)
    float a0 = 0.0f, a1 = 0.0f, c0 = 0.0f, c1 = 0.0f;
    for (int b = threadIdx.y; b < n; b += 8) {
        float d0 = dy[2 * b], d1 = dy[2 * b + 1];
        if (j < W) {
            float h = __bfloat162float(H[(size_t)b * W + j]);
            a0 = fmaf(d0, h, a0);
            a1 = fmaf(d1, h, a1);
        }
        c0 += d0;
        c1 += d1;
    }
    s0[threadIdx.y][threadIdx.x] = a0;
    s1[threadIdx.y][threadIdx.x] = a1;
    __syncthreads();
    if (threadIdx.y == 0 && j < W) {
        float t0 = 0.0f, t1 = 0.0f;
        for (int k = 0; k < 8; k++) { t0 += s0[k][threadIdx.x]; t1 += s1[k][threadIdx.x]; }
        gWh[j] = t0;
        gWh[W + j] = t1;
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        s0[threadIdx.y][threadIdx.x] = c0;
        s1[threadIdx.y][threadIdx.x] = c1;
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            // every thread of a column saw the same rows: one column's partials suffice
            float t0 = 0.0f, t1 = 0.0f;
            for (int k = 0; k < 8; k++) { t0 += s0[k][0]; t1 += s1[k][0]; }
            gbh[0] = t0;
            gbh[1] = t1;
        }
    }
}

// dZ[b][j] = (dy[b][0] Wh[0][j] + dy[b][1] Wh[1][j]) * (H[b][j] > 0), BF16
__global__ void k_head_dgrad(const __nv_bfloat16* __restrict__ H, const float* __restrict__ dy, int64_t n, int W,
                             const float* __restrict__ Wh, __nv_bfloat16* __restrict__ dZ) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * W) return;
    int64_t b = k / W;
    int j = (int)(k - b * W);
    float g = dy[2 * b] * Wh[j] + dy[2 * b + 1] * Wh[W + j];
    dZ[k] = __float2bfloat16_rn(__bfloat162float(H[k]) > 0.0f ? g : 0.0f);
}

// dZ = dH * (H > 0), FP32 -> BF16
__global__ void k_relu_bwd(const float* __restrict__ dH, const __nv_bfloat16* __restrict__ H, int64_t n,
                           __nv_bfloat16* __restrict__ dZ) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dZ[k] = __float2bfloat16_rn(__bfloat162float(H[k]) > 0.0f ? dH[k] : 0.0f);
}

// out[c][r] = in[r][c], BF16, 32 x 32 tiles
__global__ void k_transpose(const __nv_bfloat16* __restrict__ in, int R, int C, __nv_bfloat16* __restrict__ out) {
    __shared__ __nv_bfloat16 t[32][34];
    int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        if (r0 + k < R && c < C) t[k][threadIdx.x] = in[(size_t)(r0 + k) * C + c];
    __syncthreads();
    int r = r0 + threadIdx.x, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        if (c0 + k < C && r < R) out[(size_t)(c0 + k) * R + r] = t[threadIdx.x][k];
}

// g[j] = sum_b dZ[b][j]
__global__ void k_colsum(const __nv_bfloat16* __restrict__ dZ, int n, int W, float* __restrict__ g) {
    __shared__ float s[8][33];
    int j = blockIdx.x * 32 + threadIdx.x;
    float a = 0.0f;
    if (j < W)
        for (int b = threadIdx.y; b < n; b += 8) a += __bfloat162float(dZ[(size_t)b * W + j]);
    s[threadIdx.y][threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.y == 0 && j < W) {
        float t = 0.0f;
        for (int k = 0; k < 8; k++) t += s[k][threadIdx.x];
        g[j] = t;
    }
}

// Adam (Kingma & Ba 2015); then BF16 copies W [out x in] and W^T [in x out]
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int64_t n, int in_dim, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wtb) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float gk = g[k];
    float mk_ = b1 * m[k] + (1.0f - b1) * gk;
    float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk_;
    v[k] = vk;
    float x = w[k] - lr * (mk_ / c1) / (sqrtf(vk / c2) + eps);
    w[k] = x;
    if (wb) {
        wb[k] = __float2bfloat16_rn(x);
        int64_t o = k / in_dim, i = k - o * in_dim;
        int64_t out_dim = n / in_dim;
        wtb[i * out_dim + o] = __float2bfloat16_rn(x);
    }
}

__global__ void k_to_bf16(const float* __restrict__ w, int64_t n, int in_dim, __nv_bfloat16* __restrict__ wb,
                          __nv_bfloat16* __restrict__ wtb) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    wb[k] = __float2bfloat16_rn(w[k]);
    int64_t o = k / in_dim, i = k - o * in_dim, out_dim = n / in_dim;
    wtb[i * out_dim + o] = __float2bfloat16_rn(w[k]);
}

// ------------------------------------------------------ fused inference
// All layers for a pair of 128-query tiles (A, B; one query per row) in a
// persistent CTA, with warp roles and mbarrier handshakes:
//   warp 8 (one lane)  streams each layer's weights by TMA in K-chunks
//                      (W output rows x 64 inputs) through a ring of NS
//                      slots; every chunk serves both tiles, so weight
//                      traffic per query is half of a one-tile design;
//   warp 9 (one lane)  issues tcgen05.mma (M = 128, N = W, K = 16) per chunk,
//                      first for tile A then for tile B, into TMEM columns
//                      [0, W) and [W, 2W); commits each slot back to the
//                      producer and each tile's last chunk to its epilogue;
//   warps 0-3 / 4-7    tile A / tile B: the Fourier features, then per layer
//                      the epilogue: read the accumulator (one TMEM lane
//                      quarter per warp), add the bias, apply ReLU, round to
//                      BF16 and write the next layer's input in place
//                      (128-byte-swizzled K-major, the layout TMA produces);
//                      after the last layer the 2-wide head.
// Tile A's epilogue overlaps tile B's last chunk, tile B's epilogue overlaps
// tile A's next layer. Every wait is bounded; after a timeout all roles
// skip their remaining work.
constexpr int FM_MAX_L = 16;
constexpr int FM_NS = 2;          // weight ring slots (W x 64 BF16 each)
constexpr int FM_THREADS = 320;   // 8 epilogue warps + producer + MMA issuer
struct alignas(64) FusedMaps {
    CUtensorMap w[FM_MAX_L];  // BF16 weights [W x K_l], box 64 x W
};

struct FusedArgs {
    const float* x;      // [n x 6]
    float* out;          // [n x 2]
    int64_t n;
    int F, W, L;
    const float* Bf;     // [F x 6]
    const float* lo;
    const float* hi;
    const float* const* bias;  // [L] device pointers to [W]
    const float* head_w;       // [2 x W]
    const float* head_b;       // [2]
    float db_scale, db_offset;
    float lam;           // free-space baseline wavelength (0 = none)
    unsigned* err;
};

__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
    // byte offset of element (r, c) inside a 64-column K-chunk (128 B rows)
    return (uint32_t)r * 128u + ((((uint32_t)c >> 3) ^ ((uint32_t)r & 7u)) << 4) + (((uint32_t)c & 7u) << 1);
}

// Shared-memory layout (offsets from a 1024-aligned base).
struct FusedLayout {
    uint32_t act_bytes, act0, act1, ring, bias, head, bf, bars;
    __host__ __device__ FusedLayout(int F, int W, int L) {
        const int kmax = (2 * F > W ? 2 * F : W) / 64;
        act_bytes = (uint32_t)kmax * 16384u;
        act0 = 0;
        act1 = act_bytes;
        ring = 2 * act_bytes;
        bias = ring + FM_NS * (uint32_t)W * 128u;
        head = bias + 4u * (uint32_t)(L * W);
        bf = head + 4u * (uint32_t)(2 * W + 2);
        bars = (bf + 4u * (uint32_t)(6 * F + 12) + 7u) & ~7u;
    }
    // ring full/empty, per tile: MMA done, input ready; MMA drain
    __host__ __device__ uint32_t bytes() const { return bars + 8u * (2 * FM_NS + 5); }
};

__global__ void __launch_bounds__(FM_THREADS, 1) k_mlp_fused(const __grid_constant__ FusedMaps maps, FusedArgs a) {
    extern __shared__ uint8_t dyn[];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    const int W = a.W, L = a.L, F = a.F;
    const FusedLayout lay(F, W, L);
    uint8_t* act[2] = {base + lay.act0, base + lay.act1};   // tile A, tile B
    uint8_t* ring = base + lay.ring;
    float* s_bias = (float*)(base + lay.bias);
    float* s_head = (float*)(base + lay.head);
    float* s_bf = (float*)(base + lay.bf);
    uint64_t* bars = (uint64_t*)(base + lay.bars);
    const uint32_t full0 = su32(bars), empty0 = su32(bars + FM_NS);
    const uint32_t mma_done0 = su32(bars + 2 * FM_NS), in_ready0 = su32(bars + 2 * FM_NS + 2);
    const uint32_t drain = su32(bars + 2 * FM_NS + 4);
    const uint32_t slot_bytes = (uint32_t)W * 128u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < L * W; i += FM_THREADS) s_bias[i] = a.bias[i / W][i % W];
    for (int i = tid; i < 2 * W; i += FM_THREADS) s_head[i] = a.head_w[i];
    if (tid < 2) s_head[2 * W + tid] = a.head_b[tid];
    for (int i = tid; i < 6 * F; i += FM_THREADS) s_bf[i] = a.Bf[i];
    if (tid < 6) {
        s_bf[6 * F + tid] = a.lo[tid];
        s_bf[6 * F + 6 + tid] = a.hi[tid];
    }
    const uint32_t tcols = 2u * (uint32_t)W <= 256u ? 256u : 512u;
    if (warp == 0) {
        tmem_alloc(su32(&tmem_slot), tcols);
        tmem_relinquish();
    }
    if (tid == 32) {
        for (int s = 0; s < FM_NS; s++) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int t = 0; t < 2; t++) {
            mbar_init(mma_done0 + 8 * t, 1);
            mbar_init(in_ready0 + 8 * t, 128);
        }
        mbar_init(drain, 1);
        mbar_fence_init();
        abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int64_t ntiles = (a.n + 127) / 128;
    const int64_t npairs = (ntiles + 1) / 2;
    auto fail = [&]() { abort_flag = 1; };

    if (warp == 8) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t pr = blockIdx.x; pr < npairs && !abort_flag; pr += gridDim.x) {
                for (int l = 0; l < L && !abort_flag; l++) {
                    const int nkc = (l == 0 ? 2 * F : W) / 64;
                    for (int kc = 0; kc < nkc; kc++, it++) {
                        const uint32_t s = it % FM_NS, ph = (it / FM_NS) & 1u;
                        if (it >= FM_NS && !mbar_wait(empty0 + 8 * s, ph ^ 1u, a.err)) {
                            fail();
                            break;
                        }
                        mbar_expect_tx(full0 + 8 * s, slot_bytes);
                        tma_load_2d(su32(ring + s * slot_bytes), &maps.w[l], kc * 64, 0, full0 + 8 * s);
                    }
                }
            }
            // drain: the last loads issued have landed before the CTA ends
            for (uint32_t j = it > FM_NS ? it - FM_NS : 0; j < it; j++)
                mbar_wait(full0 + 8 * (j % FM_NS), (j / FM_NS) & 1u, a.err);
        }
    } else if (warp == 9) {
        // -------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, W);
            uint32_t it = 0, in_ph[2] = {0, 0};
            for (int64_t pr = blockIdx.x; pr < npairs && !abort_flag; pr += gridDim.x) {
                for (int l = 0; l < L && !abort_flag; l++) {
                    const int nkc = (l == 0 ? 2 * F : W) / 64;
                    for (int kc = 0; kc < nkc; kc++, it++) {
                        const uint32_t s = it % FM_NS, ph = (it / FM_NS) & 1u;
                        if (!mbar_wait(full0 + 8 * s, ph, a.err)) { fail(); break; }
                        bool okk = true;
                        for (int t = 0; t < 2; t++) {
                            // a layer's input (features for layer 0) and free TMEM columns
                            if (kc == 0) {
                                if (!mbar_wait(in_ready0 + 8 * t, in_ph[t], a.err)) { okk = false; break; }
                                in_ph[t] ^= 1u;
                            }
                            tc_fence_after();
#pragma unroll
                            for (int k = 0; k < 4; k++)
                                mma_bf16(tmem + (uint32_t)(t * W), desc_sw128(su32(act[t] + kc * 16384) + k * 32),
                                         desc_sw128(su32(ring + s * slot_bytes) + k * 32), idesc,
                                         (kc | k) != 0 ? 1u : 0u);
                            if (kc == nkc - 1) mma_commit(mma_done0 + 8 * t);
                        }
                        mma_commit(empty0 + 8 * s);
                        if (!okk) { fail(); break; }
                    }
                }
            }
            // drain: every MMA issued has completed before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, a.err);
        }
    } else {
        // ---------------------------------------- features + epilogue, per tile
        const int t = warp >> 2;                       // 0: tile A, 1: tile B
        const int row = (warp & 3) * 32 + lane;        // query row = TMEM lane
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const uint32_t col0 = (uint32_t)(t * W);
        uint8_t* buf = act[t];
        uint32_t done_ph = 0;
        for (int64_t pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
            const int64_t q = (2 * pr + t) * 128 + row;
            {
                float xn[6];
                for (int k = 0; k < 6; k++) {
                    float xv = q < a.n ? a.x[6 * q + k] : 0.0f;
                    xn[k] = 2.0f * (xv - s_bf[6 * F + k]) / (s_bf[6 * F + 6 + k] - s_bf[6 * F + k]) - 1.0f;
                }
                for (int j = 0; j < F; j += 2) {
                    float s2[2], c2[2];
                    for (int hh = 0; hh < 2; hh++) {
                        float v = 0.0f;
                        for (int k = 0; k < 6; k++) v = fmaf(s_bf[6 * (j + hh) + k], xn[k], v);
                        v -= rintf(v);
                        feature_sincos(v, &s2[hh], &c2[hh]);
                    }
                    *(uint32_t*)(buf + (j / 64) * 16384 + sw128_off(row, j % 64)) = pack_bf16(s2[0], s2[1]);
                    *(uint32_t*)(buf + ((F + j) / 64) * 16384 + sw128_off(row, (F + j) % 64)) =
                        pack_bf16(c2[0], c2[1]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(in_ready0 + 8 * t);
            float h0 = 0.0f, h1 = 0.0f;
            bool ok = true;
            for (int l = 0; l < L; l++) {
                bool got = !abort_flag && mbar_wait(mma_done0 + 8 * t, done_ph, a.err);
                done_ph ^= 1u;
                got = __all_sync(0xffffffffu, got);
                if (!got) { fail(); ok = false; break; }
                tc_fence_after();
                for (int cc = 0; cc < W; cc += 64) {
                    // two 32-column loads in flight per wait
                    uint32_t r2[2][32];
                    tmem_ld32(tmem + lane_base + col0 + (uint32_t)cc, r2[0]);
                    tmem_ld32(tmem + lane_base + col0 + (uint32_t)cc + 32u, r2[1]);
                    tmem_wait_ld();
#pragma unroll
                    for (int hh = 0; hh < 2; hh++) {
                    const int c0 = cc + 32 * hh;
                    const uint32_t* r = r2[hh];
                    uint32_t packed[16];
                    const float4* bv = reinterpret_cast<const float4*>(s_bias + l * W + c0);
#pragma unroll
                    for (int j4 = 0; j4 < 8; j4++) {
                        const float4 b = bv[j4];
                        const int j = 4 * j4;
                        packed[2 * j4] = add2_relu_bf16x2(__uint_as_float(r[j]), b.x, __uint_as_float(r[j + 1]), b.y);
                        packed[2 * j4 + 1] =
                            add2_relu_bf16x2(__uint_as_float(r[j + 2]), b.z, __uint_as_float(r[j + 3]), b.w);
                    }
                    if (l == L - 1) {
#pragma unroll
                        for (int j = 0; j < 32; j += 2) {
                            __nv_bfloat162 b2 = *reinterpret_cast<__nv_bfloat162*>(&packed[j / 2]);
                            float r0 = __low2float(b2), r1 = __high2float(b2);
                            h0 = fmaf(r0, s_head[c0 + j], fmaf(r1, s_head[c0 + j + 1], h0));
                            h1 = fmaf(r0, s_head[W + c0 + j], fmaf(r1, s_head[W + c0 + j + 1], h1));
                        }
                    }
                    if (l < L - 1) {
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int c = c0 + 8 * u;
                            *(uint4*)(buf + (c / 64) * 16384 + sw128_off(row, c % 64)) =
                                make_uint4(packed[4 * u], packed[4 * u + 1], packed[4 * u + 2], packed[4 * u + 3]);
                        }
                    }
                    }
                }
                if (l < L - 1) {
                    // the next layer's input is in place and this tile's TMEM columns are free
                    fence_async_smem();
                    tc_fence_before();
                    mbar_arrive(in_ready0 + 8 * t);
                }
            }
            if (!ok) break;
            if (q < a.n) {
                a.out[2 * q] = h0 + s_head[2 * W];
                a.out[2 * q + 1] = (h1 + s_head[2 * W + 1]) * a.db_scale + a.db_offset + fspl_db(a.x + 6 * q, a.lam);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tcols);
}

// ------------------------------------------------------------- tensor maps
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled g_encode = nullptr;

bool load_encoder() {
    if (g_encode) return true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    g_encode = (EncodeTiled)fn;
    return true;
}

// BF16 row-major [rows x cols] (cols % 8 == 0), box = 64 columns x box_rows rows, 128-byte swizzle
bool make_map(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    if (!load_encoder()) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int pick_bn(int N) { return N <= 64 ? 64 : (N <= 128 ? 128 : 256); }

template <int BN>
size_t gemm_smem() {
    return (size_t)GSTAGES * (GM * GK * 2 + BN * GK * 2) + 1024;
}

template <int BN>
cudaError_t launch_gemm_t(cudaStream_t st, const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K,
                          const float* bias, int relu, int out_bf16, void* C, int ldc, unsigned* err) {
    size_t smem = gemm_smem<BN>();
    cudaError_t e = ensure_smem_attr((const void*)k_gemm<BN>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((M + GM - 1) / GM), (unsigned)((N + BN - 1) / BN));
    k_gemm<BN><<<grid, 128, smem, st>>>(ta, tb, M, N, K, bias, relu, out_bf16, C, ldc, err);
    return cudaGetLastError();
}

}  // namespace

// C = act(A B^T + bias): A [M x K], B [N x K] BF16 row-major (device), M, N,
// K with K % 8 == 0 and N % 8 == 0 (TMA strides); C FP32 or BF16 [M x N].
cudaError_t gemm_bf16(cudaStream_t st, const void* A, const void* B, int M, int N, int K, const float* bias, int relu,
                      int out_bf16, void* C, int ldc, unsigned* err) {
    const int BN = pick_bn(N);
    alignas(64) CUtensorMap ta, tb;
    if (!make_map(&ta, A, M, K, GM) || !make_map(&tb, B, N, K, BN)) return cudaErrorInvalidValue;
    if (BN == 64) return launch_gemm_t<64>(st, ta, tb, M, N, K, bias, relu, out_bf16, C, ldc, err);
    if (BN == 128) return launch_gemm_t<128>(st, ta, tb, M, N, K, bias, relu, out_bf16, C, ldc, err);
    return launch_gemm_t<256>(st, ta, tb, M, N, K, bias, relu, out_bf16, C, ldc, err);
}

// ------------------------------------------------------------- MLP object
struct rt_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    int F = 32, W = 256, L = 8;  // Fourier frequencies, width, hidden layers
    float db_scale = 20.0f, db_offset = -100.0f;
    float lam = 0.0f;            // free-space baseline wavelength (0 = none)
    std::string err;
    DevBuf Bf, lo, hi, errw, loss;
    std::vector<DevBuf> w, b, mw, vw, mb, vb, gw, gb, wbf, wtbf;  // per layer, head = index L
    std::vector<DevBuf> H;                                         // H[0] features, H[l] hidden outputs
    DevBuf bias_ptrs;                                              // [L] device pointers (fused kernel)
    DevBuf y, dy, dZ, dH, dZt, Ht;
    int64_t cap = 0;
    int step = 0;
    int in_dim(int l) const { return l == 0 ? 2 * F : W; }
    int out_dim(int l) const { return l == L ? 2 : W; }
};

static int mlp_err(rt_mlp* m, int code, const std::string& s) {
    m->err = s;
    return code;
}
#define MT(expr)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) return mlp_err(m, e_ == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, \
                                              std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static int mlp_reserve(rt_mlp* m, int64_t B) {
    if (B <= m->cap) return RT_OK;
    m->H.resize(m->L + 1);
    for (int l = 0; l <= m->L; l++)
        MT(buf_reserve(m->H[l], sizeof(__nv_bfloat16) * B * (l == 0 ? 2 * m->F : m->W)));
    MT(buf_reserve(m->y, sizeof(float) * 2 * B));
    MT(buf_reserve(m->dy, sizeof(float) * 2 * B));
    MT(buf_reserve(m->dZ, sizeof(__nv_bfloat16) * B * m->W));
    MT(buf_reserve(m->dH, sizeof(float) * B * m->W));
    MT(buf_reserve(m->dZt, sizeof(__nv_bfloat16) * B * m->W));
    MT(buf_reserve(m->Ht, sizeof(__nv_bfloat16) * B * m->W));
    m->cap = B;
    return RT_OK;
}

static int mlp_forward(rt_mlp* m, const float* x, int64_t B) {
    cudaStream_t st = m->stream;
    unsigned* err = bp<unsigned>(m->errw);
    dim3 fb(32, 8);
    k_features<<<(unsigned)((B + 7) / 8), fb, 0, st>>>(x, B, bp<float>(m->Bf), m->F, bp<float>(m->lo),
                                                       bp<float>(m->hi), bp<__nv_bfloat16>(m->H[0]));
    MT(cudaGetLastError());
    for (int l = 0; l < m->L; l++)
        MT(gemm_bf16(st, m->H[l].p, m->wbf[l].p, (int)B, m->W, m->in_dim(l), bp<float>(m->b[l]), 1, 1, m->H[l + 1].p,
                     m->W, err));
    k_head<<<(unsigned)((B + 7) / 8), 256, 0, st>>>(bp<__nv_bfloat16>(m->H[m->L]), B, m->W, bp<float>(m->w[m->L]),
                                                    bp<float>(m->b[m->L]), bp<float>(m->y));
    MT(cudaGetLastError());
    return RT_OK;
}

extern "C" {

int rt_mlp_create(rt_mlp** out, int device, void* stream, int32_t n_freq, int32_t width, int32_t n_hidden,
                  float sigma, uint64_t seed, const float* lo_host, const float* hi_host) {
    if (!out || n_freq < 4 || n_freq % 4 || width < 64 || width > 256 || width % 64 || n_hidden < 1 ||
        n_hidden > 16 || !lo_host || !hi_host)
        return RT_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return RT_ERR_INVALID_ARG;
    rt_mlp* m = new rt_mlp();
    m->device = device;
    m->stream = (cudaStream_t)stream;
    m->F = n_freq;
    m->W = width;
    m->L = n_hidden;
    if (!load_encoder()) {
        delete m;
        return RT_ERR_CUDA;
    }
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.0f, sigma);
    std::vector<float> Bf(6 * n_freq);
    for (auto& v : Bf) v = nd(rng);
    int n = m->L + 1;
    for (auto* v : {&m->w, &m->b, &m->mw, &m->vw, &m->mb, &m->vb, &m->gw, &m->gb}) v->resize(n);
    m->wbf.resize(m->L);
    m->wtbf.resize(m->L);
    int rc = RT_OK;
    auto up = [&](DevBuf& d, const std::vector<float>& h) -> int {
        if (buf_reserve(d, sizeof(float) * h.size()) != cudaSuccess) return RT_ERR_OOM;
        return cudaMemcpy(d.p, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice) == cudaSuccess ? RT_OK
                                                                                                          : RT_ERR_CUDA;
    };
    rc |= up(m->Bf, Bf);
    rc |= up(m->lo, std::vector<float>(lo_host, lo_host + 6));
    rc |= up(m->hi, std::vector<float>(hi_host, hi_host + 6));
    for (int l = 0; l < n && !rc; l++) {
        int fi = m->in_dim(l), fo = m->out_dim(l);
        float bound = std::sqrt(6.0f / fi) * (l == m->L ? 0.1f : 1.0f);  // He-uniform; small head
        std::uniform_real_distribution<float> ud(-bound, bound);
        std::vector<float> wv((size_t)fi * fo), zero_w((size_t)fi * fo, 0.0f), zero_b(fo, 0.0f);
        for (auto& v : wv) v = ud(rng);
        rc |= up(m->w[l], wv);
        rc |= up(m->mw[l], zero_w);
        rc |= up(m->vw[l], zero_w);
        rc |= up(m->gw[l], zero_w);
        rc |= up(m->b[l], zero_b);
        rc |= up(m->mb[l], zero_b);
        rc |= up(m->vb[l], zero_b);
        rc |= up(m->gb[l], zero_b);
        if (l < m->L && !rc) {
            if (buf_reserve(m->wbf[l], 2 * wv.size()) != cudaSuccess || buf_reserve(m->wtbf[l], 2 * wv.size()) != cudaSuccess)
                rc = RT_ERR_OOM;
            else
                k_to_bf16<<<(unsigned)((wv.size() + 255) / 256), 256>>>(bp<float>(m->w[l]), (int64_t)wv.size(), fi,
                                                                          bp<__nv_bfloat16>(m->wbf[l]),
                                                                          bp<__nv_bfloat16>(m->wtbf[l]));
        }
    }
    if (!rc && (buf_reserve(m->errw, 64) != cudaSuccess || buf_reserve(m->loss, 64) != cudaSuccess)) rc = RT_ERR_OOM;
    if (!rc) {
        cudaMemset(m->errw.p, 0, 64);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = RT_ERR_CUDA;
    }
    if (rc) {
        rt_mlp_destroy(m);
        return rc < 0 ? rc : RT_ERR_CUDA;
    }
    *out = m;
    return RT_OK;
}

int rt_mlp_destroy(rt_mlp* m) {
    if (!m) return RT_OK;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (auto* v : {&m->w, &m->b, &m->mw, &m->vw, &m->mb, &m->vb, &m->gw, &m->gb, &m->wbf, &m->wtbf, &m->H})
        for (auto& d : *v) buf_free(d);
    for (DevBuf* d : {&m->Bf, &m->lo, &m->hi, &m->errw, &m->loss, &m->y, &m->dy, &m->dZ, &m->dH, &m->dZt, &m->Ht,
                      &m->bias_ptrs})
        buf_free(*d);
    delete m;
    return RT_OK;
}

int rt_mlp_set_stream(rt_mlp* m, void* stream) {
    if (!m) return RT_ERR_INVALID_ARG;
    m->stream = (cudaStream_t)stream;
    return RT_OK;
}

int rt_mlp_last_error(const rt_mlp* m, char* buf, size_t len) {
    if (!m || !buf || !len) return RT_ERR_INVALID_ARG;
    size_t n = std::min(len - 1, m->err.size());
    memcpy(buf, m->err.data(), n);
    buf[n] = 0;
    return RT_OK;
}

int rt_mlp_infer(rt_mlp* m, const float* x, int64_t n, float* out) {
    if (!m || (n > 0 && (!x || !out))) return RT_ERR_INVALID_ARG;
    if (cudaSetDevice(m->device) != cudaSuccess) return RT_ERR_CUDA;
    if ((2 * m->F) % 64 || m->W % 64 || m->L > FM_MAX_L) return rt_mlp_infer_layers(m, x, n, out);
    if (n == 0) return RT_OK;
    alignas(64) FusedMaps maps;
    for (int l = 0; l < m->L; l++)
        if (!make_map(&maps.w[l], m->wbf[l].p, m->W, m->in_dim(l), m->W))
            return mlp_err(m, RT_ERR_CUDA, "tensor map of a weight matrix");
    if (!m->bias_ptrs.p) {
        std::vector<const float*> bp_h(m->L);
        for (int l = 0; l < m->L; l++) bp_h[l] = bp<float>(m->b[l]);
        MT(buf_reserve(m->bias_ptrs, sizeof(float*) * m->L));
        MT(cudaMemcpy(m->bias_ptrs.p, bp_h.data(), sizeof(float*) * m->L, cudaMemcpyHostToDevice));
    }
    FusedArgs a;
    a.x = x;
    a.out = out;
    a.n = n;
    a.F = m->F;
    a.W = m->W;
    a.L = m->L;
    a.Bf = bp<float>(m->Bf);
    a.lo = bp<float>(m->lo);
    a.hi = bp<float>(m->hi);
    a.bias = (const float* const*)m->bias_ptrs.p;
    a.head_w = bp<float>(m->w[m->L]);
    a.head_b = bp<float>(m->b[m->L]);
    a.db_scale = m->db_scale;
    a.db_offset = m->db_offset;
    a.lam = m->lam;
    a.err = bp<unsigned>(m->errw);
    const size_t smem = 1024 + FusedLayout(m->F, m->W, m->L).bytes();
    if (smem > 227 * 1024) return rt_mlp_infer_layers(m, x, n, out);
    MT(ensure_smem_attr((const void*)k_mlp_fused, smem));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
    int64_t npairs = ((n + 127) / 128 + 1) / 2;
    int grid = (int)std::min<int64_t>(npairs, sms);
    k_mlp_fused<<<grid, FM_THREADS, smem, m->stream>>>(maps, a);
    MT(cudaGetLastError());
    return RT_OK;
}

// Layer-by-layer inference through the generic GEMM (activations in HBM):
// the reference path the fused kernel is checked against.
int rt_mlp_infer_layers(rt_mlp* m, const float* x, int64_t n, float* out) {
    if (!m || (n > 0 && (!x || !out))) return RT_ERR_INVALID_ARG;
    if (cudaSetDevice(m->device) != cudaSuccess) return RT_ERR_CUDA;
    const int64_t chunk = 1 << 18;
    int rc = mlp_reserve(m, std::min<int64_t>(std::max<int64_t>(n, 128), chunk));
    if (rc) return rc;
    for (int64_t s = 0; s < n; s += chunk) {
        int64_t c = std::min(chunk, n - s);
        rc = mlp_forward(m, x + 6 * s, c);
        if (rc) return rc;
        k_head_out<<<(unsigned)((c + 255) / 256), 256, 0, m->stream>>>(bp<float>(m->y), x + 6 * s, c, m->db_scale,
                                                                       m->db_offset, m->lam, out + 2 * s);
        MT(cudaGetLastError());
    }
    return RT_OK;
}

int rt_mlp_set_baseline(rt_mlp* m, float wavelength) {
    if (!m || !(wavelength >= 0.0f)) return RT_ERR_INVALID_ARG;
    m->lam = wavelength;
    return RT_OK;
}

int rt_mlp_train_step(rt_mlp* m, const float* x, const float* target, int32_t B, float lr, float* loss_out) {
    if (!m || !x || !target || B < 128 || B % 128) return RT_ERR_INVALID_ARG;
    if (cudaSetDevice(m->device) != cudaSuccess) return RT_ERR_CUDA;
    int rc = mlp_reserve(m, B);
    if (rc) return rc;
    cudaStream_t st = m->stream;
    unsigned* err = bp<unsigned>(m->errw);
    rc = mlp_forward(m, x, B);
    if (rc) return rc;
    float* loss = loss_out ? loss_out : bp<float>(m->loss);
    k_loss<<<(B + 255) / 256, 256, 0, st>>>(bp<float>(m->y), target, x, B, m->db_scale, m->db_offset, m->lam,
                                           bp<float>(m->dy), loss);
    const int W = m->W, L = m->L;
    k_head_wgrad<<<(W + 31) / 32, dim3(32, 8), 0, st>>>(bp<__nv_bfloat16>(m->H[L]), bp<float>(m->dy), B, W,
                                                         bp<float>(m->gw[L]), bp<float>(m->gb[L]));
    k_head_dgrad<<<(unsigned)(((int64_t)B * W + 255) / 256), 256, 0, st>>>(
        bp<__nv_bfloat16>(m->H[L]), bp<float>(m->dy), B, W, bp<float>(m->w[L]), bp<__nv_bfloat16>(m->dZ));
    MT(cudaGetLastError());
    for (int l = L - 1; l >= 0; l--) {
        const int K = m->in_dim(l);
        // dW_l = dZ^T H_l  (GEMM over the batch)
        k_transpose<<<dim3(W / 32, B / 32), dim3(32, 8), 0, st>>>(bp<__nv_bfloat16>(m->dZ), B, W,
                                                                  bp<__nv_bfloat16>(m->dZt));
        k_transpose<<<dim3(K / 32, B / 32), dim3(32, 8), 0, st>>>(bp<__nv_bfloat16>(m->H[l]), B, K,
                                                                  bp<__nv_bfloat16>(m->Ht));
        MT(cudaGetLastError());
        MT(gemm_bf16(st, m->dZt.p, m->Ht.p, W, K, B, nullptr, 0, 0, m->gw[l].p, K, err));
        k_colsum<<<(W + 31) / 32, dim3(32, 8), 0, st>>>(bp<__nv_bfloat16>(m->dZ), B, W, bp<float>(m->gb[l]));
        MT(cudaGetLastError());
        if (l > 0) {
            // dH_{l} = dZ W_l, then through the ReLU of layer l's input
            MT(gemm_bf16(st, m->dZ.p, m->wtbf[l].p, B, K, W, nullptr, 0, 0, m->dH.p, K, err));
            k_relu_bwd<<<(unsigned)(((int64_t)B * K + 255) / 256), 256, 0, st>>>(
                bp<float>(m->dH), bp<__nv_bfloat16>(m->H[l]), (int64_t)B * K, bp<__nv_bfloat16>(m->dZ));
            MT(cudaGetLastError());
        }
    }
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
    for (int l = 0; l <= L; l++) {
        int64_t nw = (int64_t)m->in_dim(l) * m->out_dim(l);
        k_adam<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(
            bp<float>(m->w[l]), bp<float>(m->mw[l]), bp<float>(m->vw[l]), bp<float>(m->gw[l]), nw, m->in_dim(l), lr,
            b1, b2, eps, c1, c2, l < L ? bp<__nv_bfloat16>(m->wbf[l]) : nullptr,
            l < L ? bp<__nv_bfloat16>(m->wtbf[l]) : nullptr);
        k_adam<<<(m->out_dim(l) + 255) / 256, 256, 0, st>>>(bp<float>(m->b[l]), bp<float>(m->mb[l]),
                                                           bp<float>(m->vb[l]), bp<float>(m->gb[l]), m->out_dim(l), 1,
                                                           lr, b1, b2, eps, c1, c2, nullptr, nullptr);
    }
    MT(cudaGetLastError());
    return RT_OK;
}

int rt_mlp_num_params(const rt_mlp* m, int64_t* n) {
    if (!m || !n) return RT_ERR_INVALID_ARG;
    int64_t s = 0;
    for (int l = 0; l <= m->L; l++) s += (int64_t)m->in_dim(l) * m->out_dim(l) + m->out_dim(l);
    *n = s + 6 * m->F;
    return RT_OK;
}

// Parameters as one FP32 vector: per layer W [out x in] then b [out], then
// the Fourier matrix [F x 6]. dir 0: model -> dst, 1: src -> model.
static int mlp_params(rt_mlp* m, float* p, int dir) {
    if (!m || !p) return RT_ERR_INVALID_ARG;
    if (cudaSetDevice(m->device) != cudaSuccess) return RT_ERR_CUDA;
    cudaStream_t st = m->stream;
    int64_t o = 0;
    for (int l = 0; l <= m->L; l++) {
        size_t nw = (size_t)m->in_dim(l) * m->out_dim(l), nb = m->out_dim(l);
        if (dir == 0) {
            MT(cudaMemcpyAsync(p + o, m->w[l].p, 4 * nw, cudaMemcpyDeviceToDevice, st));
            MT(cudaMemcpyAsync(p + o + nw, m->b[l].p, 4 * nb, cudaMemcpyDeviceToDevice, st));
        } else {
            MT(cudaMemcpyAsync(m->w[l].p, p + o, 4 * nw, cudaMemcpyDeviceToDevice, st));
            MT(cudaMemcpyAsync(m->b[l].p, p + o + nw, 4 * nb, cudaMemcpyDeviceToDevice, st));
            if (l < m->L)
                k_to_bf16<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(bp<float>(m->w[l]), (int64_t)nw, m->in_dim(l),
                                                                       bp<__nv_bfloat16>(m->wbf[l]),
                                                                       bp<__nv_bfloat16>(m->wtbf[l]));
        }
        o += nw + nb;
    }
    if (dir == 0)
        MT(cudaMemcpyAsync(p + o, m->Bf.p, 4 * 6 * m->F, cudaMemcpyDeviceToDevice, st));
    else
        MT(cudaMemcpyAsync(m->Bf.p, p + o, 4 * 6 * m->F, cudaMemcpyDeviceToDevice, st));
    MT(cudaGetLastError());
    return RT_OK;
}

int rt_mlp_get_params(rt_mlp* m, float* dst) { return mlp_params(m, dst, 0); }
int rt_mlp_set_params(rt_mlp* m, const float* src) { return mlp_params(m, const_cast<float*>(src), 1); }

// Serialised model (rt_mlp_save / rt_mlp_load), little-endian host bytes:
//   "RTMLP001" | int32 F, W, L, 0 | float lo[6], hi[6], lam, db_scale,
//   db_offset, 0 | int64 n_params | float params[n_params] (the
//   rt_mlp_get_params layout) | uint64 FNV-1a hash of everything before it.
namespace {
constexpr char MLP_MAGIC[8] = {'R', 'T', 'M', 'L', 'P', '0', '0', '1'};
constexpr size_t MLP_HDR = 8 + 4 * 4 + 16 * 4 + 8;

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}
}  // namespace

int rt_mlp_save(rt_mlp* m, void* buf, int64_t cap, int64_t* size_out) {
    if (!m || !size_out) return RT_ERR_INVALID_ARG;
    int64_t np = 0;
    rt_mlp_num_params(m, &np);
    const size_t need = MLP_HDR + 4 * (size_t)np + 8;
    *size_out = (int64_t)need;
    if (!buf) return RT_OK;
    if (cap < (int64_t)need) return mlp_err(m, RT_ERR_CAPACITY, "mlp_save: buffer smaller than the size query");
    if (cudaSetDevice(m->device) != cudaSuccess) return RT_ERR_CUDA;
    unsigned char* out = (unsigned char*)buf;
    std::memcpy(out, MLP_MAGIC, 8);
    const int32_t dims[4] = {m->F, m->W, m->L, 0};
    std::memcpy(out + 8, dims, sizeof(dims));
    float box[16] = {0};
    MT(cudaMemcpyAsync(box, m->lo.p, 24, cudaMemcpyDeviceToHost, m->stream));
    MT(cudaMemcpyAsync(box + 6, m->hi.p, 24, cudaMemcpyDeviceToHost, m->stream));
    float* params = (float*)(out + MLP_HDR);
    int64_t o = 0;
    for (int l = 0; l <= m->L; l++) {
        size_t nw = (size_t)m->in_dim(l) * m->out_dim(l), nb = m->out_dim(l);
        MT(cudaMemcpyAsync(params + o, m->w[l].p, 4 * nw, cudaMemcpyDeviceToHost, m->stream));
        MT(cudaMemcpyAsync(params + o + nw, m->b[l].p, 4 * nb, cudaMemcpyDeviceToHost, m->stream));
        o += nw + nb;
    }
    MT(cudaMemcpyAsync(params + o, m->Bf.p, 4 * 6 * m->F, cudaMemcpyDeviceToHost, m->stream));
    MT(cudaStreamSynchronize(m->stream));
    box[12] = m->lam;
    box[13] = m->db_scale;
    box[14] = m->db_offset;
    std::memcpy(out + 8 + 16, box, sizeof(box));
    std::memcpy(out + 8 + 16 + 64, &np, 8);
    const uint64_t h = fnv1a(out, need - 8);
    std::memcpy(out + need - 8, &h, 8);
    return RT_OK;
}

int rt_mlp_load(rt_mlp** out, int device, void* cuda_stream, const void* buf, int64_t size) {
    if (!out || !buf || size < (int64_t)(MLP_HDR + 8)) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    const unsigned char* in = (const unsigned char*)buf;
    if (std::memcmp(in, MLP_MAGIC, 8) != 0) return RT_ERR_INVALID_ARG;
    int32_t dims[4];
    float box[16];
    int64_t np = 0;
    std::memcpy(dims, in + 8, sizeof(dims));
    std::memcpy(box, in + 8 + 16, sizeof(box));
    std::memcpy(&np, in + 8 + 16 + 64, 8);
    if (np < 0 || size != (int64_t)(MLP_HDR + 4 * (size_t)np + 8)) return RT_ERR_INVALID_ARG;
    uint64_t h = 0;
    std::memcpy(&h, in + size - 8, 8);
    if (h != fnv1a(in, (size_t)size - 8)) return RT_ERR_INVALID_ARG;
    rt_mlp* m = nullptr;
    int rc = rt_mlp_create(&m, device, cuda_stream, dims[0], dims[1], dims[2], 1.0f, 0, box, box + 6);
    if (rc) return rc;
    int64_t want = 0;
    rt_mlp_num_params(m, &want);
    if (want != np) {
        rt_mlp_destroy(m);
        return RT_ERR_INVALID_ARG;
    }
    DevBuf tmp;
    if (buf_reserve(tmp, 4 * (size_t)np) != cudaSuccess) {
        rt_mlp_destroy(m);
        return RT_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(tmp.p, in + MLP_HDR, 4 * (size_t)np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) rc = mlp_params(m, bp<float>(tmp), 1);
    if (e == cudaSuccess && !rc) e = cudaStreamSynchronize(m->stream);
    buf_free(tmp);
    if (e != cudaSuccess || rc) {
        rt_mlp_destroy(m);
        return rc ? rc : RT_ERR_CUDA;
    }
    m->lam = box[12];
    m->db_scale = box[13];
    m->db_offset = box[14];
    *out = m;
    return RT_OK;
}

// Gradients of the last rt_mlp_train_step (before its Adam update), same
// layout as the parameters (Fourier matrix entries are 0: not trained).
int rt_mlp_get_grads(rt_mlp* m, float* dst) {
    if (!m || !dst) return RT_ERR_INVALID_ARG;
    if (cudaSetDevice(m->device) != cudaSuccess) return RT_ERR_CUDA;
    int64_t o = 0;
    for (int l = 0; l <= m->L; l++) {
        size_t nw = (size_t)m->in_dim(l) * m->out_dim(l), nb = m->out_dim(l);
        MT(cudaMemcpyAsync(dst + o, m->gw[l].p, 4 * nw, cudaMemcpyDeviceToDevice, m->stream));
        MT(cudaMemcpyAsync(dst + o + nw, m->gb[l].p, 4 * nb, cudaMemcpyDeviceToDevice, m->stream));
        o += nw + nb;
    }
    MT(cudaMemsetAsync(dst + o, 0, 4 * 6 * m->F, m->stream));
    return RT_OK;
}

int rt_mlp_status(rt_mlp* m, uint32_t* status) {
    if (!m || !status) return RT_ERR_INVALID_ARG;
    MT(cudaMemcpy(status, m->errw.p, 4, cudaMemcpyDeviceToHost));
    return RT_OK;
}

int rt_gemm_bf16(void* stream, const void* A, const void* B, int32_t M, int32_t N, int32_t K, const float* bias,
                 int32_t relu, int32_t out_bf16, void* C, uint32_t* status) {
    if (!A || !B || !C || M < 1 || N < 8 || K < 8 || N % 8 || K % 8) return RT_ERR_INVALID_ARG;
    cudaError_t e = gemm_bf16((cudaStream_t)stream, A, B, M, N, K, bias, relu, out_bf16, C, N, status);
    return e == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

}  // extern "C"
