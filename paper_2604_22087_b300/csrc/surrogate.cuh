// MLP constitutive surrogate: parameter layout, BF16 operand images and the tensor-core
// forward / input-Jacobian pass shared by the standalone evaluation kernel and the fused
// element kernels.
//
// Network (a reading of the paper's remark that a surrogate model can replace the explicit
// material function, Section III-B): x = [E_voigt / in_scale (6), one-hot phase (2)] ->
// 3 x (Linear 64 + SiLU) -> Linear 6 -> normalised S; S_c = y_c * out_scale[p][c] +
// out_shift[p][c].  The tangent dS/dE is the input-Jacobian, propagated forward through the
// layers as 6 tangent vectors per point: T1 = silu'(z1) (.) W1[:, :6], T_l = silu'(z_l) (.)
// (W_l T_{l-1}), J = W4 T3.  For a tile of 128 points every hidden layer is one GEMM for the
// activations plus six for the tangents (M = 128, N = 64, K = 64, BF16 in, FP32 accumulate in
// TMEM).
#pragma once

#include <cstddef>

#include <cuda_bf16.h>
#include <stdint.h>

#include "tc.cuh"

namespace jetsci {

constexpr int kMlpIn = 8, kMlpH = 64, kMlpOut = 6;
// FP32 parameter vector: W1[64][8], b1[64], W2[64][64], b2, W3[64][64], b3, W4[6][64], b4[6].
constexpr int kOffW1 = 0, kOffB1 = 512, kOffW2 = 576, kOffB2 = 4672, kOffW3 = 4736, kOffB3 = 8832,
              kOffW4 = 8896, kOffB4 = 9280, kNumParams = 9286;
// BF16 operand image (bytes), K-major core-matrix tiles: W1p [64 n][16 k] (k >= 8 zero),
// W2, W3 [64][64], W4p [16 n][64 k] (n >= 6 zero), W4Tp [64 n][16 k] (k >= 6 zero),
// W3T, W2T [64][64] (transposes for the backward pass).
constexpr int kImgW1 = 0, kImgW2 = 2048, kImgW3 = 10240, kImgW4 = 18432, kImgW4T = 20480, kImgW3T = 22528,
              kImgW2T = 30720, kImgBytes = 38912, kImgFwdBytes = 20480;

struct SurrogateConfig {
    float in_scale;
    float range;
    float out_scale[2][6];
    float out_shift[2][6];
};

// SiLU a = z s and its derivative s (1 + z (1 - s)) = s + a (1 - s) with s = 1 / (1 + e^-z),
// from the fast exponential and a fast reciprocal: their few-ulp FP32 errors are far below the
// BF16 rounding (2^-9) every activation and tangent goes through, and an IEEE-rounded division
// here made the epilogues several times slower.  The derivative reuses a: one FMA after 1 - s.
__device__ __forceinline__ float sigmoid_f(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }
__device__ __forceinline__ float silu_prime_f(float z) {
    const float s = sigmoid_f(z);
    return fmaf(z * s, 1.0f - s, s);
}
__device__ __forceinline__ void silu_and_prime(float z, float &a, float &ds) {
    const float s = sigmoid_f(z);
    a = z * s;
    ds = fmaf(a, 1.0f - s, s);
}

// Shared-memory workspace of one 128-point tile for the forward + input-Jacobian pass.  The
// six Jacobian directions run in two rounds of three (the forward pass is recomputed in the
// second round), so a tile needs 256 TMEM columns and about 91 KB of shared memory and two
// CTAs fit on one SM.  The forward pass alone (the residual) uses everything before `tan`
// (kMlpFwdSmem, about 43 KB) and 64 TMEM columns, so five CTAs fit.
constexpr int kMlpTmemCols = 256;
constexpr int kMlpFwdTmemCols = 64;

struct __align__(128) MlpTileSmem {
    unsigned char w[kImgFwdBytes];       // W1p, W2, W3, W4p
    float b[3][64];
    float b4[8];
    float w1t[8][64];                    // FP32 W1 transposed (tangent seeds), [input][unit]
    uint64_t mbar;
    uint32_t tmem_base;
    alignas(128) unsigned char x[128 * 16 * 2];  // inputs [128][16]; x, act and tan are contiguous
    unsigned char act[128 * 64 * 2];             // activations [128][64]
    unsigned char tan[3][128 * 64 * 2];          // tangent rows of the round's three directions
};
constexpr size_t kMlpFwdSmem = offsetof(MlpTileSmem, tan);

// Cooperative load of the forward weights into shared memory (all 128 threads).
__device__ __forceinline__ void mlp_load_weights(MlpTileSmem &sm, const unsigned char *__restrict__ img,
                                                 const float *__restrict__ params) {
    const int t = threadIdx.x;
    const uint4 *src = reinterpret_cast<const uint4 *>(img);
    uint4 *dst = reinterpret_cast<uint4 *>(sm.w);
    for (int i = t; i < kImgFwdBytes / 16; i += blockDim.x) dst[i] = src[i];
    for (int i = t; i < 64; i += blockDim.x) {
        sm.b[0][i] = params[kOffB1 + i];
        sm.b[1][i] = params[kOffB2 + i];
        sm.b[2][i] = params[kOffB3 + i];
    }
    for (int i = t; i < 8; i += blockDim.x) sm.b4[i] = i < 6 ? params[kOffB4 + i] : 0.0f;
    for (int i = t; i < 512; i += blockDim.x) sm.w1t[i & 7][i >> 3] = params[kOffW1 + i];
}

// 16 consecutive FP32 values from 16-byte aligned shared memory (four vector loads; the
// bias and seed rows are read by every thread of the tile, a broadcast).
__device__ __forceinline__ void ld_f32x16(const float *p, float (&v)[16]) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float4 q = reinterpret_cast<const float4 *>(p)[k];
        v[4 * k] = q.x, v[4 * k + 1] = q.y, v[4 * k + 2] = q.z, v[4 * k + 3] = q.w;
    }
}

// Stores 8 consecutive values (columns 8*c8 .. 8*c8+7 of row r) as one 16-byte core-matrix
// row; a quarter-warp's eight rows then cover 128 contiguous bytes (no bank conflicts).
__device__ __forceinline__ void st_bf16x8(unsigned char *tile, int r, int c8, int K, const float *v) {
    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 p1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]);
    __nv_bfloat162 p3 = __floats2bfloat162_rn(v[6], v[7]);
    uint4 q;
    q.x = *reinterpret_cast<uint32_t *>(&p0);
    q.y = *reinterpret_cast<uint32_t *>(&p1);
    q.z = *reinterpret_cast<uint32_t *>(&p2);
    q.w = *reinterpret_cast<uint32_t *>(&p3);
    *reinterpret_cast<uint4 *>(tile + tc::core_offset(r, 8 * c8, K)) = q;
}

// Commits the MMAs issued by thread 0 and waits (all threads) with a bound.  `phase` is a
// per-thread copy of the mbarrier's completed-phase count, advanced in lockstep by every
// thread.  Returns false on timeout.
__device__ __forceinline__ bool mma_sync_bounded(uint64_t *mbar, uint32_t &phase) {
    if (threadIdx.x == 0) tc::mma_commit(mbar);
    bool ok = tc::mbar_wait_bounded(mbar, phase & 1);
    phase++;
    tc::fence_after_sync();
    return ok;
}

__device__ __forceinline__ void smem_to_tensor_sync() {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Forward pass only (the residual needs S, not dS/dE) for the tile whose inputs are already in
// sm.x: on return thread t holds y[6] (normalised outputs).  Returns false if a tensor-core wait
// timed out.
__device__ inline bool mlp_forward(MlpTileSmem &sm, uint32_t &phase, float y[6]) {
    const int t = threadIdx.x;
    const uint32_t tm = sm.tmem_base;
    smem_to_tensor_sync();
    if (t == 0) tc::gemm_bf16_128xN(tm, sm.x, sm.w + kImgW1, 64, 16);
    bool ok = mma_sync_bounded(&sm.mbar, phase);
#pragma unroll 1
    for (int layer = 0; layer < 3; layer++) {
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float z[16], a[16], bias[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, c0), z);
            ld_f32x16(&sm.b[layer][c0], bias);
#pragma unroll
            for (int j = 0; j < 16; j++) a[j] = silu_f(z[j] + bias[j]);
            st_bf16x8(sm.act, t, c0 / 8, 64, a);
            st_bf16x8(sm.act, t, c0 / 8 + 1, 64, a + 8);
        }
        smem_to_tensor_sync();
        if (t == 0) {
            const unsigned char *W = sm.w + (layer == 0 ? kImgW2 : layer == 1 ? kImgW3 : kImgW4);
            tc::gemm_bf16_128xN(tm, sm.act, W, layer < 2 ? 64 : 16, 64);
        }
        ok = mma_sync_bounded(&sm.mbar, phase) && ok;
    }
    float v[16];
    tc::tmem_ld16(tc::tmem_lane_addr(tm, 0), v);
#pragma unroll
    for (int c = 0; c < 6; c++) y[c] = v[c] + sm.b4[c];
    return ok;
}

// One round of the forward and input-Jacobian pass: directions 3 ROUND .. 3 ROUND + 2.  The
// round is a template parameter, so the columns of Jm that the round fills are fixed at
// compile time (a single copy of this code with the round chosen at run time returned the
// second round's middle direction in both rounds' middle column from the evaluation kernel).
template <int ROUND>
__device__ __forceinline__ bool mlp_jacobian_round(MlpTileSmem &sm, uint32_t &phase, float y[6], float Jm[6][6]) {
    const int t = threadIdx.x;
    const uint32_t tm = sm.tmem_base;
    constexpr int round = ROUND;
    bool ok = true;
    smem_to_tensor_sync();
    // layer 1: z1 = x W1^T (K = 16, zero-padded)
    if (t == 0) tc::gemm_bf16_128xN(tm, sm.x, sm.w + kImgW1, 64, 16);
    ok = mma_sync_bounded(&sm.mbar, phase) && ok;
#pragma unroll 1
    for (int layer = 0; layer < 3; layer++) {
        // epilogue of layer `layer`: activation, silu' and the three tangent rows
        float s[64];
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float z[16], a[16], bias[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, c0), z);
            ld_f32x16(&sm.b[layer][c0], bias);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                silu_and_prime(z[j] + bias[j], a[j], s[c0 + j]);
            }
            st_bf16x8(sm.act, t, c0 / 8, 64, a);
            st_bf16x8(sm.act, t, c0 / 8 + 1, 64, a + 8);
        }
#pragma unroll
        for (int dl = 0; dl < 3; dl++) {
            const int d = 3 * round + dl;
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                float u[16];
                if (layer == 0) {
                    ld_f32x16(&sm.w1t[d][c0], u);
#pragma unroll
                    for (int j = 0; j < 16; j++) u[j] *= s[c0 + j];
                } else {
                    tc::tmem_ld16(tc::tmem_lane_addr(tm, 64 * (dl + 1) + c0), u);
#pragma unroll
                    for (int j = 0; j < 16; j++) u[j] *= s[c0 + j];
                }
                st_bf16x8(sm.tan[dl], t, c0 / 8, 64, u);
                st_bf16x8(sm.tan[dl], t, c0 / 8 + 1, 64, u + 8);
            }
        }
        smem_to_tensor_sync();
        if (t == 0) {
            const unsigned char *W = sm.w + (layer == 0 ? kImgW2 : layer == 1 ? kImgW3 : kImgW4);
            const int N = layer < 2 ? 64 : 16;
            tc::gemm_bf16_128xN(tm, sm.act, W, N, 64);
            for (int dl = 0; dl < 3; dl++) tc::gemm_bf16_128xN(tm + 64 * (dl + 1), sm.tan[dl], W, N, 64);
        }
        ok = mma_sync_bounded(&sm.mbar, phase) && ok;
    }
    float v[16];
    if (ROUND == 0) {
        tc::tmem_ld16(tc::tmem_lane_addr(tm, 0), v);
#pragma unroll
        for (int c = 0; c < 6; c++) y[c] = v[c] + sm.b4[c];
    }
#pragma unroll
    for (int dl = 0; dl < 3; dl++) {
        tc::tmem_ld16(tc::tmem_lane_addr(tm, 64 * (dl + 1)), v);
#pragma unroll
        for (int c = 0; c < 6; c++) Jm[c][3 * ROUND + dl] = v[c];
    }
    return ok;
}

// Runs the forward and input-Jacobian pass for the tile whose inputs are already in sm.x
// (row t = point t).  On return thread t holds y[6] (normalised outputs) and Jm[6][6]
// (dy/dx, column d = input direction d).  Returns false if a tensor-core wait timed out.
__device__ inline bool mlp_forward_jacobian(MlpTileSmem &sm, uint32_t &phase, float y[6], float Jm[6][6]) {
    const bool ok0 = mlp_jacobian_round<0>(sm, phase, y, Jm);
    const bool ok1 = mlp_jacobian_round<1>(sm, phase, y, Jm);
    return ok0 && ok1;
}

}  // namespace jetsci
