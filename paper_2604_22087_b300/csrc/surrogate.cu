// MLP constitutive surrogate: labels from the plain neo-Hookean update, on-device training
// (BF16 tensor-core forward/backward, FP32 weight gradients and Adam), evaluation of S and
// dS/dE, and attachment to a mesh for the fused element kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <string>

#include "jetsci_internal.h"
#include "surrogate.cuh"

struct jetsci_surrogate_s {
    int device = 0;
    jetsci::SurrogateConfig cfg;
    float *d_params = nullptr;  // [kNumParams] FP32 master weights
    float *d_m = nullptr, *d_v = nullptr;
    unsigned char *d_img = nullptr;  // [kImgBytes] BF16 operand image
    float *d_partial = nullptr;      // [max_ctas][kNumParams]
    float *d_partial_loss = nullptr; // [max_ctas]
    uint32_t *d_err = nullptr;
    int max_ctas = 0;
    int64_t adam_t = 0;
};

namespace jetsci {

jetsci_surrogate mesh_surrogate(jetsci_mesh m) { return m->surrogate; }
const unsigned char *surrogate_image(jetsci_surrogate s) { return s->d_img; }
const float *surrogate_params(jetsci_surrogate s) { return s->d_params; }
SurrogateConfig surrogate_config(jetsci_surrogate s) { return s->cfg; }

// ------------------------------------------------------------------ weight image
__global__ void k_pack_weights(const float *__restrict__ p, unsigned char *__restrict__ img) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 7 * 4096; i += gridDim.x * blockDim.x) {
        int r, k;
        float v = 0.0f;
        unsigned char *tile;
        int K;
        if (i < 1024) {  // W1p [64][16]
            r = i / 16; k = i % 16; K = 16; tile = img + kImgW1;
            v = k < 8 ? p[kOffW1 + r * 8 + k] : 0.0f;
        } else if (i < 1024 + 4096) {  // W2 [64][64]
            int j = i - 1024; r = j / 64; k = j % 64; K = 64; tile = img + kImgW2; v = p[kOffW2 + r * 64 + k];
        } else if (i < 1024 + 8192) {  // W3
            int j = i - 1024 - 4096; r = j / 64; k = j % 64; K = 64; tile = img + kImgW3; v = p[kOffW3 + r * 64 + k];
        } else if (i < 1024 + 8192 + 1024) {  // W4p [16][64]
            int j = i - 1024 - 8192; r = j / 64; k = j % 64; K = 64; tile = img + kImgW4;
            v = r < 6 ? p[kOffW4 + r * 64 + k] : 0.0f;
        } else if (i < 1024 + 8192 + 2048) {  // W4Tp [64][16]: W4T[n][k] = W4[k][n]
            int j = i - 1024 - 8192 - 1024; r = j / 16; k = j % 16; K = 16; tile = img + kImgW4T;
            v = k < 6 ? p[kOffW4 + k * 64 + r] : 0.0f;
        } else if (i < 1024 + 8192 + 2048 + 4096) {  // W3T[n][k] = W3[k][n]
            int j = i - 1024 - 8192 - 2048; r = j / 64; k = j % 64; K = 64; tile = img + kImgW3T; v = p[kOffW3 + k * 64 + r];
        } else if (i < 1024 + 8192 + 2048 + 8192) {  // W2T
            int j = i - 1024 - 8192 - 2048 - 4096; r = j / 64; k = j % 64; K = 64; tile = img + kImgW2T; v = p[kOffW2 + k * 64 + r];
        } else {
            continue;
        }
        *reinterpret_cast<__nv_bfloat16 *>(tile + tc::core_offset(r, k, K)) = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------------------------------ labels
// S of the compressible neo-Hookean law at Green-Lagrange strain E (Voigt, tensor shear):
// C = I + 2E, J = sqrt(det C), S = mu (I - C^-1) + lambda ln J C^-1, in FP64.
struct LameTable {
    double lam[2], mu[2];
};

__global__ void k_nh_labels(const double *__restrict__ E6, const int32_t *__restrict__ phase, int64_t n,
                            LameTable lm, double *__restrict__ S6, uint32_t *__restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *e = E6 + 6 * i;
    int p = phase[i];
    if (p != 0 && p != 1) {
        atomicOr(err, 2u);
        p = 0;
    }
    const double lam = lm.lam[p], mu = lm.mu[p];
    double C00 = 1 + 2 * e[0], C11 = 1 + 2 * e[1], C22 = 1 + 2 * e[2];
    double C12 = 2 * e[3], C02 = 2 * e[4], C01 = 2 * e[5];
    double a00 = C11 * C22 - C12 * C12, a11 = C00 * C22 - C02 * C02, a22 = C00 * C11 - C01 * C01;
    double a12 = C01 * C02 - C00 * C12, a02 = C01 * C12 - C11 * C02, a01 = C02 * C12 - C01 * C22;
    double det = C00 * a00 + C01 * a01 + C02 * a02;
    if (!(det > 0.0)) {
        atomicOr(err, 4u);
        det = 1.0;
    }
    double r = 1.0 / det;
    double lnJ = 0.5 * log(det);
    double c = lam * lnJ - mu;
    double *s = S6 + 6 * i;
    s[0] = mu + c * a00 * r;
    s[1] = mu + c * a11 * r;
    s[2] = mu + c * a22 * r;
    s[3] = c * a12 * r;
    s[4] = c * a02 * r;
    s[5] = c * a01 * r;
}

// ------------------------------------------------------------------ training step
struct __align__(128) TrainSmem {
    unsigned char w[kImgBytes];
    unsigned char x[128 * 16 * 2];
    unsigned char act[3][128 * 64 * 2];
    unsigned char dy[128 * 16 * 2];
    unsigned char dz[128 * 64 * 2];
    float dzf[128][65];
    float dyf[128][8];
    float xf[128][8];
    float b[3][64];
    float b4[8];
    float red[128];
    uint64_t mbar;
    uint32_t tmem_base;
};

__device__ __forceinline__ void sync_all() {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Gradient of sum over the CTA's 128 samples of mean-squared-error contributions
// (normalised by the whole batch) for layer outputs; writes the CTA's partial gradient.
__device__ __forceinline__ void weight_grad(const float (*dzf)[65], int n_out, const unsigned char *act_tile,
                                            int n_in, int K_tile, const float *xin, float *out_W, float *out_b) {
    const int t = threadIdx.x;
    for (int o = t; o < n_out * n_in; o += blockDim.x) {
        const int r = o / n_in, j = o % n_in;
        float s = 0.0f;
        for (int m = 0; m < 128; m++) {
            float a = xin ? xin[m * 8 + j] : tc::ld_bf16(act_tile, m, j, K_tile);
            s = fmaf(dzf[m][r], a, s);
        }
        out_W[o] = s;
    }
    for (int r = t; r < n_out; r += blockDim.x) {
        float s = 0.0f;
        for (int m = 0; m < 128; m++) s += dzf[m][r];
        out_b[r] = s;
    }
}

__global__ void __launch_bounds__(128) k_mlp_train(const unsigned char *__restrict__ img, const float *__restrict__ params,
                                                   const double *__restrict__ E6, const int32_t *__restrict__ phase,
                                                   const double *__restrict__ S6, const int32_t *__restrict__ order,
                                                   int64_t n_samples, int64_t offset, int batch, SurrogateConfig cfg,
                                                   float *__restrict__ partial, float *__restrict__ partial_loss,
                                                   uint32_t *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TrainSmem &sm = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int t = threadIdx.x;
    if (t < 32) tc::tmem_alloc(&sm.tmem_base, 512);
    if (t == 0) {
        tc::mbar_init(&sm.mbar, 1);
        tc::fence_mbar_init();
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(img);
        uint4 *dst = reinterpret_cast<uint4 *>(sm.w);
        for (int i = t; i < kImgBytes / 16; i += 128) dst[i] = src[i];
        for (int i = t; i < 64; i += 128) {
            sm.b[0][i] = params[kOffB1 + i];
            sm.b[1][i] = params[kOffB2 + i];
            sm.b[2][i] = params[kOffB3 + i];
        }
        if (t < 8) sm.b4[t] = t < 6 ? params[kOffB4 + t] : 0.0f;
    }
    // sample of this thread
    int64_t idx = order[offset + (int64_t)blockIdx.x * 128 + t];
    if (idx < 0 || idx >= n_samples) {
        atomicOr(err, 2u);
        idx = 0;
    }
    int ph = phase[idx];
    if (ph != 0 && ph != 1) {
        atomicOr(err, 2u);
        ph = 0;
    }
    float tgt[6];
    float xin[8];
#pragma unroll
    for (int c = 0; c < 6; c++) {
        xin[c] = (float)(E6[6 * idx + c] / (double)cfg.in_scale);
        tgt[c] = (float)((S6[6 * idx + c] - (double)cfg.out_shift[ph][c]) / (double)cfg.out_scale[ph][c]);
    }
    xin[6] = ph == 0 ? 1.0f : 0.0f;
    xin[7] = ph == 1 ? 1.0f : 0.0f;
#pragma unroll
    for (int k = 0; k < 16; k++) tc::st_bf16(sm.x, t, k, 16, k < 8 ? xin[k] : 0.0f);
    // the BF16-rounded inputs, as the forward pass sees them (for dW1)
#pragma unroll
    for (int k = 0; k < 8; k++) sm.xf[t][k] = tc::ld_bf16(sm.x, t, k, 16);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = sm.tmem_base;
    uint32_t phase_ctr = 0;
    bool ok = true;
    sync_all();
    // ---------------- forward
    if (t == 0) tc::gemm_bf16_128xN(tm, sm.x, sm.w + kImgW1, 64, 16);
    ok = mma_sync_bounded(&sm.mbar, phase_ctr) && ok;
    for (int layer = 0; layer < 3; layer++) {
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float z[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, 64 * layer + c0), z);
#pragma unroll
            for (int j = 0; j < 16; j++) tc::st_bf16(sm.act[layer], t, c0 + j, 64, silu_f(z[j] + sm.b[layer][c0 + j]));
        }
        sync_all();
        if (t == 0) {
            if (layer < 2)
                tc::gemm_bf16_128xN(tm + 64 * (layer + 1), sm.act[layer], sm.w + (layer == 0 ? kImgW2 : kImgW3), 64, 64);
            else
                tc::gemm_bf16_128xN(tm + 192, sm.act[2], sm.w + kImgW4, 16, 64);
        }
        ok = mma_sync_bounded(&sm.mbar, phase_ctr) && ok;
    }
    // ---------------- loss and dLoss/dy
    float loss = 0.0f;
    {
        float v[16];
        tc::tmem_ld16(tc::tmem_lane_addr(tm, 192), v);
        const float sc = 2.0f / (float)(batch * 6);
#pragma unroll
        for (int c = 0; c < 16; c++) {
            float d = 0.0f;
            if (c < 6) {
                float diff = v[c] + sm.b4[c] - tgt[c];
                loss += diff * diff;
                d = sc * diff;
            }
            if (c < 8) sm.dyf[t][c] = d;
            tc::st_bf16(sm.dy, t, c, 16, d);
        }
    }
    sm.red[t] = loss;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (t < w) sm.red[t] += sm.red[t + w];
        __syncthreads();
    }
    if (t == 0) partial_loss[blockIdx.x] = sm.red[0];
    sync_all();
    float *pg = partial + (int64_t)blockIdx.x * kNumParams;
    // ---------------- backward: dW4, db4 from dy and a3
    {
        const int n_out = 6, n_in = 64;
        for (int o = t; o < n_out * n_in; o += 128) {
            const int r = o / n_in, j = o % n_in;
            float s = 0.0f;
            for (int m = 0; m < 128; m++) s = fmaf(sm.dyf[m][r], tc::ld_bf16(sm.act[2], m, j, 64), s);
            pg[kOffW4 + o] = s;
        }
        if (t < 6) {
            float s = 0.0f;
            for (int m = 0; m < 128; m++) s += sm.dyf[m][t];
            pg[kOffB4 + t] = s;
        }
    }
    // d a3 = dy W4  (A = dy [128][16], B = W4T [64][16])
    if (t == 0) tc::gemm_bf16_128xN(tm + 256, sm.dy, sm.w + kImgW4T, 64, 16);
    ok = mma_sync_bounded(&sm.mbar, phase_ctr) && ok;
    for (int layer = 2; layer >= 0; layer--) {
        // dz_l = da_l * silu'(z_l)
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float da[16], z[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, 256 + c0), da);
            tc::tmem_ld16(tc::tmem_lane_addr(tm, 64 * layer + c0), z);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                float g = da[j] * silu_prime_f(z[j] + sm.b[layer][c0 + j]);
                sm.dzf[t][c0 + j] = g;
                tc::st_bf16(sm.dz, t, c0 + j, 64, g);
            }
        }
        sync_all();
        if (layer > 0) {
            // next: da_{l-1} = dz_l W_l  (B = W_l^T)
            if (t == 0) tc::gemm_bf16_128xN(tm + 256, sm.dz, sm.w + (layer == 2 ? kImgW3T : kImgW2T), 64, 64);
            weight_grad(sm.dzf, 64, sm.act[layer - 1], 64, 64, nullptr, pg + (layer == 2 ? kOffW3 : kOffW2),
                        pg + (layer == 2 ? kOffB3 : kOffB2));
            ok = mma_sync_bounded(&sm.mbar, phase_ctr) && ok;
            __syncthreads();  // dzf is overwritten next
        } else {
            weight_grad(sm.dzf, 64, nullptr, 8, 16, &sm.xf[0][0], pg + kOffW1, pg + kOffB1);
        }
    }
    if (!ok && t == 0) atomicOr(err, 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tm, 512);
}

// Sum of the CTAs' partial gradients in a fixed order, then (if lr > 0) one Adam step.
__global__ void k_reduce_adam(const float *__restrict__ partial, int n_cta, const float *__restrict__ partial_loss,
                              float *__restrict__ params, float *__restrict__ m, float *__restrict__ v,
                              float lr, float c1, float c2, float *__restrict__ grad_out, float *__restrict__ loss_out,
                              int batch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNumParams) {
        float g = 0.0f;
        for (int c = 0; c < n_cta; c++) g += partial[(int64_t)c * kNumParams + i];
        if (grad_out) grad_out[i] = g;
        if (lr > 0.0f) {
            const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
            float mi = b1 * m[i] + (1.0f - b1) * g;
            float vi = b2 * v[i] + (1.0f - b2) * g * g;
            m[i] = mi;
            v[i] = vi;
            params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        }
    }
    if (i == 0 && loss_out) {
        float s = 0.0f;
        for (int c = 0; c < n_cta; c++) s += partial_loss[c];
        loss_out[0] = s / (float)(batch * 6);
    }
}

// ------------------------------------------------------------------ evaluation
__global__ void __launch_bounds__(128) k_mlp_eval(const unsigned char *__restrict__ img, const float *__restrict__ params,
                                                  SurrogateConfig cfg, const double *__restrict__ E6,
                                                  const int32_t *__restrict__ phase, int64_t n, double *__restrict__ S6,
                                                  double *__restrict__ D36, uint32_t *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpTileSmem &sm = *reinterpret_cast<MlpTileSmem *>(smem_raw);
    const int t = threadIdx.x;
    if (t < 32) tc::tmem_alloc(&sm.tmem_base, kMlpTmemCols);
    if (t == 0) {
        tc::mbar_init(&sm.mbar, 1);
        tc::fence_mbar_init();
    }
    mlp_load_weights(sm, img, params);
    const int64_t i = (int64_t)blockIdx.x * 128 + t;
    const bool active = i < n;
    int ph = active ? phase[i] : 0;
    if (ph != 0 && ph != 1) {
        atomicOr(err, 2u);
        ph = 0;
    }
#pragma unroll
    for (int k = 0; k < 16; k++) {
        float xv = 0.0f;
        if (active && k < 6) xv = (float)(E6[6 * i + k] / (double)cfg.in_scale);
        if (k == 6) xv = ph == 0 ? 1.0f : 0.0f;
        if (k == 7) xv = ph == 1 ? 1.0f : 0.0f;
        tc::st_bf16(sm.x, t, k, 16, xv);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t phase_ctr = 0;
    float y[6], Jm[6][6];
    bool ok = mlp_forward_jacobian(sm, phase_ctr, y, Jm);
    if (active) {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const float sc = ph ? cfg.out_scale[1][c] : cfg.out_scale[0][c];
            S6[6 * i + c] = (double)(y[c] * sc + (ph ? cfg.out_shift[1][c] : cfg.out_shift[0][c]));
            if (D36)
#pragma unroll
                for (int d = 0; d < 6; d++) D36[36 * i + 6 * c + d] = (double)(Jm[c][d] * sc / cfg.in_scale);
        }
    }
    if (!ok && t == 0) atomicOr(err, 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(sm.tmem_base, kMlpTmemCols);
}

}  // namespace jetsci

using namespace jetsci;

namespace {

void free_surrogate(jetsci_surrogate s) {
    if (!s) return;
    cudaFree(s->d_params);
    cudaFree(s->d_m);
    cudaFree(s->d_v);
    cudaFree(s->d_img);
    cudaFree(s->d_partial);
    cudaFree(s->d_partial_loss);
    cudaFree(s->d_err);
    delete s;
}

jetsci_status enter_s(jetsci_surrogate s) {
    if (!s) return fail(JETSCI_ERR_ARG, "surrogate is NULL");
    int cur = -1;
    JETSCI_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != s->device) JETSCI_CUDA_TRY(cudaSetDevice(s->device));
    return JETSCI_OK;
}

jetsci_status check_err(jetsci_surrogate s, cudaStream_t st) {
    uint32_t e = 0;
    JETSCI_CUDA_TRY(cudaMemcpyAsync(&e, s->d_err, sizeof(e), cudaMemcpyDeviceToHost, st));
    JETSCI_CUDA_TRY(cudaStreamSynchronize(st));
    if (e) {
        cudaMemsetAsync(s->d_err, 0, sizeof(uint32_t), st);
        return fail(e & 1u ? JETSCI_ERR_CUDA : JETSCI_ERR_ARG,
                    e & 1u ? "tensor-core wait timed out in a surrogate kernel"
                           : "sample index or phase out of range in a surrogate kernel");
    }
    return JETSCI_OK;
}

}  // namespace

extern "C" jetsci_status jetsci_surrogate_create(const double *params_host, const jetsci_surrogate_config *cfg,
                                                 void *stream, jetsci_surrogate *out) {
    if (!out) return fail(JETSCI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!params_host || !cfg) return fail(JETSCI_ERR_ARG, "params or config is NULL");
    if (!(cfg->in_scale > 0) || !(cfg->range > 0)) return fail(JETSCI_ERR_ARG, "in_scale and range must be > 0");
    for (int p = 0; p < 2; p++)
        for (int c = 0; c < 6; c++)
            if (!(cfg->out_scale[p][c] != 0.0) || !std::isfinite(cfg->out_scale[p][c]) || !std::isfinite(cfg->out_shift[p][c]))
                return fail(JETSCI_ERR_ARG, "invalid output normalisation");
    for (int i = 0; i < kNumParams; i++)
        if (!std::isfinite(params_host[i])) return fail(JETSCI_ERR_ARG, "non-finite parameter");
    jetsci_surrogate s = new (std::nothrow) jetsci_surrogate_s();
    if (!s) return fail(JETSCI_ERR_OOM, "host allocation failed");
    cudaStream_t st = (cudaStream_t)stream;
    auto bail = [&](cudaError_t e, const char *what) {
        free_surrogate(s);
        return cuda_fail(e, what);
    };
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return bail(e, "cudaGetDevice");
    s->cfg.in_scale = (float)cfg->in_scale;
    s->cfg.range = (float)cfg->range;
    for (int p = 0; p < 2; p++)
        for (int c = 0; c < 6; c++) {
            s->cfg.out_scale[p][c] = (float)cfg->out_scale[p][c];
            s->cfg.out_shift[p][c] = (float)cfg->out_shift[p][c];
        }
    s->max_ctas = 1024;
    if ((e = cudaMalloc(&s->d_params, kNumParams * sizeof(float)))) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->d_m, kNumParams * sizeof(float)))) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->d_v, kNumParams * sizeof(float)))) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->d_img, kImgBytes))) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->d_partial, (size_t)s->max_ctas * kNumParams * sizeof(float)))) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->d_partial_loss, s->max_ctas * sizeof(float)))) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&s->d_err, sizeof(uint32_t)))) return bail(e, "cudaMalloc");
    float hp[kNumParams];
    for (int i = 0; i < kNumParams; i++) hp[i] = (float)params_host[i];
    if ((e = cudaMemcpyAsync(s->d_params, hp, sizeof(hp), cudaMemcpyHostToDevice, st))) return bail(e, "upload");
    if ((e = cudaMemsetAsync(s->d_m, 0, kNumParams * sizeof(float), st))) return bail(e, "memset");
    if ((e = cudaMemsetAsync(s->d_v, 0, kNumParams * sizeof(float), st))) return bail(e, "memset");
    if ((e = cudaMemsetAsync(s->d_img, 0, kImgBytes, st))) return bail(e, "memset");
    if ((e = cudaMemsetAsync(s->d_err, 0, sizeof(uint32_t), st))) return bail(e, "memset");
    k_pack_weights<<<28, 1024, 0, st>>>(s->d_params, s->d_img);
    if ((e = cudaGetLastError())) return bail(e, "k_pack_weights");
    if ((e = cudaStreamSynchronize(st))) return bail(e, "sync");
    static bool attr_done[128] = {};
    if (s->device < 128 && !attr_done[s->device]) {
        if ((e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem))))
            return bail(e, "smem attribute");
        if ((e = cudaFuncSetAttribute(k_mlp_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpTileSmem))))
            return bail(e, "smem attribute");
        attr_done[s->device] = true;
    }
    *out = s;
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_surrogate_destroy(jetsci_surrogate s) {
    if (!s) return JETSCI_OK;
    cudaDeviceSynchronize();
    free_surrogate(s);
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_surrogate_get_params(jetsci_surrogate s, double *params_host) {
    jetsci_status st = enter_s(s);
    if (st) return st;
    if (!params_host) return fail(JETSCI_ERR_ARG, "params_host is NULL");
    float hp[kNumParams];
    JETSCI_CUDA_TRY(cudaDeviceSynchronize());
    JETSCI_CUDA_TRY(cudaMemcpy(hp, s->d_params, sizeof(hp), cudaMemcpyDeviceToHost));
    for (int i = 0; i < kNumParams; i++) params_host[i] = hp[i];
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_surrogate_label(const jetsci_material *mats, int32_t n_mats, const double *E6,
                                                const int32_t *phase, int64_t n, double *S6, uint32_t *err_flag,
                                                void *stream) {
    if (!mats || n_mats < 1 || n_mats > 2) return fail(JETSCI_ERR_ARG, "need 1 or 2 materials");
    if (n < 0 || (n > 0 && (!E6 || !phase || !S6))) return fail(JETSCI_ERR_ARG, "invalid label arguments");
    if (n == 0) return JETSCI_OK;
    LameTable lm;
    for (int p = 0; p < 2; p++) {
        const jetsci_material &mt = mats[p < n_mats ? p : 0];
        double E = mt.E, nu = mt.nu;
        if (!(E > 0) || !(nu > -1 && nu < 0.5)) return fail(JETSCI_ERR_ARG, "invalid material");
        lm.lam[p] = E * nu / ((1 + nu) * (1 - 2 * nu));
        lm.mu[p] = E / (2 * (1 + nu));
    }
    if (!err_flag) return fail(JETSCI_ERR_ARG, "err_flag_dev is NULL");
    k_nh_labels<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(E6, phase, n, lm, S6, err_flag);
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

static jetsci_status train_steps(jetsci_surrogate s, const double *E6, const int32_t *phase, const double *S6,
                                 int64_t n_samples, const int32_t *order, int64_t order_len, int64_t n_steps, int32_t batch, double lr_max,
                                 double lr_min, float *loss_dev, float *grad_out, cudaStream_t st) {
    if (batch <= 0 || batch % 128 != 0 || batch / 128 > s->max_ctas)
        return fail(JETSCI_ERR_ARG, "batch must be a positive multiple of 128 up to 131072");
    if (n_steps < 0 || n_steps * (int64_t)batch > order_len) return fail(JETSCI_ERR_ARG, "order too short for the steps");
    if (!E6 || !phase || !S6 || !order || n_samples <= 0) return fail(JETSCI_ERR_ARG, "NULL or empty training buffer");
    const int n_cta = batch / 128;
    for (int64_t k = 0; k < n_steps; k++) {
        k_mlp_train<<<n_cta, 128, sizeof(TrainSmem), st>>>(s->d_img, s->d_params, E6, phase, S6, order, n_samples,
                                                           k * batch, batch,
                                                           s->cfg, s->d_partial, s->d_partial_loss, s->d_err);
        float lr = 0.0f, c1 = 1.0f, c2 = 1.0f;
        if (!grad_out) {
            double frac = n_steps > 1 ? (double)k / (double)(n_steps - 1) : 0.0;
            lr = (float)(lr_min + 0.5 * (lr_max - lr_min) * (1.0 + std::cos(M_PI * frac)));
            s->adam_t++;
            c1 = (float)(1.0 - std::pow(0.9, (double)s->adam_t));
            c2 = (float)(1.0 - std::pow(0.999, (double)s->adam_t));
        }
        k_reduce_adam<<<(kNumParams + 255) / 256, 256, 0, st>>>(s->d_partial, n_cta, s->d_partial_loss, s->d_params, s->d_m,
                                                                s->d_v, lr, c1, c2, grad_out,
                                                                loss_dev ? loss_dev + k : nullptr, batch);
        if (!grad_out) k_pack_weights<<<28, 1024, 0, st>>>(s->d_params, s->d_img);
        JETSCI_CUDA_TRY(cudaGetLastError());
    }
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_surrogate_train(jetsci_surrogate s, const double *E6, const int32_t *phase,
                                                const double *S6, int64_t n_samples, const int32_t *order,
                                                int64_t order_len,
                                                int64_t n_steps, int32_t batch, double lr_max, double lr_min,
                                                float *loss_dev, void *stream) {
    jetsci_status st = enter_s(s);
    if (st) return st;
    if (!(lr_max > 0) || !(lr_min >= 0)) return fail(JETSCI_ERR_ARG, "invalid learning rates");
    st = train_steps(s, E6, phase, S6, n_samples, order, order_len, n_steps, batch, lr_max, lr_min, loss_dev, nullptr,
                     (cudaStream_t)stream);
    if (st) return st;
    return check_err(s, (cudaStream_t)stream);
}

extern "C" jetsci_status jetsci_surrogate_gradient(jetsci_surrogate s, const double *E6, const int32_t *phase,
                                                   const double *S6, int64_t n_samples, const int32_t *order,
                                                   int32_t batch,
                                                   float *grad_dev, float *loss_dev, void *stream) {
    jetsci_status st = enter_s(s);
    if (st) return st;
    if (!grad_dev) return fail(JETSCI_ERR_ARG, "grad_dev is NULL");
    st = train_steps(s, E6, phase, S6, n_samples, order, batch, 1, batch, 0.0, 0.0, loss_dev, grad_dev,
                     (cudaStream_t)stream);
    if (st) return st;
    return check_err(s, (cudaStream_t)stream);
}

extern "C" jetsci_status jetsci_surrogate_eval(jetsci_surrogate s, const double *E6, const int32_t *phase, int64_t n,
                                               double *S6, double *D36, void *stream) {
    jetsci_status st = enter_s(s);
    if (st) return st;
    if (n < 0 || (n > 0 && (!E6 || !phase || !S6))) return fail(JETSCI_ERR_ARG, "invalid eval arguments");
    if (n == 0) return JETSCI_OK;
    cudaStream_t cs = (cudaStream_t)stream;
    k_mlp_eval<<<(unsigned)((n + 127) / 128), 128, sizeof(MlpTileSmem), cs>>>(s->d_img, s->d_params, s->cfg, E6, phase, n,
                                                                               S6, D36, s->d_err);
    JETSCI_CUDA_TRY(cudaGetLastError());
    return check_err(s, cs);
}

extern "C" jetsci_status jetsci_mesh_set_surrogate(jetsci_mesh m, jetsci_surrogate s) {
    if (!m) return fail(JETSCI_ERR_ARG, "mesh is NULL");
    if (s && s->device != m->device) return fail(JETSCI_ERR_ARG, "surrogate and mesh on different devices");
    m->surrogate = s;
    return JETSCI_OK;
}
