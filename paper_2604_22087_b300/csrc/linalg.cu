// Sparse product with the assembled CSR tangent and the deterministic FP64 norm.
#include <cuda_runtime.h>

#include "jetsci_internal.h"

namespace jetsci {

// y = K v.  Four lanes per node (eight nodes per warp): the node's three rows 3n, 3n+1,
// 3n+2 are contiguous in the CSR arrays and share one column list (node-interleaved
// DOFs), so each column index and each v entry is loaded once for three rows, and four
// lanes still read whole 32-byte sectors of each row.  Each lane sums a fixed strided
// subset and two fixed xor steps combine the lanes, so the result is reproducible.  Few
// lanes per node keep the cross-lane reduction small: on B300 every FP64 add of a warp
// shuffle reduction occupies the narrow FP64 pipe as much as a product does.  AT is the
// accumulation type (FP64 for FP64 values, FP32 for FP32 values).
constexpr int kSpmvLanes = 4;
constexpr int kSpmvDepth = 4;

template <typename VT, typename AT>
__global__ void __launch_bounds__(256) k_spmv(int64_t n_nodes, const int64_t *__restrict__ rowptr,
                                              const int32_t *__restrict__ col, const VT *__restrict__ vals,
                                              const double *__restrict__ v, double *__restrict__ y) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t node = gid / kSpmvLanes;
    const int lane = (int)(gid % kSpmvLanes);
    const bool active = node < n_nodes;
    AT s0 = 0, s1 = 0, s2 = 0;
    if (active) {
        const int64_t r0 = rowptr[3 * node];
        const int len = (int)(rowptr[3 * node + 1] - r0);
        const VT *v0 = vals + r0;
        const VT *v1 = v0 + len;
        const VT *v2 = v1 + len;
        const int32_t *c = col + r0;
        // kSpmvDepth strided entries are loaded before any is used (the column -> v -> product
        // chain of one entry would otherwise leave each lane with one load in flight); the sums
        // still take the lane's entries in order, so the result does not depend on the depth.
        int t = lane;
        for (; t + (kSpmvDepth - 1) * kSpmvLanes < len; t += kSpmvDepth * kSpmvLanes) {
            int32_t cj[kSpmvDepth];
            AT x[kSpmvDepth], a0[kSpmvDepth], a1[kSpmvDepth], a2[kSpmvDepth];
#pragma unroll
            for (int j = 0; j < kSpmvDepth; j++) cj[j] = __ldg(c + t + j * kSpmvLanes);
#pragma unroll
            for (int j = 0; j < kSpmvDepth; j++) {
                x[j] = (AT)__ldg(v + cj[j]);
                a0[j] = (AT)__ldg(v0 + t + j * kSpmvLanes);
                a1[j] = (AT)__ldg(v1 + t + j * kSpmvLanes);
                a2[j] = (AT)__ldg(v2 + t + j * kSpmvLanes);
            }
#pragma unroll
            for (int j = 0; j < kSpmvDepth; j++) {
                s0 += a0[j] * x[j];
                s1 += a1[j] * x[j];
                s2 += a2[j] * x[j];
            }
        }
        for (; t < len; t += kSpmvLanes) {
            const AT x = (AT)__ldg(v + __ldg(c + t));
            s0 += (AT)__ldg(v0 + t) * x;
            s1 += (AT)__ldg(v1 + t) * x;
            s2 += (AT)__ldg(v2 + t) * x;
        }
    }
#pragma unroll
    for (int o = kSpmvLanes / 2; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o, kSpmvLanes);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o, kSpmvLanes);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o, kSpmvLanes);
    }
    if (active && lane == 0) {
        y[3 * node] = (double)s0;
        y[3 * node + 1] = (double)s1;
        y[3 * node + 2] = (double)s2;
    }
}

jetsci_status launch_spmv(jetsci_mesh m, const void *vals, bool fp32, const double *v, double *y,
                          cudaStream_t s) {
    if (m->n_nodes == 0) return JETSCI_OK;
    unsigned grid = (unsigned)((m->n_nodes * kSpmvLanes + 255) / 256);
    if (fp32)
        k_spmv<float, float><<<grid, 256, 0, s>>>(m->n_nodes, m->d_rowptr, m->d_col, (const float *)vals, v, y);
    else
        k_spmv<double, double><<<grid, 256, 0, s>>>(m->n_nodes, m->d_rowptr, m->d_col, (const double *)vals, v, y);
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

// First pass: block b sums x[t]^2 over its chunk [b*kNormChunk, (b+1)*kNormChunk) in a
// fixed order (thread-strided, then a fixed shared-memory tree).
__global__ void __launch_bounds__(256) k_norm_partial(const double *__restrict__ x, int64_t n,
                                                      double *__restrict__ partials) {
    __shared__ double red[256];
    const int64_t base = (int64_t)blockIdx.x * kNormChunk;
    const int64_t end = min(n, base + (int64_t)kNormChunk);
    double s = 0.0;
    for (int64_t t = base + threadIdx.x; t < end; t += 256) {
        double v = x[t];
        s = fma(v, v, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// Second pass: one block sums the partials in the same fixed pattern and takes the root.
__global__ void __launch_bounds__(256) k_norm_final(const double *__restrict__ partials, int64_t np,
                                                    double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < np; t += 256) s += partials[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(red[0]);
}

jetsci_status launch_norm2(const double *x, int64_t n, double *partials, int64_t cap, double *out,
                           cudaStream_t s) {
    int64_t np = (n + kNormChunk - 1) / kNormChunk;
    if (np > cap) return fail(JETSCI_ERR_ARG, "vector too long for the norm scratch");
    if (np > 0) k_norm_partial<<<(unsigned)np, 256, 0, s>>>(x, n, partials);
    k_norm_final<<<1, 256, 0, s>>>(partials, np, out);
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

}  // namespace jetsci
