// Sparse product with the assembled CSR tangent and the deterministic FP64 norm.
#include <cuda_runtime.h>

#include "jetsci_internal.h"

namespace jetsci {

// y = K v, one warp per row; each lane sums a fixed strided subset, then a fixed xor tree.
template <typename VT>
__global__ void __launch_bounds__(256) k_spmv(int64_t n_rows, const int64_t *__restrict__ rowptr,
                                              const int32_t *__restrict__ col, const VT *__restrict__ vals,
                                              const double *__restrict__ v, double *__restrict__ y) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n_rows) return;  // uniform per warp
    double s = 0.0;
    const int64_t end = rowptr[row + 1];
    for (int64_t t = rowptr[row] + lane; t < end; t += 32) s += (double)vals[t] * v[col[t]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

jetsci_status launch_spmv(jetsci_mesh m, const void *vals, bool fp32, const double *v, double *y,
                          cudaStream_t s) {
    if (m->n_dof == 0) return JETSCI_OK;
    unsigned grid = (unsigned)((m->n_dof * 32 + 255) / 256);
    if (fp32)
        k_spmv<float><<<grid, 256, 0, s>>>(m->n_dof, m->d_rowptr, m->d_col, (const float *)vals, v, y);
    else
        k_spmv<double><<<grid, 256, 0, s>>>(m->n_dof, m->d_rowptr, m->d_col, (const double *)vals, v, y);
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
