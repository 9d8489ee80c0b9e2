// Device Newton iteration with a Jacobi-preconditioned conjugate-gradient linear solve, used
// to drive the assembly end to end (the paper solves R(u) = 0 by Newton's method with a
// Krylov solve of K du = -R per step, Section II-A and Section V; it hands the linear solve to
// PETSc, which is not reproduced here).  Dirichlet conditions are imposed by a DOF mask: the
// residual and every Krylov vector vanish on constrained DOFs, so CG runs on the free block of
// K.  The residual and its norm are FP64 in every precision; the tangent may be FP64, FP32 or
// TF32 (an inexact Newton method).  Dot products use the fixed-shape two-pass reduction, so a
// solve is bitwise reproducible.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "jetsci_internal.h"

namespace jetsci {

__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                              double *__restrict__ partials) {
    __shared__ double red[256];
    const int64_t base = (int64_t)blockIdx.x * kNormChunk;
    const int64_t end = min(n, base + (int64_t)kNormChunk);
    double s = 0.0;
    for (int64_t t = base + threadIdx.x; t < end; t += 256) s = fma(a[t], b[t], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_dot_final(const double *__restrict__ partials, int64_t np, double *__restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < np; t += 256) s += partials[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Scalars of one CG iteration, kept on the device.
struct CgScalars {
    double rz, rz_new, pq, rr;
};

__global__ void k_zero_masked(double *__restrict__ x, const uint8_t *__restrict__ fixed, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && fixed[i]) x[i] = 0.0;
}

// Jacobi: dinv = 1 / K_ii on free DOFs, 0 on constrained ones.
template <typename VT>
__global__ void k_jacobi(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, const VT *__restrict__ vals,
                         const uint8_t *__restrict__ fixed, int64_t n, double *__restrict__ dinv) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double d = 0.0;
    int64_t lo = rowptr[r], hi = rowptr[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] == r) { d = (double)vals[mid]; break; }
        if (col[mid] < r) lo = mid + 1; else hi = mid - 1;
    }
    dinv[r] = (fixed[r] || d == 0.0) ? 0.0 : 1.0 / d;
}

// x = dinv .* r ; p = x (first iteration)
__global__ void k_precond(const double *__restrict__ dinv, const double *__restrict__ r, double *__restrict__ z,
                          double *__restrict__ p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = dinv[i] * r[i];
    z[i] = v;
    if (p) p[i] = v;
}

// x += alpha p ; r -= alpha q with alpha = rz / pq
__global__ void k_cg_update_xr(const CgScalars *__restrict__ s, const double *__restrict__ p, const double *__restrict__ q,
                               double *__restrict__ x, double *__restrict__ r, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = s->pq != 0.0 ? s->rz / s->pq : 0.0;
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
}

// p = z + beta p with beta = rz_new / rz
__global__ void k_cg_update_p(const CgScalars *__restrict__ s, const double *__restrict__ z, double *__restrict__ p,
                              int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double beta = s->rz != 0.0 ? s->rz_new / s->rz : 0.0;
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void k_cg_shift(CgScalars *s) { s->rz = s->rz_new; }

__global__ void k_axpy(double a, const double *__restrict__ x, double *__restrict__ y, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(a, x[i], y[i]);
}

__global__ void k_set_bc(const int64_t *__restrict__ dofs, const double *__restrict__ vals, int64_t nbc, int64_t n,
                         double *__restrict__ u, uint8_t *__restrict__ fixed) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbc) return;
    int64_t d = dofs[i];
    if (d < 0 || d >= n) return;  // validated on the host
    u[d] = vals[i];
    fixed[d] = 1;
}

}  // namespace jetsci

using namespace jetsci;

namespace {

struct Workspace {
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x = nullptr, *dinv = nullptr, *R = nullptr;
    double *partials = nullptr, *scal_norm = nullptr;
    CgScalars *sc = nullptr;
    uint8_t *fixed = nullptr;
    void *vals = nullptr;
    // events bracketing the residual, tangent and solve phases of a Newton step
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ~Workspace() {
        cudaFree(r); cudaFree(z); cudaFree(p); cudaFree(q); cudaFree(x); cudaFree(dinv); cudaFree(R);
        cudaFree(partials); cudaFree(scal_norm); cudaFree(sc); cudaFree(fixed); cudaFree(vals);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

// Adds the device time between two recorded events (seconds) to *acc.
static jetsci_status add_elapsed(cudaEvent_t a, cudaEvent_t b, double *acc) {
    float ms = 0.0f;
    JETSCI_CUDA_TRY(cudaEventSynchronize(b));
    JETSCI_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    *acc += 1e-3 * (double)ms;
    return JETSCI_OK;
}

inline unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

jetsci_status dot(const double *a, const double *b, int64_t n, double *partials, double *out, cudaStream_t s) {
    int64_t np = (n + kNormChunk - 1) / kNormChunk;
    if (np > 0) k_dot_partial<<<(unsigned)np, 256, 0, s>>>(a, b, n, partials);
    k_dot_final<<<1, 256, 0, s>>>(partials, np, out);
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

}  // namespace

extern "C" jetsci_status jetsci_newton_solve(jetsci_mesh m, double *u, int64_t n_bc, const int64_t *bc_dofs,
                                             const double *bc_vals, int32_t tangent_precision, double rtol,
                                             int32_t max_newton, double cg_rtol, int32_t max_cg, void *stream,
                                             jetsci_newton_info *info) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (!u || !info || (n_bc > 0 && (!bc_dofs || !bc_vals)) || n_bc < 0) return fail(JETSCI_ERR_ARG, "invalid arguments");
    if (tangent_precision != JETSCI_FP64 && tangent_precision != JETSCI_FP32 && tangent_precision != JETSCI_TF32)
        return fail(JETSCI_ERR_ARG, "tangent precision must be FP64, FP32 or TF32");
    if (!(rtol > 0) || !(cg_rtol > 0) || max_newton < 1 || max_cg < 1) return fail(JETSCI_ERR_ARG, "invalid tolerances");
    const int64_t n = m->n_dof;
    if ((n + kNormChunk - 1) / kNormChunk > kNormMaxPartials) return fail(JETSCI_ERR_ARG, "system too large");
    *info = jetsci_newton_info{};
    if (n == 0) return JETSCI_OK;
    {
        std::vector<int64_t> hb(n_bc);
        if (n_bc) JETSCI_CUDA_TRY(cudaMemcpy(hb.data(), bc_dofs, n_bc * sizeof(int64_t), cudaMemcpyDefault));
        for (int64_t v : hb)
            if (v < 0 || v >= n) return fail(JETSCI_ERR_ARG, "boundary DOF out of range");
    }
    Workspace w;
    const bool f32 = tangent_precision != JETSCI_FP64;
    JETSCI_CUDA_TRY(cudaMalloc(&w.r, n * 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.z, n * 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.p, n * 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.q, n * 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.x, n * 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.dinv, n * 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.R, n * 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.partials, kNormMaxPartials * 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.scal_norm, 8));
    JETSCI_CUDA_TRY(cudaMalloc(&w.sc, sizeof(CgScalars)));
    JETSCI_CUDA_TRY(cudaMalloc(&w.fixed, n));
    JETSCI_CUDA_TRY(cudaMalloc(&w.vals, m->nnz * (f32 ? 4 : 8) + 8));
    for (cudaEvent_t &e : w.ev) JETSCI_CUDA_TRY(cudaEventCreate(&e));
    JETSCI_CUDA_TRY(cudaMemsetAsync(w.fixed, 0, n, s));
    if (n_bc) k_set_bc<<<blocks(n_bc), 256, 0, s>>>(bc_dofs, bc_vals, n_bc, n, u, w.fixed);
    double nrm0 = 0.0;
    int total_cg = 0;
    for (int it = 0; it <= max_newton; it++) {
        // FP64 residual on the free DOFs decides convergence
        JETSCI_CUDA_TRY(cudaEventRecord(w.ev[0], s));
        if ((st = launch_residual(m, u, w.R, JETSCI_FP64, nullptr, s))) return st;
        k_zero_masked<<<blocks(n), 256, 0, s>>>(w.R, w.fixed, n);
        if ((st = launch_norm2(w.R, n, w.partials, kNormMaxPartials, w.scal_norm, s))) return st;
        JETSCI_CUDA_TRY(cudaEventRecord(w.ev[1], s));
        double nrm = 0.0;
        JETSCI_CUDA_TRY(cudaMemcpyAsync(&nrm, w.scal_norm, 8, cudaMemcpyDeviceToHost, s));
        JETSCI_CUDA_TRY(cudaStreamSynchronize(s));
        if ((st = add_elapsed(w.ev[0], w.ev[1], &info->seconds_residual))) return st;
        if (!std::isfinite(nrm)) return fail(JETSCI_ERR_NONFINITE, "non-finite residual norm");
        if (it == 0) nrm0 = nrm;
        const double rel = nrm0 > 0 ? nrm / nrm0 : 0.0;
        if (it < 32) info->residual_history[it] = rel;
        info->newton_iters = it;
        info->final_rel_residual = rel;
        info->cg_iters_total = total_cg;
        if (rel <= rtol || nrm == 0.0) return JETSCI_OK;
        if (it == max_newton) break;
        // tangent and Jacobi preconditioner
        JETSCI_CUDA_TRY(cudaEventRecord(w.ev[2], s));
        if ((st = launch_tangent(m, u, w.vals, nullptr, tangent_precision, nullptr, s))) return st;
        if (f32)
            k_jacobi<float><<<blocks(n), 256, 0, s>>>(m->d_rowptr, m->d_col, (const float *)w.vals, w.fixed, n, w.dinv);
        else
            k_jacobi<double><<<blocks(n), 256, 0, s>>>(m->d_rowptr, m->d_col, (const double *)w.vals, w.fixed, n, w.dinv);
        JETSCI_CUDA_TRY(cudaEventRecord(w.ev[3], s));
        if ((st = add_elapsed(w.ev[2], w.ev[3], &info->seconds_tangent))) return st;
        // CG on K x = -R (free block), x0 = 0
        JETSCI_CUDA_TRY(cudaMemsetAsync(w.x, 0, n * 8, s));
        JETSCI_CUDA_TRY(cudaMemcpyAsync(w.r, w.R, n * 8, cudaMemcpyDeviceToDevice, s));
        k_axpy<<<blocks(n), 256, 0, s>>>(-2.0, w.R, w.r, n);  // r = -R
        k_precond<<<blocks(n), 256, 0, s>>>(w.dinv, w.r, w.z, w.p, n);
        if ((st = dot(w.r, w.z, n, w.partials, &w.sc->rz, s))) return st;
        double rr0 = nrm * nrm;
        int k = 0;
        for (; k < max_cg; k++) {
            if ((st = launch_spmv(m, w.vals, f32, w.p, w.q, s))) return st;
            k_zero_masked<<<blocks(n), 256, 0, s>>>(w.q, w.fixed, n);
            if ((st = dot(w.p, w.q, n, w.partials, &w.sc->pq, s))) return st;
            k_cg_update_xr<<<blocks(n), 256, 0, s>>>(w.sc, w.p, w.q, w.x, w.r, n);
            k_precond<<<blocks(n), 256, 0, s>>>(w.dinv, w.r, w.z, nullptr, n);
            if ((st = dot(w.r, w.z, n, w.partials, &w.sc->rz_new, s))) return st;
            if ((k + 1) % 10 == 0) {
                if ((st = dot(w.r, w.r, n, w.partials, &w.sc->rr, s))) return st;
                double rr = 0.0;
                JETSCI_CUDA_TRY(cudaMemcpyAsync(&rr, &w.sc->rr, 8, cudaMemcpyDeviceToHost, s));
                JETSCI_CUDA_TRY(cudaStreamSynchronize(s));
                if (!std::isfinite(rr)) return fail(JETSCI_ERR_NONFINITE, "CG diverged");
                if (rr <= cg_rtol * cg_rtol * rr0) {
                    k++;
                    break;
                }
            }
            k_cg_update_p<<<blocks(n), 256, 0, s>>>(w.sc, w.z, w.p, n);
            k_cg_shift<<<1, 1, 0, s>>>(w.sc);
        }
        total_cg += k;
        if (k >= max_cg) info->cg_capped++;
        k_axpy<<<blocks(n), 256, 0, s>>>(1.0, w.x, u, n);
        JETSCI_CUDA_TRY(cudaEventRecord(w.ev[0], s));
        if ((st = add_elapsed(w.ev[3], w.ev[0], &info->seconds_solve))) return st;
        JETSCI_CUDA_TRY(cudaGetLastError());
    }
    info->cg_iters_total = total_cg;
    return fail(JETSCI_ERR_NOT_CONVERGED, "Newton did not reach the tolerance in max_newton steps");
}
