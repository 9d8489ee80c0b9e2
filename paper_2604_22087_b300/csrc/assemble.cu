// Element kernels: residual, consistent tangent into CSR, matrix-free tangent product and
// the material-gradient (adjoint) pass.  All scatters are coloured read-modify-writes:
// within one colour no two elements share a node, colours run in a fixed order, so the
// sums are race-free without atomics and bitwise reproducible.
#include <cuda_runtime.h>

#include <type_traits>

#include "element.cuh"
#include "jetsci_internal.h"

namespace jetsci {

struct ElemArgs {
    const int32_t *__restrict__ conn;
    const double *__restrict__ coords;
    const int32_t *__restrict__ phase;
    const Material *__restrict__ mats;
    const double *__restrict__ E_elem;
    const int32_t *__restrict__ elems;  // element ids of one colour (NULL = identity)
    int64_t n;                          // number of elements in the list
    uint32_t *flags;
};

template <typename T>
__device__ __forceinline__ bool finite3(const T f[3]) {
    return isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]);
}

__device__ __forceinline__ void raise_flag(uint32_t *flags, uint32_t bits) {
    if (bits) atomicOr(flags, bits);
}

// Upper-triangle node pairs (a <= b) of the 8x8 block structure of K_e.
__constant__ int8_t kPairA[36] = {0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2,
                                  2, 2, 2, 3, 3, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 6, 6, 7};
__constant__ int8_t kPairB[36] = {0, 1, 2, 3, 4, 5, 6, 7, 1, 2, 3, 4, 5, 6, 7, 2, 3, 4,
                                  5, 6, 7, 3, 4, 5, 6, 7, 4, 5, 6, 7, 5, 6, 7, 6, 7, 7};
// Reference coordinates (+-1) of the hex8 local nodes, packed as bits (xi, eta, zeta).
__constant__ int8_t kNodeBits[8] = {0, 1, 3, 2, 4, 5, 7, 6};

// ---------------------------------------------------------------------------- residual
// R_e(a,i) = sum_q w detJ P_iJ G_aJ, scattered into R (FP64 in every precision).
template <typename T>
__global__ void __launch_bounds__(128) k_residual(ElemArgs A, const double *__restrict__ u,
                                                  double *__restrict__ R) {
    const int l = threadIdx.x & 7;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool active = slot < A.n;
    const int64_t e = A.elems ? A.elems[active ? slot : A.n - 1] : (active ? slot : A.n - 1);
    int32_t node;
    GaussKinematics<T> K;
    T cu[3];
    gauss_kinematics<T>(A.conn, A.coords, u, e, l, node, K, cu);
    ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, false);
    Constitutive<T> c;
    constitutive<T>(mt.law, from_double<T>(mt.lam), from_double<T>(mt.mu), K.H, c, false);
    T f[3];
    nodal_force(c.P, K, l, f);
    if (active) {
        uint32_t bits = (K.dJ > T(0) ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (c.ok ? 0u : JETSCI_FLAG_BAD_STATE) |
                        (finite3(f) ? 0u : JETSCI_FLAG_NONFINITE);
        raise_flag(A.flags, bits);
#pragma unroll
        for (int i = 0; i < 3; i++) R[3 * (int64_t)node + i] += to_double(f[i]);
    }
}

// ---------------------------------------------------------------------------- tangent
// Phase 1 (8 lanes per element, lane = Gauss point): kinematics and constitutive update;
// per Gauss point the spatial gradients g_a = F^-T G_a of the eight shape functions,
// tg_a = c (tau + m I) g_a, and c lam, c m, c tau_R into shared memory (c = w detJ,
// tau = F S F^T the Kirchhoff stress; tau_R = tau for the neo-Hookean law and sigma for the
// linear law, where tau = 0 in the tangent).  Phase 2 (one thread per element and node pair
// a <= b):
//   K_ab,ik = sum_q [ c lam g_ai g_bk + c m g_ak g_bi + delta_ik g_a . tg_b ]
// which is the push-forward of sum_q w detJ G_aJ (delta_ik S_JL + F_iI CC_IJKL F_kK) G_bL
// for the neo-Hookean CC (F CC F = lam I(x)I + 2 m Isym, m = mu - lam lnJ; the linear law has
// g = G, m = mu, tau = 0); the diagonal-pair thread (a == b) also forms the residual
// R_a = sum_q c tau_R g_a (= sum_q w detJ P G_a).
constexpr int kTanElems = 16;  // elements per 128-thread block

template <typename T>
struct TangentSmem {
    T g[kTanElems][8][8][3];   // [elem][q][node a][component]
    T tg[kTanElems][8][8][3];  // c (tau + m I) g_a
    T coef[kTanElems][8][8];   // [elem][q]: c lam, c m, c tau_R (00,11,22,12,02,01)
    int32_t node[kTanElems][8];
    int32_t elem[kTanElems];
};

template <typename T, typename VT>
__global__ void __launch_bounds__(128) k_tangent(ElemArgs A, const double *__restrict__ u,
                                                 const int64_t *__restrict__ rowptr,
                                                 const uint8_t *__restrict__ slotmap,
                                                 VT *__restrict__ vals, double *__restrict__ R) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TangentSmem<T> &sm = *reinterpret_cast<TangentSmem<T> *>(smem_raw);
    const int l = threadIdx.x & 7;
    const int es = threadIdx.x >> 3;
    const int64_t slot = (int64_t)blockIdx.x * kTanElems + es;
    const bool active = slot < A.n;
    const int64_t e = A.elems ? A.elems[active ? slot : A.n - 1] : (active ? slot : A.n - 1);
    {
        int32_t node;
        GaussKinematics<T> K;
        T cu[3];
        gauss_kinematics<T>(A.conn, A.coords, u, e, l, node, K, cu);
        ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, false);
        Constitutive<T> c;
        constitutive<T>(mt.law, from_double<T>(mt.lam), from_double<T>(mt.mu), K.H, c, true);
        if (active) {
            uint32_t bits = (K.dJ > T(0) ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (c.ok ? 0u : JETSCI_FLAG_BAD_STATE);
            raise_flag(A.flags, bits);
        }
        const bool lin = mt.law == JETSCI_LINEAR_ELASTIC;
        const T rdJ = my_rcp(K.dJ);
        const T cw = K.dJ * T(1.0 / 512.0);
        // W = (F Jp)^-1 = Jp^-1 F^-1 = adj(Jp) F^-1 / det(Jp)
        T W[3][3];
#pragma unroll
        for (int d = 0; d < 3; d++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                W[d][j] = (K.aJ[d][0] * c.Fi[0][j] + K.aJ[d][1] * c.Fi[1][j] + K.aJ[d][2] * c.Fi[2][j]) * rdJ;
        const T cl = cw * c.lam, cm = cw * c.m;
        // c (tau + m I), tau = 0 in the linear law's tangent
        const T t00 = cw * c.tau[0][0] + cm, t11 = cw * c.tau[1][1] + cm, t22 = cw * c.tau[2][2] + cm;
        const T t12 = cw * c.tau[1][2], t02 = cw * c.tau[0][2], t01 = cw * c.tau[0][1];
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const int bits_a = kNodeBits[a];
            const T s0 = (bits_a & 1) ? T(1) : T(-1), s1 = (bits_a & 2) ? T(1) : T(-1), s2 = (bits_a & 4) ? T(1) : T(-1);
            const T fx = T(1) + s0 * K.xi, fy = T(1) + s1 * K.eta, fz = T(1) + s2 * K.zeta;
            const T n0 = s0 * fy * fz, n1 = fx * s1 * fz, n2 = fx * fy * s2;
            T g[3];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                g[j] = W[0][j] * n0 + W[1][j] * n1 + W[2][j] * n2;
                sm.g[es][l][a][j] = g[j];
            }
            sm.tg[es][l][a][0] = t00 * g[0] + t01 * g[1] + t02 * g[2];
            sm.tg[es][l][a][1] = t01 * g[0] + t11 * g[1] + t12 * g[2];
            sm.tg[es][l][a][2] = t02 * g[0] + t12 * g[1] + t22 * g[2];
        }
        sm.coef[es][l][0] = cl;
        sm.coef[es][l][1] = cm;
        if (lin) {
            // tau_R = sigma = P for the linear law
            sm.coef[es][l][2] = cw * c.P[0][0];
            sm.coef[es][l][3] = cw * c.P[1][1];
            sm.coef[es][l][4] = cw * c.P[2][2];
            sm.coef[es][l][5] = cw * c.P[1][2];
            sm.coef[es][l][6] = cw * c.P[0][2];
            sm.coef[es][l][7] = cw * c.P[0][1];
        } else {
            sm.coef[es][l][2] = cw * c.tau[0][0];
            sm.coef[es][l][3] = cw * c.tau[1][1];
            sm.coef[es][l][4] = cw * c.tau[2][2];
            sm.coef[es][l][5] = cw * c.tau[1][2];
            sm.coef[es][l][6] = cw * c.tau[0][2];
            sm.coef[es][l][7] = cw * c.tau[0][1];
        }
        sm.node[es][hex_node_of_lane(l)] = node;
        if (l == 0) sm.elem[es] = active ? (int32_t)e : -1;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < kTanElems * 36; it += blockDim.x) {
        const int ee = it / 36, p = it - 36 * (it / 36);
        const int32_t eid = sm.elem[ee];
        if (eid < 0) continue;
        const int a = kPairA[p], b = kPairB[p];
        T Kab[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) Kab[i][k] = T(0);
        T Ra0 = T(0), Ra1 = T(0), Ra2 = T(0);
#pragma unroll 2
        for (int q = 0; q < 8; q++) {
            const T *ga = sm.g[ee][q][a];
            const T *gb = sm.g[ee][q][b];
            const T *tb = sm.tg[ee][q][b];
            const T *cf = sm.coef[ee][q];
            const T a0 = ga[0], a1 = ga[1], a2 = ga[2], b0 = gb[0], b1 = gb[1], b2 = gb[2];
            const T lam = cf[0], m = cf[1];
            const T s = fma_t(a0, tb[0], fma_t(a1, tb[1], a2 * tb[2]));
            const T la0 = lam * a0, la1 = lam * a1, la2 = lam * a2;
            const T ma0 = m * a0, ma1 = m * a1, ma2 = m * a2;
            Kab[0][0] = fma_t(la0, b0, fma_t(ma0, b0, Kab[0][0] + s));
            Kab[0][1] = fma_t(la0, b1, fma_t(ma1, b0, Kab[0][1]));
            Kab[0][2] = fma_t(la0, b2, fma_t(ma2, b0, Kab[0][2]));
            Kab[1][0] = fma_t(la1, b0, fma_t(ma0, b1, Kab[1][0]));
            Kab[1][1] = fma_t(la1, b1, fma_t(ma1, b1, Kab[1][1] + s));
            Kab[1][2] = fma_t(la1, b2, fma_t(ma2, b1, Kab[1][2]));
            Kab[2][0] = fma_t(la2, b0, fma_t(ma0, b2, Kab[2][0]));
            Kab[2][1] = fma_t(la2, b1, fma_t(ma1, b2, Kab[2][1]));
            Kab[2][2] = fma_t(la2, b2, fma_t(ma2, b2, Kab[2][2] + s));
            if (R && a == b) {
                Ra0 = fma_t(cf[2], a0, fma_t(cf[7], a1, fma_t(cf[6], a2, Ra0)));
                Ra1 = fma_t(cf[7], a0, fma_t(cf[3], a1, fma_t(cf[5], a2, Ra1)));
                Ra2 = fma_t(cf[6], a0, fma_t(cf[5], a1, fma_t(cf[4], a2, Ra2)));
            }
        }
        const int32_t na = sm.node[ee][a], nb = sm.node[ee][b];
        const int64_t sbase = 64 * (int64_t)eid;
        const int sab = slotmap[sbase + 8 * a + b];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            VT *dst = vals + rowptr[3 * (int64_t)na + i] + 3 * sab;
#pragma unroll
            for (int k = 0; k < 3; k++) dst[k] += store_as<VT>(Kab[i][k]);
        }
        if (a != b) {
            const int sba = slotmap[sbase + 8 * b + a];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                VT *dst = vals + rowptr[3 * (int64_t)nb + k] + 3 * sba;
#pragma unroll
                for (int i = 0; i < 3; i++) dst[i] += store_as<VT>(Kab[i][k]);
            }
        } else if (R) {
            const bool fin = isfinite(Ra0) && isfinite(Ra1) && isfinite(Ra2);
            if (!fin) raise_flag(A.flags, JETSCI_FLAG_NONFINITE);
            R[3 * (int64_t)na] += to_double(Ra0);
            R[3 * (int64_t)na + 1] += to_double(Ra1);
            R[3 * (int64_t)na + 2] += to_double(Ra2);
        }
    }
}

// ---------------------------------------------------------------------------- K v, matrix-free
// y_a += sum_q w detJ [ (Hv S) + tau' F^-T ] G_a with Hv = grad_X v, h = Hv F^-1,
// tau' = lam tr(h) I + m (h + h^T)  (neo-Hookean);  y_a += sum_q w detJ sigma(Hv) G_a (linear).
template <typename T>
__global__ void __launch_bounds__(128) k_apply_mf(ElemArgs A, const double *__restrict__ u,
                                                  const double *__restrict__ v, double *__restrict__ y) {
    const int l = threadIdx.x & 7;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool active = slot < A.n;
    const int64_t e = A.elems ? A.elems[active ? slot : A.n - 1] : (active ? slot : A.n - 1);
    int32_t node;
    GaussKinematics<T> K;
    T cu[3];
    gauss_kinematics<T>(A.conn, A.coords, u, e, l, node, K, cu);
    ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, false);
    T Hv[3][3];
    field_gradient<T>(v, node, l, K, Hv);
    T Y[3][3];
    bool ok = true;
    if (mt.law == JETSCI_LINEAR_ELASTIC) {
        T lam = from_double<T>(mt.lam), mu = from_double<T>(mt.mu);
        T tr = Hv[0][0] + Hv[1][1] + Hv[2][2];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) Y[i][j] = mu * (Hv[i][j] + Hv[j][i]) + ((i == j) ? lam * tr : T(0));
    } else {
        Constitutive<T> c;
        constitutive<T>(mt.law, from_double<T>(mt.lam), from_double<T>(mt.mu), K.H, c, false);
        ok = c.ok;
        T h[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) h[i][j] = Hv[i][0] * c.Fi[0][j] + Hv[i][1] * c.Fi[1][j] + Hv[i][2] * c.Fi[2][j];
        T trh = h[0][0] + h[1][1] + h[2][2];
        T tp[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) tp[i][j] = c.m * (h[i][j] + h[j][i]) + ((i == j) ? c.lam * trh : T(0));
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int J2 = 0; J2 < 3; J2++)
                Y[i][J2] = Hv[i][0] * c.S[0][J2] + Hv[i][1] * c.S[1][J2] + Hv[i][2] * c.S[2][J2] +
                           tp[i][0] * c.Fi[J2][0] + tp[i][1] * c.Fi[J2][1] + tp[i][2] * c.Fi[J2][2];
    }
    T f[3];
    nodal_force(Y, K, l, f);
    if (active) {
        uint32_t bits = (K.dJ > T(0) ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (ok ? 0u : JETSCI_FLAG_BAD_STATE) |
                        (finite3(f) ? 0u : JETSCI_FLAG_NONFINITE);
        raise_flag(A.flags, bits);
#pragma unroll
        for (int i = 0; i < 3; i++) y[3 * (int64_t)node + i] += to_double(f[i]);
    }
}

// ---------------------------------------------------------------------------- adjoint
// dL/dE_e = R[dofs_e] . R_e(u; E = 1) for L = 1/2 ||R||^2 (stress linear in E at fixed nu).
template <typename T>
__global__ void __launch_bounds__(128) k_material_grad(ElemArgs A, const double *__restrict__ u,
                                                       const double *__restrict__ R, double *__restrict__ g) {
    const int l = threadIdx.x & 7;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool active = slot < A.n;
    const int64_t e = active ? slot : A.n - 1;
    int32_t node;
    GaussKinematics<T> K;
    T cu[3];
    gauss_kinematics<T>(A.conn, A.coords, u, e, l, node, K, cu);
    ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, true);
    Constitutive<T> c;
    constitutive<T>(mt.law, from_double<T>(mt.lam), from_double<T>(mt.mu), K.H, c, false);
    T f[3];
    nodal_force(c.P, K, l, f);
    double d = R[3 * (int64_t)node] * to_double(f[0]) + R[3 * (int64_t)node + 1] * to_double(f[1]) +
               R[3 * (int64_t)node + 2] * to_double(f[2]);
    d = allreduce8(d);
    if (active && l == 0) {
        uint32_t bits = (K.dJ > T(0) ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (c.ok ? 0u : JETSCI_FLAG_BAD_STATE) |
                        (isfinite(d) ? 0u : JETSCI_FLAG_NONFINITE);
        raise_flag(A.flags, bits);
        g[e] = d;
    }
}

// ---------------------------------------------------------------------------- launchers
static ElemArgs make_args(jetsci_mesh m, const double *E_elem) {
    ElemArgs A;
    A.conn = m->d_conn;
    A.coords = m->d_coords;
    A.phase = m->d_phase;
    A.mats = m->d_mats;
    A.E_elem = E_elem;
    A.elems = nullptr;
    A.n = 0;
    A.flags = m->d_flags;
    return A;
}

template <typename T>
static void residual_colours(jetsci_mesh m, ElemArgs A, const double *u, double *R, cudaStream_t s) {
    for (int c = 0; c < m->n_colours; c++) {
        A.elems = m->d_colour_elems + m->colour_ptr[c];
        A.n = m->colour_ptr[c + 1] - m->colour_ptr[c];
        if (A.n == 0) continue;
        unsigned grid = (unsigned)((8 * A.n + 127) / 128);
        k_residual<T><<<grid, 128, 0, s>>>(A, u, R);
    }
}

jetsci_status launch_residual(jetsci_mesh m, const double *u, double *R, int precision,
                              const double *E_elem, cudaStream_t s) {
    JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
    ElemArgs A = make_args(m, E_elem);
    if (precision == JETSCI_FP64)
        residual_colours<double>(m, A, u, R, s);
    else if (precision == JETSCI_FP32 || precision == JETSCI_TF32)
        residual_colours<float>(m, A, u, R, s);
    else if (precision == JETSCI_DF64)
        residual_colours<df64>(m, A, u, R, s);
    else if (precision == JETSCI_SURROGATE)
        return launch_surrogate(m, u, nullptr, R, s);
    else
        return fail(JETSCI_ERR_UNSUPPORTED, "precision not implemented for the residual");
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

template <typename T, typename VT>
static jetsci_status tangent_colours(jetsci_mesh m, ElemArgs A, const double *u, VT *vals, double *R,
                                     cudaStream_t s) {
    const size_t smem = sizeof(TangentSmem<T>);
    JETSCI_CUDA_TRY(cudaFuncSetAttribute(k_tangent<T, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // One launch per colour.  Splitting colours into L2-sized chunks (chunk-major order) was
    // measured slower at 128^3 for every precision: the 8x more, smaller launches lose more
    // in launch tails than the L2-resident read-modify-writes gain.
    for_colour_chunks(m, 1, [&](const int32_t *elems, int64_t n) {
        A.elems = elems;
        A.n = n;
        unsigned grid = (unsigned)((A.n + kTanElems - 1) / kTanElems);
        k_tangent<T, VT><<<grid, 128, smem, s>>>(A, u, m->d_rowptr, m->d_slot, vals, R);
    });
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

jetsci_status launch_tangent(jetsci_mesh m, const double *u, void *vals, double *R, int precision,
                             const double *E_elem, cudaStream_t s) {
    ElemArgs A = make_args(m, E_elem);
    if (precision == JETSCI_FP64) {
        JETSCI_CUDA_TRY(cudaMemsetAsync(vals, 0, m->nnz * sizeof(double), s));
        if (R) JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
        return tangent_colours<double, double>(m, A, u, (double *)vals, R, s);
    }
    if (precision == JETSCI_FP32) {
        JETSCI_CUDA_TRY(cudaMemsetAsync(vals, 0, m->nnz * sizeof(float), s));
        if (R) JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
        return tangent_colours<float, float>(m, A, u, (float *)vals, R, s);
    }
    if (precision == JETSCI_DF64) {
        JETSCI_CUDA_TRY(cudaMemsetAsync(vals, 0, m->nnz * sizeof(double), s));
        if (R) JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
        return tangent_colours<df64, double>(m, A, u, (double *)vals, R, s);
    }
    if (precision == JETSCI_TF32) return launch_tf32(m, u, nullptr, (float *)vals, R, nullptr, E_elem, s);
    if (precision == JETSCI_SURROGATE) return launch_surrogate(m, u, (float *)vals, R, s);
    return fail(JETSCI_ERR_UNSUPPORTED, "precision not implemented for the tangent");
}

template <typename T>
static void apply_colours(jetsci_mesh m, ElemArgs A, const double *u, const double *v, double *y,
                          cudaStream_t s) {
    for (int c = 0; c < m->n_colours; c++) {
        A.elems = m->d_colour_elems + m->colour_ptr[c];
        A.n = m->colour_ptr[c + 1] - m->colour_ptr[c];
        if (A.n == 0) continue;
        unsigned grid = (unsigned)((8 * A.n + 127) / 128);
        k_apply_mf<T><<<grid, 128, 0, s>>>(A, u, v, y);
    }
}

jetsci_status launch_apply_mf(jetsci_mesh m, const double *u, const double *v, double *y, int precision,
                              const double *E_elem, cudaStream_t s) {
    if (precision == JETSCI_TF32) return launch_tf32(m, u, v, nullptr, nullptr, y, E_elem, s);
    JETSCI_CUDA_TRY(cudaMemsetAsync(y, 0, m->n_dof * sizeof(double), s));
    ElemArgs A = make_args(m, E_elem);
    if (precision == JETSCI_FP64)
        apply_colours<double>(m, A, u, v, y, s);
    else if (precision == JETSCI_FP32)
        apply_colours<float>(m, A, u, v, y, s);
    else if (precision == JETSCI_DF64)
        apply_colours<df64>(m, A, u, v, y, s);
    else
        return fail(JETSCI_ERR_UNSUPPORTED, "precision not implemented for the matrix-free product");
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

jetsci_status launch_material_grad(jetsci_mesh m, const double *u, const double *E_elem, const double *R,
                                   double *g, int precision, cudaStream_t s) {
    ElemArgs A = make_args(m, E_elem);
    A.n = m->n_elem;
    unsigned grid = (unsigned)((8 * A.n + 127) / 128);
    if (precision == JETSCI_FP64)
        k_material_grad<double><<<grid, 128, 0, s>>>(A, u, R, g);
    else if (precision == JETSCI_FP32 || precision == JETSCI_TF32)
        k_material_grad<float><<<grid, 128, 0, s>>>(A, u, R, g);
    else if (precision == JETSCI_DF64)
        k_material_grad<df64><<<grid, 128, 0, s>>>(A, u, R, g);
    else
        return fail(JETSCI_ERR_UNSUPPORTED, "precision not implemented for the material gradient");
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

}  // namespace jetsci
