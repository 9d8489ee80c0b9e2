// Element residual and tangent with the MLP surrogate fused into the element kernel.
//
// One CTA = 16 elements x 8 Gauss points = one 128-point tile.  Phase 1 (thread = Gauss
// point, FP32): kinematics, Green-Lagrange strain E = 1/2 (F^T F - I), surrogate inputs.
// Phase 2: the MLP forward and input-Jacobian pass on the tensor cores (BF16, FP32
// accumulate in TMEM) gives S and D = dS/dE; points with any |E_ij| > range take S and D of
// the plain neo-Hookean law instead.  Phase 3a (thread = Gauss point): residual
// contribution and, per node b, B_b = dE/du_b (Voigt, tensor components), c W D and c S
// (c = w detJ, W = diag(1,1,1,2,2,2)) into shared memory.  Phase 3b (thread = element node
// a): K_ab = sum_q [ B_a^T (c W D) B_b + (G_a . c S G_b) I ], the consistent tangent
// sum_q w detJ G_aJ (delta_ik S_JL + F_iI CC_IJKL F_kK) G_bL written with the Voigt
// tangent; it is not symmetric for the surrogate, so all 64 node pairs are formed.
#include <cuda_runtime.h>

#include "element.cuh"
#include "jetsci_internal.h"
#include "surrogate.cuh"

struct jetsci_surrogate_s;

namespace jetsci {

jetsci_surrogate mesh_surrogate(jetsci_mesh m);
const unsigned char *surrogate_image(jetsci_surrogate s);
const float *surrogate_params(jetsci_surrogate s);
SurrogateConfig surrogate_config(jetsci_surrogate s);

struct SurArgs {
    const int32_t *__restrict__ conn;
    const double *__restrict__ coords;
    const int32_t *__restrict__ phase;
    const Material *__restrict__ mats;
    const int32_t *__restrict__ elems;
    int64_t n;
    uint32_t *flags;
    uint32_t *fallback_count;  // number of Gauss points that used the plain law (may be NULL)
};

// Per-point phase-3 record in the (reused) activation / tangent region of the tile smem.
struct PointRec {
    float G[8][3];
    float B[8][6][3];
    float cWD[6][6];
    float cS[6];
};
static_assert(sizeof(PointRec) * 128 <= 128 * 16 * 2 + 128 * 64 * 2 + 6 * 128 * 64 * 2, "phase-3 records do not fit");

__constant__ int8_t kVoigtI[6] = {0, 1, 2, 1, 0, 0};
__constant__ int8_t kVoigtJ[6] = {0, 1, 2, 2, 2, 1};

template <bool TANGENT>
__global__ void __launch_bounds__(128) k_elem_surrogate(SurArgs A, const double *__restrict__ u,
                                                        const unsigned char *__restrict__ img,
                                                        const float *__restrict__ params, SurrogateConfig cfg,
                                                        const int64_t *__restrict__ rowptr,
                                                        const uint8_t *__restrict__ slotmap, float *__restrict__ vals,
                                                        double *__restrict__ R) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpTileSmem &sm = *reinterpret_cast<MlpTileSmem *>(smem_raw);
    __shared__ int32_t s_node[16][8];
    __shared__ int32_t s_elem[16];
    const int t = threadIdx.x;
    const int l = t & 7, es = t >> 3;
    if (t < 32) tc::tmem_alloc(&sm.tmem_base, 512);
    if (t == 0) {
        tc::mbar_init(&sm.mbar, 1);
        tc::fence_mbar_init();
    }
    mlp_load_weights(sm, img, params);
    const int64_t slot = (int64_t)blockIdx.x * 16 + es;
    const bool active = slot < A.n;
    const int64_t e = A.elems[active ? slot : A.n - 1];
    // ---------------- phase 1
    int32_t node;
    GaussKinematics<float> K;
    float cu[3];
    gauss_kinematics<float>(A.conn, A.coords, u, e, l, node, K, cu);
    const Material mt = A.mats[A.phase[e]];
    int ph = A.phase[e];
    float F[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) F[i][j] = (i == j ? 1.0f : 0.0f) + K.H[i][j];
    float E6[6];
#pragma unroll
    for (int a = 0; a < 6; a++) {
        const int I = kVoigtI[a], Jj = kVoigtJ[a];
        float c = F[0][I] * F[0][Jj] + F[1][I] * F[1][Jj] + F[2][I] * F[2][Jj];
        E6[a] = 0.5f * (c - (I == Jj ? 1.0f : 0.0f));
    }
    bool in_range = ph == 0 || ph == 1;
#pragma unroll
    for (int a = 0; a < 6; a++) in_range = in_range && fabsf(E6[a]) <= cfg.range;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        float xv = 0.0f;
        if (k < 6) xv = E6[k] / cfg.in_scale;
        if (k == 6) xv = ph == 0 ? 1.0f : 0.0f;
        if (k == 7) xv = ph == 1 ? 1.0f : 0.0f;
        tc::st_bf16(sm.x, t, k, 16, xv);
    }
    s_node[es][hex_node_of_lane(l)] = node;
    if (l == 0) s_elem[es] = active ? (int32_t)e : -1;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---------------- phase 2
    uint32_t phase_ctr = 0;
    float y[6], Jm[6][6];
    bool ok = mlp_forward_jacobian(sm, phase_ctr, y, Jm);
    float S[6], D[6][6];
    bool ok_state = true;
    const int phs = ph == 1 ? 1 : 0;
    if (in_range) {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const float sc = cfg.out_scale[phs][c];
            S[c] = y[c] * sc + cfg.out_shift[phs][c];
#pragma unroll
            for (int d = 0; d < 6; d++) D[c][d] = Jm[c][d] * sc / cfg.in_scale;
        }
    } else {
        // plain compressible neo-Hookean: S = mu I + (lam lnJ - mu) C^-1,
        // D_ab = dS_a/dE_b = lam Ci_a Ci_b + m (Ci_IK Ci_JL + Ci_IL Ci_JK) * (2 if b is shear)
        const float lam = (float)mt.lam, mu = (float)mt.mu;
        float aF[3][3];
        adj3(F, aF);
        float Jd = F[0][0] * aF[0][0] + F[0][1] * aF[1][0] + F[0][2] * aF[2][0];
        ok_state = Jd > 0.0f;
        if (!ok_state) Jd = 1.0f;
        const float rJ = 1.0f / Jd, lnJ = logf(Jd);
        float Fi[3][3], Ci[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) Fi[i][j] = aF[i][j] * rJ;
#pragma unroll
        for (int I = 0; I < 3; I++)
#pragma unroll
            for (int Kk = 0; Kk < 3; Kk++) Ci[I][Kk] = Fi[I][0] * Fi[Kk][0] + Fi[I][1] * Fi[Kk][1] + Fi[I][2] * Fi[Kk][2];
        const float m = mu - lam * lnJ;
#pragma unroll
        for (int a = 0; a < 6; a++) {
            const int I = kVoigtI[a], Jj = kVoigtJ[a];
            S[a] = (lam * lnJ - mu) * Ci[I][Jj] + (I == Jj ? mu : 0.0f);
#pragma unroll
            for (int b = 0; b < 6; b++) {
                const int Kk = kVoigtI[b], L = kVoigtJ[b];
                float v = lam * Ci[I][Jj] * Ci[Kk][L] + m * (Ci[I][Kk] * Ci[Jj][L] + Ci[I][L] * Ci[Jj][Kk]);
                D[a][b] = (Kk == L) ? v : 2.0f * v;
            }
        }
        if (active && A.fallback_count) atomicAdd(A.fallback_count, 1u);
    }
    // ---------------- phase 3a: residual and per-point records
    float Smat[3][3] = {{S[0], S[5], S[4]}, {S[5], S[1], S[3]}, {S[4], S[3], S[2]}};
    float P[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int J2 = 0; J2 < 3; J2++) P[i][J2] = F[i][0] * Smat[0][J2] + F[i][1] * Smat[1][J2] + F[i][2] * Smat[2][J2];
    float f[3];
    nodal_force(P, K, l, f);
    if (active) {
        uint32_t bits = (K.dJ > 0.0f ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (ok_state ? 0u : JETSCI_FLAG_BAD_STATE) |
                        (isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]) ? 0u : JETSCI_FLAG_NONFINITE) |
                        (ok ? 0u : JETSCI_FLAG_NONFINITE);
        if (bits) atomicOr(A.flags, bits);
        if (R)
#pragma unroll
            for (int i = 0; i < 3; i++) R[3 * (int64_t)node + i] += (double)f[i];
    }
    if (!TANGENT) {
        tc::fence_before_sync();
        __syncthreads();
        if (t < 32) tc::tmem_dealloc(sm.tmem_base, 512);
        return;
    }
    __syncthreads();  // all MLP tiles consumed: the region becomes the point records
    PointRec *rec = reinterpret_cast<PointRec *>(sm.x);
    PointRec &me = rec[t];
    {
        const float rdJ = 1.0f / K.dJ;
        const float c = K.dJ * (1.0f / 512.0f);
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const int nb = hex_node_of_lane(a);  // the map is an involution: also node -> sign bits
            const float s0 = (nb & 1) ? 1.0f : -1.0f, s1 = (nb & 2) ? 1.0f : -1.0f, s2 = (nb & 4) ? 1.0f : -1.0f;
            const float fx = 1.0f + s0 * K.xi, fy = 1.0f + s1 * K.eta, fz = 1.0f + s2 * K.zeta;
            const float n0 = s0 * fy * fz, n1 = fx * s1 * fz, n2 = fx * fy * s2;
            float G[3];
#pragma unroll
            for (int j = 0; j < 3; j++) G[j] = (K.aJ[0][j] * n0 + K.aJ[1][j] * n1 + K.aJ[2][j] * n2) * rdJ;
#pragma unroll
            for (int j = 0; j < 3; j++) me.G[a][j] = G[j];
#pragma unroll
            for (int v = 0; v < 6; v++) {
                const int I = kVoigtI[v], Jj = kVoigtJ[v];
#pragma unroll
                for (int i = 0; i < 3; i++) me.B[a][v][i] = 0.5f * (F[i][I] * G[Jj] + F[i][Jj] * G[I]);
            }
        }
#pragma unroll
        for (int v = 0; v < 6; v++) {
            const float w = v < 3 ? c : 2.0f * c;
#pragma unroll
            for (int b = 0; b < 6; b++) me.cWD[v][b] = w * D[v][b];
            me.cS[v] = c * S[v];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(sm.tmem_base, 512);
    // ---------------- phase 3b: thread = (element es, node a = l)
    const int32_t eid = s_elem[es];
    if (eid < 0) return;
    const int a = l;
    float Kab[8][3][3];
#pragma unroll
    for (int b = 0; b < 8; b++)
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) Kab[b][i][k] = 0.0f;
    for (int q = 0; q < 8; q++) {
        const PointRec &r = rec[8 * es + q];
        float Y[3][6];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int bb = 0; bb < 6; bb++) {
                float s = 0.0f;
#pragma unroll
                for (int v = 0; v < 6; v++) s += r.B[a][v][i] * r.cWD[v][bb];
                Y[i][bb] = s;
            }
        const float ga0 = r.G[a][0], ga1 = r.G[a][1], ga2 = r.G[a][2];
        const float sg0 = r.cS[0] * ga0 + r.cS[5] * ga1 + r.cS[4] * ga2;
        const float sg1 = r.cS[5] * ga0 + r.cS[1] * ga1 + r.cS[3] * ga2;
        const float sg2 = r.cS[4] * ga0 + r.cS[3] * ga1 + r.cS[2] * ga2;
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const float geo = sg0 * r.G[b][0] + sg1 * r.G[b][1] + sg2 * r.G[b][2];
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    float s = (i == k) ? geo : 0.0f;
#pragma unroll
                    for (int v = 0; v < 6; v++) s += Y[i][v] * r.B[b][v][k];
                    Kab[b][i][k] += s;
                }
        }
    }
    const int32_t na = s_node[es][a];
    const uint8_t *sl = slotmap + 64 * (int64_t)eid + 8 * a;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float *row = vals + rowptr[3 * (int64_t)na + i];
#pragma unroll
        for (int b = 0; b < 8; b++) {
            float *dst = row + 3 * (int)sl[b];
#pragma unroll
            for (int k = 0; k < 3; k++) dst[k] += Kab[b][i][k];
        }
    }
}

jetsci_status launch_surrogate(jetsci_mesh m, const double *u, float *vals, double *R, cudaStream_t s) {
    jetsci_surrogate sg = mesh_surrogate(m);
    if (!sg) return fail(JETSCI_ERR_ARG, "no surrogate attached to the mesh (jetsci_mesh_set_surrogate)");
    for (int p = 0; p < m->n_mats; p++)
        if (m->mats[p].law != JETSCI_NEO_HOOKEAN || p > 1)
            return fail(JETSCI_ERR_UNSUPPORTED, "the surrogate path needs at most two neo-Hookean phases");
    SurArgs A;
    A.conn = m->d_conn;
    A.coords = m->d_coords;
    A.phase = m->d_phase;
    A.mats = m->d_mats;
    A.flags = m->d_flags;
    A.fallback_count = m->d_fallback;
    const size_t smem = sizeof(MlpTileSmem);
    if (vals) {
        JETSCI_CUDA_TRY(cudaFuncSetAttribute(k_elem_surrogate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        JETSCI_CUDA_TRY(cudaMemsetAsync(vals, 0, m->nnz * sizeof(float), s));
    } else {
        JETSCI_CUDA_TRY(cudaFuncSetAttribute(k_elem_surrogate<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (R) JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
    JETSCI_CUDA_TRY(cudaMemsetAsync(m->d_fallback, 0, sizeof(uint32_t), s));
    const SurrogateConfig cfg = surrogate_config(sg);
    for (int c = 0; c < m->n_colours; c++) {
        A.elems = m->d_colour_elems + m->colour_ptr[c];
        A.n = m->colour_ptr[c + 1] - m->colour_ptr[c];
        if (A.n == 0) continue;
        unsigned grid = (unsigned)((A.n + 15) / 16);
        if (vals)
            k_elem_surrogate<true><<<grid, 128, smem, s>>>(A, u, surrogate_image(sg), surrogate_params(sg), cfg,
                                                           m->d_rowptr, m->d_slot, vals, R);
        else
            k_elem_surrogate<false><<<grid, 128, smem, s>>>(A, u, surrogate_image(sg), surrogate_params(sg), cfg,
                                                            m->d_rowptr, m->d_slot, nullptr, R);
    }
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

}  // namespace jetsci
