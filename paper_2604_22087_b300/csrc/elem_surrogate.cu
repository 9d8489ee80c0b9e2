// Element residual and tangent with the MLP surrogate fused into the element kernel.
//
// One CTA = 16 elements x 8 Gauss points = one 128-point tile (two CTAs per SM).  Phase 1
// (thread = Gauss point, FP32): kinematics, Green-Lagrange strain E = 1/2 (F^T F - I),
// surrogate inputs.  Phase 2: the MLP forward and input-Jacobian pass on the tensor cores
// (BF16, FP32 accumulate in TMEM) gives S and D = dS/dE; points with any |E_ij| > range take
// S and D of the plain neo-Hookean law instead.  Phase 3a (thread = Gauss point): residual
// contribution, and the reference gradients G_b (all nodes) and the first elasticity tensor
//   A_iJkL = c (F_iI CC_IJKL F_kK + delta_ik S_JL)   (c = w detJ, CC_IJKL from D = dS/dE)
// into shared memory.  Phase 3b (thread = element node a):
//   K_ab[i][k] = sum_q sum_L M[i][k][L] G_bL,  M[i][k][L] = sum_J G_aJ A_iJkL,
// the consistent tangent sum_q w detJ G_aJ (delta_ik S_JL + F_iI CC_IJKL F_kK) G_bL.  Forming
// A once per point (about 430 multiply-adds) leaves 81 + 8 x 27 per node and point, against
// about 530 when each node contracted B_a^T (c W D) B_b itself.  The tangent is not symmetric
// for the surrogate, so all 64 node pairs are formed.
//
// The tangent (TANGENT) runs over all elements in order in one launch and writes each element's
// 24 x 24 rows and nodal forces to the row-gather workspace (gather.cu forms the CSR rows and R).
// The residual alone runs the forward pass only (no Jacobian directions: 64 TMEM columns and the
// forward part of the tile's shared memory, five CTAs per SM) and scatters R by colour.
#include <cuda_runtime.h>

#include "blocks.cuh"
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
    uint32_t *fallback_count;  // Gauss points that used the plain law (may be NULL)
};

// Per-point phase-3 record, in the (reused) input / activation / tangent region of the tile:
// G[8][3] (reference shape gradients of the eight nodes), then the point's first elasticity
// tensor times c = w detJ,
//   A[i][J][k][L] = c (F_iI CC_IJKL F_kK + delta_ik S_JL),
// as three 28-float blocks (one per i, [J][k][L], the last float padding) so that phase 3b
// reads each block with seven 16-byte loads.  Points are kRec floats apart and every element's
// eight points a further 4 floats, which puts the four elements a warp reads in phase 3b on
// distinct banks.
constexpr int kRec = 108, kRecA = 24, kRecBlk = 28;
__device__ __forceinline__ int rec_off(int p) { return p * kRec + (p >> 3) * 4; }
static_assert((128 * kRec + 16 * 4) * 4 <= 128 * 16 * 2 + 128 * 64 * 2 + 3 * 128 * 64 * 2, "phase-3 records do not fit");

// Voigt index of the tensor component (I, J): [11, 22, 33, 23, 13, 12].
__host__ __device__ constexpr int voigt_of(int I, int J) { return I == J ? I : 6 - I - J; }

template <bool TANGENT>
__global__ void __launch_bounds__(128, 2) k_elem_surrogate(SurArgs A, const double *__restrict__ u,
                                                           const unsigned char *__restrict__ img,
                                                           const float *__restrict__ params, SurrogateConfig cfg,
                                                           float *__restrict__ vals, double *__restrict__ R) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpTileSmem &sm = *reinterpret_cast<MlpTileSmem *>(smem_raw);
    __shared__ int32_t s_node[16][8];
    __shared__ int32_t s_elem[16];
    const int t = threadIdx.x;
    const int l = t & 7, es = t >> 3;
    constexpr uint32_t kCols = TANGENT ? kMlpTmemCols : kMlpFwdTmemCols;
    if (t < 32) tc::tmem_alloc(&sm.tmem_base, kCols);
    if (t == 0) {
        tc::mbar_init(&sm.mbar, 1);
        tc::fence_mbar_init();
    }
    mlp_load_weights(sm, img, params);
    const int64_t slot = (int64_t)blockIdx.x * 16 + es;
    const bool active = slot < A.n;
    const int64_t e = A.elems ? A.elems[active ? slot : A.n - 1] : (active ? slot : A.n - 1);
    // ---------------- phase 1
    int32_t node;
    GaussKinematics<float> K;
    float cu[3];
    gauss_kinematics_coords<float>(A.conn, A.coords, u, e, l, node, K, cu);
    const int ph = A.phase[e];
    const Material mt = A.mats[ph];
    float H[3][3], F[3][3];
    displacement_gradient(K, H);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) F[i][j] = (i == j ? 1.0f : 0.0f) + H[i][j];
    float E6[6];
#pragma unroll
    for (int a = 0; a < 6; a++) {
        const int I = voigt_i(a), Jj = voigt_j(a);
        const float c = F[0][I] * F[0][Jj] + F[1][I] * F[1][Jj] + F[2][I] * F[2][Jj];
        E6[a] = 0.5f * (c - (I == Jj ? 1.0f : 0.0f));
    }
    bool in_range = ph == 0 || ph == 1;
#pragma unroll
    for (int a = 0; a < 6; a++) in_range = in_range && fabsf(E6[a]) <= cfg.range;
    // one reciprocal for the input and Jacobian scalings (IEEE divisions there cost about 400
    // instructions per point)
    const float rin = 1.0f / cfg.in_scale;
    {
        float xv[16];
#pragma unroll
        for (int k = 0; k < 16; k++) xv[k] = 0.0f;
#pragma unroll
        for (int k = 0; k < 6; k++) xv[k] = E6[k] * rin;
        xv[6] = ph == 0 ? 1.0f : 0.0f;
        xv[7] = ph == 1 ? 1.0f : 0.0f;
        st_bf16x8(sm.x, t, 0, 16, xv);
        st_bf16x8(sm.x, t, 1, 16, xv + 8);
    }
    s_node[es][hex_node_of_lane(l)] = node;
    if (l == 0) s_elem[es] = active ? (int32_t)e : -1;
    // ---------------- phase 2
    uint32_t phase_ctr = 0;
    float y[6], Jm[6][6];
    // the residual needs S only: the Jacobian's six directions run for the tangent alone
    const bool ok = TANGENT ? mlp_forward_jacobian(sm, phase_ctr, y, Jm) : mlp_forward(sm, phase_ctr, y);
    float S[6], D[6][6];
    bool ok_state = true;
    const int phs = ph == 1 ? 1 : 0;
    if (in_range) {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const float sc = phs ? cfg.out_scale[1][c] : cfg.out_scale[0][c];
            S[c] = y[c] * sc + (phs ? cfg.out_shift[1][c] : cfg.out_shift[0][c]);
            if (TANGENT) {
                const float scd = sc * rin;
#pragma unroll
                for (int d = 0; d < 6; d++) D[c][d] = Jm[c][d] * scd;
            }
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
            const int I = voigt_i(a), Jj = voigt_j(a);
            S[a] = (lam * lnJ - mu) * Ci[I][Jj] + (I == Jj ? mu : 0.0f);
            if (TANGENT)
#pragma unroll
            for (int b = 0; b < 6; b++) {
                const int Kk = voigt_i(b), L = voigt_j(b);
                const float v = lam * Ci[I][Jj] * Ci[Kk][L] + m * (Ci[I][Kk] * Ci[Jj][L] + Ci[I][L] * Ci[Jj][Kk]);
                D[a][b] = (Kk == L) ? v : 2.0f * v;
            }
        }
        if (active && A.fallback_count) atomicAdd(A.fallback_count, 1u);
    }
    // ---------------- phase 3a: residual and per-point records
    {
        const float Smat[3][3] = {{S[0], S[5], S[4]}, {S[5], S[1], S[3]}, {S[4], S[3], S[2]}};
        float P[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int J2 = 0; J2 < 3; J2++)
                P[i][J2] = F[i][0] * Smat[0][J2] + F[i][1] * Smat[1][J2] + F[i][2] * Smat[2][J2];
        float f[3];
        nodal_force(P, K, l, f);
        if (active) {
            const uint32_t bits = (K.dJ > 0.0f ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (ok_state ? 0u : JETSCI_FLAG_BAD_STATE) |
                                  (isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]) ? 0u : JETSCI_FLAG_NONFINITE) |
                                  (ok ? 0u : JETSCI_FLAG_NONFINITE);
            if (bits) atomicOr(A.flags, bits);
            if (R) {
                if (TANGENT)  // the workspace's residual part [element][local node][3]
#pragma unroll
                    for (int i = 0; i < 3; i++) R[3 * (8 * e + hex_node_of_lane(l)) + i] = to_double(f[i]);
                else
#pragma unroll
                    for (int i = 0; i < 3; i++) R[3 * (int64_t)node + i] += to_double(f[i]);
            }
        }
    }
    if (!TANGENT) {
        tc::fence_before_sync();
        __syncthreads();
        if (t < 32) tc::tmem_dealloc(sm.tmem_base, kCols);
        return;
    }
    __syncthreads();  // every MLP tile consumed: the region becomes the point records
    float *recs = reinterpret_cast<float *>(sm.x);
    {
        float *me = recs + rec_off(t);
        const float rdJ = 1.0f / K.dJ;
        const float c = K.dJ * (1.0f / 512.0f);
        float Gv[24];
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const int nb = hex_node_of_lane(a);  // the map is an involution: node -> sign bits
            const float s0 = (nb & 1) ? 1.0f : -1.0f, s1 = (nb & 2) ? 1.0f : -1.0f, s2 = (nb & 4) ? 1.0f : -1.0f;
            const float fx = 1.0f + s0 * K.xi, fy = 1.0f + s1 * K.eta, fz = 1.0f + s2 * K.zeta;
            const float n0 = s0 * fy * fz, n1 = fx * s1 * fz, n2 = fx * fy * s2;
#pragma unroll
            for (int j = 0; j < 3; j++) Gv[3 * a + j] = (K.aJ[0][j] * n0 + K.aJ[1][j] * n1 + K.aJ[2][j] * n2) * rdJ;
        }
#pragma unroll
        for (int c4 = 0; c4 < 6; c4++)
            reinterpret_cast<float4 *>(me)[c4] = make_float4(Gv[4 * c4], Gv[4 * c4 + 1], Gv[4 * c4 + 2], Gv[4 * c4 + 3]);
        // c CC in Voigt pairs: D differentiates w.r.t. tensor components with a shear column
        // standing for both E_KL and E_LK, so CC_IJKL = D[IJ][KL] / 2 for K != L
        float Cv[6][6];
#pragma unroll
        for (int v = 0; v < 6; v++)
#pragma unroll
            for (int d = 0; d < 6; d++) Cv[v][d] = (d < 3 ? c : 0.5f * c) * D[v][d];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            // Z[J][KL] = sum_I F_iI c CC_IJKL
            float Z[3][6];
#pragma unroll
            for (int J = 0; J < 3; J++)
#pragma unroll
                for (int d = 0; d < 6; d++)
                    Z[J][d] = F[i][0] * Cv[voigt_of(0, J)][d] + F[i][1] * Cv[voigt_of(1, J)][d] +
                              F[i][2] * Cv[voigt_of(2, J)][d];
            float Ai[kRecBlk];
#pragma unroll
            for (int J = 0; J < 3; J++)
#pragma unroll
                for (int k = 0; k < 3; k++)
#pragma unroll
                    for (int L = 0; L < 3; L++) {
                        float sacc = F[k][0] * Z[J][voigt_of(0, L)] + F[k][1] * Z[J][voigt_of(1, L)] +
                                     F[k][2] * Z[J][voigt_of(2, L)];
                        if (k == i) sacc += c * S[voigt_of(J, L)];
                        Ai[9 * J + 3 * k + L] = sacc;
                    }
            Ai[27] = 0.0f;
#pragma unroll
            for (int c4 = 0; c4 < kRecBlk / 4; c4++)
                reinterpret_cast<float4 *>(me + kRecA + kRecBlk * i)[c4] =
                    make_float4(Ai[4 * c4], Ai[4 * c4 + 1], Ai[4 * c4 + 2], Ai[4 * c4 + 3]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(sm.tmem_base, kCols);
    // ---------------- phase 3b: thread = (element es, node a = l)
    //   K_ab[i][k] += sum_L M[i][k][L] G_bL,  M[i][k][L] = sum_J G_aJ A[i][J][k][L]
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
#pragma unroll 1
    for (int q = 0; q < 8; q++) {
        const float *r = recs + rec_off(8 * es + q);
        const float ga0 = r[3 * a], ga1 = r[3 * a + 1], ga2 = r[3 * a + 2];
        float M[3][3][3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            float Ai[kRecBlk];
#pragma unroll
            for (int c4 = 0; c4 < kRecBlk / 4; c4++) {
                const float4 x = reinterpret_cast<const float4 *>(r + kRecA + kRecBlk * i)[c4];
                Ai[4 * c4] = x.x, Ai[4 * c4 + 1] = x.y, Ai[4 * c4 + 2] = x.z, Ai[4 * c4 + 3] = x.w;
            }
#pragma unroll
            for (int k = 0; k < 3; k++)
#pragma unroll
                for (int L = 0; L < 3; L++)
                    M[i][k][L] = fmaf(ga0, Ai[3 * k + L], fmaf(ga1, Ai[9 + 3 * k + L], ga2 * Ai[18 + 3 * k + L]));
        }
        float Gb[24];
#pragma unroll
        for (int c4 = 0; c4 < 6; c4++) {
            const float4 x = reinterpret_cast<const float4 *>(r)[c4];
            Gb[4 * c4] = x.x, Gb[4 * c4 + 1] = x.y, Gb[4 * c4 + 2] = x.z, Gb[4 * c4 + 3] = x.w;
        }
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const float g0 = Gb[3 * b], g1 = Gb[3 * b + 1], g2 = Gb[3 * b + 2];
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int k = 0; k < 3; k++)
                    Kab[b][i][k] = fmaf(M[i][k][0], g0, fmaf(M[i][k][1], g1, fmaf(M[i][k][2], g2, Kab[b][i][k])));
        }
    }
    // rows 3a .. 3a+2 of K_e: 72 contiguous values of the workspace [element][24][24]
    float4 *dst = reinterpret_cast<float4 *>(vals + 576 * (int64_t)eid + 72 * a);
#pragma unroll
    for (int c = 0; c < 18; c++) {
        float x[4];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int v = 4 * c + h, i = v / 24, b = (v % 24) / 3, k = v % 3;
            x[h] = Kab[b][i][k];
        }
        dst[c] = make_float4(x[0], x[1], x[2], x[3]);
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
    JETSCI_CUDA_TRY(cudaMemsetAsync(m->d_fallback, 0, sizeof(uint32_t), s));
    const SurrogateConfig cfg = surrogate_config(sg);
    if (vals) {
        // row-gather assembly: element rows (one launch, elements in order), then the row pass
        void *ws = nullptr;
        double *Re = nullptr;
        if (jetsci_status st = ensure_block_workspace(m, blk_full_bytes(m->n_elem, sizeof(float)), s, &ws, &Re))
            return st;
        if (!R) Re = nullptr;
        if (m->n_elem > 0) {
            if (jetsci_status st = kernel_attrs_once<k_elem_surrogate<true>>(smem, false)) return st;
            A.elems = nullptr;
            A.n = m->n_elem;
            const unsigned grid = (unsigned)((A.n + 15) / 16);
            k_elem_surrogate<true><<<grid, 128, smem, s>>>(A, u, surrogate_image(sg), surrogate_params(sg), cfg,
                                                           (float *)ws, Re);
            JETSCI_CUDA_TRY(cudaGetLastError());
        }
        return launch_gather_rows<float>(m, (const float *)ws, Re, vals, R, s);
    }
    // residual only: the forward pass needs the tile's first kMlpFwdSmem bytes (five CTAs per SM)
    if (jetsci_status st = kernel_attrs_once<k_elem_surrogate<false>>(kMlpFwdSmem, false)) return st;
    if (R) JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
    for_each_colour(m, [&](const int32_t *elems, int64_t n) {
        A.elems = elems;
        A.n = n;
        unsigned grid = (unsigned)((A.n + 15) / 16);
        k_elem_surrogate<false><<<grid, 128, kMlpFwdSmem, s>>>(A, u, surrogate_image(sg), surrogate_params(sg), cfg,
                                                        nullptr, R);
    });
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

}  // namespace jetsci
