// Element stiffness on the tensor cores in TF32 (FP32 accumulate in TMEM): CSR assembly and
// the matrix-free product K.v.
//
// For one element, K_e = sum_q B_q^T (c_q W D_q) B_q + geometric term, where B_q (6 x 24) maps
// nodal displacements to the Voigt tensor components of the Green-Lagrange strain increment,
// D_q = dS/dE (6 x 6) and W = diag(1,1,1,2,2,2).  Stacking the 8 Gauss points gives one
// contraction over K = 48 = (q, Voigt component): K_mat = Bt^T Zt with Bt, Zt of 48 x 24 and
// Zt = blockdiag(c W D) Bt.  Four elements share one tcgen05.mma of M = 128 (96 rows used),
// N = 96, K = 48 (6 instructions of K = 8); of its output only the four diagonal 24 x 24 blocks
// are kept.  The geometric term delta_ik (G_a . c S G_b) is added in the epilogue.
//
// One CTA = one such group: each warp evaluates the 4 elements x 8 Gauss points and forms the
// operand rows of two of the eight nodes, the MMA runs, and all four warps read one accumulator
// row each.  At about 53 KB of shared memory and
// 128 TMEM columns four CTAs share an SM; 16 elements per CTA (one CTA per SM) was 1.65x slower.
#include <cuda_runtime.h>

#include "blocks.cuh"
#include "element.cuh"
#include "jetsci_internal.h"
#include "tc.cuh"

namespace jetsci {

constexpr int kTfElems = 4;            // elements per CTA
constexpr int kTfGroups = 1;           // MMA groups of 4 elements per CTA
constexpr uint32_t kTfTmemCols = 128;  // 96 accumulator columns per group, allocated as a power of 2
constexpr int kTfK = 48;               // 8 Gauss points x 6 Voigt components
// Operand tiles use padded core-matrix strides: 144 B between core matrices along K (16 B of
// padding) and 12 x 144 B between 8-row blocks.  With the fill pattern below (four elements x
// eight Gauss points per warp, one 4-byte store per lane) this leaves at most 2-way shared-
// memory bank conflicts instead of 16-way with the dense 128 B / 1536 B strides.
constexpr uint32_t kTfLBO = 144;
constexpr uint32_t kTfSBO = (kTfK / 4) * kTfLBO;
constexpr int kTfATile = 16 * kTfSBO;  // 128 rows (rows 96..127 zero)
constexpr int kTfBTile = 12 * kTfSBO;  // 96 rows

struct __align__(128) Tf32Smem {
    unsigned char A[kTfGroups][kTfATile];
    unsigned char B[kTfGroups][kTfBTile];
    float G[kTfElems][8][8][3];  // [elem][q][node][comp]
    float cS[kTfElems][8][6];
    float vnode[kTfElems][8][3];  // v at the element's nodes (matrix-free mode), FP32
    float geo[kTfElems][8][8];    // sum_q G_a . c S G_b (symmetric in a, b)
    int32_t node[kTfElems][8];
    int32_t elem[kTfElems];
    uint64_t mbar;
    uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t tf32_offset(int r, int k) {
    // K-major core matrices of 8 rows x 16 bytes (4 x 32-bit); 12 core matrices along K = 48
    return (uint32_t)((r >> 3) * kTfSBO + (k >> 2) * kTfLBO + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}


struct Tf32Args {
    const int32_t *__restrict__ conn;
    const double *__restrict__ coords;
    const int32_t *__restrict__ phase;
    const Material *__restrict__ mats;
    const double *__restrict__ E_elem;
    const int32_t *__restrict__ elems;
    int64_t n;
    uint32_t *flags;
};

// MODE 0: element pass of the row-gather assembly -- the element's 24 x 24 stiffness rows go to
// vals = the workspace [element][24][24] (elements in order, one launch) and, if R is given, its
// nodal forces to R = the workspace's residual part [element][local node][3];
// MODE 1: y += K_e v_e (matrix-free, one launch per colour).
template <int MODE>
__global__ void __launch_bounds__(128) k_tf32(Tf32Args A, const double *__restrict__ u, const double *__restrict__ v,
                                              float *__restrict__ vals, double *__restrict__ R, double *__restrict__ y) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Tf32Smem &sm = *reinterpret_cast<Tf32Smem *>(smem_raw);
    static_assert(kTfElems == 4 && kTfGroups == 1, "one MMA group of four elements per CTA");
    const int t = threadIdx.x;
    // Every warp covers all four elements (lane = element slot x Gauss point); warp w forms the
    // operand rows of nodes 2w and 2w+1, warp 0 also the residual and the per-element records.
    const int w = t >> 5, l = t & 7, es = (t >> 3) & 3;
    const int grp = 0, el = es;
    if (t < 32) tc::tmem_alloc(&sm.tmem_base, kTfTmemCols);
    if (t == 0) {
        tc::mbar_init(&sm.mbar, 1);
        tc::fence_mbar_init();
    }
    // zero the padding rows 96..127 of every A tile (4 row blocks)
    for (int i = t; i < kTfGroups * 32 * kTfK; i += 128) {
        const int g = i / (32 * kTfK), rem = i % (32 * kTfK);
        *reinterpret_cast<float *>(sm.A[g] + tf32_offset(96 + rem / kTfK, rem % kTfK)) = 0.0f;
    }
    // ---------------- phase 1: thread = (element, Gauss point) in every warp
    {
        const int64_t slot = (int64_t)blockIdx.x * kTfElems + es;
        const bool active = slot < A.n;
        const int64_t e = A.elems ? A.elems[active ? slot : A.n - 1] : (active ? slot : A.n - 1);
        int32_t node;
        GaussKinematics<float> K;
        float cu[3];
        gauss_kinematics<float>(A.conn, A.coords, u, e, l, node, K, cu);
        ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, false);
        float H[3][3];
        displacement_gradient(K, H);
        Constitutive<float> c;
        constitutive<float>(mt.law, (float)mt.lam, (float)mt.mu, H, c);
        const bool lin = mt.law == JETSCI_LINEAR_ELASTIC;
        if (MODE == 0 && R && w == 0) {
            float f[3];
            nodal_force(c.P, K, l, f);
            if (active)
#pragma unroll
                for (int i = 0; i < 3; i++) R[3 * (8 * e + hex_node_of_lane(l)) + i] = to_double(f[i]);
        }
        if (active && w == 0) {
            uint32_t bits = (K.dJ > 0.0f ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (c.ok ? 0u : JETSCI_FLAG_BAD_STATE);
            if (bits) atomicOr(A.flags, bits);
        }
        // Voigt tangent D (dS/dE w.r.t. tensor components) and the kinematic F of B
        float D[6][6];
        if (lin) {
#pragma unroll
            for (int a = 0; a < 6; a++)
#pragma unroll
                for (int b = 0; b < 6; b++)
                    D[a][b] = (a < 3 && b < 3 ? c.lam : 0.0f) + (a == b ? 2.0f * c.m : 0.0f);
        } else {
            float Ci[3][3];
#pragma unroll
            for (int I = 0; I < 3; I++)
#pragma unroll
                for (int Kk = 0; Kk < 3; Kk++)
                    Ci[I][Kk] = c.Fi[I][0] * c.Fi[Kk][0] + c.Fi[I][1] * c.Fi[Kk][1] + c.Fi[I][2] * c.Fi[Kk][2];
#pragma unroll
            for (int a = 0; a < 6; a++) {
                const int I = voigt_i(a), Jj = voigt_j(a);
#pragma unroll
                for (int b = 0; b < 6; b++) {
                    const int Kk = voigt_i(b), L = voigt_j(b);
                    float w = c.lam * Ci[I][Jj] * Ci[Kk][L] + c.m * (Ci[I][Kk] * Ci[Jj][L] + Ci[I][L] * Ci[Jj][Kk]);
                    D[a][b] = (Kk == L) ? w : 2.0f * w;
                }
            }
        }
        const float cw = K.dJ * (1.0f / 512.0f);
        const float rdJ = 1.0f / K.dJ;
        if (w == 0)
#pragma unroll
            for (int a = 0; a < 6; a++) sm.cS[es][l][a] = lin ? 0.0f : cw * c.S[voigt_i(a)][voigt_j(a)];
        // B_b and Z_b = c W D B_b for this warp's nodes b, written at k = 6q + alpha
        unsigned char *At = sm.A[grp];
        unsigned char *Bt = sm.B[grp];
#pragma unroll
        for (int bi = 0; bi < 2; bi++) {
            const int b = 2 * w + bi;
            const int nb = hex_node_of_lane(b);
            const float s0 = (nb & 1) ? 1.0f : -1.0f, s1 = (nb & 2) ? 1.0f : -1.0f, s2 = (nb & 4) ? 1.0f : -1.0f;
            const float fx = 1.0f + s0 * K.xi, fy = 1.0f + s1 * K.eta, fz = 1.0f + s2 * K.zeta;
            const float n0 = s0 * fy * fz, n1 = fx * s1 * fz, n2 = fx * fy * s2;
            float G[3];
#pragma unroll
            for (int j = 0; j < 3; j++) G[j] = (K.aJ[0][j] * n0 + K.aJ[1][j] * n1 + K.aJ[2][j] * n2) * rdJ;
#pragma unroll
            for (int j = 0; j < 3; j++) sm.G[es][l][b][j] = G[j];
            float Bb[6][3];
#pragma unroll
            for (int a = 0; a < 6; a++) {
                const int I = voigt_i(a), Jj = voigt_j(a);
#pragma unroll
                for (int i = 0; i < 3; i++) Bb[a][i] = 0.5f * (c.F[i][I] * G[Jj] + c.F[i][Jj] * G[I]);
            }
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const int row = 24 * el + 3 * b + i;
#pragma unroll
                for (int a = 0; a < 6; a++) {
                    float z = 0.0f;
#pragma unroll
                    for (int bb = 0; bb < 6; bb++) z += D[a][bb] * Bb[bb][i];
                    const float wgt = a < 3 ? cw : 2.0f * cw;
                    *reinterpret_cast<float *>(At + tf32_offset(row, 6 * l + a)) = to_tf32(Bb[a][i]);
                    *reinterpret_cast<float *>(Bt + tf32_offset(row, 6 * l + a)) = to_tf32(wgt * z);
                }
            }
        }
        if (w == 0) {
            sm.node[es][hex_node_of_lane(l)] = node;
            if (MODE == 1)
#pragma unroll
                for (int k = 0; k < 3; k++)
                    sm.vnode[es][hex_node_of_lane(l)][k] = from_double<float>(v[3 * (int64_t)node + k]);
            if (l == 0) sm.elem[es] = active ? (int32_t)e : -1;
        }
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = sm.tmem_base;
    if (t == 0) {
        const uint32_t id = tc::idesc_tf32(128, 96);
        for (int g = 0; g < kTfGroups; g++) {
            const uint32_t a0 = tc::smem_addr(sm.A[g]), b0 = tc::smem_addr(sm.B[g]);
            // one MMA of K = 8 covers two core matrices along K
            for (int kk = 0; kk < kTfK / 8; kk++)
                tc::mma_tf32(tm + 96 * g, tc::smem_desc(a0 + kk * 2 * kTfLBO, kTfLBO, kTfSBO),
                             tc::smem_desc(b0 + kk * 2 * kTfLBO, kTfLBO, kTfSBO), id, kk > 0 ? 1u : 0u);
        }
    }
    uint32_t ph = 0;
    if (t == 0) tc::mma_commit(&sm.mbar);
    // While the MMA runs: the geometric term of every element and node pair a <= b (row a of
    // the upper triangle starts at 8a - a(a-1)/2), once per pair instead of once per row.
    for (int it = t; it < kTfElems * 36; it += blockDim.x) {
        const int ee = it / 36, p = it - 36 * (it / 36);
        const int a = (p >= 8) + (p >= 15) + (p >= 21) + (p >= 26) + (p >= 30) + (p >= 33) + (p >= 35);
        const int b = p - (8 * a - (a * (a - 1)) / 2) + a;
        float g = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float *s6 = sm.cS[ee][q];
            const float *ga = sm.G[ee][q][a];
            const float *gb = sm.G[ee][q][b];
            const float sg0 = s6[0] * ga[0] + s6[5] * ga[1] + s6[4] * ga[2];
            const float sg1 = s6[5] * ga[0] + s6[1] * ga[1] + s6[3] * ga[2];
            const float sg2 = s6[4] * ga[0] + s6[3] * ga[1] + s6[2] * ga[2];
            g += sg0 * gb[0] + sg1 * gb[1] + sg2 * gb[2];
        }
        sm.geo[ee][a][b] = g;
        sm.geo[ee][b][a] = g;
    }
    const bool ok = tc::mbar_wait_bounded(&sm.mbar, ph & 1);
    tc::fence_after_sync();
    __syncthreads();  // geometric terms of all threads visible to the epilogue
    if (!ok && t == 0) atomicOr(A.flags, JETSCI_FLAG_NONFINITE);
    // ---------------- epilogue: thread t owns row t of each group's accumulator
    // tcgen05.ld is warp-collective with one column address per warp, and a warp's 32 rows
    // straddle at most two element slots: load each slot's 24 columns uniformly, keep own.
    const int warp = t >> 5;
    const int elr_lo = min((32 * warp) / 24, 3), elr_hi = min((32 * warp + 31) / 24, 3);
    for (int g = 0; g < kTfGroups; g++) {
        float rowv[24];
        const int elr = min(t / 24, 3);  // element slot of this row (rows >= 96 are padding)
#pragma unroll
        for (int pass = 0; pass < 2; pass++) {
            const int slot_e = pass == 0 ? elr_lo : elr_hi;
            if (pass == 1 && elr_hi == elr_lo) break;  // warp-uniform condition
            float v16[16], v8[8];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, 96 * g + 24 * slot_e), v16);
            tc::tmem_ld8(tc::tmem_lane_addr(tm, 96 * g + 24 * slot_e + 16), v8);
            if (elr == slot_e) {
#pragma unroll
                for (int j = 0; j < 16; j++) rowv[j] = v16[j];
#pragma unroll
                for (int j = 0; j < 8; j++) rowv[16 + j] = v8[j];
            }
        }
        if (t >= 96) continue;
        const int ee = 4 * g + elr;
        const int32_t eid = sm.elem[ee];
        if (eid < 0) continue;
        const int a = (t % 24) / 3, i = t % 3;
        // geometric term on the diagonal of each 3x3 block
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const float geo = sm.geo[ee][a][b];
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (k == i) rowv[3 * b + k] += geo;  // compile-time index, predicated
        }
        const int32_t na = sm.node[ee][a];
        if (MODE == 0) {
            // row 3a + i of K_e: 96 contiguous bytes; a warp writes 32 consecutive rows
            float4 *dst = reinterpret_cast<float4 *>(vals + 576 * (int64_t)eid + 24 * (3 * a + i));
#pragma unroll
            for (int c = 0; c < 6; c++)
                dst[c] = make_float4(rowv[4 * c], rowv[4 * c + 1], rowv[4 * c + 2], rowv[4 * c + 3]);
        } else {
            float s = 0.0f;
#pragma unroll
            for (int b = 0; b < 8; b++)
#pragma unroll
                for (int k = 0; k < 3; k++) s += rowv[3 * b + k] * sm.vnode[ee][b][k];
            y[3 * (int64_t)na + i] += to_double(s);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tm, kTfTmemCols);
}

jetsci_status launch_tf32(jetsci_mesh m, const double *u, const double *v, float *vals, double *R, double *y,
                          const double *E_elem, cudaStream_t s) {
    Tf32Args A;
    A.conn = m->d_conn;
    A.coords = m->d_coords;
    A.phase = m->d_phase;
    A.mats = m->d_mats;
    A.E_elem = E_elem;
    A.flags = m->d_flags;
    const size_t smem = sizeof(Tf32Smem);
    if (vals) {
        // row-gather assembly: element rows (one launch, elements in order), then the row pass
        void *ws = nullptr;
        double *Re = nullptr;
        if (jetsci_status st = ensure_block_workspace(m, blk_full_bytes(m->n_elem, sizeof(float)), s, &ws, &Re))
            return st;
        if (!R) Re = nullptr;
        if (m->n_elem > 0) {
            JETSCI_CUDA_TRY(cudaFuncSetAttribute(k_tf32<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            A.elems = nullptr;
            A.n = m->n_elem;
            const unsigned grid = (unsigned)((A.n + kTfElems - 1) / kTfElems);
            k_tf32<0><<<grid, 128, smem, s>>>(A, u, nullptr, (float *)ws, Re, nullptr);
            JETSCI_CUDA_TRY(cudaGetLastError());
        }
        return launch_gather_rows<float>(m, (const float *)ws, true, Re, vals, R, s);
    }
    JETSCI_CUDA_TRY(cudaFuncSetAttribute(k_tf32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    JETSCI_CUDA_TRY(cudaMemsetAsync(y, 0, m->n_dof * sizeof(double), s));
    for_each_colour(m, [&](const int32_t *elems, int64_t n) {
        A.elems = elems;
        A.n = n;
        unsigned grid = (unsigned)((A.n + kTfElems - 1) / kTfElems);
        k_tf32<1><<<grid, 128, smem, s>>>(A, u, v, nullptr, nullptr, y);
    });
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

}  // namespace jetsci
