// Element stiffness on the tensor cores in TF32 (FP32 accumulate in TMEM): the element rows of
// the row-gather tangent assembly.
//
// The tangent in pair form, as the CUDA-core kernels use it:
//   K_ab,ik = sum_q [ c lam g_ai g_bk + c m g_ak g_bi ] + delta_ik mu L_ab
// with g_a = F^-T G_a the spatial shape-function gradients at Gauss point q, c = w detJ,
// m = mu - lam lnJ (mu for Hooke) and L_ab = sum_q detJ G_a . G_b the element's reference
// Laplacian (the geometric term sum_q c g_a^T (tau + m I) g_b equals mu L_ab for both laws; the
// mesh caches L_ab, element.cuh kLap*).  The two rank-8 parts are contractions over the Gauss
// points: with P[(a,i), q] = g_ai,
//   T1 = P diag(c lam) P^T,   T2 = P diag(c m) P^T,   K_ab,ik = T1[(a,i),(b,k)] + T2[(a,k),(b,i)] + ...
// Four elements share one tcgen05.mma (kind::tf32, M = 128, N = 48, K = 32, as four MMAs of
// K = 8): A holds P of the four elements block-diagonally (row (e,a,i), column (e,q), zero
// outside the element's eight columns) and B the columns c lam g_b | c m g_b (row (term,b,k),
// column (e,q)).  Accumulator row (e,a,i) so receives T1 and T2 of its own element only, in 48
// TMEM columns.  The epilogue adds mu L_ab on the diagonal of each 3 x 3 block.
//
// Persistent CTAs (two per SM, as TMEM allows: 256 columns each) loop over batches of 16
// elements = four groups of four; warp w evaluates group w (lane = element x Gauss point) and
// writes its operand columns, one thread issues the 16 MMAs, then every warp reads its TMEM lane
// quarter of each group's accumulator and T2 is transposed within node blocks through shared
// memory.  Per CTA the zeros of the block-diagonal A tiles are written once (a lane only ever
// writes its own element's rows), and the gathers of the next batch are issued before the
// current batch's arithmetic: the connectivity two batches ahead, the coordinates and
// displacements one batch ahead.
#include <cuda_runtime.h>

#include <algorithm>

#include "blocks.cuh"
#include "element.cuh"
#include "jetsci_internal.h"
#include "tc.cuh"

namespace jetsci {

constexpr int kTgGroups = 4;                   // MMA groups per CTA (one per warp)
constexpr int kTgElems = 4 * kTgGroups;        // elements per CTA
constexpr int kTgK = 32;                       // 4 elements x 8 Gauss points
constexpr int kTgN = 48;                       // 2 terms x 8 nodes x 3 components
constexpr uint32_t kTgCols = 64;               // TMEM columns per group (48 used)
constexpr uint32_t kTgTmemCols = kTgGroups * kTgCols;
// K-major core matrices (8 rows x 16 bytes) with 144 B between core matrices along K (16 B of
// padding): a warp's 32 lanes (8 element columns x 4 per core matrix) write one row of a tile
// on 32 distinct banks.
constexpr uint32_t kTgLBO = 144;
constexpr uint32_t kTgSBO = (kTgK / 4) * kTgLBO;  // 8-row blocks
constexpr int kTgATile = 12 * kTgSBO;             // rows 0..95 (M = 128: see below)
constexpr int kTgBTile = 6 * kTgSBO;              // 48 rows
constexpr int kTgT2Stride = 25;                   // floats per row of the T2 transposition buffer

// The MMA reads 128 rows of A; rows 96..127 (row blocks 12..15) fall on the next tile or on the
// B tiles and produce accumulator rows that are never read, so they need neither zeros nor room.
constexpr int kTgT2Groups = 2;  // groups whose T2 rows the transposition buffer holds at once
struct __align__(128) TgSmem {
    unsigned char A[kTgGroups][kTgATile];
    unsigned char B[kTgGroups][kTgBTile];
    float t2[kTgT2Groups][96 * kTgT2Stride];  // T2 rows of two groups, [row][kTgT2Stride]
    float geo[kTgElems][kLapPairs];           // mu L_ab of each element (kLap* order)
    int32_t elem[kTgElems];
    uint64_t mbar;
    uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t tg_offset(int r, int k) {
    return (uint32_t)((r >> 3) * kTgSBO + (k >> 2) * kTgLBO + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// index of node pair (a, b) in an element's L_ab (element.cuh, kLap*): the pairs a < b row by
// row, then the diagonal
__device__ __forceinline__ int tg_lap(int a, int b) {
    if (a == b) return kLapDiag + a;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return 7 * lo - (lo * (lo - 1)) / 2 + (hi - lo - 1);
}

struct Tf32Args {
    const int32_t *__restrict__ conn;
    const double *__restrict__ coords;
    const int32_t *__restrict__ phase;
    const Material *__restrict__ mats;
    const double *__restrict__ E_elem;
    const double *__restrict__ lap;  // per-element L_ab (kLap* order)
    int64_t n;         // elements 0 .. n - 1
    uint32_t *flags;
};

// What a lane gathers for one batch: its element, its node, the node's coordinates and
// displacement, the element's phase and modulus.
struct Tf32Gather {
    int64_t e;
    int32_t node, ph;
    double E;
    double X[3], U[3];
};

// element of the lane in batch b (the last element for the slots past the end), and whether
// the slot is one
__device__ __forceinline__ int64_t tf32_elem(const Tf32Args &A, int64_t b, int es, bool &active) {
    const int64_t slot = b * kTgElems + es;
    active = slot < A.n;
    return active ? slot : A.n - 1;
}

__device__ __forceinline__ void tf32_gather_conn(const Tf32Args &A, int64_t b, int es, int l, Tf32Gather &g) {
    bool active;
    g.e = tf32_elem(A, b, es, active);
    g.node = __ldg(A.conn + 8 * g.e + hex_node_of_lane(l));
    g.ph = __ldg(A.phase + g.e);
    g.E = A.E_elem ? __ldg(A.E_elem + g.e) : 0.0;
}

__device__ __forceinline__ void tf32_gather_values(const Tf32Args &A, const double *__restrict__ u, Tf32Gather &g) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
        g.X[i] = __ldg(A.coords + 3 * (int64_t)g.node + i);
        g.U[i] = u ? __ldg(u + 3 * (int64_t)g.node + i) : 0.0;
    }
}

// Element pass of the row-gather assembly: the element's 24 x 24 stiffness rows go to vals = the
// workspace [element][24][24] and, if R is given, its nodal forces to R = the workspace's residual
// part [element][local node][3].
__global__ void __launch_bounds__(128) k_tf32(Tf32Args A, const double *__restrict__ u, float *__restrict__ vals,
                                              double *__restrict__ R) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TgSmem &sm = *reinterpret_cast<TgSmem *>(smem_raw);
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int el = lane >> 3, l = lane & 7;  // element in the group, Gauss point
    const int es = t >> 3;                   // element slot in the batch (= 4 w + el)
    if (w == 0) tc::tmem_alloc(&sm.tmem_base, kTgTmemCols);
    if (t == 0) {
        tc::mbar_init(&sm.mbar, 1);
        tc::fence_mbar_init();
    }
    // zeros of the A tiles, once: every lane later writes only its own element's rows in its
    // column, so the other elements' rows there stay zero
    {
        uint4 *z = reinterpret_cast<uint4 *>(&sm.A[0][0]);
        for (int i = t; i < (int)(sizeof(sm.A) / 16); i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = sm.tmem_base;
    const int64_t n_batches = (A.n + kTgElems - 1) / kTgElems;
    const int64_t G = gridDim.x;
    int64_t b = blockIdx.x;
    Tf32Gather cur, nxt;
    if (b < n_batches) {
        tf32_gather_conn(A, b, es, l, cur);
        tf32_gather_values(A, u, cur);
    }
    if (b + G < n_batches) tf32_gather_conn(A, b + G, es, l, nxt);
    uint32_t it = 0;
    for (; b < n_batches; b += G, it++) {
        // ---------------- phase 1: thread = (element, Gauss point)
        bool active;
        (void)tf32_elem(A, b, es, active);
        const int64_t e = cur.e;
        {
            GaussKinematics<float> K;
            float cu[3];
            gauss_kinematics_of<float>(cur.X, cur.U, l, K, cu);
            const Material &mat = A.mats[cur.ph];
            const float lam = A.E_elem ? (float)(cur.E * mat.lam1) : (float)mat.lam;
            const float mu = A.E_elem ? (float)(cur.E * mat.mu1) : (float)mat.mu;
            // W with g_a = W^T (8 dN_a/dxi), m, and the residual moment Q
            float W[3][3], Q[3][3], m;
            bool ok = true;
            if (mat.law == JETSCI_LINEAR_ELASTIC) {
                const float rdJ = 1.0f / K.dJ;
#pragma unroll
                for (int d = 0; d < 3; d++)
#pragma unroll
                    for (int j = 0; j < 3; j++) W[d][j] = K.aJ[d][j] * rdJ;
                float H[3][3], sg[3][3];
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++) H[i][j] = K.Du[i][0] * W[0][j] + K.Du[i][1] * W[1][j] + K.Du[i][2] * W[2][j];
                const float ltr = lam * (H[0][0] + H[1][1] + H[2][2]);
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++) sg[i][j] = mu * (H[i][j] + H[j][i]) + ((i == j) ? ltr : 0.0f);
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        Q[i][d] = sg[i][0] * K.aJ[d][0] + sg[i][1] * K.aJ[d][1] + sg[i][2] * K.aJ[d][2];
                m = mu;
            } else {
                NeoHookeanState<float> st;
                neo_hookean_state(K, lam, mu, st);
                ok = st.ok;
                m = st.m;
                const float sc = K.dJ * st.rdj;
#pragma unroll
                for (int d = 0; d < 3; d++)
#pragma unroll
                    for (int j = 0; j < 3; j++) W[d][j] = st.aj[d][j] * st.rdj;
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int d = 0; d < 3; d++)
                        Q[i][d] = sc * (st.tau[i][0] * st.aj[d][0] + st.tau[i][1] * st.aj[d][1] + st.tau[i][2] * st.aj[d][2]);
            }
            if (active) {
                const uint32_t bits = (K.dJ > 0.0f ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (ok ? 0u : JETSCI_FLAG_BAD_STATE);
                if (bits) atomicOr(A.flags, bits);
            }
            const float cw = K.dJ * (1.0f / 512.0f);
            const float cl = cw * lam, cm = cw * m;
            const float xp = 1.0f + K.xi, xm = 1.0f - K.xi, yp = 1.0f + K.eta, ym = 1.0f - K.eta;
            const float zp = 1.0f + K.zeta, zm = 1.0f - K.zeta;
            unsigned char *At = sm.A[w];
            unsigned char *Bt = sm.B[w];
            const int kc = 8 * el + l;  // this lane's column of A and B
#pragma unroll
            for (int a = 0; a < 8; a++) {
                const int bits = hex_bits_of_node(a);
                const float fx = (bits & 1) ? xp : xm, fy = (bits & 2) ? yp : ym, fz = (bits & 4) ? zp : zm;
                const float yz = fy * fz, xz = fx * fz, xy = fx * fy;
                const float n0 = (bits & 1) ? yz : -yz, n1 = (bits & 2) ? xz : -xz, n2 = (bits & 4) ? xy : -xy;
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const float g = W[0][i] * n0 + W[1][i] * n1 + W[2][i] * n2;
                    // A: the element's own row block (the other elements' rows of this column
                    // hold the zeros written at the start)
                    *reinterpret_cast<float *>(At + tg_offset(24 * el + 3 * a + i, kc)) = to_tf32(g);
                    *reinterpret_cast<float *>(Bt + tg_offset(3 * a + i, kc)) = to_tf32(cl * g);
                    *reinterpret_cast<float *>(Bt + tg_offset(24 + 3 * a + i, kc)) = to_tf32(cm * g);
                }
            }
            // geometric term: mu L_ab of the element, lane l holding pairs l, l + 8, ...
            {
                const double *le = A.lap + (int64_t)kLapPairs * e;
#pragma unroll
                for (int j = l; j < kLapPairs; j += 8) sm.geo[es][j] = mu * (float)__ldg(le + j);
            }
            // residual: nodal forces of the lane's node
            float f[3];
            nodal_force_of_moment(Q, K, l, f);
            if (R && active)
#pragma unroll
                for (int i = 0; i < 3; i++) R[3 * (8 * e + hex_node_of_lane(l)) + i] = to_double(f[i]);
            if (l == 0) sm.elem[es] = active ? (int32_t)e : -1;
        }
        // the next batch's coordinates and displacements (its connectivity has arrived)
        if (b + G < n_batches) tf32_gather_values(A, u, nxt);
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
            const uint32_t id = tc::idesc_tf32(128, kTgN);
            for (int g = 0; g < kTgGroups; g++) {
                const uint32_t a0 = tc::smem_addr(sm.A[g]), b0 = tc::smem_addr(sm.B[g]);
                // one MMA of K = 8 covers two core matrices along K
                for (int kk = 0; kk < kTgK / 8; kk++)
                    tc::mma_tf32(tm + kTgCols * g, tc::smem_desc(a0 + kk * 2 * kTgLBO, kTgLBO, kTgSBO),
                                 tc::smem_desc(b0 + kk * 2 * kTgLBO, kTgLBO, kTgSBO), id, kk > 0 ? 1u : 0u);
            }
            tc::mma_commit(&sm.mbar);
        }
        const bool ok = tc::mbar_wait_bounded(&sm.mbar, it & 1);
        tc::fence_after_sync();
        if (!ok && t == 0) atomicOr(A.flags, JETSCI_FLAG_NONFINITE);
        // ---------------- epilogue: thread t owns accumulator row r = t of each group (TMEM lane
        // t); rows 96..127 (warp 3) carry nothing.  Two groups at a time: their T2 rows into the
        // transposition buffer, then each row
        //   K[(a,i),(b,k)] = T1[(a,i),(b,k)] + T2[(b,i),(a,k)] + delta_ik geo(a,b)
        // (T2 is symmetric: its entry ((a,k),(b,i)) is row (b,i), column (a,k)).
        const int r = t, rel = r / 24, ra = (r % 24) / 3, ri = r % 3;
        for (int g0 = 0; g0 < kTgGroups; g0 += kTgT2Groups) {
            if (w < 3) {
#pragma unroll
                for (int gg = 0; gg < kTgT2Groups; gg++) {
                    float v16[16], v8[8];
                    tc::tmem_ld16(tc::tmem_lane_addr(tm, kTgCols * (g0 + gg) + 24), v16);
                    tc::tmem_ld8(tc::tmem_lane_addr(tm, kTgCols * (g0 + gg) + 40), v8);
                    float *dst = sm.t2[gg] + r * kTgT2Stride;
#pragma unroll
                    for (int c = 0; c < 16; c++) dst[c] = v16[c];
#pragma unroll
                    for (int c = 0; c < 8; c++) dst[16 + c] = v8[c];
                }
            }
            __syncthreads();
            if (w < 3) {
#pragma unroll 1
                for (int gg = 0; gg < kTgT2Groups; gg++) {
                    const int g = g0 + gg;
                    float rowv[24];
                    {
                        float v16[16], v8[8];
                        tc::tmem_ld16(tc::tmem_lane_addr(tm, kTgCols * g), v16);
                        tc::tmem_ld8(tc::tmem_lane_addr(tm, kTgCols * g + 16), v8);
#pragma unroll
                        for (int c = 0; c < 16; c++) rowv[c] = v16[c];
#pragma unroll
                        for (int c = 0; c < 8; c++) rowv[16 + c] = v8[c];
                    }
                    const int ee = 4 * g + rel;
                    const int32_t eid = sm.elem[ee];
                    if (eid < 0) continue;
                    const float *t2e = sm.t2[gg] + 24 * rel * kTgT2Stride;
#pragma unroll
                    for (int bb = 0; bb < 8; bb++) {
                        const float geo = sm.geo[ee][tg_lap(ra, bb)];
#pragma unroll
                        for (int k = 0; k < 3; k++)
                            rowv[3 * bb + k] += t2e[(3 * bb + ri) * kTgT2Stride + 3 * ra + k] + (k == ri ? geo : 0.0f);
                    }
                    // row 3a + i of K_e: 96 contiguous bytes
                    float4 *dst = reinterpret_cast<float4 *>(vals + 576 * (int64_t)eid + 24 * (3 * ra + ri));
#pragma unroll
                    for (int c = 0; c < 6; c++)
                        dst[c] = make_float4(rowv[4 * c], rowv[4 * c + 1], rowv[4 * c + 2], rowv[4 * c + 3]);
                }
            }
            tc::fence_before_sync();
            __syncthreads();  // the buffer, geo and elem are reused; the next MMA overwrites TMEM
            tc::fence_after_sync();
        }
        cur = nxt;
        if (b + 2 * G < n_batches) tf32_gather_conn(A, b + 2 * G, es, l, nxt);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tm, kTgTmemCols);
}

jetsci_status launch_tf32(jetsci_mesh m, const double *u, float *vals, double *R, const double *E_elem,
                          cudaStream_t s) {
    Tf32Args A;
    A.conn = m->d_conn;
    A.coords = m->d_coords;
    A.phase = m->d_phase;
    A.mats = m->d_mats;
    A.E_elem = E_elem;
    A.lap = m->d_lap;
    A.flags = m->d_flags;
    const size_t smem = sizeof(TgSmem);
    // row-gather assembly: element rows (one persistent launch, elements in order), then the row pass
    void *ws = nullptr;
    double *Re = nullptr;
    if (jetsci_status st = ensure_block_workspace(m, blk_full_bytes(m->n_elem, sizeof(float)), s, &ws, &Re))
        return st;
    if (!R) Re = nullptr;
    if (m->n_elem > 0) {
        if (jetsci_status st = kernel_attrs_once<k_tf32>(smem, false)) return st;
        int sms = 0;
        JETSCI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
        A.n = m->n_elem;
        const int64_t n_batches = (A.n + kTgElems - 1) / kTgElems;
        // two CTAs per SM: 256 TMEM columns and about 104 KB of shared memory each
        const unsigned grid = (unsigned)std::min<int64_t>(n_batches, 2 * (int64_t)std::max(sms, 1));
        k_tf32<<<grid, 128, smem, s>>>(A, u, (float *)ws, Re);
        JETSCI_CUDA_TRY(cudaGetLastError());
    }
    return launch_gather_rows<float>(m, (const float *)ws, Re, vals, R, s);
}

}  // namespace jetsci
