// Element stiffness on the tensor cores in TF32 (FP32 accumulate in TMEM): the element rows of
// the row-gather tangent assembly.
//
// The tangent in pair form, as the CUDA-core kernels use it:
//   K_ab,ik = sum_q [ c lam g_ai g_bk + c m g_ak g_bi ] + delta_ik mu L_ab
// with g_a = F^-T G_a the spatial shape-function gradients at Gauss point q, c = w detJ,
// m = mu - lam lnJ (mu for Hooke) and L_ab = sum_q detJ G_a . G_b the element's reference
// Laplacian (the geometric term sum_q c g_a^T (tau + m I) g_b equals mu L_ab for both laws; the
// mesh caches L_ab, element.cuh kLap*).  With g_a = W^T n_a, where n_a = 8 dN_a/dxi at the point
// is the same for every element (W = j^-1, j = 8 dx/dxi), the two material terms become
//   K_ab,ik = sum_{q,r,s} n_ar n_bs V_q[(r,s),(i,k)],   V_q[(r,s),(i,k)] = c lam W_ri W_sk + c m W_rk W_si:
// one product of a constant matrix N[(a,b),(r,s,q)] = n_ar n_bs (64 node pairs x 72) with the
// elements' V (nine rows (i,k) per element, 72 columns (r,s,q)).  Twenty-four elements share one
// tcgen05.mma chain (kind::tf32, M = 128 of which the 64 pair rows are used, N = 224 of which 216
// are used, K = 72): accumulator row (a,b), column 8 (3 (3i + k) + o) + j holds K_ab,ik of element
// 8 o + j (o = octet) without the geometric term, so
// the epilogue needs no transposition and adds mu L_ab on the diagonal of each 3 x 3 block.  N is
// split into two TF32 parts (hi + lo, two MMAs per K step), which leaves the rounding of V as the
// only TF32 rounding (N itself is formed in FP32); every V entry is dense (no block-diagonal
// zeros).
//
// Persistent CTAs (six warps, two CTAs per SM: 256 TMEM columns and about 105 KB of shared
// memory each) loop over batches of 24 elements: thread = element x Gauss point writes its
// point's 81 V entries, one thread issues the 18 MMAs, then the four warps that see TMEM lanes
// 0-63 (warps 0, 1, 4 and 5; each reads the lanes of its quarter) read the accumulator rows of
// the 64 node pairs, one octet of elements per 8-column load, into the element matrices, laid
// out in shared memory over the V tile; one bulk asynchronous copy writes them out while the
// next batch's kinematics run (phase 1 waits for its reads before storing V).  The
// gathers of the next batch are issued before the current batch's arithmetic: the connectivity
// two batches ahead, the coordinates and displacements one batch ahead.
#include <cuda_runtime.h>

#include <algorithm>

#include "blocks.cuh"
#include "element.cuh"
#include "jetsci_internal.h"
#include "tc.cuh"

namespace jetsci {

constexpr int kTnE = 24;                           // elements per batch (three octets)
constexpr int kTnThreads = 8 * kTnE;               // thread = element x Gauss point in phase 1
constexpr int kTnK = 72;                           // columns (r, s, q): 8 (3 r + s) + q
constexpr int kTnCols = 9 * kTnE;                  // accumulator columns 8 (3 (3 i + k) + octet) + element
constexpr int kTnN = (kTnCols + 15) / 16 * 16;     // the MMA's N (a multiple of 16; the last rows unused)
constexpr uint32_t kTnTmemCols = 256;
// K-major core matrices (8 rows x 16 bytes), no padding: LBO = step along K, SBO = 8-row step
constexpr uint32_t kTnLBO = 128;
constexpr uint32_t kTnSBO = (kTnK / 4) * kTnLBO;
constexpr int kTnATile = 8 * kTnSBO;               // the 64 pair rows of N
constexpr int kTnBTile = (kTnN / 8) * kTnSBO;      // 224 rows of V (216 used)

// The MMA reads 128 rows of A; rows 64..127 fall on the next bytes of shared memory (the lo part,
// then the V tile) and produce accumulator rows that are never read.
struct __align__(128) TnSmem {
    unsigned char A[2][kTnATile];       // N, hi and lo TF32 parts
    unsigned char B[kTnBTile];          // V of the batch's 24 elements
    float geo[kTnE][kLapPairs];         // mu L_ab of each element (kLap* order)
    int32_t elem[kTnE];
    uint64_t mbar;
    uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t tn_offset(int r, int k) {
    return (uint32_t)((r >> 3) * kTnSBO + (k >> 2) * kTnLBO + (r & 7) * 16 + (k & 3) * 4);
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

// n_a,r = 8 dN_a/dxi_r at Gauss point q (lane bits of q: xi, eta, zeta signs), in FP32: each
// factor 1 +- g where the node's and the point's signs agree or differ
__device__ __forceinline__ float tn_nref(int q, int a, int r) {
    const int bits = hex_bits_of_node(a);
    const float f[3] = {((bits ^ q) & 1) ? (float)kGaussM : (float)kGaussP,
                        ((bits ^ q) & 2) ? (float)kGaussM : (float)kGaussP,
                        ((bits ^ q) & 4) ? (float)kGaussM : (float)kGaussP};
    const float sgn = (bits >> r) & 1 ? 1.0f : -1.0f;
    return sgn * f[(r + 1) % 3] * f[(r + 2) % 3];
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
    const int64_t slot = b * kTnE + es;
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
__global__ void __launch_bounds__(kTnThreads, 2) k_tf32(Tf32Args A, const double *__restrict__ u, float *__restrict__ vals,
                                              double *__restrict__ R) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TnSmem &sm = *reinterpret_cast<TnSmem *>(smem_raw);
    const int t = threadIdx.x, w = t >> 5;
    const int l = t & 7;   // Gauss point
    const int es = t >> 3; // element slot in the batch
    if (w == 0) tc::tmem_alloc(&sm.tmem_base, kTnTmemCols);
    if (t == 0) {
        tc::mbar_init(&sm.mbar, 1);
        tc::fence_mbar_init();
    }
    // the constant operand N[(a,b), 8 (3 r + s) + q] = n_ar n_bs at point q, as hi + lo TF32 parts
    for (int idx = t; idx < 64 * kTnK; idx += kTnThreads) {
        const int row = idx / kTnK, col = idx - kTnK * row;
        const int a = row >> 3, b = row & 7, rs = col >> 3, q = col & 7;
        const float x = tn_nref(q, a, rs / 3) * tn_nref(q, b, rs % 3);
        const float hi = to_tf32(x);
        const float lo = to_tf32(x - hi);  // (exact: x - hi has at most 13 significant bits)
        *reinterpret_cast<float *>(sm.A[0] + tn_offset(row, col)) = hi;
        *reinterpret_cast<float *>(sm.A[1] + tn_offset(row, col)) = lo;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = sm.tmem_base;
    const int64_t n_batches = (A.n + kTnE - 1) / kTnE;
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
            // V_q[(r,s),(i,k)] = c lam W_ri W_sk + c m W_rk W_si at row 8 (3 (3 i + k) + octet) + j,
            // column 8 (3 r + s) + q; the entry of ((s,r),(k,i)) is the same
            float Lw[3][3], Mw[3][3];
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int i = 0; i < 3; i++) Lw[r][i] = cl * W[r][i], Mw[r][i] = cm * W[r][i];
            // the previous batch's rows have left the V tile (their bulk copy read it)
            if (t == 0) tc::bulk_wait_read();
            __syncthreads();
            unsigned char *Bt = sm.B;
            // V row (= accumulator column) of component c of this element
            auto vrow = [&](int c) { return 8 * (3 * c + (es >> 3)) + (es & 7); };
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int s2 = 0; s2 < 3; s2++)
#pragma unroll
                    for (int i = 0; i < 3; i++)
#pragma unroll
                        for (int k = 0; k < 3; k++) {
                            const int self = 9 * (3 * r + s2) + 3 * i + k, mirror = 9 * (3 * s2 + r) + 3 * k + i;
                            if (self > mirror) continue;
                            const float v = to_tf32(fmaf(Lw[r][i], W[s2][k], Mw[r][k] * W[s2][i]));
                            *reinterpret_cast<float *>(Bt + tn_offset(vrow(3 * i + k), 8 * (3 * r + s2) + l)) = v;
                            if (mirror != self)
                                *reinterpret_cast<float *>(Bt + tn_offset(vrow(3 * k + i), 8 * (3 * s2 + r) + l)) = v;
                        }
            // geometric term: mu L_ab of the element, lane l holding pairs l, l + 8, ...
            {
                const double *le = A.lap + (int64_t)kLapPairs * e;
#pragma unroll
                for (int j = l; j < kLapPairs; j += 8) sm.geo[es][j] = mu * (float)__ldg(le + j);  // (a cast: the FP64 pipe is idle here; the integer conversion measured 6% slower)
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
            const uint32_t id = tc::idesc_tf32(128, kTnN);
            const uint32_t b0 = tc::smem_addr(sm.B);
            // one MMA of K = 8 covers two core matrices along K; N's hi and lo parts in turn
            for (int kk = 0; kk < kTnK / 8; kk++)
                for (int part = 0; part < 2; part++)
                    tc::mma_tf32(tm, tc::smem_desc(tc::smem_addr(sm.A[part]) + kk * 2 * kTnLBO, kTnLBO, kTnSBO),
                                 tc::smem_desc(b0 + kk * 2 * kTnLBO, kTnLBO, kTnSBO), id, (kk | part) ? 1u : 0u);
            tc::mma_commit(&sm.mbar);
        }
        const bool ok = tc::mbar_wait_bounded(&sm.mbar, it & 1);
        tc::fence_after_sync();
        if (!ok && t == 0) atomicOr(A.flags, JETSCI_FLAG_NONFINITE);
        // ---------------- epilogue: thread t < 64 owns accumulator row t = node pair (a, b); the
        // batch's element matrices are laid out in [element][24][24] order over the V tile (free
        // once the MMAs completed: conflict-free stores), then every thread copies them out, one
        // contiguous span of 16-byte stores
        float *stage = reinterpret_cast<float *>(sm.B);
        if ((w & 3) < 2) {  // warps 0, 1: components 0-4; warps 4, 5: components 5-8
            const int pr = 32 * (w & 1) + (t & 31), pa = pr >> 3, pb = pr & 7, li = tg_lap(pa, pb);
            float *dst = stage + 24 * (3 * pa) + 3 * pb;
            const int c0 = w < 4 ? 0 : 5, c1 = w < 4 ? 5 : 9;
#pragma unroll 1
            for (int c = c0; c < c1; c++) {
                const int i = c / 3, k = c - 3 * i;
#pragma unroll 1
                for (int o = 0; o < kTnE / 8; o++) {
                    float v[8];
                    tc::tmem_ld8(tc::tmem_lane_addr(tm, 8 * (3 * c + o)), v);
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const int el = 8 * o + j;
                        dst[576 * el + 24 * i + k] = (i == k) ? v[j] + sm.geo[el][li] : v[j];
                    }
                }
            }
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();  // the element matrices are laid out; the next MMA may overwrite TMEM
        tc::fence_after_sync();
        if (t == 0) {  // one bulk copy of the batch's contiguous rows; it drains during the next phase 1
            const int64_t e0 = b * kTnE;
            const int n_el = (int)(A.n - e0 < kTnE ? A.n - e0 : kTnE);
            tc::bulk_store(vals + 576 * e0, stage, (uint32_t)n_el * 576u * (uint32_t)sizeof(float));
            tc::bulk_commit();
        }
        cur = nxt;
        if (b + 2 * G < n_batches) tf32_gather_conn(A, b + 2 * G, es, l, nxt);
    }
    if (t == 0) tc::bulk_wait();  // the last batch's rows are written before the CTA exits
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tm, kTnTmemCols);
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
    const size_t smem = sizeof(TnSmem);
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
        const int64_t n_batches = (A.n + kTnE - 1) / kTnE;
        // two CTAs per SM: 256 TMEM columns and about 105 KB of shared memory each
        const unsigned grid = (unsigned)std::min<int64_t>(n_batches, 2 * (int64_t)std::max(sms, 1));
        k_tf32<<<grid, kTnThreads, smem, s>>>(A, u, (float *)ws, Re);
        JETSCI_CUDA_TRY(cudaGetLastError());
    }
    return launch_gather_rows<float>(m, (const float *)ws, Re, vals, R, s);
}

}  // namespace jetsci
