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
// elements' V (72 columns (r,s,q)).  Since K_ba,ki = K_ab,ik, only the six components i <= k are
// formed: six rows of V per element, and the epilogue takes K_ab,ik for i > k from the row of
// pair (b,a).  Forty elements share one tcgen05.mma chain (kind::tf32, M = 128 of which the 64
// pair rows are used, N = 240, K = 72): accumulator row (a,b), column 8 (5 c + o) + j holds
// component c of K_ab of element 8 o + j (o = octet) without the geometric term, which the
// epilogue adds (mu L_ab) on the diagonal of each 3 x 3 block.  N is split into two TF32 parts
// (hi + lo, two MMAs per K step), which leaves the rounding of V as the only TF32 rounding (N
// itself is formed in FP32); every V entry is dense (no block-diagonal zeros).
//
// Persistent CTAs (ten warps, two CTAs per SM: 256 TMEM columns and about 110 KB of shared
// memory each) loop over batches of 40 elements: thread = element x Gauss point writes its
// point's 54 V entries, one thread issues the 18 MMAs, then the six warps that see TMEM lanes
// 0-63 (warps 0, 1, 4, 5, 8 and 9; each reads the lanes of its quarter, two components each)
// read the accumulator rows of the 64 node pairs, one octet of elements per 8-column load, into
// the element matrices, laid out in shared memory over the V tile three octets at a time; one
// bulk asynchronous copy per chunk writes them out, the last one while the next batch's
// kinematics run (V stores wait for its reads).  The gathers of the next batch are issued
// before the current batch's arithmetic: the connectivity two batches ahead, the coordinates
// and displacements one batch ahead.
#include <cuda_runtime.h>

#include <algorithm>

#include "blocks.cuh"
#include "element.cuh"
#include "jetsci_internal.h"
#include "tc.cuh"

namespace jetsci {

constexpr int kTnE = 40;                           // elements per batch (five octets)
constexpr int kTnOct = kTnE / 8;
constexpr int kTnThreads = 8 * kTnE;               // thread = element x Gauss point in phase 1
constexpr int kTnK = 72;                           // columns (r, s, q): 8 (3 r + s) + q
constexpr int kTnComp = 6;                         // components (i, k), i <= k
constexpr int kTnN = kTnComp * kTnE;               // accumulator columns 8 (5 c + octet) + element (240)
constexpr uint32_t kTnTmemCols = 256;
// K-major core matrices (8 rows x 16 bytes), no padding: LBO = step along K, SBO = 8-row step
constexpr uint32_t kTnLBO = 128;
constexpr uint32_t kTnSBO = (kTnK / 4) * kTnLBO;
constexpr int kTnATile = 8 * kTnSBO;               // the 64 pair rows of N
constexpr int kTnBTile = (kTnN / 8) * kTnSBO;      // 240 rows of V
static_assert(kTnN % 16 == 0 && kTnN <= (int)kTnTmemCols, "MMA N");
static_assert(kTnThreads == 320, "the epilogue gives two components to each of the six warps on TMEM lanes 0-63");
// octets of element rows staged over the V tile at a time (each written by one bulk copy)
constexpr int kTnStageOct = kTnBTile / (8 * 576 * 4);
static_assert(kTnStageOct >= 1, "an octet of element rows fits over the V tile");

// Component c of the accumulator: (i, k) = (0,0) (1,1) (2,2) (0,1) (0,2) (1,2)
__host__ __device__ constexpr int tn_comp_i(int c) { return c < 3 ? c : (c < 5 ? 0 : 1); }
__host__ __device__ constexpr int tn_comp_k(int c) { return c < 3 ? c : (c == 3 ? 1 : 2); }

// The MMA reads 128 rows of A; rows 64..127 fall on the next bytes of shared memory (the lo part,
// then the V tile) and produce accumulator rows that are never read.
struct __align__(128) TnSmem {
    unsigned char A[2][kTnATile];       // N, hi and lo TF32 parts
    unsigned char B[kTnBTile];          // V of the batch's elements; then up to three octets of their rows
    float geo[kTnE][kLapPairs];         // mu L_ab of each element (kLap* order)
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
            // V_q[(r,s),(i,k)] = c lam W_ri W_sk + c m W_rk W_si for the components i <= k, at row
            // 8 (5 c + octet) + j, column 8 (3 r + s) + q.  The diagonal components are
            // (c lam + c m) W_ri W_si, the same for (r,s) and (s,r).
            float Lw[3][3], Mw[3][3];
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int i = 0; i < 3; i++) Lw[r][i] = cl * W[r][i], Mw[r][i] = cm * W[r][i];
            const float cs = cl + cm;
            // the previous batch's rows have left the V tile (their bulk copy read it)
            if (t == 0) tc::bulk_wait_read();
            __syncthreads();
            unsigned char *Bt = sm.B;
            // V row (= accumulator column) of component c of this element
            auto vrow = [&](int c) { return 8 * (kTnOct * c + (es >> 3)) + (es & 7); };
            auto vput = [&](int c, int r, int s2, float v) {
                *reinterpret_cast<float *>(Bt + tn_offset(vrow(c), 8 * (3 * r + s2) + l)) = v;
            };
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int s2 = r; s2 < 3; s2++) {
                        const float v = to_tf32(cs * W[r][i] * W[s2][i]);
                        vput(i, r, s2, v);
                        if (s2 != r) vput(i, s2, r, v);
                    }
#pragma unroll
            for (int c = 3; c < kTnComp; c++) {
                const int i = tn_comp_i(c), k = tn_comp_k(c);
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int s2 = 0; s2 < 3; s2++) vput(c, r, s2, to_tf32(fmaf(Lw[r][i], W[s2][k], Mw[r][k] * W[s2][i])));
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
        // ---------------- epilogue, kTnStageOct octets of the batch at a time: the thread of
        // TMEM lane t < 64 owns accumulator row t = node pair (a, b).  Its component (i, k),
        // i <= k, is K_ab,ik, and for i < k also K_ba,ki.  The chunk's element matrices are laid
        // out in [element][24][24] order over the V tile (free once the MMAs completed), then one
        // bulk asynchronous copy writes them out as one contiguous span; the next chunk waits
        // until that copy has read the tile, the next batch's V stores until the last one's.
        float *stage = reinterpret_cast<float *>(sm.B);
        const int64_t eb = b * kTnE;
#pragma unroll 1
        for (int o0 = 0; o0 < kTnOct; o0 += kTnStageOct) {
            const int64_t e0 = eb + 8 * o0;
            if (e0 >= A.n) break;  // (uniform over the CTA)
            const int nco = kTnOct - o0 < kTnStageOct ? kTnOct - o0 : kTnStageOct;
            const int n_el = (int)(A.n - e0 < 8 * nco ? A.n - e0 : 8 * nco);
            if (o0 > 0) {
                if (t == 0) tc::bulk_wait_read();
                __syncthreads();
            }
            if ((w & 3) < 2) {  // warps 0 and 1, 4 and 5, 8 and 9 (TMEM lanes 0-63): two components each
                const int pr = 32 * (w & 1) + (t & 31), pa = pr >> 3, pb = pr & 7, li = tg_lap(pa, pb);
#pragma unroll 1
                for (int cc = 0; cc < 2; cc++) {
                    const int c = 2 * (w >> 2) + cc, i = tn_comp_i(c), k = tn_comp_k(c);
                    const bool dg = c < 3;
                    float *dst = stage + 24 * (3 * pa + i) + 3 * pb + k;
                    float *dsT = stage + 24 * (3 * pb + k) + 3 * pa + i;
#pragma unroll
                    for (int oo = 0; oo < kTnStageOct; oo++) {
                        if (oo >= nco) break;
                        float v[8];
                        tc::tmem_ld8(tc::tmem_lane_addr(tm, 8 * (kTnOct * c + o0 + oo)), v);
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            const int el = 8 * oo + j;
                            if (dg) {
                                dst[576 * el] = v[j] + sm.geo[8 * o0 + el][li];
                            } else {
                                dst[576 * el] = v[j];
                                dsT[576 * el] = v[j];
                            }
                        }
                    }
                }
            }
            tc::fence_smem_to_async();
            tc::fence_before_sync();
            __syncthreads();  // the chunk's element matrices are laid out (after the last: the next MMA may overwrite TMEM)
            tc::fence_after_sync();
            if (t == 0) {  // the last copy drains during the next batch's phase 1
                tc::bulk_store(vals + 576 * e0, stage, (uint32_t)n_el * 576u * (uint32_t)sizeof(float));
                tc::bulk_commit();
            }
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
        // two CTAs per SM: 256 TMEM columns and about 112 KB of shared memory each
        const unsigned grid = (unsigned)std::min<int64_t>(n_batches, 2 * (int64_t)std::max(sms, 1));
        k_tf32<<<grid, kTnThreads, smem, s>>>(A, u, (float *)ws, Re);
        JETSCI_CUDA_TRY(cudaGetLastError());
    }
    return launch_gather_rows<float>(m, (const float *)ws, Re, vals, R, s);
}

}  // namespace jetsci
