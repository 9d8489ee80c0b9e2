// Element kernels: residual, consistent tangent into CSR, matrix-free tangent product and
// the material-gradient (adjoint) pass.  Their scatters are coloured read-modify-writes:
// within one colour no two elements share a node, colours run in a fixed order, so the
// sums are race-free without atomics and bitwise reproducible.  The FP32 tangent instead
// writes element rows for the row-gather assembly (gather.cu), as do the TF32 and surrogate
// element passes.  FP64 and two-float kernels read the mesh's reference-geometry cache
// (element.cuh), filled here at mesh creation.
#include <cuda_runtime.h>

#include <type_traits>

#include "blocks.cuh"
#include "element.cuh"
#include "jetsci_internal.h"

namespace jetsci {

struct ElemArgs {
    const int32_t *__restrict__ conn;
    const double *__restrict__ coords;
    const double *__restrict__ geom;    // per-element reference geometry (read by the FP64 kernels)
    const double *__restrict__ lap;     // per-element L_ab (element.cuh, kLap*; read by the tangent)
    double *lin;                        // FP64 linearisation store (element.cuh, kLin*): written by
                                        // the FP64 residual and tangent when set
    double *re;                         // element residual store [n_elem][8][3]: written by the
                                        // residual when set (for the material gradient)
    const int32_t *__restrict__ phase;
    const Material *__restrict__ mats;
    const double *__restrict__ E_elem;
    const int32_t *__restrict__ elems;  // element ids of one colour (NULL = identity)
    const uint8_t *__restrict__ order;  // FP64 tangent: the colour's off-diagonal item order (or NULL)
    int64_t n;                          // number of elements in the list
    uint32_t *flags;
};

template <typename T>
__device__ __forceinline__ bool finite3(const T f[3]) {
    return finite_t(f[0]) && finite_t(f[1]) && finite_t(f[2]);
}

__device__ __forceinline__ void raise_flag(uint32_t *flags, uint32_t bits) {
    if (bits) atomicOr(flags, bits);
}

// CSR scatter of one 3 x 3 block at slot s of node n's rows (kTrans: the transpose): the first
// writer of a block stores (no read), later writers add.  The choice is made once per block: a
// lane-wise choice per value was executed as predicated additions, which occupy the FP64 pipe
// whether or not a lane adds.
template <typename VT, typename T, bool kTrans>
__device__ __forceinline__ void put_or_add_block(VT *__restrict__ vals, const int64_t *__restrict__ rowptr,
                                                 int32_t n, int s, const T K[3][3], bool first) {
    VT *row[3];
#pragma unroll
    for (int i = 0; i < 3; i++) row[i] = vals + rowptr[3 * (int64_t)n + i] + 3 * s;
    if (first) {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) row[i][k] = store_as<VT>(kTrans ? K[k][i] : K[i][k]);
    } else {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) row[i][k] += store_as<VT>(kTrans ? K[k][i] : K[i][k]);
    }
}

// ---------------------------------------------------------------------------- residual
// R_e(a,i) = sum_q w detJ P_iJ G_aJ, scattered into R (FP64 in every precision); the stress
// moment comes from residual_moment (spatial form for the neo-Hookean law).  kKeep: also
// writes each element's R_e to A.re (a separate instantiation: the FP32 kernel without it stays
// at 56 registers, one block per SM more than with it).
template <typename T, bool kKeep>
__global__ void __launch_bounds__(128) k_residual(ElemArgs A, const double *__restrict__ u,
                                                  double *__restrict__ R) {
    const int l = threadIdx.x & 7;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool active = slot < A.n;
    const int64_t e = A.elems ? A.elems[active ? slot : A.n - 1] : (active ? slot : A.n - 1);
    int32_t node;
    GaussKinematics<T> K;
    T cu[3];
    gauss_kinematics<T>(A.conn, A.coords, u, e, l, node, K, cu, A.geom);
    ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, false);
    T Q[3][3];
    NeoHookeanState<T> st;
    const T lam = from_double<T>(mt.lam), mu = from_double<T>(mt.mu);
    const bool ok = residual_moment<T>(K, mt.law, lam, mu, Q, &st);
    if constexpr (!std::is_same<T, float>::value)  // FP64 and two-float calls store the state
        if (A.lin && active && mt.law != JETSCI_LINEAR_ELASTIC) {
            LinCoeffs<T> c;
            lin_coeffs(st.aj, st.rdj, K.dJ, st.lnJ, from_double<T>(element_lam_mu(A.mats, A.phase, e)), c);
            lin_store_t<T>(A.lin, e, l, c);
        }
    T f[3];
    nodal_force_of_moment(Q, K, l, f);
    if (active) {
        uint32_t bits = (positive(K.dJ) ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (ok ? 0u : JETSCI_FLAG_BAD_STATE) |
                        (finite3(f) ? 0u : JETSCI_FLAG_NONFINITE);
        raise_flag(A.flags, bits);
#pragma unroll
        for (int i = 0; i < 3; i++) R[3 * (int64_t)node + i] += to_double(f[i]);
        if constexpr (kKeep)
#pragma unroll
            for (int i = 0; i < 3; i++) A.re[24 * e + 3 * hex_node_of_lane(l) + i] = to_double(f[i]);
    }
}

// ---------------------------------------------------------------------------- tangent
// Phase 1 (8 lanes per element, lane = Gauss point): kinematics and constitutive update; per
// Gauss point the spatial gradients g_a = F^-T G_a of the eight shape functions and the
// coefficients c lam, c m and c Tg go to shared memory (c = w detJ, Tg the stress paired with g
// in the residual: the Kirchhoff stress tau = F S F^T for the neo-Hookean law, sigma for the
// linear one; m = mu - lam lnJ, and the linear law has g = G and m = mu).  Phase 2 (one thread
// per element and node pair a <= b):
//   K_ab,ik = sum_q [ c lam g_ai g_bk + c m g_ak g_bi ] + delta_ik mu L_ab
// which is the push-forward of sum_q w detJ G_aJ (delta_ik S_JL + F_iI CC_IJKL F_kK) G_bL for
// the neo-Hookean CC (F CC F = lam I(x)I + 2 m Isym); L_ab = sum_q detJ G_a . G_b is the
// element's reference Laplacian from the mesh's cache (element.cuh, kLap*), because the
// geometric term sum_q c g_a^T (tau + m I) g_b equals mu L_ab for both laws.  The diagonal-pair
// thread (a == b) also forms the residual R_a = sum_q c Tg g_a (= sum_q w detJ P G_a).
//
// With h_a = (c lam + c m)/2 g_a and d_a = (c lam - c m)/2 g_a (so c lam g_a = h_a + d_a and
// c m g_a = h_a - d_a), the block is, for i != k, K_ab,ik = A_ik + B_ik with
//   A_ik = sum_q h_ai g_bk + h_ak g_bi  (symmetric),   B_ik = sum_q d_ai g_bk - d_ak g_bi  (skew),
// and K_ab,ii = 2 sum_q h_ai g_bi + mu L_ab: 15 multiply-adds per Gauss point, against 21 for
// accumulating c lam g_ai g_bk, c m g_ak g_bi and the geometric term tg_a . g_b separately.
// FP32 and two-float elements form h_a and d_a from g_a and two coefficients, keeping the
// smaller record, which leaves room for more resident blocks.  FP64 elements, bound by B300's
// FP64 pipe, store l_a = c lam g_a, m_a = c m g_a and s_a = l_a + m_a and accumulate the entries
// directly, K_ab,ik = sum_q l_ai g_bk + m_ak g_bi (i != k) and sum_q s_ai g_bi + mu L_ab
// (i == k): also 15 multiply-adds per Gauss point, with the sums of the diagonal entries
// starting from mu L_ab and no finishing operations (the A +- B and 2 A + mu L_ab of the
// symmetric/skew form: 9 per off-diagonal pair), for 3 more multiplies per node and point.

// Shared memory: one array per per-node vector (g and, for FP64, l, m and s), each
// [element][Gauss point][node][3], nodes 3 entries apart, so that the eight nodes of an element
// read in phase 2 fall on distinct banks.  Elements are 200 entries apart (8 mod 32 words for
// FP32, 16 mod 32 for 8-byte types), which also spreads the up to four elements of one warp
// over distinct banks.  For 8-byte types points are 25 entries apart (the eight Gauss-point
// lanes of phase 1 on distinct banks); for FP32 24, keeping each lane's 24 values 16-byte
// aligned for vector stores.
template <typename T>
struct TangentLayout {
    static constexpr bool kPre = std::is_same<T, double>::value;
    // Elements per block (phase 1: one thread per element and Gauss point).  Measured at 128^3:
    // 8 is 4-5% faster than 16 for FP64 and FP32; the two-float kernel needs 16.  The FP64 block
    // adds four warps that only join the pair loop (phase 2): 6% faster again (two warps: 5%,
    // six: slower; the two-float kernel: slower with any).
    static constexpr int kElems = std::is_same<T, df64>::value ? 16 : 8;
    // The FP32 element pass (rows mode) adds one warp to the pair loop too: its items' blocks
    // are held in registers until the matrices are assembled, and three items per thread
    // instead of five were 5% faster (four warps: slower).
    static constexpr int kThreads = kPre ? 192 : (std::is_same<T, float>::value ? 96 : 8 * kElems);
    // Blocks per SM the kernels are compiled for: FP64 4 (56 KB of shared memory; 80 registers
    // with a 12-byte spill, where the compiler's own choice of 96 registers allowed three: 28.19
    // -> 27.99 ms at 128^3), FP32 12 (56 registers; at 10 the compiler took 64 and the element
    // pass ran 4% slower), two-float 5 (96 registers, its own choice; at 6, 80 registers with a
    // 16-byte spill, the tangent ran 18.15 -> 18.40 ms).
    static constexpr int kMinBlocks = kPre ? 4 : (std::is_same<T, float>::value ? 12 : 5);
    static constexpr int kNumVec = kPre ? 4 : 1;
    static constexpr int kPoint = sizeof(T) == 4 ? 24 : 25;
    static constexpr int kElem = 200;
    static constexpr int kArr = kElems * kElem;
    // per (element, Gauss point): (c lam + c m)/2, (c lam - c m)/2, c Tg (00,11,22,12,02,01); odd stride
    static constexpr int kCoef = 9;
    enum { kG = 0, kLG = 1, kMG = 2, kSG = 3 };  // g, c lam g, c m g, (c lam + c m) g (FP64)
    // FP64 values: each CSR block's first writer stores and no clearing pass is needed (saves
    // the 4 GB memset at 128^3).  The two-float kernel was measured slower that way (the
    // partial-sector first stores and the divergent store/accumulate paths cost more than the
    // clearing pass), so it clears the array and accumulates; FP32 values are assembled by row
    // gather instead of by scatter.
    static constexpr bool kFirstWrites = std::is_same<T, double>::value;
};

template <typename T>
struct TangentSmem {
    T v[TangentLayout<T>::kNumVec * TangentLayout<T>::kArr];
    T coef[TangentLayout<T>::kElems * 8 * TangentLayout<T>::kCoef];
    int32_t node[TangentLayout<T>::kElems][8];
    int32_t elem[TangentLayout<T>::kElems];
    T mu[TangentLayout<T>::kElems];
    uint8_t first[TangentLayout<T>::kElems][8];  // first-writer bits of each node's blocks (FP64)
};

// Work items, per group of 8 elements: first the 28 off-diagonal node pairs (a < b) of each
// element (7 warps), then their 8 diagonal pairs (2 warps).  Each warp holds items of one kind,
// so neither the residual (diagonal pairs only) nor the symmetric diagonal block leaves lanes
// predicated off, and an element's diagonal blocks follow its other blocks closely.
constexpr int kGroup = 8, kGroupItems = kGroup * 36, kGroupOff = kGroup * 28;

// Off-diagonal block K_ab (a < b) of element slot ee from the phase-1 records.
template <typename T, int kUnrollQ>
__device__ __forceinline__ void offdiag_block(const TangentSmem<T> &sm, int ee, int a, int b, T gs, T Kab[3][3]) {
    using L = TangentLayout<T>;
    const T *pa = sm.v + ee * L::kElem + 3 * a;
    const T *pb = sm.v + ee * L::kElem + 3 * b;
    if constexpr (L::kPre) {
        // FP64: K_ab,ik = sum_q l_ai g_bk + m_ak g_bi for i != k and sum_q s_ai g_bi + mu L_ab
        // for i == k (l = c lam g, m = c m g, s = l + m): 15 multiply-adds per Gauss point and no
        // finishing operations (the diagonal sums start from mu L_ab)
        T K00 = gs, K11 = gs, K22 = gs, K01 = T(0), K10 = T(0), K02 = T(0), K20 = T(0), K12 = T(0), K21 = T(0);
#pragma unroll kUnrollQ
        for (int q = 0; q < 8; q++) {
            const T *qa = pa + q * L::kPoint;
            const T *qb = pb + q * L::kPoint;
            const T b0 = qb[0], b1 = qb[1], b2 = qb[2];
            const T *la = qa + L::kLG * L::kArr, *ma = qa + L::kMG * L::kArr, *sa = qa + L::kSG * L::kArr;
            const T l0 = la[0], l1 = la[1], l2 = la[2], m0 = ma[0], m1 = ma[1], m2 = ma[2];
            K00 = acc_t(sa[0], b0, K00);
            K11 = acc_t(sa[1], b1, K11);
            K22 = acc_t(sa[2], b2, K22);
            K01 = acc_t(l0, b1, acc_t(m1, b0, K01));
            K10 = acc_t(l1, b0, acc_t(m0, b1, K10));
            K02 = acc_t(l0, b2, acc_t(m2, b0, K02));
            K20 = acc_t(l2, b0, acc_t(m0, b2, K20));
            K12 = acc_t(l1, b2, acc_t(m2, b1, K12));
            K21 = acc_t(l2, b1, acc_t(m1, b2, K21));
        }
        Kab[0][0] = K00, Kab[1][1] = K11, Kab[2][2] = K22;
        Kab[0][1] = K01, Kab[1][0] = K10, Kab[0][2] = K02, Kab[2][0] = K20, Kab[1][2] = K12, Kab[2][1] = K21;
        return;
    }
    const T *pc = sm.coef + ee * 8 * L::kCoef;
    T A00 = T(0), A11 = T(0), A22 = T(0), A01 = T(0), A02 = T(0), A12 = T(0);
    T B01 = T(0), B02 = T(0), B12 = T(0);
#pragma unroll kUnrollQ
    for (int q = 0; q < 8; q++) {
        const T *qa = pa + q * L::kPoint;
        const T *qb = pb + q * L::kPoint;
        const T b0 = qb[0], b1 = qb[1], b2 = qb[2];
        const T *cf = pc + q * L::kCoef;
        const T ch = cf[0], cd = cf[1], a0 = qa[0], a1 = qa[1], a2 = qa[2];
        const T h0 = ch * a0, h1 = ch * a1, h2 = ch * a2, d0 = cd * a0, d1 = cd * a1, d2 = cd * a2;
        A00 = acc_t(h0, b0, A00);
        A11 = acc_t(h1, b1, A11);
        A22 = acc_t(h2, b2, A22);
        A01 = acc_t(h0, b1, acc_t(h1, b0, A01));
        A02 = acc_t(h0, b2, acc_t(h2, b0, A02));
        A12 = acc_t(h1, b2, acc_t(h2, b1, A12));
        B01 = acc_t(d0, b1, acc_t(-d1, b0, B01));
        B02 = acc_t(d0, b2, acc_t(-d2, b0, B02));
        B12 = acc_t(d1, b2, acc_t(-d2, b1, B12));
    }
    // (two-float running sums are normalised once, here)
    A00 = acc_norm(A00), A11 = acc_norm(A11), A22 = acc_norm(A22);
    A01 = acc_norm(A01), A02 = acc_norm(A02), A12 = acc_norm(A12);
    B01 = acc_norm(B01), B02 = acc_norm(B02), B12 = acc_norm(B12);
    Kab[0][0] = fma_t(T(2), A00, gs);
    Kab[1][1] = fma_t(T(2), A11, gs);
    Kab[2][2] = fma_t(T(2), A22, gs);
    Kab[0][1] = A01 + B01, Kab[1][0] = A01 - B01;
    Kab[0][2] = A02 + B02, Kab[2][0] = A02 - B02;
    Kab[1][2] = A12 + B12, Kab[2][1] = A12 - B12;
}

// Diagonal block K_aa,ik = 2 sum_q h_ai g_ak + delta_ik gs (gs = mu L_aa) of element slot ee and,
// with want_r, the residual R_a = sum_q c Tg g_a.
template <typename T, int kUnrollQ>
__device__ __forceinline__ void diag_block(const TangentSmem<T> &sm, int ee, int a, bool want_r, T gs, T Kab[3][3],
                                           T Ra[3]) {
    using L = TangentLayout<T>;
    const T *pa = sm.v + ee * L::kElem + 3 * a;
    const T *pc = sm.coef + ee * 8 * L::kCoef;
    T Ra0 = T(0), Ra1 = T(0), Ra2 = T(0);
    if constexpr (L::kPre) {
        // FP64: K_aa,ik = sum_q s_ai g_ak + delta_ik mu L_aa (s = (c lam + c m) g)
        T k00 = gs, k11 = gs, k22 = gs, k12 = T(0), k02 = T(0), k01 = T(0);
#pragma unroll kUnrollQ
        for (int q = 0; q < 8; q++) {
            const T *qa = pa + q * L::kPoint;
            const T *cf = pc + q * L::kCoef;
            const T b0 = qa[0], b1 = qa[1], b2 = qa[2];
            const T *sa = qa + L::kSG * L::kArr;
            const T s0 = sa[0], s1 = sa[1], s2 = sa[2];
            k00 = acc_t(s0, b0, k00);
            k11 = acc_t(s1, b1, k11);
            k22 = acc_t(s2, b2, k22);
            k12 = acc_t(s1, b2, k12);
            k02 = acc_t(s0, b2, k02);
            k01 = acc_t(s0, b1, k01);
            if (want_r) {
                Ra0 = acc_t(cf[2], b0, acc_t(cf[7], b1, acc_t(cf[6], b2, Ra0)));
                Ra1 = acc_t(cf[7], b0, acc_t(cf[3], b1, acc_t(cf[5], b2, Ra1)));
                Ra2 = acc_t(cf[6], b0, acc_t(cf[5], b1, acc_t(cf[4], b2, Ra2)));
            }
        }
        Kab[0][0] = k00, Kab[1][1] = k11, Kab[2][2] = k22;
        Kab[1][2] = Kab[2][1] = k12;
        Kab[0][2] = Kab[2][0] = k02;
        Kab[0][1] = Kab[1][0] = k01;
        Ra[0] = Ra0, Ra[1] = Ra1, Ra[2] = Ra2;
        return;
    }
    T k00 = T(0), k11 = T(0), k22 = T(0), k12 = T(0), k02 = T(0), k01 = T(0);
#pragma unroll kUnrollQ
    for (int q = 0; q < 8; q++) {
        const T *qa = pa + q * L::kPoint;
        const T *cf = pc + q * L::kCoef;
        const T b0 = qa[0], b1 = qa[1], b2 = qa[2];
        const T ch = cf[0];
        const T h0 = ch * b0, h1 = ch * b1, h2 = ch * b2;
        k00 = acc_t(h0, b0, k00);
        k11 = acc_t(h1, b1, k11);
        k22 = acc_t(h2, b2, k22);
        k12 = acc_t(h1, b2, k12);
        k02 = acc_t(h0, b2, k02);
        k01 = acc_t(h0, b1, k01);
        if (want_r) {
            Ra0 = acc_t(cf[2], b0, acc_t(cf[7], b1, acc_t(cf[6], b2, Ra0)));
            Ra1 = acc_t(cf[7], b0, acc_t(cf[3], b1, acc_t(cf[5], b2, Ra1)));
            Ra2 = acc_t(cf[6], b0, acc_t(cf[5], b1, acc_t(cf[4], b2, Ra2)));
        }
    }
    k00 = acc_norm(k00), k11 = acc_norm(k11), k22 = acc_norm(k22);
    k12 = acc_norm(k12), k02 = acc_norm(k02), k01 = acc_norm(k01);
    Kab[0][0] = fma_t(T(2), k00, gs);
    Kab[1][1] = fma_t(T(2), k11, gs);
    Kab[2][2] = fma_t(T(2), k22, gs);
    Kab[1][2] = Kab[2][1] = k12 + k12;
    Kab[0][2] = Kab[2][0] = k02 + k02;
    Kab[0][1] = Kab[1][0] = k01 + k01;
    Ra[0] = acc_norm(Ra0);
    Ra[1] = acc_norm(Ra1);
    Ra[2] = acc_norm(Ra2);
}

// Work item `it` of a group (element slot ee, nodes a <= b, off = a < b; li = the pair's index in
// the element's L_ab, element.cuh kLap*).
__device__ __forceinline__ void item_nodes(int it, int &ee, int &a, int &b, bool &off, int &li) {
    const int grp = it / kGroupItems, r = it - kGroupItems * grp;
    off = r < kGroupOff;
    if (off) {
        const int eg = r / 28;
        const int p = r - 28 * eg;
        ee = kGroup * grp + eg;
        // p -> (a, b), a < b, in row order: row a starts at 7a - a(a-1)/2
        a = (p >= 7) + (p >= 13) + (p >= 18) + (p >= 22) + (p >= 25) + (p >= 27);
        b = p - (7 * a - (a * (a - 1)) / 2) + a + 1;
        li = p;
    } else {
        const int j = r - kGroupOff;
        ee = kGroup * grp + (j >> 3);
        a = b = j & 7;
        li = kLapDiag + a;
    }
}

// The geometric term mu L_ab of item (ee, li) (an inactive slot reads element 0's entry).
template <typename T>
__device__ __forceinline__ T item_gs(const TangentSmem<T> &sm, const double *__restrict__ lap, int ee, int li) {
    const int64_t eid = sm.elem[ee] < 0 ? 0 : sm.elem[ee];
    return sm.mu[ee] * from_double<T>(__ldg(lap + kLapPairs * eid + li));
}

// Block K_ab of work item `it` from the phase-1 records; for a diagonal item with want_r also
// the residual R_a.
template <typename T>
__device__ __forceinline__ void tangent_item(const TangentSmem<T> &sm, const double *__restrict__ lap, int it,
                                             bool want_r, T Kab[3][3], T Ra[3], int &ee, int &a, int &b, bool &off) {
    int li;
    item_nodes(it, ee, a, b, off, li);
    const T gs = item_gs(sm, lap, ee, li);
    if (off)
        offdiag_block<T, 2>(sm, ee, a, b, gs, Kab);
    else
        diag_block<T, 2>(sm, ee, a, want_r, gs, Kab, Ra);
}

// Shared memory of the rows mode: the block's element matrices [element][24][24], as in the
// workspace, laid over the phase-1 records once every item has read them (a padded row stride
// of 28 was measured 3% slower at 128^3: more shared memory per block).
template <typename T>
constexpr size_t tangent_smem_bytes(bool rows) {
    const size_t mat = (size_t)TangentLayout<T>::kElems * 576 * sizeof(T);
    return rows && mat > sizeof(TangentSmem<T>) ? mat : sizeof(TangentSmem<T>);
}

// kRows = false: scatter into the CSR values (vals) and R, one launch per colour.
// kRows = true: the element pass of the row-gather assembly, over all elements in order in one
// launch: vals is the workspace [element][24][24] (blocks.cuh) and R its residual part.  Each
// thread keeps its items' blocks in registers until every item has read the phase-1 records;
// then the block's element matrices are assembled over those records in shared memory and
// written out as one contiguous span.
template <typename T, typename VT, bool kRows>
__device__ __forceinline__ void tangent_element_pass(ElemArgs A, const double *__restrict__ u,
                                                     const int64_t *__restrict__ rowptr,
                                                     const uint8_t *__restrict__ slotmap,
                                                     const uint8_t *__restrict__ first,
                                                     VT *__restrict__ vals, double *__restrict__ R) {
    using L = TangentLayout<T>;
    constexpr bool kFirst = L::kFirstWrites && !kRows;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TangentSmem<T> &sm = *reinterpret_cast<TangentSmem<T> *>(smem_raw);
    const int l = threadIdx.x & 7;
    const int es = threadIdx.x >> 3;
    const int64_t slot = (int64_t)blockIdx.x * L::kElems + es;
    const bool active = slot < A.n;
    const int64_t e = A.elems ? A.elems[active ? slot : A.n - 1] : (active ? slot : A.n - 1);
    if (es < L::kElems) {  // warps beyond the element slots join in phase 2 only
        int32_t node;
        GaussKinematics<T> K;
        T cu[3];
        gauss_kinematics<T, false, false>(A.conn, A.coords, u, e, l, node, K, cu, A.geom);
        ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, false);
        const T lam = from_double<T>(mt.lam), mu = from_double<T>(mt.mu);
        // Per law: W with g_a = W^T (8 dN_a/dxi), Tg (the stress paired with g in the residual) and m.
        T W[3][3], Tg[3][3], m;
        bool ok = true;
        if (mt.law == JETSCI_LINEAR_ELASTIC) {
            // g = G: W = Jp^-1; sigma = lam tr(H) I + mu (H + H^T), H = Du Jp^-1
            const T rdJ = my_rcp(K.dJ);
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int j = 0; j < 3; j++) W[d][j] = K.aJ[d][j] * rdJ;
            T H[3][3];
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) H[i][j] = K.Du[i][0] * W[0][j] + K.Du[i][1] * W[1][j] + K.Du[i][2] * W[2][j];
            const T ltr = lam * (H[0][0] + H[1][1] + H[2][2]);
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    Tg[i][j] = mu * (H[i][j] + H[j][i]) + ((i == j) ? ltr : T(0));
                }
            m = mu;
        } else {
            // Neo-Hookean: W = (F Jp)^-1 = j^-1 with j = Jp + Du the deformed Jacobian.
            NeoHookeanState<T> st;
            neo_hookean_state(K, lam, mu, st);
            ok = st.ok;
            m = st.m;
            if constexpr (!std::is_same<T, float>::value)  // FP64 and two-float calls store the state
                if (A.lin && active) {
                    LinCoeffs<T> c;
                    lin_coeffs(st.aj, st.rdj, K.dJ, st.lnJ, from_double<T>(element_lam_mu(A.mats, A.phase, e)), c);
                    lin_store_t<T>(A.lin, e, l, c);
                }
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    W[d][j] = st.aj[d][j] * st.rdj;
                    Tg[d][j] = st.tau[d][j];
                }
        }
        if (active) {
            uint32_t bits = (positive(K.dJ) ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (ok ? 0u : JETSCI_FLAG_BAD_STATE);
            raise_flag(A.flags, bits);
        }
        const T cw = K.dJ * T(1.0 / 512.0);
        const T cl = cw * lam, cm = cw * m;
        const T ch = T(0.5) * (cl + cm), cd = T(0.5) * (cl - cm), cs = cl + cm;
        // 1 +- xi, 1 +- eta, 1 +- zeta at the lane's Gauss point (selected for FP64: element.cuh)
        T xp, xm, yp, ym, zp, zm;
        if constexpr (std::is_same<T, double>::value) {
            xp = (l & 1) ? kGaussP : kGaussM, xm = (l & 1) ? kGaussM : kGaussP;
            yp = (l & 2) ? kGaussP : kGaussM, ym = (l & 2) ? kGaussM : kGaussP;
            zp = (l & 4) ? kGaussP : kGaussM, zm = (l & 4) ? kGaussM : kGaussP;
        } else {
            xp = T(1) + K.xi, xm = T(1) - K.xi, yp = T(1) + K.eta, ym = T(1) - K.eta;
            zp = T(1) + K.zeta, zm = T(1) - K.zeta;
        }
        T *pv = sm.v + es * L::kElem + l * L::kPoint;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const int bits = hex_bits_of_node(a);
            T yz, xz, xy;
            if constexpr (std::is_same<T, double>::value) {
                // each product of two of 1 +- g is (1+g)^2, (1+g)(1-g) or (1-g)^2: selected, not
                // multiplied (the node's factor is 1 + g where its sign matches the point's)
                const bool mx = ((bits ^ l) & 1) == 0, my = ((bits ^ l) & 2) == 0, mz = ((bits ^ l) & 4) == 0;
                yz = my ? (mz ? kGaussPP : kGaussPM) : (mz ? kGaussPM : kGaussMM);
                xz = mx ? (mz ? kGaussPP : kGaussPM) : (mz ? kGaussPM : kGaussMM);
                xy = mx ? (my ? kGaussPP : kGaussPM) : (my ? kGaussPM : kGaussMM);
            } else {
                const T fx = (bits & 1) ? xp : xm, fy = (bits & 2) ? yp : ym, fz = (bits & 4) ? zp : zm;
                yz = fy * fz, xz = fx * fz, xy = fx * fy;
            }
            // 8 dN_a/dxi at the Gauss point
            const T n0 = (bits & 1) ? yz : -yz, n1 = (bits & 2) ? xz : -xz, n2 = (bits & 4) ? xy : -xy;
            T *r = pv + 3 * a;
            T g[3];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                g[j] = W[0][j] * n0 + W[1][j] * n1 + W[2][j] * n2;
                r[L::kG * L::kArr + j] = g[j];
                if constexpr (L::kPre) {
                    r[L::kLG * L::kArr + j] = cl * g[j];
                    r[L::kMG * L::kArr + j] = cm * g[j];
                    r[L::kSG * L::kArr + j] = cs * g[j];
                }
            }
        }
        T *pc = sm.coef + (es * 8 + l) * L::kCoef;
        pc[0] = ch;
        pc[1] = cd;
        pc[2] = cw * Tg[0][0];
        pc[3] = cw * Tg[1][1];
        pc[4] = cw * Tg[2][2];
        pc[5] = cw * Tg[1][2];
        pc[6] = cw * Tg[0][2];
        pc[7] = cw * Tg[0][1];
        sm.node[es][hex_node_of_lane(l)] = node;
        sm.first[es][hex_node_of_lane(l)] = kFirst ? first[8 * e + hex_node_of_lane(l)] : 0;
        if (l == 0) {
            sm.elem[es] = active ? (int32_t)e : -1;
            sm.mu[es] = mu;
        }
    }
    __syncthreads();
    static_assert(L::kElems % kGroup == 0 && kGroupOff % 32 == 0 && kGroupItems % 32 == 0,
                  "items of one kind per warp");
    if constexpr (!kRows) {
        // (Gauss-point loops unrolled by 2; by 1 for two-float elements, whose long unrolled
        // arithmetic otherwise stalls on instruction fetch: 0.9% faster at 128^3)
        constexpr int kUnrollQ = std::is_same<T, df64>::value ? 1 : 2;
        for (int it = threadIdx.x; it < L::kElems * 36; it += blockDim.x) {
            int ee, a, b, li;
            bool off;
            int itm = it;
            if (kFirst && A.order) {  // (first-writer pairs grouped into whole warps)
                const int grp = it / kGroupItems, r = it - kGroupItems * grp;
                if (r < kGroupOff) itm = kGroupItems * grp + A.order[r];
            }
            item_nodes(itm, ee, a, b, off, li);
            const int32_t eid = sm.elem[ee];
            if (eid < 0) continue;
            const T gs = item_gs(sm, A.lap, ee, li);
            const int32_t na = sm.node[ee][a];
            const int64_t sbase = 64 * (int64_t)eid;
            T Kab[3][3];
            if (off) {
                offdiag_block<T, kUnrollQ>(sm, ee, a, b, gs, Kab);
                {
                    const int32_t nb = sm.node[ee][b];
                    const int sab = slotmap[sbase + 8 * a + b];
                    const int sba = slotmap[sbase + 8 * b + a];
                    // the block's first writer (lowest colour) stores, later colours accumulate;
                    // one choice per block, so a warp whose lanes all store issues no additions
                    const bool fab = kFirst && ((sm.first[ee][a] >> b) & 1);
                    const bool fba = kFirst && ((sm.first[ee][b] >> a) & 1);
                    put_or_add_block<VT, T, false>(vals, rowptr, na, sab, Kab, fab);
                    put_or_add_block<VT, T, true>(vals, rowptr, nb, sba, Kab, fba);
                }
            } else {
                T Ra[3];
                diag_block<T, kUnrollQ>(sm, ee, a, R != nullptr, gs, Kab, Ra);
                const T Ra0 = Ra[0], Ra1 = Ra[1], Ra2 = Ra[2];
                {
                    const int saa = slotmap[sbase + 9 * a];
                    const bool faa = kFirst && ((sm.first[ee][a] >> a) & 1);
                    put_or_add_block<VT, T, false>(vals, rowptr, na, saa, Kab, faa);
                }
                if (R) {
                    const bool fin = finite_t(Ra0) && finite_t(Ra1) && finite_t(Ra2);
                    if (!fin) raise_flag(A.flags, JETSCI_FLAG_NONFINITE);
                    R[3 * (int64_t)na] += to_double(Ra0);
                    R[3 * (int64_t)na + 1] += to_double(Ra1);
                    R[3 * (int64_t)na + 2] += to_double(Ra2);
                }
            }
        }
    } else {
        constexpr int kItems = L::kElems * 36;
        constexpr int kIters = (kItems + L::kThreads - 1) / L::kThreads;
        VT res[kIters][9];
#pragma unroll
        for (int j = 0; j < kIters; j++) {
            const int it = threadIdx.x + j * L::kThreads;
            if (it < kItems) {  // warp-uniform (kItems is a multiple of 32)
                T Kab[3][3], Ra[3];
                int ee, a, b;
                bool off;
                tangent_item<T>(sm, A.lap, it, R != nullptr, Kab, Ra, ee, a, b, off);
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int k = 0; k < 3; k++) res[j][3 * i + k] = store_as<VT>(Kab[i][k]);
                const int32_t eid = sm.elem[ee];
                if (!off && R && eid >= 0) {
                    const bool fin = finite_t(Ra[0]) && finite_t(Ra[1]) && finite_t(Ra[2]);
                    if (!fin) raise_flag(A.flags, JETSCI_FLAG_NONFINITE);
#pragma unroll
                    for (int i = 0; i < 3; i++) R[3 * (8 * (int64_t)eid + a) + i] = to_double(Ra[i]);
                }
            }
        }
        __syncthreads();  // every item has read the phase-1 records: lay the matrices over them
        VT *mat = reinterpret_cast<VT *>(smem_raw);
#pragma unroll
        for (int j = 0; j < kIters; j++) {
            const int it = threadIdx.x + j * L::kThreads;
            if (it < kItems) {
                int ee, a, b, li;
                bool off;
                item_nodes(it, ee, a, b, off, li);
                VT *me = mat + (size_t)ee * 576;
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        me[(3 * a + i) * 24 + 3 * b + k] = res[j][3 * i + k];
                        me[(3 * b + k) * 24 + 3 * a + i] = res[j][3 * i + k];  // K_ba = K_ab^T
                    }
            }
        }
        __syncthreads();
        // the block's element matrices, in order: one contiguous span of the workspace
        const int64_t e0 = (int64_t)blockIdx.x * L::kElems;
        const int n_vec = (int)((A.n - e0 < L::kElems ? A.n - e0 : L::kElems) * 576 * sizeof(VT) / 16);
        uint4 *dst = reinterpret_cast<uint4 *>(vals + 576 * e0);
        const uint4 *src = reinterpret_cast<const uint4 *>(mat);
        for (int c = threadIdx.x; c < n_vec; c += blockDim.x) dst[c] = src[c];
    }
}

template <typename T, typename VT, bool kRows>
__global__ void __launch_bounds__(TangentLayout<T>::kThreads, TangentLayout<T>::kMinBlocks)
    k_tangent(ElemArgs A, const double *__restrict__ u,
                                                 const int64_t *__restrict__ rowptr,
                                                 const uint8_t *__restrict__ slotmap,
                                                 const uint8_t *__restrict__ first,
                                                 VT *__restrict__ vals, double *__restrict__ R) {
    tangent_element_pass<T, VT, kRows>(A, u, rowptr, slotmap, first, vals, R);
}


// ---------------------------------------------------------------------------- K v, matrix-free
// y_a += sum_q w detJ Y G_a with Y the linearised first Piola-Kirchhoff stress in the direction
// Hv = grad_X v:  Y = sigma(Hv) for the linear law;  for the neo-Hookean law, with
// S = mu I - m C^-1 (m = mu - lam lnJ), C^-1 = F^-1 F^-T and h = Hv F^-1,
//   Y = Hv S + (lam tr(h) I + m (h + h^T)) F^-T = mu Hv + (m h^T + lam tr(h) I) F^-T.
// The neo-Hookean branch works with the deformed Jacobian j = Jp + Du = 8 dx/dxi, so that
// F^-1 = Jp j^-1, J = det j / det Jp and h = Dv j^-1 (Dv = 8 dv/dxi), and forms the moment
// Q = Y adj(Jp)^T directly:
//   Q = (mu / det Jp) Dv adj(Jp) adj(Jp)^T + (det Jp / det j^2) M' adj(j)^T,
//   M' = m h'^T + lam tr(h') I,  h' = Dv adj(j) = det j h,
// i.e. Q = mu [Dv A0' + (alpha h'^T + beta tr(h') I) adj(j)^T] with A0' = adj(Jp) adj(Jp)^T /
// det Jp from the geometry cache and the per-point coefficients alpha = (m / mu) det Jp / det j^2,
// beta = (lam / mu) det Jp / det j^2 (element.cuh, lin_coeffs).  The nodal forces are linear in
// Q and mu is the element's, so mu multiplies the three forces of a lane after the sum over the
// Gauss points instead of each of the nine entries of Q at every point.
// kReuse (FP64 and two-float): the coefficients come from the mesh's linearisation store (the
// last FP64 or two-float residual or tangent, at its u) instead of u; u is not read.
template <typename T, bool kReuse>
__device__ __forceinline__ void apply_mf_element(ElemArgs A, const double *__restrict__ u,
                                                 const double *__restrict__ v, double *__restrict__ y) {
    const int l = threadIdx.x & 7;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool active = slot < A.n;
    const int64_t e = A.elems ? A.elems[active ? slot : A.n - 1] : (active ? slot : A.n - 1);
    int32_t node;
    GaussKinematics<T> K;
    if constexpr (kReuse) {
        static_assert(!std::is_same<T, float>::value, "the linearisation store serves FP64 and two-float products");
        gauss_geometry<T>(A.conn, A.geom, e, l, node, K);
    } else {
        T cu[3];
        gauss_kinematics<T>(A.conn, A.coords, u, e, l, node, K, cu, A.geom);
    }
    ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, false);
    const T lam = from_double<T>(mt.lam), mu = from_double<T>(mt.mu);
    T Dv[3][3];
    field_ref_gradient<T>(v, node, l, K, Dv);
    T Q[3][3];
    bool ok = true;
    if (mt.law == JETSCI_LINEAR_ELASTIC) {
        const T rdJ = my_rcp(K.dJ);
        T Hv[3][3], Y[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                Hv[i][j] = (Dv[i][0] * K.aJ[0][j] + Dv[i][1] * K.aJ[1][j] + Dv[i][2] * K.aJ[2][j]) * rdJ;
        const T tr = Hv[0][0] + Hv[1][1] + Hv[2][2];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) Y[i][j] = mu * (Hv[i][j] + Hv[j][i]) + ((i == j) ? lam * tr : T(0));
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int d = 0; d < 3; d++) Q[i][d] = Y[i][0] * K.aJ[d][0] + Y[i][1] * K.aJ[d][1] + Y[i][2] * K.aJ[d][2];
    } else if constexpr (std::is_same<T, float>::value) {
        // FP32: Q = s1 Dv adj(Jp) adj(Jp)^T + (alpha h'^T + beta tr(h') I) adj(j)^T with
        // s1 = mu / det Jp, alpha = m det Jp / det j^2, beta = lam det Jp / det j^2 (no cache; the
        // mu-scaled form below took this issue-bound kernel from 56 to 64 registers, 0.86 -> 0.92 ms)
        NeoHookeanState<T> st;
        neo_hookean_state(K, lam, mu, st);
        ok = st.ok;
        const T s2 = K.dJ * st.rdj * st.rdj, al = s2 * st.m, be = s2 * lam, s1 = mu * st.rdJ;
        T A0[3][3];
        adj_gram(K.aJ, A0);
        T hp[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) hp[i][k] = Dv[i][0] * st.aj[0][k] + Dv[i][1] * st.aj[1][k] + Dv[i][2] * st.aj[2][k];
        const T btr = be * (hp[0][0] + hp[1][1] + hp[2][2]);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const T M0 = fma_t(al, hp[0][i], (i == 0) ? btr : T(0));
            const T M1 = fma_t(al, hp[1][i], (i == 1) ? btr : T(0));
            const T M2 = fma_t(al, hp[2][i], (i == 2) ? btr : T(0));
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const T p1 = Dv[i][0] * A0[0][d] + Dv[i][1] * A0[1][d] + Dv[i][2] * A0[2][d];
                T q = s1 * p1;
                q = fma_t(M0, st.aj[d][0], q);
                q = fma_t(M1, st.aj[d][1], q);
                Q[i][d] = fma_t(M2, st.aj[d][2], q);
            }
        }
    } else {
        LinCoeffs<T> c;
        T A0[3][3];  // adj(Jp) adj(Jp)^T / det Jp (symmetric; from the geometry cache)
        {
            const double *p = geom_point(A.geom, e, l);
            const double2 a01 = geom_pair(p, kGeomA0 / 2), a23 = geom_pair(p, kGeomA0 / 2 + 1),
                          a45 = geom_pair(p, kGeomA0 / 2 + 2);  // 00 11 | 22 12 | 02 01
            A0[0][0] = from_double<T>(a01.x), A0[1][1] = from_double<T>(a01.y), A0[2][2] = from_double<T>(a23.x);
            A0[1][2] = A0[2][1] = from_double<T>(a23.y);
            A0[0][2] = A0[2][0] = from_double<T>(a45.x);
            A0[0][1] = A0[1][0] = from_double<T>(a45.y);
        }
        if constexpr (kReuse) {
            lin_load_t<T>(A.lin, e, l, c);  // (states outside the law were flagged when stored)
        } else {
            NeoHookeanState<T> st;
            neo_hookean_state(K, lam, mu, st);
            ok = st.ok;
            lin_coeffs(st.aj, st.rdj, K.dJ, st.lnJ, from_double<T>(element_lam_mu(A.mats, A.phase, e)), c);
        }
        T hp[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) hp[i][k] = Dv[i][0] * c.aj[0][k] + Dv[i][1] * c.aj[1][k] + Dv[i][2] * c.aj[2][k];
        const T btr = c.beta * (hp[0][0] + hp[1][1] + hp[2][2]);
        // Q / mu = Dv A0 + (alpha h'^T + beta tr(h') I) adj(j)^T; mu is applied to the nodal forces
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const T M0 = fma_t(c.alpha, hp[0][i], (i == 0) ? btr : T(0));
            const T M1 = fma_t(c.alpha, hp[1][i], (i == 1) ? btr : T(0));
            const T M2 = fma_t(c.alpha, hp[2][i], (i == 2) ? btr : T(0));
#pragma unroll
            for (int d = 0; d < 3; d++) {
                T q = Dv[i][0] * A0[0][d];
                q = fma_t(Dv[i][1], A0[1][d], q);
                q = fma_t(Dv[i][2], A0[2][d], q);
                q = fma_t(M0, c.aj[d][0], q);
                q = fma_t(M1, c.aj[d][1], q);
                Q[i][d] = fma_t(M2, c.aj[d][2], q);
            }
        }
    }
    T f[3];
    nodal_force_of_moment(Q, K, l, f);
    if constexpr (!std::is_same<T, float>::value)
        if (mt.law != JETSCI_LINEAR_ELASTIC)  // (the neo-Hookean moment above is Q / mu: mu is the element's)
#pragma unroll
            for (int i = 0; i < 3; i++) f[i] = mu * f[i];
    if (active) {
        uint32_t bits = (positive(K.dJ) ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (ok ? 0u : JETSCI_FLAG_BAD_STATE) |
                        (finite3(f) ? 0u : JETSCI_FLAG_NONFINITE);
        raise_flag(A.flags, bits);
#pragma unroll
        for (int i = 0; i < 3; i++) y[3 * (int64_t)node + i] += to_double(f[i]);
    }
}

template <typename T, bool kReuse>
__global__ void __launch_bounds__(128) k_apply_mf(ElemArgs A, const double *__restrict__ u,
                                                  const double *__restrict__ v, double *__restrict__ y) {
    apply_mf_element<T, kReuse>(A, u, v, y);
}

// The product at the stored linearisation asks for six blocks per SM (80 registers, 16 bytes
// spilled): 7.93 -> 7.85 ms at 128^3 against five at 92 registers; seven (72 registers, 64
// bytes spilled) measured 7.94 ms.  The other instantiations keep the compiler's own choice: an
// explicit minimum of one block let it take far more registers (the FP32 product 0.90 -> 1.08 ms).
template <>
__global__ void __launch_bounds__(128, 6) k_apply_mf<double, true>(ElemArgs A, const double *__restrict__ u,
                                                                   const double *__restrict__ v,
                                                                   double *__restrict__ y) {
    apply_mf_element<double, true>(A, u, v, y);
}

// The FP32 product (FP32 and TF32 calls) is issue-bound: compiled for ten blocks per SM (48
// registers, a 28-byte spill) it runs 0.860 -> 0.847 ms at 128^3 against nine at 56 registers.
template <>
__global__ void __launch_bounds__(128, 10) k_apply_mf<float, false>(ElemArgs A, const double *__restrict__ u,
                                                                    const double *__restrict__ v,
                                                                    double *__restrict__ y) {
    apply_mf_element<float, false>(A, u, v, y);
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
    gauss_kinematics<T>(A.conn, A.coords, u, e, l, node, K, cu, A.geom);
    ElemMaterial mt = element_material(A.mats, A.phase, A.E_elem, e, true);
    T Q[3][3];
    const bool ok = residual_moment<T>(K, mt.law, from_double<T>(mt.lam), from_double<T>(mt.mu), Q);
    T f[3];
    nodal_force_of_moment(Q, K, l, f);
    double d = R[3 * (int64_t)node] * to_double(f[0]) + R[3 * (int64_t)node + 1] * to_double(f[1]) +
               R[3 * (int64_t)node + 2] * to_double(f[2]);
    d = allreduce8(d);
    if (active && l == 0) {
        uint32_t bits = (positive(K.dJ) ? 0u : JETSCI_FLAG_BAD_ELEMENT) | (ok ? 0u : JETSCI_FLAG_BAD_STATE) |
                        (finite_t(d) ? 0u : JETSCI_FLAG_NONFINITE);
        raise_flag(A.flags, bits);
        g[e] = d;
    }
}

// The same gradient from the element vectors a residual call with E_elem kept: R_e(u; E) =
// E_e R_e(u; 1), so dL/dE_e = R[dofs_e] . R_e / E_e, a gather and a dot per element (lane =
// local node) with no element arithmetic.
__global__ void __launch_bounds__(128) k_material_grad_stored(const int32_t *__restrict__ conn,
                                                              const double *__restrict__ re,
                                                              const double *__restrict__ E_elem, int64_t n,
                                                              const double *__restrict__ R, double *__restrict__ g,
                                                              uint32_t *flags) {
    const int a = threadIdx.x & 7;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool active = slot < n;
    const int64_t e = active ? slot : n - 1;
    const int64_t node = conn[8 * e + a];
    const double *r = re + 24 * e + 3 * a;
    double d = R[3 * node] * r[0] + R[3 * node + 1] * r[1] + R[3 * node + 2] * r[2];
    d = allreduce8(d);
    if (active && a == 0) {
        const double ge = d / E_elem[e];
        if (!isfinite(ge)) raise_flag(flags, JETSCI_FLAG_NONFINITE);
        g[e] = ge;
    }
}

// ---------------------------------------------------------------------------- geometry cache
// Fills the mesh's per-element reference geometry (element.cuh) with the same arithmetic the
// kernels use when they form it from the coordinates.
__global__ void __launch_bounds__(128) k_fill_geom(const int32_t *__restrict__ conn, const double *__restrict__ coords,
                                                   int64_t n, double *__restrict__ geom) {
    const int l = threadIdx.x & 7;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool active = slot < n;
    const int64_t e = active ? slot : n - 1;
    int32_t node;
    GaussKinematics<double> K;
    double cu[3];
    gauss_kinematics_coords<double>(conn, coords, nullptr, e, l, node, K, cu);
    double A0[3][3];
    adj_gram(K.aJ, A0);
    const double rdJ = 1.0 / K.dJ;  // (the cache holds A0 / det Jp)
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) A0[i][j] *= rdJ;
    if (!active) return;
    double *p = geom + (int64_t)kGeomFields * 8 * e + 2 * l;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            *geom_field(p, kGeomJp + 3 * i + j) = K.Jp[i][j];
            *geom_field(p, kGeomAJ + 3 * i + j) = K.aJ[i][j];
        }
    *geom_field(p, kGeomDJ) = K.dJ;
    *geom_field(p, kGeomDJ + 1) = 0.0;
    *geom_field(p, kGeomA0 + 0) = A0[0][0];
    *geom_field(p, kGeomA0 + 1) = A0[1][1];
    *geom_field(p, kGeomA0 + 2) = A0[2][2];
    *geom_field(p, kGeomA0 + 3) = A0[1][2];
    *geom_field(p, kGeomA0 + 4) = A0[0][2];
    *geom_field(p, kGeomA0 + 5) = A0[0][1];
}

// L_ab (element.cuh, kLap*): each lane forms its Gauss point's share detJ G_a . G_b =
// (adj(Jp)^T n_a) . (adj(Jp)^T n_b) / (512 det Jp), n_a = 8 dN_a/dxi, and the element's 8 lanes
// sum the shares by butterfly (the same sum in every lane); lane l writes pairs l, l + 8, ...
__global__ void __launch_bounds__(128) k_fill_lap(const int32_t *__restrict__ conn, const double *__restrict__ coords,
                                                  int64_t n, double *__restrict__ lap) {
    const int l = threadIdx.x & 7;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool active = slot < n;
    const int64_t e = active ? slot : n - 1;
    int32_t node;
    GaussKinematics<double> K;
    double cu[3];
    gauss_kinematics_coords<double>(conn, coords, nullptr, e, l, node, K, cu);
    const double xp = (l & 1) ? kGaussP : kGaussM, xm = (l & 1) ? kGaussM : kGaussP;
    const double yp = (l & 2) ? kGaussP : kGaussM, ym = (l & 2) ? kGaussM : kGaussP;
    const double zp = (l & 4) ? kGaussP : kGaussM, zm = (l & 4) ? kGaussM : kGaussP;
    double v[8][3];
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const int bits = hex_bits_of_node(a);
        const double fx = (bits & 1) ? xp : xm, fy = (bits & 2) ? yp : ym, fz = (bits & 4) ? zp : zm;
        const double n0 = (bits & 1) ? fy * fz : -fy * fz, n1 = (bits & 2) ? fx * fz : -fx * fz;
        const double n2 = (bits & 4) ? fx * fy : -fx * fy;
#pragma unroll
        for (int j = 0; j < 3; j++) v[a][j] = K.aJ[0][j] * n0 + K.aJ[1][j] * n1 + K.aJ[2][j] * n2;
    }
    const double w = 1.0 / (512.0 * K.dJ);
    double *out = lap + (int64_t)kLapPairs * e;
    int p = 0;
#pragma unroll
    for (int a = 0; a < 8; a++)
#pragma unroll
        for (int b = a; b < 8; b++) {
            const int idx = (a == b) ? kLapDiag + a : p++;
            double x = (v[a][0] * v[b][0] + v[a][1] * v[b][1] + v[a][2] * v[b][2]) * w;
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            x += __shfl_xor_sync(0xffffffffu, x, 4);
            if (active && (idx & 7) == l) out[idx] = x;
        }
}

jetsci_status launch_fill_geom(jetsci_mesh m, cudaStream_t s) {
    if (m->n_elem == 0) return JETSCI_OK;
    const unsigned grid = (unsigned)((8 * m->n_elem + 127) / 128);
    k_fill_geom<<<grid, 128, 0, s>>>(m->d_conn, m->d_coords, m->n_elem, m->d_geom);
    JETSCI_CUDA_TRY(cudaGetLastError());
    k_fill_lap<<<grid, 128, 0, s>>>(m->d_conn, m->d_coords, m->n_elem, m->d_lap);
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

// ---------------------------------------------------------------------------- block insertion
// Caller blocks Ke[e][24][24] go through the row pass of the row-gather assembly: each CSR row
// is the element-ordered sum of its blocks, written once (no clearing, no colouring).
jetsci_status launch_insert_blocks(jetsci_mesh m, const void *Ke, void *vals, bool fp32, cudaStream_t s) {
    if (reinterpret_cast<uintptr_t>(Ke) % 16 != 0) return fail(JETSCI_ERR_ARG, "Ke_dev must be 16-byte aligned");
    if (fp32) return launch_gather_rows<float>(m, (const float *)Ke, nullptr, (float *)vals, nullptr, s);
    return launch_gather_rows<double>(m, (const double *)Ke, nullptr, (double *)vals, nullptr, s);
}

// ---------------------------------------------------------------------------- launchers
static ElemArgs make_args(jetsci_mesh m, const double *E_elem) {
    ElemArgs A;
    A.conn = m->d_conn;
    A.coords = m->d_coords;
    A.geom = m->d_geom;
    A.lap = m->d_lap;
    A.lin = nullptr;
    A.order = nullptr;
    A.re = nullptr;
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
    // One launch per colour.  Running all colours of an element-id chunk before the next chunk
    // (so that the nodal data the colours share stays in L2) was measured slower at every chunk
    // size at 128^3 (FP32 residual 0.70 ms against 0.72 / 0.98 / 2.08 ms for chunks of 2^20 /
    // 2^18 / 2^16 elements; matrix-free FP32 0.90 against 0.95 / 1.21 / 2.28 ms): the launches
    // and their tails cost more than the DRAM re-reads of a colour-major order.
    for_each_colour(m, [&](const int32_t *elems, int64_t n) {
        A.elems = elems;
        A.n = n;
        unsigned grid = (unsigned)((8 * A.n + 127) / 128);
        if (A.re)
            k_residual<T, true><<<grid, 128, 0, s>>>(A, u, R);
        else
            k_residual<T, false><<<grid, 128, 0, s>>>(A, u, R);
    });
}

jetsci_status launch_residual(jetsci_mesh m, const double *u, double *R, int precision,
                              const double *E_elem, cudaStream_t s) {
    JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
    ElemArgs A = make_args(m, E_elem);
    if (E_elem) {
        // keep R_e for jetsci_material_grad at this state (u = NULL there); the surrogate
        // residual keeps none, so it leaves no element vectors to use
        m->re_valid = precision != JETSCI_SURROGATE;
        m->re_E = E_elem;
        m->re_prec = precision == JETSCI_TF32 ? JETSCI_FP32 : precision;
        if (m->re_valid) A.re = m->d_re;
    }
    if (precision == JETSCI_FP64) {
        A.lin = m->d_lin;  // the linearisation at u, for matrix-free products at this state
        m->lin_valid = true;
        m->lin_E = E_elem;
        residual_colours<double>(m, A, u, R, s);
    }
    else if (precision == JETSCI_FP32 || precision == JETSCI_TF32)
        residual_colours<float>(m, A, u, R, s);
    else if (precision == JETSCI_DF64) {
        A.lin = m->d_lin;  // the linearisation at u (two-float values rounded to double)
        m->lin_valid = true;
        m->lin_E = E_elem;
        residual_colours<df64>(m, A, u, R, s);
    }
    else if (precision == JETSCI_SURROGATE)
        return launch_surrogate(m, u, nullptr, R, s);
    else
        return fail(JETSCI_ERR_UNSUPPORTED, "precision not implemented for the residual");
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

template <typename T, typename VT, bool kRows>
static jetsci_status tangent_setup(size_t smem) {
    // The FP64 tangent needs 56 KB of shared memory per 8-element block: take the largest carveout.
    return kernel_attrs_once<k_tangent<T, VT, kRows>>(smem, true);
}

template <typename T, typename VT>
static jetsci_status tangent_colours(jetsci_mesh m, ElemArgs A, const double *u, VT *vals, double *R,
                                     cudaStream_t s) {
    const size_t smem = tangent_smem_bytes<T>(false);
    if (jetsci_status st = tangent_setup<T, VT, false>(smem)) return st;
    // One launch per colour.  Splitting colours into L2-sized chunks (chunk-major order) was
    // measured slower at 128^3 for every precision: the 8x more, smaller launches lose more
    // in launch tails than the L2-resident read-modify-writes gain.
    for (int c = 0; c < m->n_colours; c++) {
        const int64_t n = m->colour_ptr[c + 1] - m->colour_ptr[c];
        if (n <= 0) continue;
        A.elems = m->d_colour_elems + m->colour_ptr[c];
        A.n = n;
        A.order = m->d_item_order + 224 * (int64_t)c;
        unsigned grid = (unsigned)((A.n + TangentLayout<T>::kElems - 1) / TangentLayout<T>::kElems);
        k_tangent<T, VT, false><<<grid, TangentLayout<T>::kThreads, smem, s>>>(A, u, m->d_rowptr, m->d_slot,
                                                                              m->d_first, vals, R);
    }
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

// Row-gather assembly: the element pass writes every element's 24 x 24 rows and residual
// vectors to the mesh's workspace in one launch, the row pass forms each CSR row and R entry once.
// (Running both passes chunk by chunk, one slab of 16,384 elements at a time with the element
// rows in a ring that L2 holds, was measured slower at 128^3: 5.93 ms against 4.19 ms for the FP32
// tangent, 5.55 / 7.86 ms with chunks of 32,768 / 8,192 elements.  The row pass is bound by load
// latency, not DRAM, so reading from L2 gains little, and 256 launches of one or two waves each
// add their tails.)
template <typename T, typename VT>
static jetsci_status tangent_rows(jetsci_mesh m, ElemArgs A, const double *u, VT *vals, double *R,
                                  cudaStream_t s) {
    void *ws = nullptr;
    double *Re = nullptr;
    if (jetsci_status st = ensure_block_workspace(m, blk_full_bytes(m->n_elem, sizeof(VT)), s, &ws, &Re)) return st;
    if (!R) Re = nullptr;
    if (m->n_elem > 0) {
        using L = TangentLayout<T>;
        const size_t smem = tangent_smem_bytes<T>(true);
        if (jetsci_status st = tangent_setup<T, VT, true>(smem)) return st;
        A.elems = nullptr;
        A.n = m->n_elem;
        const unsigned grid = (unsigned)((A.n + L::kElems - 1) / L::kElems);
        k_tangent<T, VT, true><<<grid, L::kThreads, smem, s>>>(A, u, nullptr, nullptr, nullptr, (VT *)ws, Re);
        JETSCI_CUDA_TRY(cudaGetLastError());
    }
    return launch_gather_rows<VT>(m, (const VT *)ws, Re, vals, R, s);
}

jetsci_status launch_tangent(jetsci_mesh m, const double *u, void *vals, double *R, int precision,
                             const double *E_elem, cudaStream_t s) {
    ElemArgs A = make_args(m, E_elem);
    // FP64 needs no clearing of vals (first writers store, TangentLayout::kFirstWrites).
    if (precision == JETSCI_FP64) {
        if (R) JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
        A.lin = m->d_lin;  // the linearisation at u, for matrix-free products at this state
        m->lin_valid = true;
        m->lin_E = E_elem;
        return tangent_colours<double, double>(m, A, u, (double *)vals, R, s);
    }
    if (precision == JETSCI_FP32) return tangent_rows<float, float>(m, A, u, (float *)vals, R, s);
    if (precision == JETSCI_DF64) {
        JETSCI_CUDA_TRY(cudaMemsetAsync(vals, 0, m->nnz * sizeof(double), s));
        if (R) JETSCI_CUDA_TRY(cudaMemsetAsync(R, 0, m->n_dof * sizeof(double), s));
        A.lin = m->d_lin;  // the linearisation at u (two-float values rounded to double)
        m->lin_valid = true;
        m->lin_E = E_elem;
        return tangent_colours<df64, double>(m, A, u, (double *)vals, R, s);
    }
    if (precision == JETSCI_TF32) return launch_tf32(m, u, (float *)vals, R, E_elem, s);
    if (precision == JETSCI_SURROGATE) return launch_surrogate(m, u, (float *)vals, R, s);
    return fail(JETSCI_ERR_UNSUPPORTED, "precision not implemented for the tangent");
}

template <typename T, bool kReuse = false>
static void apply_colours(jetsci_mesh m, ElemArgs A, const double *u, const double *v, double *y,
                          cudaStream_t s) {
    for_each_colour(m, [&](const int32_t *elems, int64_t n) {  // (one launch per colour: see residual_colours)
        A.elems = elems;
        A.n = n;
        unsigned grid = (unsigned)((8 * A.n + 127) / 128);
        k_apply_mf<T, kReuse><<<grid, 128, 0, s>>>(A, u, v, y);
    });
}

// The matrix-free product forms no element stiffness: per Gauss point it is 3 x 3 algebra between
// the sum-factorised gradient of v and the nodal forces, with no contraction for the tensor cores
// to take.  TF32 therefore runs the FP32 product (as the TF32 residual runs the FP32 residual);
// forming K_e on the tensor cores to multiply it by v_e was measured 5.8x slower at 128^3.
jetsci_status launch_apply_mf(jetsci_mesh m, const double *u, const double *v, double *y, int precision,
                              const double *E_elem, cudaStream_t s) {
    if (precision == JETSCI_TF32) precision = JETSCI_FP32;
    JETSCI_CUDA_TRY(cudaMemsetAsync(y, 0, m->n_dof * sizeof(double), s));
    ElemArgs A = make_args(m, E_elem);
    if (!u) {  // at the stored linearisation (checked by the caller), in FP64 or two-float arithmetic
        A.lin = m->d_lin;
        if (precision == JETSCI_DF64)
            apply_colours<df64, true>(m, A, nullptr, v, y, s);
        else
            apply_colours<double, true>(m, A, nullptr, v, y, s);
    } else if (precision == JETSCI_FP64)
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
    if (!u) {  // from the element vectors of the last residual call with E_elem (checked by the caller)
        k_material_grad_stored<<<grid, 128, 0, s>>>(m->d_conn, m->d_re, E_elem, A.n, R, g, m->d_flags);
        JETSCI_CUDA_TRY(cudaGetLastError());
        return JETSCI_OK;
    }
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
