// Device-side element arithmetic for hex8 / 2x2x2 Gauss, shared by the assembly,
// matrix-free and adjoint kernels.
//
// Layout: eight consecutive lanes of a warp own one element.  Lane l (0..7) stands for
// Gauss point q = l (xi = +-g by bit 0, eta by bit 1, zeta by bit 2, g = 1/sqrt 3; the
// paper's per-element quadrature, Section III-B) and, for gathers and scatters, for the
// element node whose reference coordinates carry the same bit pattern, i.e. hex8 local
// node kPerm[l].
//
// Geometry and displacement fields are trilinear, f(xi) = sum_m c_m mono_m(xi) over the
// monomials m in {1, xi, eta, xi eta, zeta, xi zeta, eta zeta, xi eta zeta} (bit pattern
// of m = which coordinates appear).  A 3-stage shuffle butterfly over the eight lanes
// turns nodal values into 8*c_m held by lane m; it runs in FP64 on the gathered data, so
// the differences that carry the element's small size and strain are exact before any
// conversion to a lower-precision element type.  Reference derivatives at the lane's
// Gauss point then need four coefficients per direction.  The transposed butterfly
// turns per-Gauss-point stress moments back into nodal forces.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

#include "df64.cuh"
#include "jetsci_internal.h"

namespace jetsci {

constexpr unsigned kFull = 0xffffffffu;

// Voigt component a in [11, 22, 33, 23, 13, 12] -> tensor indices (I, J); constexpr so that
// unrolled loops index register arrays with compile-time indices.
__host__ __device__ constexpr int voigt_i(int a) { return a == 1 ? 1 : a == 2 ? 2 : a == 3 ? 1 : 0; }
__host__ __device__ constexpr int voigt_j(int a) { return a == 0 ? 0 : a == 1 ? 1 : a == 5 ? 1 : 2; }

__device__ __forceinline__ int hex_node_of_lane(int l) {
    // binary (xi, eta, zeta) bit pattern -> hex8 local node number
    return (0x67542310 >> (4 * l)) & 0xF;
}

template <typename T>
__device__ __forceinline__ T shfl8(T v, int src) {
    return __shfl_sync(kFull, v, src, 8);
}

template <typename T>
__device__ __forceinline__ T shfl_xor8(T v, int mask) {
    return __shfl_xor_sync(kFull, v, mask, 8);
}

template <>
__device__ __forceinline__ df64 shfl8<df64>(df64 v, int src) {
    return shfl_df(v, src, 8);
}

template <>
__device__ __forceinline__ df64 shfl_xor8<df64>(df64 v, int mask) {
    return shfl_xor_df(v, mask, 8);
}

// x with its sign flipped when neg: by integer sign-bit operations, so that the butterflies below
// (x - p on some lanes of a warp, x + p on the others) issue one addition of the partner's value
// with the sign each lane needs; x - p is x + (-p) exactly, so the results are unchanged.
__device__ __forceinline__ float neg_if(float x, bool neg) {
    return __uint_as_float(__float_as_uint(x) ^ (neg ? 0x80000000u : 0u));
}
__device__ __forceinline__ double neg_if(double x, bool neg) {
    return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}
__device__ __forceinline__ df64 neg_if(df64 x, bool neg) { return df64(neg_if(x.h, neg), neg_if(x.l, neg)); }

// x > 0 and isfinite(x).  For doubles these test the bit pattern with integer operations: an
// FP64 comparison issues on the FP64 pipe, whose slots the FP64 element kernels need for their
// arithmetic.  positive is false for NaN and for both zeros, as the comparison is.
__device__ __forceinline__ bool positive(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool positive(float x) { return x > 0.0f; }
__device__ __forceinline__ bool positive(df64 x) { return x.h > 0.0f || (x.h == 0.0f && x.l > 0.0f); }
__device__ __forceinline__ bool finite_t(double x) { return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff; }
__device__ __forceinline__ bool finite_t(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_t(df64 x) { return isfinite(x); }

// Nodal values (lane = node in binary order) -> 8 * monomial coefficient (lane = monomial).
__device__ __forceinline__ double butterfly_forward(double v, int l) {
#pragma unroll
    for (int s = 1; s < 8; s <<= 1) {
        const double p = shfl_xor8(v, s);
        v = v + neg_if(p, (l & s) != 0);  // v - p where bit s of l is set, v + p elsewhere
    }
    return v;
}

// Conversions between double storage and the element type T.  For FP32 and two-float
// elements they use integer/FP32 instructions only (B300's FP64 pipe is 1/64 of FP32).
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return f2d_bits(x); }
__device__ __forceinline__ double to_double(df64 x) { return df_to_double(x); }

template <typename T>
__device__ __forceinline__ T from_double(double x);
template <>
__device__ __forceinline__ double from_double<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_double<float>(double x) {
    const df64 s = split_double(x);
    return __fadd_rn(s.h, s.l);
}
template <>
__device__ __forceinline__ df64 from_double<df64>(double x) { return split_double(x); }

template <typename VT, typename T>
__device__ __forceinline__ VT store_as(T x) { return (VT)x; }
template <>
__device__ __forceinline__ double store_as<double, df64>(df64 x) { return df_to_double(x); }

// 8 * monomial coefficient (lane = monomial) in the element type from nodal doubles (lane =
// node).  FP64: the butterfly in FP64.  Two-float: FP64 butterfly, integer split.  FP32: the
// butterfly in FP32 of the values less the element's first one (below), so the coefficients
// (differences of nearby nodal values) keep full FP32 relative accuracy.
template <typename T>
__device__ __forceinline__ T monomial_coeff(double v, int l);
template <>
__device__ __forceinline__ double monomial_coeff<double>(double v, int l) { return butterfly_forward(v, l); }
template <>
__device__ __forceinline__ df64 monomial_coeff<df64>(double v, int l) { return split_double(butterfly_forward(v, l)); }
// FP32 elements take the butterfly of v - v_0, v_0 the value at the element's lane 0: every
// coefficient but the constant one (lane 0, which no caller reads) sums the nodes with weights
// of zero sum, so the shift leaves it unchanged.  v - v_0 is of the element's size, one FP64
// subtraction exact to 2^-53 of |v|, so one rounding to FP32 and a plain FP32 butterfly keep
// FP32 accuracy at about 20 instructions per value, against about 55 for the two-float
// butterfly of v.
template <>
__device__ __forceinline__ float monomial_coeff<float>(double v, int l) {
    const double v0 = __shfl_sync(kFull, v, 0, 8);
    float x = from_double<float>(v - v0);
#pragma unroll
    for (int s = 1; s < 8; s <<= 1) {
        const float p = shfl_xor8(x, s);
        x = x + neg_if(p, (l & s) != 0);  // x - p where bit s of l is set, x + p elsewhere
    }
    return x;
}

// Transpose of the forward butterfly: lane m holds a monomial moment, result at lane l
// (node in binary order) is sum_m mono_m(node l) * moment_m.
template <typename T>
__device__ __forceinline__ T butterfly_transpose(T v, int l) {
#pragma unroll
    for (int s = 1; s < 8; s <<= 1) {
        const T p = shfl_xor8(v, s);
        v = v + neg_if(p, (l & s) == 0);  // v + p where bit s of l is set, v - p elsewhere
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T allreduce8(T v) {
    v += shfl_xor8(v, 1);
    v += shfl_xor8(v, 2);
    v += shfl_xor8(v, 4);
    return v;
}

// Reduce-scatter over the eight lanes of an element: lane l receives sum over lanes of v[l].
// Each exchange stage keeps the half of the vector selected by one bit of l and adds the
// partner's copy of it, so 7 additions and 7 exchanges replace 8 separate all-reduces.
template <typename T>
__device__ __forceinline__ T reduce_scatter8(const T v[8], int l) {
    const bool h4 = l & 4, h2 = l & 2, h1 = l & 1;
    T r4[4], r2[2];
#pragma unroll
    for (int j = 0; j < 4; j++) r4[j] = (h4 ? v[4 + j] : v[j]) + shfl_xor8(h4 ? v[j] : v[4 + j], 4);
#pragma unroll
    for (int j = 0; j < 2; j++) r2[j] = (h2 ? r4[2 + j] : r4[j]) + shfl_xor8(h2 ? r4[j] : r4[2 + j], 2);
    return (h1 ? r2[1] : r2[0]) + shfl_xor8(h1 ? r2[0] : r2[1], 1);
}

// Reference-coordinate bit pattern (xi, eta, zeta) of hex8 local node a: {0,1,3,2,4,5,7,6}.
__host__ __device__ constexpr int hex_bits_of_node(int a) { return a ^ ((a >> 1) & 1); }

// Gauss coordinate g = 1/sqrt 3 and the values that products of two of the lane's Gauss
// coordinates (each +-g) and the factors 1 +- g take, rounded as the FP64 operations round them.
// FP64 elements select these by sign instead of computing them: B300's FP64 pipe bounds the
// FP64 kernels, and the selection runs on the integer pipes with bit-identical results.
constexpr double kGaussG = 0.57735026918962576451;
constexpr double kGaussG2 = kGaussG * kGaussG;                      // (+-g)(+-g) = +-g^2
constexpr double kGaussP = 1.0 + kGaussG, kGaussM = 1.0 - kGaussG;  // 1 +- g
constexpr double kGaussPP = kGaussP * kGaussP, kGaussPM = kGaussP * kGaussM, kGaussMM = kGaussM * kGaussM;

// a b for two Gauss coordinates a, b in {+g, -g}: +-g^2 with the sign of a b.
template <typename T>
__device__ __forceinline__ T gauss_coord_product(T a, T b) { return a * b; }
template <>
__device__ __forceinline__ double gauss_coord_product<double>(double a, double b) {
    const int s = (__double2hiint(a) ^ __double2hiint(b)) & (int)0x80000000;
    return __hiloint2double(__double2hiint(kGaussG2) | s, __double2loint(kGaussG2));
}

// 8 * reference derivatives at the lane's Gauss point from 8 * monomial coefficients held
// by lanes 1..7 (component held by the calling lane in `c`):
//   d/dxi   = c_xi   + c_xieta eta + c_xizeta zeta + c_xietazeta eta zeta
//   d/deta  = c_eta  + c_xieta xi  + c_etazeta zeta + c_xietazeta xi zeta
//   d/dzeta = c_zeta + c_xizeta xi + c_etazeta eta  + c_xietazeta xi eta
template <typename T>
__device__ __forceinline__ void ref_gradient(T c, T xi, T eta, T zeta, T out[3]) {
    T c1 = shfl8(c, 1), c2 = shfl8(c, 2), c3 = shfl8(c, 3), c4 = shfl8(c, 4);
    T c5 = shfl8(c, 5), c6 = shfl8(c, 6), c7 = shfl8(c, 7);
    out[0] = c1 + c3 * eta + c5 * zeta + c7 * gauss_coord_product(eta, zeta);
    out[1] = c2 + c3 * xi + c6 * zeta + c7 * gauss_coord_product(xi, zeta);
    out[2] = c4 + c5 * xi + c6 * eta + c7 * gauss_coord_product(xi, eta);
}

template <typename T>
__device__ __forceinline__ T det3(const T A[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
           A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// Adjugate (transpose of the cofactor matrix): A^-1 = adj / det.
template <typename T>
__device__ __forceinline__ void adj3(const T A[3][3], T B[3][3]) {
    B[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    B[0][1] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
    B[0][2] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
    B[1][0] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    B[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    B[1][2] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
    B[2][0] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    B[2][1] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
    B[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
}

template <typename T>
__device__ __forceinline__ T my_log(T x);
// FP64 ln x.  Near 1, where the volume ratios of these elements lie (|x - 1| < 1/16), the
// alternating series ln(1 + t) = t - t^2/2 + t^3/3 - ... in t = x - 1 (exact there, Sterbenz),
// thirteen terms by Horner's rule: the truncation t^13/14 is below 2^-53 of ln(1 + t), and it
// costs 14 FP64 operations against about 35 FP64-pipe slots for the library log, which serves
// every other x.  The range test reads the bit pattern (no FP64 comparison).
template <>
__device__ __forceinline__ double my_log<double>(double x) {
    const double t = x - 1.0;
    if ((__double_as_longlong(t) & 0x7fffffffffffffffll) < 0x3fb0000000000000ll) {  // |t| < 1/16
        double p = 1.0 / 13.0;
#pragma unroll
        for (int n = 12; n >= 1; n--) p = fma(p, t, ((n & 1) ? 1.0 : -1.0) / (double)n);
        return t * p;
    }
    return log(x);
}
template <>
__device__ __forceinline__ float my_log<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ df64 my_log<df64>(df64 x) { return df_log(x); }

template <typename T>
__device__ __forceinline__ T my_rcp(T x) { return T(1) / x; }
template <>
__device__ __forceinline__ df64 my_rcp<df64>(df64 x) { return df_rcp(x); }

// a * b + c in the element type (a fused multiply-add for FP64/FP32, one renormalisation
// for two-float values).
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ df64 fma_t(df64 a, df64 b, df64 c) { return df_fma(a, b, c); }
// Running-sum steps (acc_t) and their final normalisation (acc_norm): fma_t for FP64 and FP32;
// two-float sums skip the per-step renormalisation (df64.cuh, df_fma_acc).
__device__ __forceinline__ double acc_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float acc_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ df64 acc_t(df64 a, df64 b, df64 c) { return df_fma_acc(a, b, c); }
__device__ __forceinline__ double acc_norm(double a) { return a; }
__device__ __forceinline__ float acc_norm(float a) { return a; }
__device__ __forceinline__ df64 acc_norm(df64 a) { return df_acc_norm(a); }

// Material of element e as (law, lambda, mu) in T.
struct ElemMaterial {
    int law;
    double lam, mu;
};

// lam / mu of element e's phase (the same for any E at the phase's nu), read where it is used.
__device__ __forceinline__ double element_lam_mu(const Material *__restrict__ mats, const int32_t *__restrict__ phase,
                                                 int64_t e) {
    return __ldg(&mats[__ldg(phase + e)].lam_mu);
}

__device__ __forceinline__ ElemMaterial element_material(const Material *__restrict__ mats,
                                                         const int32_t *__restrict__ phase,
                                                         const double *__restrict__ E_elem,
                                                         int64_t e, bool unit_modulus) {
    const Material &mt = mats[phase[e]];
    ElemMaterial r;
    r.law = mt.law;
    if (unit_modulus) {
        r.lam = mt.lam1;
        r.mu = mt.mu1;
    } else if (E_elem) {
        double E = E_elem[e];
        r.lam = E * mt.lam1;
        r.mu = E * mt.mu1;
    } else {
        r.lam = mt.lam;
        r.mu = mt.mu;
    }
    return r;
}

// Per-lane kinematics at the lane's Gauss point.
//   Jp = 8 dX/dxi, aJ = adj(Jp), dJ = det(Jp)   (detJ = dJ / 512),  Du = 8 du/dxi
template <typename T>
struct GaussKinematics {
    T xi, eta, zeta;
    T Jp[3][3], aJ[3][3], dJ;
    T Du[3][3];  // 8 du/dxi
};

// Reference geometry of an element at its 8 Gauss points, kept per mesh for the FP64 kernels
// (FP64 arithmetic is the scarce resource on this GPU, HBM bandwidth is not): fields Jp (0-8),
// adj(Jp) (9-17), det Jp (18), an unused slot (19) and A0 = adj(Jp) adj(Jp)^T / det Jp (20-25:
// 00 11 22 12 02 01; the matrix-free product's reference term), stored in pairs as [element][field / 2][Gauss point][2] doubles, so that a lane
// reads two fields with one 16-byte load and an element's 8 lanes read 128 contiguous bytes.
constexpr int kGeomJp = 0, kGeomAJ = 9, kGeomDJ = 18, kGeomA0 = 20, kGeomFields = 26;
constexpr int kGeomKinPairs = 10;  // pairs holding Jp, adj(Jp) and det Jp

__device__ __forceinline__ const double *geom_point(const double *__restrict__ geom, int64_t e, int l) {
    return geom + (int64_t)kGeomFields * 8 * e + 2 * l;
}
// field f of the lane's Gauss point (p from geom_point)
__device__ __forceinline__ double *geom_field(double *p, int f) { return p + 16 * (f >> 1) + (f & 1); }
// fields 2k and 2k + 1
__device__ __forceinline__ double2 geom_pair(const double *__restrict__ p, int k) {
    return __ldg(reinterpret_cast<const double2 *>(p + 16 * k));
}

// Reference "Laplacian" of an element, kept per mesh for the tangent kernels: per node pair
// L_ab = sum_q detJ_q G_a,q . G_b,q (G_a = dN_a/dX, the reference shape-function gradient), as
// [element][36] doubles: the 28 pairs a < b in row order (0, 1), (0, 2), ..., (6, 7), then the 8
// pairs a == b.  For both laws the geometric and identity parts of the spatial tangent combine to
// c (tau + m I) = c mu F F^T (neo-Hookean: tau + m I = mu b; linear: tau = 0, m = mu), and
// (F F^T g_a) . g_b = (F G_a) . (F^-T G_b) = G_a . G_b, so the term delta_ik sum_q tg_a . g_b of
// K_ab,ik is mu L_ab: fixed by the reference geometry, whatever the deformation.
constexpr int kLapPairs = 36, kLapDiag = 28;

// Linearisation of the neo-Hookean state at the last FP64 or two-float residual or tangent call,
// kept per mesh for matrix-free products at that state, in the form those products use
// (apply_mf_element): adj(j) (0-8), alpha = (m / mu) det Jp / det j^2 (9) and
// beta = (lam / mu) det Jp / det j^2 (10) per element and Gauss point, and one padding value, in
// pairs as [element][6][Gauss point][2] doubles.
constexpr int kLinAj = 0, kLinAlpha = 9, kLinBeta = 10, kLinPairs = 6;

template <typename T>
struct LinCoeffs {
    T aj[3][3];
    T alpha, beta;
};

// The coefficients at a neo-Hookean state: adj(j), 1 / det j (rdj), det Jp (dJ), ln J and
// lam / mu (m / mu = 1 - (lam / mu) ln J).
template <typename T>
__device__ __forceinline__ void lin_coeffs(const T aj[3][3], T rdj, T dJ, T lnJ, T lam_mu, LinCoeffs<T> &c) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) c.aj[i][k] = aj[i][k];
    const T s2 = dJ * rdj * rdj;
    c.alpha = s2 * fma_t(-lam_mu, lnJ, T(1));
    c.beta = s2 * lam_mu;
}

// The coefficients of a two-float (or FP64) neo-Hookean update, stored in FP64 (two-float values
// rounded to the nearest double, about 48 significant bits either way).
template <typename T>
__device__ __forceinline__ void lin_store_t(double *__restrict__ lin, int64_t e, int l, const LinCoeffs<T> &c) {
    const double f[2 * kLinPairs] = {to_double(c.aj[0][0]), to_double(c.aj[0][1]), to_double(c.aj[0][2]),
                                     to_double(c.aj[1][0]), to_double(c.aj[1][1]), to_double(c.aj[1][2]),
                                     to_double(c.aj[2][0]), to_double(c.aj[2][1]), to_double(c.aj[2][2]),
                                     to_double(c.alpha),    to_double(c.beta),     0.0};
    double2 *p = reinterpret_cast<double2 *>(lin + (int64_t)2 * kLinPairs * 8 * e + 2 * l);
#pragma unroll
    for (int k = 0; k < kLinPairs; k++) p[8 * k] = make_double2(f[2 * k], f[2 * k + 1]);
}

// The stored coefficients in the element type T (FP64 as stored; two-float by splitting each
// double).
template <typename T>
__device__ __forceinline__ void lin_load_t(const double *__restrict__ lin, int64_t e, int l, LinCoeffs<T> &c) {
    const double2 *p = reinterpret_cast<const double2 *>(lin + (int64_t)2 * kLinPairs * 8 * e + 2 * l);
    double f[2 * kLinPairs];
#pragma unroll
    for (int k = 0; k < kLinPairs; k++) {
        const double2 v = __ldg(p + 8 * k);
        f[2 * k] = v.x;
        f[2 * k + 1] = v.y;
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.aj[i][j] = from_double<T>(f[kLinAj + 3 * i + j]);
    c.alpha = from_double<T>(f[kLinAlpha]);
    c.beta = from_double<T>(f[kLinBeta]);
}

// Kinematics at the lane's Gauss point from the lane's node's coordinates X and nodal field
// values U (gathered by the caller): coefficients (FP64 differences, element.cuh header), Jp,
// adj(Jp), det Jp and Du.
template <typename T>
__device__ __forceinline__ void gauss_kinematics_of(const double X[3], const double U[3], int l,
                                                    GaussKinematics<T> &K, T cu[3]) {
    T cx[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        cx[i] = monomial_coeff<T>(X[i], l);
        cu[i] = monomial_coeff<T>(U[i], l);
    }
    const T g = (T)kGaussG;
    K.xi = (l & 1) ? g : -g;
    K.eta = (l & 2) ? g : -g;
    K.zeta = (l & 4) ? g : -g;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        ref_gradient(cx[i], K.xi, K.eta, K.zeta, K.Jp[i]);
        ref_gradient(cu[i], K.xi, K.eta, K.zeta, K.Du[i]);
    }
    adj3(K.Jp, K.aJ);
    K.dJ = K.Jp[0][0] * K.aJ[0][0] + K.Jp[0][1] * K.aJ[1][0] + K.Jp[0][2] * K.aJ[2][0];
}

// Gathers coordinates and one nodal field for element e, forms coefficients (FP64) and the
// kinematics at the lane's Gauss point.  `node` receives the global node of the lane.
template <typename T>
__device__ __forceinline__ void gauss_kinematics_coords(const int32_t *__restrict__ conn,
                                                        const double *__restrict__ coords,
                                                        const double *__restrict__ u, int64_t e, int l,
                                                        int32_t &node, GaussKinematics<T> &K, T cu[3]) {
    node = conn[8 * e + hex_node_of_lane(l)];
    double X[3], U[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        X[i] = coords[3 * (int64_t)node + i];
        U[i] = u ? u[3 * (int64_t)node + i] : 0.0;
    }
    gauss_kinematics_of<T>(X, U, l, K, cu);
}

// The kinematics of gauss_kinematics_coords.  FP64 and two-float elements read Jp, adj(Jp) and
// det Jp from the mesh's geometry cache `geom` (FP64, filled by gauss_kinematics_coords: the
// same values for FP64; two-float elements split them, keeping the ~48 bits their own
// arithmetic would have) and gather only the nodal field; FP32 elements form them from the
// coordinates (geom is not used).  kPairs: 16-byte loads of two fields (fewer load
// instructions) or 8-byte loads of one (fewer live registers, for the register-bound tangent).
// kCachedDf64 = false: two-float elements form the geometry from the coordinates as well (the
// issue-bound two-float tangent was 1.3% slower reading the cache).
template <typename T, bool kPairs = true, bool kCachedDf64 = true>
__device__ __forceinline__ void gauss_kinematics(const int32_t *__restrict__ conn,
                                                 const double *__restrict__ coords,
                                                 const double *__restrict__ u, int64_t e, int l,
                                                 int32_t &node, GaussKinematics<T> &K, T cu[3],
                                                 const double *__restrict__ geom) {
    if constexpr (std::is_same<T, double>::value || (kCachedDf64 && std::is_same<T, df64>::value)) {
        node = conn[8 * e + hex_node_of_lane(l)];
        const T g = (T)kGaussG;
        K.xi = (l & 1) ? g : -g;
        K.eta = (l & 2) ? g : -g;
        K.zeta = (l & 4) ? g : -g;
        const double *p = geom_point(geom, e, l);
        if constexpr (kPairs) {
            double gf[2 * kGeomKinPairs];
#pragma unroll
            for (int k = 0; k < kGeomKinPairs; k++) {
                const double2 v = geom_pair(p, k);
                gf[2 * k] = v.x;
                gf[2 * k + 1] = v.y;
            }
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    K.Jp[i][j] = from_double<T>(gf[kGeomJp + 3 * i + j]);
                    K.aJ[i][j] = from_double<T>(gf[kGeomAJ + 3 * i + j]);
                }
            K.dJ = from_double<T>(gf[kGeomDJ]);
        }
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const double Ui = u ? u[3 * (int64_t)node + i] : 0.0;
            cu[i] = monomial_coeff<T>(Ui, l);
            ref_gradient(cu[i], K.xi, K.eta, K.zeta, K.Du[i]);
            if constexpr (!kPairs)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const int fj = kGeomJp + 3 * i + j, fa = kGeomAJ + 3 * i + j;
                    K.Jp[i][j] = from_double<T>(p[16 * (fj >> 1) + (fj & 1)]);
                    K.aJ[i][j] = from_double<T>(p[16 * (fa >> 1) + (fa & 1)]);
                }
        }
        if constexpr (!kPairs) K.dJ = from_double<T>(p[16 * (kGeomDJ >> 1) + (kGeomDJ & 1)]);
    } else {
        (void)geom;
        gauss_kinematics_coords<T>(conn, coords, u, e, l, node, K, cu);
    }
}

// The reference geometry of the lane's Gauss point alone (from the FP64 cache, in the element
// type): node, xi, eta, zeta, Jp, adj(Jp), det Jp; K.Du is not formed.
template <typename T>
__device__ __forceinline__ void gauss_geometry(const int32_t *__restrict__ conn, const double *__restrict__ geom,
                                               int64_t e, int l, int32_t &node, GaussKinematics<T> &K) {
    node = conn[8 * e + hex_node_of_lane(l)];
    const T g = (T)kGaussG;
    K.xi = (l & 1) ? g : -g;
    K.eta = (l & 2) ? g : -g;
    K.zeta = (l & 4) ? g : -g;
    const double *p = geom_point(geom, e, l);
    double gf[2 * kGeomKinPairs];
#pragma unroll
    for (int k = 0; k < kGeomKinPairs; k++) {
        const double2 v = geom_pair(p, k);
        gf[2 * k] = v.x;
        gf[2 * k + 1] = v.y;
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            K.Jp[i][j] = from_double<T>(gf[kGeomJp + 3 * i + j]);
            K.aJ[i][j] = from_double<T>(gf[kGeomAJ + 3 * i + j]);
        }
    K.dJ = from_double<T>(gf[kGeomDJ]);
}

// A0 = adj(Jp) adj(Jp)^T of the matrix-free neo-Hookean product (symmetric).
template <typename T>
__device__ __forceinline__ void adj_gram(const T aJ[3][3], T A0[3][3]) {
#pragma unroll
    for (int n = 0; n < 3; n++)
#pragma unroll
        for (int d = n; d < 3; d++) {
            const T t = aJ[n][0] * aJ[d][0] + aJ[n][1] * aJ[d][1] + aJ[n][2] * aJ[d][2];
            A0[n][d] = t;
            A0[d][n] = t;
        }
}

// Displacement gradient H = grad_X u = (8 du/dxi) Jp^-1 at the lane's Gauss point.
template <typename T>
__device__ __forceinline__ void displacement_gradient(const GaussKinematics<T> &K, T H[3][3]) {
    const T rdJ = my_rcp(K.dJ);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            H[i][j] = (K.Du[i][0] * K.aJ[0][j] + K.Du[i][1] * K.aJ[1][j] + K.Du[i][2] * K.aJ[2][j]) * rdJ;
}

// Reference gradient of a second nodal field v at the lane's Gauss point: Dv = 8 dv/dxi.
template <typename T>
__device__ __forceinline__ void field_ref_gradient(const double *__restrict__ v, int32_t node, int l,
                                                   const GaussKinematics<T> &K, T Dv[3][3]) {
    T cv[3];
#pragma unroll
    for (int i = 0; i < 3; i++) cv[i] = monomial_coeff<T>(v[3 * (int64_t)node + i], l);
#pragma unroll
    for (int i = 0; i < 3; i++) ref_gradient(cv[i], K.xi, K.eta, K.zeta, Dv[i]);
}

// Gradient of a second nodal field v with the same geometry: Hv = (8 dv/dxi) Jp^-1.
template <typename T>
__device__ __forceinline__ void field_gradient(const double *__restrict__ v, int32_t node, int l,
                                               const GaussKinematics<T> &K, T Hv[3][3]) {
    T Dv[3][3];
    field_ref_gradient<T>(v, node, l, K, Dv);
    T rdJ = my_rcp(K.dJ);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            Hv[i][j] = (Dv[i][0] * K.aJ[0][j] + Dv[i][1] * K.aJ[1][j] + Dv[i][2] * K.aJ[2][j]) * rdJ;
}

// Constitutive state at one Gauss point: F, F^-1 (identity for the linear law), the second
// and first Piola-Kirchhoff stresses S and P, lam and m = mu - lam lnJ (the push-forward of
// the neo-Hookean CC is lam I(x)I + 2m Isym), ok = (J > 0).
template <typename T>
struct Constitutive {
    T P[3][3];
    T S[3][3];
    T Fi[3][3];
    T F[3][3];
    T lam, m;
    bool ok;
};

template <typename T>
__device__ __forceinline__ void constitutive(int law, T lam, T mu, const T H[3][3], Constitutive<T> &c) {
    c.ok = true;
    if (law == JETSCI_LINEAR_ELASTIC) {
        T tr = H[0][0] + H[1][1] + H[2][2];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                T s = mu * (H[i][j] + H[j][i]);
                if (i == j) s += lam * tr;
                c.P[i][j] = s;
                c.S[i][j] = s;
                c.F[i][j] = (i == j) ? T(1) : T(0);
                c.Fi[i][j] = c.F[i][j];
            }
        c.lam = lam;
        c.m = mu;
        return;
    }
    // compressible neo-Hookean: S = mu I + (lam lnJ - mu) C^-1
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.F[i][j] = ((i == j) ? T(1) : T(0)) + H[i][j];
    T aF[3][3];
    adj3(c.F, aF);
    T J = c.F[0][0] * aF[0][0] + c.F[0][1] * aF[1][0] + c.F[0][2] * aF[2][0];
    c.ok = positive(J);
    T Js = c.ok ? J : T(1);
    T rJ = my_rcp(Js);
    T lnJ = my_log(Js);
    // C^-1 = F^-1 F^-T with F^-1 = adj(F) / J
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.Fi[i][j] = aF[i][j] * rJ;
    c.lam = lam;
    c.m = mu - lam * lnJ;
    T Ci[3][3];
#pragma unroll
    for (int I = 0; I < 3; I++)
#pragma unroll
        for (int K = I; K < 3; K++) {
            T s = c.Fi[I][0] * c.Fi[K][0] + c.Fi[I][1] * c.Fi[K][1] + c.Fi[I][2] * c.Fi[K][2];
            Ci[I][K] = s;
            Ci[K][I] = s;
        }
    T a = lam * lnJ - mu;
#pragma unroll
    for (int I = 0; I < 3; I++)
#pragma unroll
        for (int K = 0; K < 3; K++) c.S[I][K] = a * Ci[I][K] + ((I == K) ? mu : T(0));
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int J2 = 0; J2 < 3; J2++)
            c.P[i][J2] = c.F[i][0] * c.S[0][J2] + c.F[i][1] * c.S[1][J2] + c.F[i][2] * c.S[2][J2];
}

// Neo-Hookean state at the lane's Gauss point from the deformed Jacobian j = Jp + Du = 8 dx/dxi:
// F = j Jp^-1, J = det j / det Jp (one reciprocal serves both determinants), m = mu - lam lnJ
// and the Kirchhoff stress tau = F S F^T = mu (F F^T - I) + lam lnJ I with F F^T formed from
// F det(Jp) = j adj(Jp).  ok = (J > 0); otherwise lnJ is taken as 0.
template <typename T>
struct NeoHookeanState {
    T jm[3][3], aj[3][3];  // j and adj(j)
    T rdj, rdJ;            // 1 / det j, 1 / det Jp
    T lnJ, m;
    T tau[3][3];
    bool ok;
};

template <typename T>
__device__ __forceinline__ void neo_hookean_state(const GaussKinematics<T> &K, T lam, T mu, NeoHookeanState<T> &s) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int d = 0; d < 3; d++) s.jm[i][d] = K.Jp[i][d] + K.Du[i][d];
    adj3(s.jm, s.aj);
    const T dj = s.jm[0][0] * s.aj[0][0] + s.jm[0][1] * s.aj[1][0] + s.jm[0][2] * s.aj[2][0];
    const T pj = K.dJ * dj;
    s.ok = positive(pj);
    const T r = my_rcp(s.ok ? pj : T(1));
    s.rdj = K.dJ * r;
    s.rdJ = dj * r;
    s.lnJ = my_log(s.ok ? dj * s.rdJ : T(1));
    s.m = mu - lam * s.lnJ;
    T Fd[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) Fd[i][k] = s.jm[i][0] * K.aJ[0][k] + s.jm[i][1] * K.aJ[1][k] + s.jm[i][2] * K.aJ[2][k];
    const T mb = mu * s.rdJ * s.rdJ, diag = lam * s.lnJ - mu;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = i; k < 3; k++) {
            const T b = Fd[i][0] * Fd[k][0] + Fd[i][1] * Fd[k][1] + Fd[i][2] * Fd[k][2];
            const T t = (i == k) ? fma_t(mb, b, diag) : mb * b;
            s.tau[i][k] = t;
            s.tau[k][i] = t;
        }
}

// Residual moment Q = P adj(Jp)^T (see nodal_force_of_moment) of the element's law at the
// lane's Gauss point.  Linear law: P = sigma(H), H = Du Jp^-1.  Neo-Hookean: P = tau F^-T and
// F^-T adj(Jp)^T = (det Jp / det j) adj(j)^T, so Q = (det Jp / det j) tau adj(j)^T.
template <typename T>
__device__ __forceinline__ bool residual_moment(const GaussKinematics<T> &K, int law, T lam, T mu, T Q[3][3],
                                                NeoHookeanState<T> *state = nullptr) {
    if (law == JETSCI_LINEAR_ELASTIC) {
        const T rdJ = my_rcp(K.dJ);
        T H[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                H[i][j] = (K.Du[i][0] * K.aJ[0][j] + K.Du[i][1] * K.aJ[1][j] + K.Du[i][2] * K.aJ[2][j]) * rdJ;
        const T ltr = lam * (H[0][0] + H[1][1] + H[2][2]);
        T Y[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) Y[i][j] = mu * (H[i][j] + H[j][i]) + ((i == j) ? ltr : T(0));
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int d = 0; d < 3; d++) Q[i][d] = Y[i][0] * K.aJ[d][0] + Y[i][1] * K.aJ[d][1] + Y[i][2] * K.aJ[d][2];
        return true;
    }
    NeoHookeanState<T> s;
    neo_hookean_state(K, lam, mu, s);
    if (state) *state = s;
    const T sc = K.dJ * s.rdj;
    T ts[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) ts[i][k] = sc * s.tau[i][k];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int d = 0; d < 3; d++) Q[i][d] = ts[i][0] * s.aj[d][0] + ts[i][1] * s.aj[d][1] + ts[i][2] * s.aj[d][2];
    return s.ok;
}

// Nodal force of the lane's node from the lane's (Gauss point's) stress moment matrix
// Q_id = sum_j Y_ij adj(Jp)_dj, i.e. (64/w) w detJ Y J^-T: returns
// f_a,i = (w/64) sum_q sum_d Q_q,id dN_a/dxi_d(q) for node a = lane (binary order).
// The Gauss coordinates are +-g, so the moment of a monomial with k factors is g^(k-1) times a
// signed sum of the Q entries (xi eta: g (s_eta Q0 + s_xi Q1), with s the point's signs).  FP64 and
// two-float elements form each moment as that sum (sign flips, no products) and apply its power
// of g once per lane after the sum over the Gauss points, together with the factor w/64 and the
// transpose's 1/8: 16 instead of 20 FP64 operations per component, fewer still in two-float
// arithmetic.  FP32 elements multiply by the coordinates (the FP32 matrix-free product took 8
// more registers the other way and ran 7% slower).
template <typename T>
__device__ __forceinline__ void nodal_force_of_moment(const T Q[3][3], const GaussKinematics<T> &K, int l,
                                                      T f[3]) {
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const T Q0 = Q[i][0], Q1 = Q[i][1], Q2 = Q[i][2];
            T mom[8];
            mom[0] = T(0);
            mom[1] = Q0;
            mom[2] = Q1;
            mom[4] = Q2;
            mom[3] = Q0 * K.eta + Q1 * K.xi;
            mom[5] = Q0 * K.zeta + Q2 * K.xi;
            mom[6] = Q1 * K.zeta + Q2 * K.eta;
            mom[7] = Q0 * gauss_coord_product(K.eta, K.zeta) + Q1 * gauss_coord_product(K.xi, K.zeta) +
                     Q2 * gauss_coord_product(K.xi, K.eta);
            const T mine = reduce_scatter8(mom, l);
            f[i] = butterfly_transpose(mine, l) * T(1.0 / 512.0);
        }
        return;
    }
    const bool nx = !(l & 1), ny = !(l & 2), nz = !(l & 4);  // xi, eta, zeta negative at this point
    // g^(k-1) / 512 for the monomial m = l this lane holds after the reduce-scatter
    const int k = __popc(l);
    const T scale = from_double<T>(k == 2 ? kGaussG / 512.0 : (k == 3 ? kGaussG2 / 512.0 : 1.0 / 512.0));
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const T Q0 = Q[i][0], Q1 = Q[i][1], Q2 = Q[i][2];
        // moment contributions of this Gauss point for monomials 0..7 (monomial 0 has none)
        T mom[8];
        mom[0] = T(0);
        mom[1] = Q0;
        mom[2] = Q1;
        mom[4] = Q2;
        mom[3] = neg_if(Q0, ny) + neg_if(Q1, nx);
        mom[5] = neg_if(Q0, nz) + neg_if(Q2, nx);
        mom[6] = neg_if(Q1, nz) + neg_if(Q2, ny);
        mom[7] = neg_if(Q0, ny != nz) + neg_if(Q1, nx != nz) + neg_if(Q2, nx != ny);
        // sum over the 8 Gauss points with moment m landing at lane m
        const T mine = reduce_scatter8(mom, l);
        f[i] = butterfly_transpose(mine * scale, l);
    }
}

// The same from the stress Y (P for the residual, the linearised P for K v).
template <typename T>
__device__ __forceinline__ void nodal_force(const T Y[3][3], const GaussKinematics<T> &K, int l,
                                            T f[3]) {
    T Q[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int d = 0; d < 3; d++) Q[i][d] = Y[i][0] * K.aJ[d][0] + Y[i][1] * K.aJ[d][1] + Y[i][2] * K.aJ[d][2];
    nodal_force_of_moment(Q, K, l, f);
}

}  // namespace jetsci
