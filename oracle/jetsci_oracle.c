/*
 * FP64 CPU oracle for hex8 finite-element residual / tangent assembly.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may include, link or
 * call this file: only the tests, the package's smoke check and the bench's CPU-baseline
 * leg use it.  It shares no code with the CUDA path.
 *
 * What it computes (the paper, Section II-A): the discrete residual R(u) = 0 of a
 * nonlinear finite-element problem and its Jacobian K = dR/du, both assembled from
 * element contributions; element Jacobians are small and dense, the global one sparse.
 * The paper obtains element Jacobians by forward-mode AD of the element residual
 * (Section III-B); the result is exactly the consistent tangent of the Galerkin
 * discretisation, so this oracle writes that definition out:
 *
 *   R_e(a,i)      = sum_q w_q detJ_q sum_J P_iJ G_aJ                      (P = F S)
 *   K_e(a,i)(b,k) = sum_q w_q detJ_q sum_{J,L} G_aJ A_iJkL G_bL
 *   A_iJkL        = delta_ik S_JL + sum_{I,K} F_iI CC_IJKL F_kK
 *
 * with G_a = J^-T dN_a/dxi the reference gradient of the trilinear shape function of
 * node a at Gauss point q (2x2x2 rule, points +-1/sqrt(3), unit weights).  The paper
 * names no element, rule or material law; the readings used here are: hex8, 2x2x2
 * Gauss, total Lagrangian, no external load (R = f_int), and per phase either
 * small-strain Hooke (sigma = lambda tr(eps) I + 2 mu eps) or compressible neo-Hookean
 * W = mu/2 (I1 - 3) - mu lnJ + lambda/2 (lnJ)^2, whose second Piola-Kirchhoff stress and
 * material tangent are
 *   S       = mu (I - C^-1) + lambda lnJ C^-1
 *   CC_IJKL = lambda Ci_IJ Ci_KL + (mu - lambda lnJ)(Ci_IK Ci_JL + Ci_IL Ci_JK),
 * with Lame constants lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)).
 * Everything is plain nested loops in FP64, no blocking or symmetry shortcuts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_BAD_ELEMENT 2   /* detJ <= 0 */
#define OR_ERR_BAD_STATE 3     /* det F <= 0 under the neo-Hookean law */
#define OR_ERR_PATTERN 4       /* a (row, col) entry missing from the CSR pattern */

#define LAW_LINEAR_ELASTIC 0
#define LAW_NEO_HOOKEAN 1

/* Reference coordinates of the 8 local nodes (xi, eta, zeta). */
static const double NODE_XI[8][3] = {
    {-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
    {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

void or_lame(double E, double nu, double *lam, double *mu) {
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    *mu = E / (2.0 * (1.0 + nu));
}

/* Gauss point q (0..7): lexicographic with xi fastest, coordinates +-1/sqrt(3). */
void or_gauss_point(int q, double xi[3]) {
    const double g = 1.0 / sqrt(3.0);
    xi[0] = (q & 1) ? g : -g;
    xi[1] = (q & 2) ? g : -g;
    xi[2] = (q & 4) ? g : -g;
}

/* Trilinear shape functions N_a = 1/8 (1 + xi_a xi)(1 + eta_a eta)(1 + zeta_a zeta)
 * and their reference derivatives dN[a][d] = dN_a / dxi_d. */
void or_shape(const double xi[3], double N[8], double dN[8][3]) {
    for (int a = 0; a < 8; a++) {
        double f0 = 1.0 + NODE_XI[a][0] * xi[0];
        double f1 = 1.0 + NODE_XI[a][1] * xi[1];
        double f2 = 1.0 + NODE_XI[a][2] * xi[2];
        N[a] = 0.125 * f0 * f1 * f2;
        dN[a][0] = 0.125 * NODE_XI[a][0] * f1 * f2;
        dN[a][1] = 0.125 * f0 * NODE_XI[a][1] * f2;
        dN[a][2] = 0.125 * f0 * f1 * NODE_XI[a][2];
    }
}

static double det3(const double A[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
         - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
         + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* Inverse by the adjugate; returns the determinant. */
static double inv3(const double A[3][3], double Ai[3][3]) {
    double d = det3(A);
    Ai[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / d;
    Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / d;
    Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / d;
    Ai[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / d;
    Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / d;
    Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / d;
    Ai[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / d;
    Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / d;
    Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / d;
    return d;
}

/* Geometry at one Gauss point: J_ij = sum_a X_a,i dN_a/dxi_j, G_a = J^-T dN_a/dxi,
 * i.e. G[a][j] = sum_k Jinv[k][j] dN[a][k]. */
int or_geometry(const double X[8][3], const double dN[8][3], double G[8][3], double *detJ) {
    double J[3][3], Ji[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int a = 0; a < 8; a++) s += X[a][i] * dN[a][j];
            J[i][j] = s;
        }
    double d = det3(J);
    *detJ = d;
    if (!(d > 0.0)) return OR_ERR_BAD_ELEMENT;
    inv3(J, Ji);
    for (int a = 0; a < 8; a++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += Ji[k][j] * dN[a][k];
            G[a][j] = s;
        }
    return OR_OK;
}

/* Small-strain Hooke: sigma from the displacement gradient H = grad u, and the
 * 4-index elasticity D_ijkl = lambda d_ij d_kl + mu (d_ik d_jl + d_il d_jk). */
void or_linear_elastic(double lam, double mu, const double H[3][3], double sig[3][3],
                       double D[3][3][3][3]) {
    double eps[3][3], tr = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) eps[i][j] = 0.5 * (H[i][j] + H[j][i]);
    for (int i = 0; i < 3; i++) tr += eps[i][i];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) sig[i][j] = lam * tr * (i == j) + 2.0 * mu * eps[i][j];
    if (D)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                for (int k = 0; k < 3; k++)
                    for (int l = 0; l < 3; l++)
                        D[i][j][k][l] = lam * (i == j) * (k == l)
                                      + mu * ((i == k) * (j == l) + (i == l) * (j == k));
}

/* Compressible neo-Hookean: S and CC from the deformation gradient F. */
int or_neo_hookean(double lam, double mu, const double F[3][3], double S[3][3],
                   double CC[3][3][3][3]) {
    double C[3][3], Ci[3][3];
    double J = det3(F);
    if (!(J > 0.0)) return OR_ERR_BAD_STATE;
    for (int I = 0; I < 3; I++)
        for (int K = 0; K < 3; K++) {
            double s = 0.0;
            for (int i = 0; i < 3; i++) s += F[i][I] * F[i][K];
            C[I][K] = s;
        }
    inv3(C, Ci);
    double lnJ = log(J);
    for (int I = 0; I < 3; I++)
        for (int K = 0; K < 3; K++) S[I][K] = mu * ((I == K) - Ci[I][K]) + lam * lnJ * Ci[I][K];
    if (CC) {
        double m = mu - lam * lnJ;
        for (int I = 0; I < 3; I++)
            for (int J2 = 0; J2 < 3; J2++)
                for (int K = 0; K < 3; K++)
                    for (int L = 0; L < 3; L++)
                        CC[I][J2][K][L] = lam * Ci[I][J2] * Ci[K][L]
                                        + m * (Ci[I][K] * Ci[J2][L] + Ci[I][L] * Ci[J2][K]);
    }
    return OR_OK;
}

/* Element residual Re[24] (index 3a+i) and, if Ke != NULL, the dense element tangent
 * Ke[24*24] (row 3a+i, column 3b+k), both in FP64. */
int or_element(int law, double lam, double mu, const double X[8][3], const double *ue,
               double *Re, double *Ke) {
    for (int r = 0; r < 24; r++) Re[r] = 0.0;
    if (Ke)
        for (int r = 0; r < 576; r++) Ke[r] = 0.0;
    for (int q = 0; q < 8; q++) {
        double xi[3], N[8], dN[8][3], G[8][3], detJ;
        or_gauss_point(q, xi);
        or_shape(xi, N, dN);
        int st = or_geometry(X, dN, G, &detJ);
        if (st) return st;
        const double w = 1.0;
        double H[3][3];
        for (int i = 0; i < 3; i++)
            for (int J = 0; J < 3; J++) {
                double s = 0.0;
                for (int a = 0; a < 8; a++) s += ue[3 * a + i] * G[a][J];
                H[i][J] = s;
            }
        double P[3][3], A[3][3][3][3];
        if (law == LAW_LINEAR_ELASTIC) {
            double sig[3][3], D[3][3][3][3];
            or_linear_elastic(lam, mu, H, sig, D);
            memcpy(P, sig, sizeof(P));
            memcpy(A, D, sizeof(A));
        } else if (law == LAW_NEO_HOOKEAN) {
            double F[3][3], S[3][3], CC[3][3][3][3];
            for (int i = 0; i < 3; i++)
                for (int J = 0; J < 3; J++) F[i][J] = (i == J) + H[i][J];
            st = or_neo_hookean(lam, mu, F, S, CC);
            if (st) return st;
            for (int i = 0; i < 3; i++)
                for (int J = 0; J < 3; J++) {
                    double s = 0.0;
                    for (int I = 0; I < 3; I++) s += F[i][I] * S[I][J];
                    P[i][J] = s;
                }
            for (int i = 0; i < 3; i++)
                for (int J = 0; J < 3; J++)
                    for (int k = 0; k < 3; k++)
                        for (int L = 0; L < 3; L++) {
                            double s = (i == k) ? S[J][L] : 0.0;
                            for (int I = 0; I < 3; I++)
                                for (int K = 0; K < 3; K++) s += F[i][I] * CC[I][J][K][L] * F[k][K];
                            A[i][J][k][L] = s;
                        }
        } else {
            return OR_ERR_ARG;
        }
        for (int a = 0; a < 8; a++)
            for (int i = 0; i < 3; i++) {
                double s = 0.0;
                for (int J = 0; J < 3; J++) s += P[i][J] * G[a][J];
                Re[3 * a + i] += w * detJ * s;
            }
        if (!Ke) continue;
        for (int a = 0; a < 8; a++)
            for (int i = 0; i < 3; i++)
                for (int b = 0; b < 8; b++)
                    for (int k = 0; k < 3; k++) {
                        double s = 0.0;
                        for (int J = 0; J < 3; J++)
                            for (int L = 0; L < 3; L++) s += G[a][J] * A[i][J][k][L] * G[b][L];
                        Ke[(3 * a + i) * 24 + 3 * b + k] += w * detJ * s;
                    }
    }
    return OR_OK;
}

/* Material parameters of element e: (law, lambda, mu).  With E_elem != NULL the
 * element's Young's modulus replaces the phase's (its Poisson ratio is kept). */
static void element_material(int64_t e, const int32_t *phase, const double *mat_E,
                             const double *mat_nu, const int32_t *mat_law, const double *E_elem,
                             int *law, double *lam, double *mu) {
    int p = phase ? phase[e] : 0;
    double E = E_elem ? E_elem[e] : mat_E[p];
    *law = mat_law[p];
    or_lame(E, mat_nu[p], lam, mu);
}

static void gather(int64_t e, const int32_t *conn, const double *coords, const double *u,
                   double X[8][3], double ue[24]) {
    for (int a = 0; a < 8; a++) {
        int64_t n = conn[8 * e + a];
        for (int i = 0; i < 3; i++) {
            X[a][i] = coords[3 * n + i];
            ue[3 * a + i] = u ? u[3 * n + i] : 0.0;
        }
    }
}

/* Element residual / tangent of element e (used for sampled rows at large sizes). */
int or_element_of(int64_t e, const int32_t *conn, const double *coords, const double *u,
                  const int32_t *phase, const double *mat_E, const double *mat_nu,
                  const int32_t *mat_law, const double *E_elem, double *Re, double *Ke) {
    double X[8][3], ue[24], lam, mu;
    int law;
    gather(e, conn, coords, u, X, ue);
    element_material(e, phase, mat_E, mat_nu, mat_law, E_elem, &law, &lam, &mu);
    return or_element(law, lam, mu, X, ue, Re, Ke);
}

/* Global residual R[n_dof] = sum_e P_e^T R_e, plain summation in element order. */
int or_residual(int64_t n_elem, int64_t n_nodes, const int32_t *conn, const double *coords,
                const double *u, const int32_t *phase, const double *mat_E,
                const double *mat_nu, const int32_t *mat_law, const double *E_elem, double *R) {
    for (int64_t r = 0; r < 3 * n_nodes; r++) R[r] = 0.0;
    for (int64_t e = 0; e < n_elem; e++) {
        double Re[24];
        int st = or_element_of(e, conn, coords, u, phase, mat_E, mat_nu, mat_law, E_elem, Re, NULL);
        if (st) return st;
        for (int a = 0; a < 8; a++)
            for (int i = 0; i < 3; i++) R[3 * (int64_t)conn[8 * e + a] + i] += Re[3 * a + i];
    }
    return OR_OK;
}

/* Position of column c in the sorted column list of one CSR row, or -1. */
static int64_t find_col(const int64_t *rowptr, const int32_t *col, int64_t r, int64_t c) {
    int64_t lo = rowptr[r], hi = rowptr[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] == c) return mid;
        if (col[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* CSR values of K (pattern given, columns sorted per row) and optionally R. */
int or_tangent_csr(int64_t n_elem, int64_t n_nodes, const int32_t *conn, const double *coords,
                   const double *u, const int32_t *phase, const double *mat_E,
                   const double *mat_nu, const int32_t *mat_law, const double *E_elem,
                   const int64_t *rowptr, const int32_t *col, double *vals, double *R) {
    int64_t n_dof = 3 * n_nodes;
    for (int64_t t = 0; t < rowptr[n_dof]; t++) vals[t] = 0.0;
    if (R)
        for (int64_t r = 0; r < n_dof; r++) R[r] = 0.0;
    double *Ke = (double *)malloc(576 * sizeof(double));
    if (!Ke) return OR_ERR_ARG;
    for (int64_t e = 0; e < n_elem; e++) {
        double Re[24];
        int st = or_element_of(e, conn, coords, u, phase, mat_E, mat_nu, mat_law, E_elem, Re, Ke);
        if (st) { free(Ke); return st; }
        for (int a = 0; a < 8; a++)
            for (int i = 0; i < 3; i++) {
                int64_t row = 3 * (int64_t)conn[8 * e + a] + i;
                if (R) R[row] += Re[3 * a + i];
                for (int b = 0; b < 8; b++)
                    for (int k = 0; k < 3; k++) {
                        int64_t c = 3 * (int64_t)conn[8 * e + b] + k;
                        int64_t pos = find_col(rowptr, col, row, c);
                        if (pos < 0) { free(Ke); return OR_ERR_PATTERN; }
                        vals[pos] += Ke[(3 * a + i) * 24 + 3 * b + k];
                    }
            }
    }
    free(Ke);
    return OR_OK;
}

/* Matrix-free tangent product y = sum_e P_e^T K_e(u) P_e v by explicit element matrices. */
int or_apply_tangent(int64_t n_elem, int64_t n_nodes, const int32_t *conn, const double *coords,
                     const double *u, const double *v, const int32_t *phase, const double *mat_E,
                     const double *mat_nu, const int32_t *mat_law, const double *E_elem, double *y) {
    for (int64_t r = 0; r < 3 * n_nodes; r++) y[r] = 0.0;
    double *Ke = (double *)malloc(576 * sizeof(double));
    if (!Ke) return OR_ERR_ARG;
    for (int64_t e = 0; e < n_elem; e++) {
        double Re[24], ve[24];
        int st = or_element_of(e, conn, coords, u, phase, mat_E, mat_nu, mat_law, E_elem, Re, Ke);
        if (st) { free(Ke); return st; }
        for (int b = 0; b < 8; b++)
            for (int k = 0; k < 3; k++) ve[3 * b + k] = v[3 * (int64_t)conn[8 * e + b] + k];
        for (int r = 0; r < 24; r++) {
            double s = 0.0;
            for (int c = 0; c < 24; c++) s += Ke[r * 24 + c] * ve[c];
            y[3 * (int64_t)conn[8 * e + r / 3] + r % 3] += s;
        }
    }
    free(Ke);
    return OR_OK;
}

/* y = K v with K in CSR form. */
void or_spmv(int64_t n_rows, const int64_t *rowptr, const int32_t *col, const double *vals,
             const double *v, double *y) {
    for (int64_t r = 0; r < n_rows; r++) {
        double s = 0.0;
        for (int64_t t = rowptr[r]; t < rowptr[r + 1]; t++) s += vals[t] * v[col[t]];
        y[r] = s;
    }
}

/* Gradient of L = 1/2 ||R(u; E)||^2 with respect to each element's Young's modulus.
 * R_e depends on E_e only, and for both laws the stress is linear in (lambda, mu), which
 * are proportional to E at fixed nu; hence dR_e/dE_e = R_e / E_e and
 * dL/dE_e = R[dofs_e] . R_e / E_e (R = the assembled residual). */
int or_material_grad(int64_t n_elem, int64_t n_nodes, const int32_t *conn, const double *coords,
                     const double *u, const int32_t *phase, const double *mat_E,
                     const double *mat_nu, const int32_t *mat_law, const double *E_elem,
                     const double *R, double *g) {
    (void)n_nodes;
    for (int64_t e = 0; e < n_elem; e++) {
        double Re[24];
        int st = or_element_of(e, conn, coords, u, phase, mat_E, mat_nu, mat_law, E_elem, Re, NULL);
        if (st) return st;
        double Ee = E_elem ? E_elem[e] : mat_E[phase ? phase[e] : 0];
        double s = 0.0;
        for (int a = 0; a < 8; a++)
            for (int i = 0; i < 3; i++) s += R[3 * (int64_t)conn[8 * e + a] + i] * Re[3 * a + i];
        g[e] = s / Ee;
    }
    return OR_OK;
}

/* Total stored energy Pi(u) = sum_e sum_q w detJ W(F) (hyperelastic laws only). */
int or_energy(int64_t n_elem, const int32_t *conn, const double *coords, const double *u,
              const int32_t *phase, const double *mat_E, const double *mat_nu,
              const int32_t *mat_law, const double *E_elem, double *out) {
    double tot = 0.0;
    for (int64_t e = 0; e < n_elem; e++) {
        double X[8][3], ue[24], lam, mu;
        int law;
        gather(e, conn, coords, u, X, ue);
        element_material(e, phase, mat_E, mat_nu, mat_law, E_elem, &law, &lam, &mu);
        for (int q = 0; q < 8; q++) {
            double xi[3], N[8], dN[8][3], G[8][3], detJ, H[3][3];
            or_gauss_point(q, xi);
            or_shape(xi, N, dN);
            int st = or_geometry(X, dN, G, &detJ);
            if (st) return st;
            for (int i = 0; i < 3; i++)
                for (int J = 0; J < 3; J++) {
                    double s = 0.0;
                    for (int a = 0; a < 8; a++) s += ue[3 * a + i] * G[a][J];
                    H[i][J] = s;
                }
            double W;
            if (law == LAW_LINEAR_ELASTIC) {
                double eps[3][3], tr = 0.0, ee = 0.0;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) eps[i][j] = 0.5 * (H[i][j] + H[j][i]);
                for (int i = 0; i < 3; i++) tr += eps[i][i];
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) ee += eps[i][j] * eps[i][j];
                W = 0.5 * lam * tr * tr + mu * ee;
            } else {
                double F[3][3], I1 = 0.0;
                for (int i = 0; i < 3; i++)
                    for (int J = 0; J < 3; J++) F[i][J] = (i == J) + H[i][J];
                for (int i = 0; i < 3; i++)
                    for (int J = 0; J < 3; J++) I1 += F[i][J] * F[i][J];
                double Jd = det3(F);
                if (!(Jd > 0.0)) return OR_ERR_BAD_STATE;
                double lnJ = log(Jd);
                W = 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ;
            }
            tot += 1.0 * detJ * W;
        }
    }
    *out = tot;
    return OR_OK;
}
