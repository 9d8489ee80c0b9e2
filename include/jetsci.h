/*
 * jetsci.h -- C ABI of the B300 (sm_103a) hex8 finite-element assembly library.
 *
 * The library evaluates, for a hex8 mesh with per-element material phases, the
 * discrete residual R(u) of a nonlinear finite-element problem and its Jacobian
 * K(u) = dR/du (JetSCI, Section II-A), assembles K into a CSR matrix whose pattern
 * is fixed once before any values are produced (Section III-B: the non-zero count is
 * precomputed, local dense element blocks are summed into a global sparse matrix),
 * applies K to vectors without assembling it (the matrix-free operator of
 * Section III-A), gives the gradient of 1/2 ||R||^2 with respect to a per-element
 * Young's modulus (the differentiable-calibration use of the Introduction), and can
 * replace the constitutive law by a learned MLP surrogate whose Jacobian provides the
 * tangent (Section III-B, last paragraph).
 *
 * Discretisation (the paper fixes none of it; these are the library's readings):
 * trilinear hex8 elements, 2x2x2 Gauss rule (points +-1/sqrt(3), unit weights,
 * lexicographic order with xi fastest), total Lagrangian kinematics, no external
 * load (R = f_int), and per phase either small-strain Hooke or the compressible
 * neo-Hookean law W = mu/2 (I1-3) - mu lnJ + lambda/2 (lnJ)^2, with Lame constants
 * from (E, nu).  Hex8 local node order: (-,-,-), (+,-,-), (+,+,-), (-,+,-),
 * (-,-,+), (+,-,+), (+,+,+), (-,+,+).  DOF of node n, component c = 3n + c.
 *
 * Conventions for every call:
 *  - Pointers named *_host are host memory; *_dev are device memory of the device
 *    that was current when the mesh was created.  All device buffers are owned and
 *    allocated by the caller unless stated; the library never frees caller memory.
 *  - Outputs are overwritten (INSERT semantics, as in the paper's MatSetValuesCOO
 *    with INSERT_ALL), never accumulated into.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) unless stated.  Only jetsci_mesh_create, jetsci_mesh_destroy,
 *    jetsci_mesh_check and the surrogate create/destroy/get calls synchronise.
 *  - Results are deterministic: element contributions are summed in a fixed
 *    (colour-major) order without atomics, so repeated calls are bitwise identical.
 *  - Every call returns a jetsci_status; on failure jetsci_last_error() gives a
 *    thread-local message.  No C++ exception crosses the ABI.  Arguments are checked
 *    on the host before any launch; kernels record inadmissible states (detJ <= 0,
 *    det F <= 0, non-finite values) in a per-mesh device flag word read by
 *    jetsci_mesh_check, and never trap.
 */
#ifndef JETSCI_H
#define JETSCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jetsci_mesh_s *jetsci_mesh;           /* opaque, library-owned */
typedef struct jetsci_surrogate_s *jetsci_surrogate; /* opaque, library-owned */

typedef enum {
    JETSCI_OK = 0,
    JETSCI_ERR_ARG = 1,           /* NULL/invalid pointer, size or enum value          */
    JETSCI_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has details)  */
    JETSCI_ERR_OOM = 3,           /* device or host allocation failed                  */
    JETSCI_ERR_MESH = 4,          /* connectivity/phase out of range, degenerate element */
    JETSCI_ERR_NONFINITE = 5,     /* a kernel met a non-finite or inadmissible value   */
    JETSCI_ERR_NOT_CONVERGED = 6, /* an iteration hit its cap                          */
    JETSCI_ERR_UNSUPPORTED = 7    /* valid request the library does not implement      */
} jetsci_status;

/* Arithmetic of the element computations.  The global residual scatter and the
 * residual norm are FP64 in every mode. */
typedef enum {
    JETSCI_FP64 = 0,      /* all element arithmetic in FP64; CSR values double        */
    JETSCI_FP32 = 1,      /* element arithmetic in FP32 (FP64 geometry differences);
                             CSR values float; R, K.v accumulated in FP64              */
    JETSCI_TF32 = 2,      /* as FP32, with the element stiffness contraction on
                             tensor cores in TF32 with FP32 accumulation (the
                             residual and the matrix-free product, which form no
                             element stiffness, run as FP32)                          */
    JETSCI_SURROGATE = 3, /* FP32 element arithmetic, stress and tangent from the
                             mesh's MLP surrogate (BF16 tensor cores, FP32 accumulate)
                             with the plain law as fallback out of range; CSR float    */
    JETSCI_DF64 = 4       /* FP64-accurate two-float arithmetic on the FP32 pipes;
                             CSR values double                                        */
} jetsci_precision;

typedef enum { JETSCI_LINEAR_ELASTIC = 0, JETSCI_NEO_HOOKEAN = 1 } jetsci_law;

typedef enum { JETSCI_MATRIX_FREE = 0, JETSCI_CSR = 1 } jetsci_apply_mode;

/* Material of one phase: Young's modulus [Pa], Poisson ratio (-1 < nu < 0.5), law. */
typedef struct {
    double E;
    double nu;
    int32_t law;
    int32_t reserved; /* must be 0 */
} jetsci_material;

/* Device flag bits reported by jetsci_mesh_check. */
#define JETSCI_FLAG_BAD_ELEMENT 0x1u /* detJ <= 0 at a Gauss point                 */
#define JETSCI_FLAG_BAD_STATE 0x2u   /* det F <= 0 under the neo-Hookean law        */
#define JETSCI_FLAG_NONFINITE 0x4u   /* NaN/Inf met in an input or an intermediate  */

/* ---------------------------------------------------------------------------
 * Mesh: geometry, connectivity, phases and materials (the element data and problem
 * structure of the paper's Fig. 1) plus everything derived once from
 * them: the CSR pattern of K (rows = DOFs; per row the columns sorted ascending;
 * DOFs of one node are interleaved so each row's columns come in node-sorted
 * 3-wide blocks), an element colouring (no two elements of one colour share a
 * node) and the element-to-CSR slot map.  It also keeps, per element, the reference
 * geometry at the 8 Gauss points (Jp, adj(Jp), det Jp and adj(Jp) adj(Jp)^T in FP64,
 * 1,664 bytes, read by the FP64 and two-float kernels instead of re-forming it from the
 * coordinates), room for one FP64 linearisation (768 bytes; see jetsci_apply_tangent) and
 * for one set of element residual vectors (192 bytes; see jetsci_material_grad).
 * Device memory at creation is about 2.8 KB per element plus 12 bytes per CSR entry
 * (column index and, allocated by the caller, FP64 values).
 *
 * coords_host [n_nodes*3] (x,y,z per node), conn_host [n_elem*8] (node ids in the
 * hex8 order above), phase_host [n_elem] (index into mats; may be NULL = all 0),
 * mats [n_mats].  n_elem may be 0 (an empty mesh; every call is then a no-op that
 * still overwrites its outputs).  Synchronises `stream`.  Errors: JETSCI_ERR_ARG
 * (NULL where required, negative sizes, bad law/nu), JETSCI_ERR_MESH (node id or
 * phase out of range, repeated node in an element, more than 255 neighbours of a
 * node or more than 64 colours), JETSCI_ERR_OOM, JETSCI_ERR_CUDA.  On error *out
 * is set to NULL and nothing is leaked.
 */
jetsci_status jetsci_mesh_create(const double *coords_host, int64_t n_nodes,
                                 const int32_t *conn_host, int64_t n_elem,
                                 const int32_t *phase_host, const jetsci_material *mats,
                                 int32_t n_mats, void *stream, jetsci_mesh *out);

/* Frees everything the mesh owns (waits for its work to finish).  NULL is a no-op. */
jetsci_status jetsci_mesh_destroy(jetsci_mesh mesh);

/* Sizes and the device CSR pattern (mesh-owned, read-only, valid until destroy).
 * Any output pointer may be NULL.  rowptr has n_dof+1 int64 entries, col nnz int32. */
jetsci_status jetsci_mesh_info(jetsci_mesh mesh, int64_t *n_dof, int64_t *nnz,
                               const int64_t **rowptr_dev, const int32_t **col_dev,
                               int32_t *n_colours);

/* Copies the CSR pattern into caller buffers rowptr [n_dof+1] int64 and col [nnz] int32,
 * which may be host or device memory (cudaMemcpyDefault).  Synchronises `stream`. */
jetsci_status jetsci_mesh_copy_pattern(jetsci_mesh mesh, int64_t *rowptr, int32_t *col, void *stream);

/* Synchronises the mesh's last stream, returns the device flag word (bits above) in
 * *flags_host and clears it.  Returns JETSCI_ERR_NONFINITE if any bit was set. */
jetsci_status jetsci_mesh_check(jetsci_mesh mesh, uint32_t *flags_host);

/* Structural check of the assembly data built at creation (the precomputed pattern and maps
 * that Section III-B's element-batched assembly and Section III-C's COO preallocation fix
 * before any values), run on the device.  counts_host [4] receives the number of violations
 * of: [0] element node ids outside [0, n_nodes); [1] the colouring (two elements of one
 * colour sharing a node, or an element not in exactly one colour); [2] the slot map (an
 * element node pair (a, b) whose slot does not hold node b's three DOF columns in each of
 * node a's three CSR rows); [3] the first-writer masks (a CSR node-pair block without exactly
 * one first writer).  All zero for a valid mesh; otherwise JETSCI_ERR_MESH with the counts in
 * the message.  A debugging aid: it allocates and frees about 4 * (n_nodes + n_elem + nnz / 9)
 * bytes of device memory and synchronises `stream`. */
jetsci_status jetsci_mesh_validate(jetsci_mesh mesh, uint64_t *counts_host, void *stream);

/* Test hook for the bounded waits of the tensor-core kernels.  Their tcgen05 MMAs signal
 * completion on an mbarrier that every thread polls a bounded number of times; a wait that runs
 * out raises JETSCI_FLAG_NONFINITE and the kernel finishes instead of hanging.  This runs that
 * wait on the current device: one block initialises an mbarrier that expects one arrival,
 * arrives on it if `arrive` is non-zero, then polls it at most max_iter times (1 .. 2^20).
 * *timed_out_host = 1 if the wait ran out (arrive = 0: nothing completes the barrier), 0 if it
 * completed.  The device stays usable either way.  Synchronises the current device's legacy
 * default stream.  JETSCI_ERR_ARG for a NULL output or max_iter out of range. */
jetsci_status jetsci_selftest_bounded_wait(uint32_t max_iter, int arrive, uint32_t *timed_out_host);

/* ---------------------------------------------------------------------------
 * Global residual R(u) = sum_e P_e^T R_e (Section II-A, R(u) = 0), with
 * R_e(a,i) = sum_q w_q detJ_q (F S)_iJ G_aJ.
 * u_dev [n_dof] FP64, R_dev [n_dof] FP64 (overwritten).  E_elem_dev [n_elem] FP64 or
 * NULL: per-element Young's modulus replacing the phase's (the phase's nu and law are
 * kept).  precision: JETSCI_FP64, FP32, DF64 or SURROGATE (TF32 acts as FP32 here).
 * With E_elem_dev given (FP64, FP32, TF32, DF64) the call also keeps its element vectors
 * R_e in the mesh (192 bytes per element, allocated with the mesh) for
 * jetsci_material_grad with u_dev = NULL; the next such call replaces them.
 */
jetsci_status jetsci_residual(jetsci_mesh mesh, const double *u_dev, double *R_dev,
                              int32_t precision, const double *E_elem_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Consistent tangent K(u) = dR/du in CSR values against the mesh's pattern
 * (Section II-A; the values the paper hands to MatSetValuesCOO, Section III-C),
 * K_e(a,i)(b,k) = sum_q w_q detJ_q sum_{J,L} G_aJ (delta_ik S_JL + F_iI CC_IJKL F_kK) G_bL.
 * vals_dev [nnz]: double for FP64/DF64, float for FP32/TF32/SURROGATE (overwritten).
 * R_dev [n_dof] FP64 or NULL: if given, the residual is produced by the same pass.
 * Assembly: FP64 and DF64 scatter element by element, one colour at a time (no two elements
 * of a colour share a node).  FP32, TF32 and SURROGATE form every element's blocks in one
 * pass into a mesh-owned workspace, then write each CSR row once, its sum taken over the
 * elements of the row's node in ascending element order (no atomics in either; results are
 * bitwise reproducible).  The first such call on a mesh allocates that workspace (2,496
 * bytes per element, kept until jetsci_mesh_destroy) and synchronises `stream`; it fails
 * with JETSCI_ERR_ARG if `stream` is being captured, so make one call before a capture.
 */
jetsci_status jetsci_tangent_csr(jetsci_mesh mesh, const double *u_dev, void *vals_dev,
                                 double *R_dev, int32_t precision, const double *E_elem_dev,
                                 void *stream);

/* ---------------------------------------------------------------------------
 * y = K(u) v.  mode JETSCI_MATRIX_FREE: element by element without forming K
 * (Section III-A's matrix-free operator); vals_dev is ignored (may be NULL).
 * mode JETSCI_CSR: sparse product with the CSR values vals_dev of the same mesh
 * (double for FP64/DF64, float for FP32/TF32/SURROGATE); u_dev is ignored.
 * u_dev, v_dev, y_dev [n_dof] FP64; y overwritten.  y must not alias u or v.
 * Matrix-free FP64 or DF64 with u_dev = NULL applies K at the linearisation stored by the mesh's
 * last FP64 or DF64 jetsci_residual or jetsci_tangent_csr call (its u; the neo-Hookean state per
 * Gauss point is kept in FP64, 768 bytes per element, so the product skips u and that state):
 * for repeated products at one Newton iterate.  E_elem_dev must be the pointer that call used;
 * the calls must be ordered on the stream(s).  Otherwise (no such call, FP32/TF32/SURROGATE,
 * another E_elem_dev) JETSCI_ERR_ARG.
 */
jetsci_status jetsci_apply_tangent(jetsci_mesh mesh, const double *u_dev, const double *v_dev,
                                   double *y_dev, int32_t mode, const void *vals_dev,
                                   int32_t precision, const double *E_elem_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Gradient of L(E) = 1/2 ||R(u; E)||^2 with respect to each element's Young's modulus
 * (differentiable calibration, Introduction).  Because the stress of both laws is
 * linear in (lambda, mu), which are proportional to E at fixed nu,
 * dL/dE_e = R[dofs_e] . R_e(u; E = 1).  R_dev must be jetsci_residual(u, E) of the
 * same mesh/precision.  E_elem_dev [n_elem] or NULL (phase moduli); dLdE_dev [n_elem]
 * FP64 (overwritten).  precision: JETSCI_FP64, FP32 or DF64.
 * u_dev = NULL: the gradient at the state of the last jetsci_residual call with a
 * per-element modulus field, from the element vectors that call kept:
 * dL/dE_e = R[dofs_e] . R_e / E_e, with no element arithmetic (the backward pass of
 * L = 1/2 ||R||^2 right after its forward residual).  E_elem_dev must be the pointer that
 * call used, with the same contents and nonzero entries, and precision the one it used;
 * otherwise (no such call, a surrogate residual since, another pointer or precision)
 * JETSCI_ERR_ARG.  The calls must be ordered on the stream(s).
 */
jetsci_status jetsci_material_grad(jetsci_mesh mesh, const double *u_dev,
                                   const double *E_elem_dev, const double *R_dev,
                                   double *dLdE_dev, int32_t precision, void *stream);

/* ---------------------------------------------------------------------------
 * ||x||_2 of x_dev [n] FP64 into out_dev[0] (device FP64), by a fixed-shape two-pass
 * reduction (chunks of 8192 entries, fixed trees), so the result is bitwise
 * reproducible.  This decides Newton convergence (the paper solves to a relative
 * residual of 1e-13, Section V-B).  Uses mesh-owned scratch, so calls on one mesh must
 * not overlap on different streams.  n may exceed n_dof up to 2^31 * 8192 - 1.
 */
jetsci_status jetsci_norm2(jetsci_mesh mesh, const double *x_dev, int64_t n, double *out_dev,
                           void *stream);

/* ---------------------------------------------------------------------------
 * MLP constitutive surrogate (the paper notes that a surrogate model can replace the
 * explicit material function and that its Jacobian is extracted the same way,
 * Section III-B).  Network: x = [E_voigt / in_scale (6), one-hot phase (2)] ->
 * 3 x (Linear 64 + SiLU) -> Linear 6 -> y; S_c = y_c * out_scale[phase][c] +
 * out_shift[phase][c] (second Piola-Kirchhoff stress, Voigt [11,22,33,23,13,12], tensor
 * shear); the tangent dS/dE (w.r.t. the tensor components of the Green-Lagrange strain E)
 * is the network's input-Jacobian.  All GEMMs run on tensor cores in BF16 with FP32
 * accumulation; master weights and Adam state are FP32.  Two phases (0, 1) are supported.
 *
 * Parameter vector (FP64 on the host, FP32 on the device), 9286 entries in this order:
 * W1 [64][8], b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [6][64], b4 [6]
 * (W[out][in]).
 */
typedef struct {
    double in_scale;         /* strain scale of the inputs (> 0)                          */
    double range;            /* fallback to the plain law if any |E_ij| > range (> 0)     */
    double out_scale[2][6];  /* per phase and component, non-zero                         */
    double out_shift[2][6];
} jetsci_surrogate_config;

#define JETSCI_MLP_PARAMS 9286

/* Creates a surrogate on the current device from params_host [9286] (copied).  Synchronises. */
jetsci_status jetsci_surrogate_create(const double *params_host, const jetsci_surrogate_config *cfg,
                                      void *stream, jetsci_surrogate *out);
jetsci_status jetsci_surrogate_destroy(jetsci_surrogate s);
/* Copies the current FP32 master weights into params_host [9286] (as double).  Synchronises. */
jetsci_status jetsci_surrogate_get_params(jetsci_surrogate s, double *params_host);

/* Training labels from the plain compressible neo-Hookean update, in FP64 on the device:
 * S6_dev [n][6] = S(E) for E6_dev [n][6] (Voigt, tensor shear) and phase_dev [n] in {0,1},
 * with the Lame constants of mats[phase] (n_mats 1 or 2).  A phase out of range or
 * det(I + 2E) <= 0 sets bits 2 / 4 in *err_flag_dev (device uint32, caller-owned). */
jetsci_status jetsci_surrogate_label(const jetsci_material *mats, int32_t n_mats, const double *E6_dev,
                                     const int32_t *phase_dev, int64_t n, double *S6_dev,
                                     uint32_t *err_flag_dev, void *stream);

/* n_steps Adam steps on minibatches of `batch` samples (a positive multiple of 128, at most
 * 131072): step k uses samples order_dev[k*batch .. (k+1)*batch) of the training set
 * (E6_dev [n_samples][6], phase_dev [n_samples], S6_dev [n_samples][6] labels).  Loss =
 * mean squared error of the normalised outputs.  Learning rate follows a cosine from lr_max
 * to lr_min over the call's steps; Adam (0.9, 0.999, 1e-8) with bias correction continues
 * across calls.  loss_dev [n_steps] (FP32, device) or NULL.  Gradients are summed over
 * 128-sample tiles in a fixed order (deterministic).  Synchronises (reads the error word). */
jetsci_status jetsci_surrogate_train(jetsci_surrogate s, const double *E6_dev, const int32_t *phase_dev,
                                     const double *S6_dev, int64_t n_samples, const int32_t *order_dev,
                                     int64_t order_len, int64_t n_steps, int32_t batch, double lr_max,
                                     double lr_min, float *loss_dev, void *stream);

/* Gradient of the loss of one minibatch (samples order_dev[0..batch)) with respect to the
 * parameter vector, into grad_dev [9286] (FP32), and the loss into loss_dev[0]; weights
 * unchanged.  Synchronises. */
jetsci_status jetsci_surrogate_gradient(jetsci_surrogate s, const double *E6_dev, const int32_t *phase_dev,
                                        const double *S6_dev, int64_t n_samples, const int32_t *order_dev,
                                        int32_t batch, float *grad_dev, float *loss_dev, void *stream);

/* Network stress S6_dev [n][6] and, if D36_dev != NULL, tangent D36_dev [n][6][6]
 * (D[c][d] = dS_c / dE_d) at E6_dev [n][6], phase_dev [n].  Synchronises. */
jetsci_status jetsci_surrogate_eval(jetsci_surrogate s, const double *E6_dev, const int32_t *phase_dev,
                                    int64_t n, double *S6_dev, double *D36_dev, void *stream);

/* Attaches (or with NULL detaches) a surrogate to a mesh; residual and tangent calls with
 * precision JETSCI_SURROGATE then take S and dS/dE from it at every Gauss point whose
 * strain is within range, and from the phase's plain law elsewhere.  The mesh does not
 * own the surrogate; keep it alive while attached. */
jetsci_status jetsci_mesh_set_surrogate(jetsci_mesh mesh, jetsci_surrogate s);

/* Number of Gauss points that fell back to the plain law (strain out of the surrogate's
 * range) in the mesh's last JETSCI_SURROGATE residual/tangent call.  Synchronises. */
jetsci_status jetsci_mesh_surrogate_fallbacks(jetsci_mesh mesh, uint32_t *count_host);

/* ---------------------------------------------------------------------------
 * Newton's method for R(u) = 0 with a Jacobi-preconditioned conjugate-gradient solve of
 * K du = -R per step (the paper's outer Newton iteration with a Krylov solve per step,
 * Sections II-A and V; the paper's PETSc solver stack itself is not reproduced).  A driver
 * for end-to-end use and iteration counts, not a tuned solver.
 * u_dev [n_dof] (in: initial guess, out: solution); the n_bc DOFs bc_dofs_dev (int64,
 * device or host) are fixed to bc_vals_dev and excluded from the residual and the Krylov
 * space.  The residual and its norm are FP64; tangent_precision (FP64, FP32 or TF32) sets
 * the tangent's arithmetic (FP32/TF32 make it an inexact Newton method).  Converged when
 * ||R_free|| <= rtol * ||R_free(u_0)||; each CG stops at ||r|| <= cg_rtol ||r_0|| or max_cg.
 * Allocates its own workspace (about 7 n_dof doubles plus one CSR value array) and
 * synchronises.  Returns JETSCI_ERR_NOT_CONVERGED after max_newton steps, with *info filled.
 * *info also splits the device time (CUDA events on `stream`) into residual evaluations,
 * tangent assembly and CG solves: the assembly-versus-solve split of the paper's timings
 * (Section V).
 */
typedef struct {
    int32_t newton_iters;         /* Newton steps taken                                  */
    int32_t cg_iters_total;       /* CG iterations over all steps                        */
    int32_t cg_capped;            /* steps whose CG hit max_cg                           */
    int32_t reserved;
    double final_rel_residual;    /* ||R_free(u)|| / ||R_free(u_0)||                      */
    double residual_history[32];  /* relative residual before step k (k < 32)            */
    double seconds_residual;      /* device time: FP64 residuals and norms               */
    double seconds_tangent;       /* device time: tangent assembly and Jacobi diagonal   */
    double seconds_solve;         /* device time: CG solves and updates                  */
} jetsci_newton_info;

jetsci_status jetsci_newton_solve(jetsci_mesh mesh, double *u_dev, int64_t n_bc, const int64_t *bc_dofs_dev,
                                  const double *bc_vals_dev, int32_t tangent_precision, double rtol,
                                  int32_t max_newton, double cg_rtol, int32_t max_cg, void *stream,
                                  jetsci_newton_info *info);

/* ---------------------------------------------------------------------------
 * Insertion of element blocks formed by the caller into the mesh's CSR pattern: the
 * counterpart of handing element-batched dense Jacobian blocks (Section III-B) to a matrix
 * preallocated with their COO pattern and setting its values with duplicates summed and
 * INSERT semantics (Section III-C).  The COO order is element-major and implied by the
 * connectivity: entry (e, 3a+i, 3b+k) goes to row 3 conn[e][a] + i, column 3 conn[e][b] + k.
 *   Ke_dev   [n_elem][24][24] row-major, local DOF 3a + i (a = local node in connectivity
 *            order, i = component); double for JETSCI_FP64, float for JETSCI_FP32; 16-byte
 *            aligned (it is read in 16-byte pieces), else JETSCI_ERR_ARG.
 *   vals_dev [nnz] of the same type, overwritten with sum_e P_e^T K_e P_e (rows of
 *            jetsci_mesh_info's pattern).  Each row is written once: its blocks are summed
 *            over the elements of the row's node in ascending element order (bitwise
 *            reproducible, no atomics, no clearing pass).
 * Other precisions -> JETSCI_ERR_ARG.  Asynchronous on `stream`.
 */
jetsci_status jetsci_assemble_element_blocks(jetsci_mesh mesh, const void *Ke_dev, void *vals_dev, int32_t precision,
                                             void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free ||x||_2 (no counterpart in the paper; a service for callers that
 * cannot allocate device memory when they need the norm -- their device memory is
 * reserved up front by another runtime's pool, or a cudaMalloc and its implicit device
 * synchronisation is not acceptable in their loop -- and that may hold no mesh).
 * Same arithmetic and fixed reduction shape as jetsci_norm2, so the results are
 * bitwise equal.  Scratch: a fixed file-scope device array of 4096 doubles (32 KiB) that
 * every GPU which loads the library holds until the process exits; the call allocates
 * nothing and frees nothing.  n is limited to 4096 * 8192 = 33,554,432 entries; larger
 * n returns JETSCI_ERR_ARG with a message.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) in the current device's context; the first call on a device may
 * load the library's device code, so make that first call before any stream capture.  The
 * address is not cached, so a cudaDeviceReset in between leaves no stale pointer.  All
 * calls on one device share the array: calls
 * that overlap on the GPU (e.g. on two streams at once) race; the array keeps the last
 * call's partial sums, which the next call overwrites before reading.
 * x_dev [n] FP64 device, out_dev[0] FP64 device.
 */
jetsci_status jetsci_norm2_static(const double *x_dev, int64_t n, double *out_dev, void *stream);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *jetsci_last_error(void);

/* Library version string. */
const char *jetsci_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JETSCI_H */
