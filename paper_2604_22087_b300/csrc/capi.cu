// C entry points of the compute calls: host-side argument checks, then the launchers.
#include <cuda_runtime.h>

#include "jetsci_internal.h"

using namespace jetsci;

namespace {

bool valid_precision(int32_t p) { return p >= JETSCI_FP64 && p <= JETSCI_DF64; }

}  // namespace

extern "C" jetsci_status jetsci_residual(jetsci_mesh m, const double *u, double *R, int32_t precision,
                                         const double *E_elem, void *stream) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (!valid_precision(precision)) return fail(JETSCI_ERR_ARG, "invalid precision");
    if (m->n_dof > 0 && (!u || !R)) return fail(JETSCI_ERR_ARG, "u or R is NULL");
    if (m->n_dof == 0) return JETSCI_OK;
    return launch_residual(m, u, R, precision, E_elem, s);
}

extern "C" jetsci_status jetsci_tangent_csr(jetsci_mesh m, const double *u, void *vals, double *R,
                                            int32_t precision, const double *E_elem, void *stream) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (!valid_precision(precision)) return fail(JETSCI_ERR_ARG, "invalid precision");
    if (m->n_dof > 0 && !u) return fail(JETSCI_ERR_ARG, "u is NULL");
    if (m->nnz > 0 && !vals) return fail(JETSCI_ERR_ARG, "vals is NULL");
    if (m->n_dof == 0) return JETSCI_OK;
    return launch_tangent(m, u, vals, R, precision, E_elem, s);
}

extern "C" jetsci_status jetsci_apply_tangent(jetsci_mesh m, const double *u, const double *v, double *y,
                                              int32_t mode, const void *vals, int32_t precision,
                                              const double *E_elem, void *stream) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (!valid_precision(precision)) return fail(JETSCI_ERR_ARG, "invalid precision");
    if (mode != JETSCI_MATRIX_FREE && mode != JETSCI_CSR) return fail(JETSCI_ERR_ARG, "invalid mode");
    if (m->n_dof == 0) return JETSCI_OK;
    if (!v || !y) return fail(JETSCI_ERR_ARG, "v or y is NULL");
    if (y == v || y == u) return fail(JETSCI_ERR_ARG, "y aliases u or v");
    if (mode == JETSCI_CSR) {
        if (m->nnz > 0 && !vals) return fail(JETSCI_ERR_ARG, "vals is NULL in CSR mode");
        bool fp32 = precision == JETSCI_FP32 || precision == JETSCI_TF32 || precision == JETSCI_SURROGATE;
        return launch_spmv(m, vals, fp32, v, y, s);
    }
    if (!u) {
        // K(u) v at the stored linearisation of the last FP64 or two-float residual or tangent call
        if (precision != JETSCI_FP64 && precision != JETSCI_DF64)
            return fail(JETSCI_ERR_ARG, "u is NULL: a stored linearisation exists for JETSCI_FP64 and JETSCI_DF64 only");
        if (!m->lin_valid)
            return fail(JETSCI_ERR_ARG,
                        "u is NULL and no FP64 or two-float residual or tangent call has stored a linearisation");
        if (E_elem != m->lin_E)
            return fail(JETSCI_ERR_ARG, "u is NULL: E_elem differs from the call that stored the linearisation");
    }
    return launch_apply_mf(m, u, v, y, precision, E_elem, s);
}

extern "C" jetsci_status jetsci_material_grad(jetsci_mesh m, const double *u, const double *E_elem,
                                              const double *R, double *g, int32_t precision, void *stream) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (!valid_precision(precision)) return fail(JETSCI_ERR_ARG, "invalid precision");
    if (m->n_elem == 0) return JETSCI_OK;
    if (!R || !g) return fail(JETSCI_ERR_ARG, "R or dLdE is NULL");
    if (!u) {
        // from the element vectors kept by the last residual call with a per-element modulus field
        if (!m->re_valid)
            return fail(JETSCI_ERR_ARG, "u is NULL and no jetsci_residual call with E_elem has kept element residuals");
        if (!E_elem || E_elem != m->re_E)
            return fail(JETSCI_ERR_ARG, "u is NULL: E_elem differs from the residual call that kept the element vectors");
        if ((precision == JETSCI_TF32 ? JETSCI_FP32 : precision) != m->re_prec)
            return fail(JETSCI_ERR_ARG, "u is NULL: precision differs from the residual call that kept the element vectors");
    }
    return launch_material_grad(m, u, E_elem, R, g, precision, s);
}

extern "C" jetsci_status jetsci_norm2(jetsci_mesh m, const double *x, int64_t n, double *out, void *stream) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (n < 0 || !out || (n > 0 && !x)) return fail(JETSCI_ERR_ARG, "invalid norm arguments");
    return launch_norm2(x, n, m->d_norm_partials, kNormMaxPartials, out, s);
}

extern "C" jetsci_status jetsci_assemble_element_blocks(jetsci_mesh m, const void *Ke, void *vals, int32_t precision,
                                                        void *stream) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (precision != JETSCI_FP64 && precision != JETSCI_FP32)
        return fail(JETSCI_ERR_ARG, "element blocks must be FP64 or FP32");
    if (m->nnz > 0 && !vals) return fail(JETSCI_ERR_ARG, "vals is NULL");
    if (m->n_elem > 0 && !Ke) return fail(JETSCI_ERR_ARG, "Ke is NULL");
    if (m->nnz == 0) return JETSCI_OK;
    return launch_insert_blocks(m, Ke, vals, precision == JETSCI_FP32, s);
}
