// Internal declarations of libjetsci (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "jetsci.h"

namespace jetsci {

// Per-phase material table as the kernels read it.  lam1/mu1 are the Lame constants
// for E = 1 (used when a per-element modulus scales them, and by the adjoint).
struct Material {
    double lam, mu;    // Lame constants of the phase's own E
    double lam1, mu1;  // Lame constants per unit E (same nu)
    double lam_mu;     // lam / mu = 2 nu / (1 - 2 nu), the same for any E at this nu
    int32_t law;
    int32_t pad;
};

constexpr int kMaxPhases = 16;
constexpr int kNormChunk = 8192;             // entries per first-pass partial
constexpr int64_t kNormMaxPartials = 65536;  // mesh-owned scratch capacity

struct Surrogate;

}  // namespace jetsci

struct jetsci_mesh_s {
    int device = 0;
    int64_t n_nodes = 0, n_elem = 0, n_dof = 0, nnz = 0;
    int32_t n_mats = 0;
    int32_t n_colours = 0;
    std::vector<int64_t> colour_ptr;  // host: offsets of each colour in d_colour_elems
    jetsci::Material mats[jetsci::kMaxPhases];

    int32_t *d_conn = nullptr;          // [n_elem*8]
    double *d_coords = nullptr;         // [n_nodes*3]
    double *d_lin = nullptr;            // [n_elem][6][8][2]: FP64 neo-Hookean linearisation (element.cuh)
    bool lin_valid = false;             // d_lin holds the state of an FP64 or two-float residual/tangent call
    const double *lin_E = nullptr;      // ... made with this per-element modulus array (or NULL)
    double *d_re = nullptr;             // [n_elem][8][3]: element residual vectors R_e kept by the last
                                        // residual call given a per-element modulus field
    bool re_valid = false;              // d_re holds such a call's R_e ...
    const double *re_E = nullptr;       // ... made with this E_elem array ...
    int32_t re_prec = -1;               // ... in this precision (TF32 recorded as FP32)
    double *d_geom = nullptr;           // [n_elem][13][8][2]: reference geometry at the Gauss points
                                        // (element.cuh, kGeom*), read by the FP64 kernels
    double *d_lap = nullptr;            // [n_elem][36]: L_ab = sum_q detJ G_a . G_b per node pair
                                        // (element.cuh, kLap*), read by the tangent kernels
    int32_t *d_phase = nullptr;         // [n_elem]
    int64_t *d_rowptr = nullptr;        // [n_dof+1]
    int32_t *d_col = nullptr;           // [nnz]
    uint8_t *d_slot = nullptr;          // [n_elem*64]: slot[a*8+b] = rank of node b among node a's neighbours
    uint8_t *d_item_order = nullptr;    // [n_colours][224]: order of the FP64 tangent's off-diagonal
                                        // work items per colour (assemble.cu, first-writer grouping)
    uint8_t *d_first = nullptr;         // [n_elem*8]: bit b of byte a set = the element writes CSR block
                                        // (node a, node b) first (lowest colour among its elements)
    int32_t *d_colour_elems = nullptr;  // [n_elem], grouped by colour, ascending within a colour
    int64_t *d_ne_ptr = nullptr;        // [n_nodes+1]: offsets into d_ne
    uint32_t *d_ne = nullptr;           // [n_elem*8]: per node, 8e + a for each element e holding it
                                        // as local node a, ascending
    void *d_blocks = nullptr;           // element-block workspace of the row-gather assembly
    size_t blocks_bytes = 0;            // (allocated on first use, kept until the mesh is destroyed)
    jetsci::Material *d_mats = nullptr; // [kMaxPhases]
    double *d_norm_partials = nullptr;  // [kNormMaxPartials]
    uint32_t *d_flags = nullptr;        // [1]
    uint32_t *d_fallback = nullptr;     // [1] Gauss points that used the plain law in the last surrogate call
    cudaStream_t last_stream = nullptr;
    jetsci_surrogate surrogate = nullptr;
};

namespace jetsci {

// Thread-local error message and helpers.
void set_error(const std::string &msg);
jetsci_status fail(jetsci_status st, const std::string &msg);
jetsci_status cuda_fail(cudaError_t err, const char *what);

#define JETSCI_CUDA_TRY(call)                                      \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::jetsci::cuda_fail(_e, #call); \
    } while (0)

// Checks that the current device is the mesh's device (switches to it) and records
// the stream; returns JETSCI_OK or an error.
jetsci_status enter(jetsci_mesh m, void *stream, cudaStream_t *s);

// Sets Kernel's dynamic shared-memory limit (if max_dyn_smem > 0) and, if asked, the largest
// shared-memory carveout, once per device: these are not stream operations, and doing them once
// keeps every later call of the library free of them (so it can run inside a CUDA graph capture).
template <auto Kernel>
inline jetsci_status kernel_attrs_once(size_t max_dyn_smem, bool max_carveout) {
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    JETSCI_CUDA_TRY(cudaGetDevice(&dev));
    const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return JETSCI_OK;
    if (max_dyn_smem > 0)
        JETSCI_CUDA_TRY(cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_dyn_smem));
    if (max_carveout)
        JETSCI_CUDA_TRY(cudaFuncSetAttribute(Kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared));
    done.fetch_or(bit, std::memory_order_release);
    return JETSCI_OK;
}

// Calls f(elems, n) for the element list of every colour in colour order.  Within one list no
// two elements share a node; the lists are launched in a fixed order on one stream, so the
// scatters stay race-free and deterministic.
template <typename Fn>
inline void for_each_colour(jetsci_mesh m, Fn f) {
    for (int c = 0; c < m->n_colours; c++) {
        const int64_t len = m->colour_ptr[c + 1] - m->colour_ptr[c];
        if (len > 0) f(m->d_colour_elems + m->colour_ptr[c], len);
    }
}

// Launch wrappers implemented in the .cu files.
jetsci_status launch_residual(jetsci_mesh m, const double *u, double *R, int precision,
                              const double *E_elem, cudaStream_t s);
jetsci_status launch_tangent(jetsci_mesh m, const double *u, void *vals, double *R,
                             int precision, const double *E_elem, cudaStream_t s);
jetsci_status launch_apply_mf(jetsci_mesh m, const double *u, const double *v, double *y,
                              int precision, const double *E_elem, cudaStream_t s);
jetsci_status launch_spmv(jetsci_mesh m, const void *vals, bool fp32, const double *v,
                          double *y, cudaStream_t s);
jetsci_status launch_norm2(const double *x, int64_t n, double *partials, int64_t cap,
                           double *out, cudaStream_t s);
jetsci_status launch_tf32(jetsci_mesh m, const double *u, float *vals, double *R, const double *E_elem,
                          cudaStream_t s);
jetsci_status launch_surrogate(jetsci_mesh m, const double *u, float *vals, double *R, cudaStream_t s);
jetsci_status launch_insert_blocks(jetsci_mesh m, const void *Ke, void *vals, bool fp32, cudaStream_t s);
// The mesh's element-block workspace (blocks.cuh): values_bytes of blocks, then the residual
// part.  Allocated on first use (synchronising the stream) or grown; fails if the stream is
// being captured and the workspace is too small.  Sets *blocks and *Re.
jetsci_status ensure_block_workspace(jetsci_mesh m, size_t values_bytes, cudaStream_t s, void **blocks, double **Re);
// Row pass of the row-gather assembly: vals (all nnz entries) and, if R != NULL, R (all n_dof
// entries) are overwritten from element rows [n_elem][24][24] (blocks.cuh) and, for R, the
// residual vectors Re [n_elem][8][3].
template <typename VT>
jetsci_status launch_gather_rows(jetsci_mesh m, const VT *blocks, const double *Re, VT *vals, double *R,
                                 cudaStream_t s);
// Fills m->d_geom (element.cuh, kGeom*) and m->d_lap (kLap*) from the connectivity and coordinates.
jetsci_status launch_fill_geom(jetsci_mesh m, cudaStream_t s);
jetsci_status launch_material_grad(jetsci_mesh m, const double *u, const double *E_elem,
                                   const double *R, double *g, int precision, cudaStream_t s);

}  // namespace jetsci
