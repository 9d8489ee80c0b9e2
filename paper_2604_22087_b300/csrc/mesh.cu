// Mesh creation: validation, CSR pattern, element colouring and the element-to-CSR
// slot map (everything the paper fixes before values are produced: its pseudocode
// precomputes the non-zero count so the assembly can be compiled once, Section III-B,
// and PETSc's COO preallocation fixes the pattern before MatSetValuesCOO, Section III-C).
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "jetsci_internal.h"

namespace jetsci {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

jetsci_status fail(jetsci_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

jetsci_status cuda_fail(cudaError_t err, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
    return err == cudaErrorMemoryAllocation ? JETSCI_ERR_OOM : JETSCI_ERR_CUDA;
}

jetsci_status enter(jetsci_mesh m, void *stream, cudaStream_t *s) {
    if (!m) return fail(JETSCI_ERR_ARG, "mesh is NULL");
    int cur = -1;
    JETSCI_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != m->device) JETSCI_CUDA_TRY(cudaSetDevice(m->device));
    *s = (cudaStream_t)stream;
    m->last_stream = *s;
    return JETSCI_OK;
}

// Expands per-node neighbour lists into CSR columns: row 3n+i holds, for each
// neighbour node t of n (ascending), the three columns 3t, 3t+1, 3t+2.
__global__ void k_expand_cols(int64_t n_nodes, const int64_t *__restrict__ nbr_ptr,
                              const int32_t *__restrict__ nbr, const int64_t *__restrict__ rowptr,
                              int32_t *__restrict__ col) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 3 * n_nodes) return;
    int64_t n = r / 3;
    int64_t b = nbr_ptr[n], e = nbr_ptr[n + 1];
    int64_t out = rowptr[r];
    for (int64_t t = b; t < e; t++) {
        int32_t c = 3 * nbr[t];
        col[out++] = c;
        col[out++] = c + 1;
        col[out++] = c + 2;
    }
}

// slot[e*64 + a*8 + b] = position of node conn[e][b] in the sorted neighbour list of
// node conn[e][a] (binary search).  Every pair is present by construction.
__global__ void k_slot_map(int64_t n_elem, const int32_t *__restrict__ conn,
                           const int64_t *__restrict__ nbr_ptr, const int32_t *__restrict__ nbr,
                           uint8_t *__restrict__ slot) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_elem * 8) return;
    int64_t e = t >> 3;
    int a = (int)(t & 7);
    int32_t na = conn[8 * e + a];
    int64_t lo0 = nbr_ptr[na], hi0 = nbr_ptr[na + 1] - 1;
    uint8_t res[8];
#pragma unroll
    for (int b = 0; b < 8; b++) {
        int32_t nb = conn[8 * e + b];
        int64_t lo = lo0, hi = hi0, pos = 0;
        while (lo <= hi) {
            int64_t mid = (lo + hi) >> 1;
            int32_t v = nbr[mid];
            if (v == nb) { pos = mid - lo0; break; }
            if (v < nb) lo = mid + 1; else hi = mid - 1;
        }
        res[b] = (uint8_t)pos;
    }
    uint2 packed;
    packed.x = res[0] | (res[1] << 8) | (res[2] << 16) | ((uint32_t)res[3] << 24);
    packed.y = res[4] | (res[5] << 8) | (res[6] << 16) | ((uint32_t)res[7] << 24);
    *reinterpret_cast<uint2 *>(slot + 8 * t) = packed;
}

// Lowest colour among the elements that contain each node-pair block of the CSR pattern; block
// ids follow the neighbour lists (block of node a and its neighbour of rank r = nbr_ptr[a] + r).
__global__ void k_block_min_colour(int64_t n_elem, const int32_t *__restrict__ conn,
                                   const int64_t *__restrict__ nbr_ptr, const uint8_t *__restrict__ slot,
                                   const uint8_t *__restrict__ colour, uint32_t *__restrict__ block_min) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_elem * 8) return;
    int64_t e = t >> 3;
    const int64_t base = nbr_ptr[conn[t]];
    const uint32_t c = colour[e];
#pragma unroll
    for (int b = 0; b < 8; b++) atomicMin(&block_min[base + slot[8 * t + b]], c);
}

// first[e*8 + a] bit b = element e is the block (a, b)'s lowest-colour element, i.e. the first
// to write it in the colour-ordered launches.
__global__ void k_first_writer(int64_t n_elem, const int32_t *__restrict__ conn,
                               const int64_t *__restrict__ nbr_ptr, const uint8_t *__restrict__ slot,
                               const uint8_t *__restrict__ colour, const uint32_t *__restrict__ block_min,
                               uint8_t *__restrict__ first) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_elem * 8) return;
    const int64_t base = nbr_ptr[conn[t]];
    const uint32_t c = colour[t >> 3];
    uint32_t bits = 0;
#pragma unroll
    for (int b = 0; b < 8; b++) bits |= (block_min[base + slot[8 * t + b]] == c ? 1u : 0u) << b;
    first[t] = (uint8_t)bits;
}

static void free_mesh(jetsci_mesh m) {
    if (!m) return;
    cudaFree(m->d_conn);
    cudaFree(m->d_coords);
    cudaFree(m->d_geom);
    cudaFree(m->d_lap);
    cudaFree(m->d_lin);
    cudaFree(m->d_re);
    cudaFree(m->d_phase);
    cudaFree(m->d_rowptr);
    cudaFree(m->d_col);
    cudaFree(m->d_slot);
    cudaFree(m->d_first);
    cudaFree(m->d_item_order);
    cudaFree(m->d_colour_elems);
    cudaFree(m->d_ne_ptr);
    cudaFree(m->d_ne);
    cudaFree(m->d_blocks);
    cudaFree(m->d_mats);
    cudaFree(m->d_norm_partials);
    cudaFree(m->d_flags);
    cudaFree(m->d_fallback);
    delete m;
}

template <typename T>
static jetsci_status dev_alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;  // keep a valid pointer for empty meshes
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    return JETSCI_OK;
}

static jetsci_status create_impl(const double *coords, int64_t n_nodes, const int32_t *conn,
                                 int64_t n_elem, const int32_t *phase, const jetsci_material *mats,
                                 int32_t n_mats, cudaStream_t s, jetsci_mesh m) {
    // ---------------- argument validation (host, before any device work)
    if (n_nodes < 0 || n_elem < 0) return fail(JETSCI_ERR_ARG, "negative size");
    if (n_nodes > 0 && !coords) return fail(JETSCI_ERR_ARG, "coords_host is NULL");
    if (n_elem > 0 && !conn) return fail(JETSCI_ERR_ARG, "conn_host is NULL");
    if (n_mats < 1 || n_mats > kMaxPhases || !mats)
        return fail(JETSCI_ERR_ARG, "need 1.." + std::to_string(kMaxPhases) + " materials");
    if (3 * n_nodes >= (int64_t)INT32_MAX) return fail(JETSCI_ERR_ARG, "too many nodes for int32 columns");
    for (int p = 0; p < n_mats; p++) {
        const jetsci_material &mt = mats[p];
        if (!(std::isfinite(mt.E) && mt.E > 0.0) || !(mt.nu > -1.0 && mt.nu < 0.5) ||
            (mt.law != JETSCI_LINEAR_ELASTIC && mt.law != JETSCI_NEO_HOOKEAN) || mt.reserved != 0)
            return fail(JETSCI_ERR_ARG, "invalid material " + std::to_string(p));
        double nu = mt.nu;
        m->mats[p].lam1 = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        m->mats[p].mu1 = 1.0 / (2.0 * (1.0 + nu));
        m->mats[p].lam = mt.E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        m->mats[p].mu = mt.E / (2.0 * (1.0 + nu));
        m->mats[p].lam_mu = 2.0 * nu / (1.0 - 2.0 * nu);
        m->mats[p].law = mt.law;
        m->mats[p].pad = 0;
    }
    for (int64_t i = 0; i < 3 * n_nodes; i++)
        if (!std::isfinite(coords[i])) return fail(JETSCI_ERR_ARG, "non-finite coordinate");
    bool bad = false;
#pragma omp parallel for reduction(|| : bad)
    for (int64_t e = 0; e < n_elem; e++) {
        for (int a = 0; a < 8; a++) {
            int32_t na = conn[8 * e + a];
            if (na < 0 || na >= n_nodes) bad = true;
            for (int b = 0; b < a; b++)
                if (conn[8 * e + b] == na) bad = true;
        }
        if (phase && (phase[e] < 0 || phase[e] >= n_mats)) bad = true;
    }
    if (bad) return fail(JETSCI_ERR_MESH, "node id or phase out of range, or repeated node in an element");

    m->n_nodes = n_nodes;
    m->n_elem = n_elem;
    m->n_dof = 3 * n_nodes;
    m->n_mats = n_mats;

    // ---------------- node -> element adjacency (counting sort): entries 8e + a (element e,
    // local node a), ascending per node; kept on the device for the row-gather assembly
    if (8 * n_elem >= (int64_t)UINT32_MAX) return fail(JETSCI_ERR_ARG, "too many elements");
    std::vector<int64_t> ne_ptr(n_nodes + 1, 0);
    for (int64_t t = 0; t < 8 * n_elem; t++) ne_ptr[conn[t] + 1]++;
    for (int64_t n = 0; n < n_nodes; n++) ne_ptr[n + 1] += ne_ptr[n];
    std::vector<uint32_t> ne_idx(std::max<int64_t>(8 * n_elem, 1));
    {
        std::vector<int64_t> fill(ne_ptr.begin(), ne_ptr.end() - 1);
        for (int64_t t = 0; t < 8 * n_elem; t++) ne_idx[fill[conn[t]]++] = (uint32_t)t;
    }

    // ---------------- node neighbour lists (sorted, unique, including the node itself)
    std::vector<int32_t> nbr_cnt(n_nodes, 0);
    bool too_many = false;
#pragma omp parallel for schedule(dynamic, 4096) reduction(|| : too_many)
    for (int64_t n = 0; n < n_nodes; n++) {
        std::vector<int32_t> cand;
        cand.reserve(8 * (ne_ptr[n + 1] - ne_ptr[n]));
        for (int64_t t = ne_ptr[n]; t < ne_ptr[n + 1]; t++)
            for (int b = 0; b < 8; b++) cand.push_back(conn[8 * (int64_t)(ne_idx[t] >> 3) + b]);
        std::sort(cand.begin(), cand.end());
        int64_t cnt = std::unique(cand.begin(), cand.end()) - cand.begin();
        if (cnt > 255) too_many = true;
        nbr_cnt[n] = (int32_t)cnt;
    }
    if (too_many) return fail(JETSCI_ERR_MESH, "a node has more than 255 neighbours");
    std::vector<int64_t> nbr_ptr(n_nodes + 1, 0);
    for (int64_t n = 0; n < n_nodes; n++) nbr_ptr[n + 1] = nbr_ptr[n] + nbr_cnt[n];
    std::vector<int32_t> nbr(std::max<int64_t>(nbr_ptr[n_nodes], 1));
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t n = 0; n < n_nodes; n++) {
        std::vector<int32_t> cand;
        cand.reserve(8 * (ne_ptr[n + 1] - ne_ptr[n]));
        for (int64_t t = ne_ptr[n]; t < ne_ptr[n + 1]; t++)
            for (int b = 0; b < 8; b++) cand.push_back(conn[8 * (int64_t)(ne_idx[t] >> 3) + b]);
        std::sort(cand.begin(), cand.end());
        auto end = std::unique(cand.begin(), cand.end());
        std::copy(cand.begin(), end, nbr.begin() + nbr_ptr[n]);
    }

    // ---------------- CSR row pointers: row 3n+i has 3*|nbr(n)| entries
    std::vector<int64_t> rowptr(m->n_dof + 1, 0);
    for (int64_t n = 0; n < n_nodes; n++)
        for (int i = 0; i < 3; i++) rowptr[3 * n + i + 1] = rowptr[3 * n + i] + 3 * (int64_t)nbr_cnt[n];
    m->nnz = rowptr[m->n_dof];

    // ---------------- greedy colouring in element order: smallest colour not used by
    // any element sharing a node (gives the 8 parity colours on structured meshes)
    std::vector<uint64_t> node_mask(n_nodes, 0);
    std::vector<int8_t> colour(n_elem);
    int n_col = 0;
    for (int64_t e = 0; e < n_elem; e++) {
        uint64_t used = 0;
        for (int a = 0; a < 8; a++) used |= node_mask[conn[8 * e + a]];
        if (used == ~0ull) return fail(JETSCI_ERR_MESH, "more than 64 colours needed");
        int c = __builtin_ctzll(~used);
        colour[e] = (int8_t)c;
        n_col = std::max(n_col, c + 1);
        for (int a = 0; a < 8; a++) node_mask[conn[8 * e + a]] |= (1ull << c);
    }
    m->n_colours = n_col;
    m->colour_ptr.assign(n_col + 1, 0);
    for (int64_t e = 0; e < n_elem; e++) m->colour_ptr[colour[e] + 1]++;
    for (int c = 0; c < n_col; c++) m->colour_ptr[c + 1] += m->colour_ptr[c];
    std::vector<int32_t> colour_elems(std::max<int64_t>(n_elem, 1));
    {
        std::vector<int64_t> fill(m->colour_ptr.begin(), m->colour_ptr.end() - 1);
        for (int64_t e = 0; e < n_elem; e++) colour_elems[fill[colour[e]]++] = (int32_t)e;
    }

    // ---------------- device upload
    jetsci_status st;
    if ((st = dev_alloc(&m->d_conn, 8 * n_elem))) return st;
    if ((st = dev_alloc(&m->d_coords, 3 * n_nodes))) return st;
    if ((st = dev_alloc(&m->d_geom, (size_t)26 * 8 * n_elem))) return st;
    if ((st = dev_alloc(&m->d_lap, (size_t)36 * n_elem))) return st;
    if ((st = dev_alloc(&m->d_lin, (size_t)12 * 8 * n_elem))) return st;
    if ((st = dev_alloc(&m->d_re, (size_t)24 * n_elem))) return st;
    if ((st = dev_alloc(&m->d_phase, n_elem))) return st;
    if ((st = dev_alloc(&m->d_rowptr, m->n_dof + 1))) return st;
    if ((st = dev_alloc(&m->d_col, m->nnz))) return st;
    if ((st = dev_alloc(&m->d_slot, 64 * n_elem))) return st;
    if ((st = dev_alloc(&m->d_first, 8 * n_elem))) return st;
    if ((st = dev_alloc(&m->d_item_order, (size_t)224 * std::max(n_col, 1)))) return st;
    if ((st = dev_alloc(&m->d_colour_elems, n_elem))) return st;
    if ((st = dev_alloc(&m->d_ne_ptr, n_nodes + 1))) return st;
    if ((st = dev_alloc(&m->d_ne, 8 * n_elem))) return st;
    if ((st = dev_alloc(&m->d_mats, kMaxPhases))) return st;
    if ((st = dev_alloc(&m->d_norm_partials, kNormMaxPartials))) return st;
    if ((st = dev_alloc(&m->d_flags, 1))) return st;
    if ((st = dev_alloc(&m->d_fallback, 1))) return st;
    int64_t *d_nbr_ptr = nullptr;
    int32_t *d_nbr = nullptr;
    uint8_t *d_colour = nullptr;
    uint32_t *d_block_min = nullptr;
    auto cleanup_tmp = [&]() { cudaFree(d_nbr_ptr); cudaFree(d_nbr); cudaFree(d_colour); cudaFree(d_block_min); };
    if ((st = dev_alloc(&d_nbr_ptr, n_nodes + 1)) || (st = dev_alloc(&d_nbr, nbr.size())) ||
        (st = dev_alloc(&d_colour, n_elem)) || (st = dev_alloc(&d_block_min, nbr.size()))) {
        cleanup_tmp();
        return st;
    }
#define UP(dst, src, bytes)                                                               \
    do {                                                                                  \
        if ((bytes) > 0) {                                                                \
            cudaError_t _e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s); \
            if (_e != cudaSuccess) { cleanup_tmp(); return cuda_fail(_e, "upload"); }     \
        }                                                                                 \
    } while (0)
    UP(m->d_conn, conn, 8 * n_elem * sizeof(int32_t));
    UP(m->d_coords, coords, 3 * n_nodes * sizeof(double));
    if (phase) {
        UP(m->d_phase, phase, n_elem * sizeof(int32_t));
    } else if (n_elem > 0) {
        cudaError_t e = cudaMemsetAsync(m->d_phase, 0, n_elem * sizeof(int32_t), s);
        if (e != cudaSuccess) { cleanup_tmp(); return cuda_fail(e, "memset phase"); }
    }
    UP(m->d_rowptr, rowptr.data(), (m->n_dof + 1) * sizeof(int64_t));
    UP(m->d_colour_elems, colour_elems.data(), n_elem * sizeof(int32_t));
    UP(m->d_ne_ptr, ne_ptr.data(), (n_nodes + 1) * sizeof(int64_t));
    UP(m->d_ne, ne_idx.data(), 8 * n_elem * sizeof(uint32_t));
    UP(m->d_mats, m->mats, sizeof(m->mats));
    UP(d_nbr_ptr, nbr_ptr.data(), (n_nodes + 1) * sizeof(int64_t));
    UP(d_nbr, nbr.data(), nbr_ptr[n_nodes] * sizeof(int32_t));
    UP(d_colour, colour.data(), n_elem * sizeof(uint8_t));
#undef UP
    {
        cudaError_t e = cudaMemsetAsync(m->d_flags, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->d_fallback, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) { cleanup_tmp(); return cuda_fail(e, "memset flags"); }
    }
    if (n_nodes > 0) {
        int64_t rows = 3 * n_nodes;
        k_expand_cols<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(n_nodes, d_nbr_ptr, d_nbr,
                                                                      m->d_rowptr, m->d_col);
    }
    if (n_elem > 0) {
        const unsigned g8 = (unsigned)((8 * n_elem + 255) / 256);
        k_slot_map<<<g8, 256, 0, s>>>(n_elem, m->d_conn, d_nbr_ptr, d_nbr, m->d_slot);
        cudaError_t e = cudaMemsetAsync(d_block_min, 0xFF, nbr.size() * sizeof(uint32_t), s);
        if (e != cudaSuccess) { cleanup_tmp(); return cuda_fail(e, "memset block colours"); }
        k_block_min_colour<<<g8, 256, 0, s>>>(n_elem, m->d_conn, d_nbr_ptr, m->d_slot, d_colour, d_block_min);
        k_first_writer<<<g8, 256, 0, s>>>(n_elem, m->d_conn, d_nbr_ptr, m->d_slot, d_colour, d_block_min,
                                          m->d_first);
        if (jetsci_status gs = launch_fill_geom(m, s)) { cleanup_tmp(); return gs; }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup_tmp();
    if (e != cudaSuccess) return cuda_fail(e, "pattern build");
    // Order of the FP64 tangent's off-diagonal work items in each colour (assemble.cu): the node
    // pairs (a < b) the colour's middle element writes first come first, for each of a block's
    // eight elements in turn, then the others.  On a structured mesh every interior element of a
    // colour has the middle element's first-writer bits, and the groups fill whole warps.
    std::vector<uint8_t> order((size_t)224 * std::max(n_col, 1));
    for (int c = 0; c < n_col; c++) {
        uint8_t mask[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const int64_t len = m->colour_ptr[c + 1] - m->colour_ptr[c];
        if (len > 0) {
            const int64_t rep = colour_elems[m->colour_ptr[c] + len / 2];
            e = cudaMemcpy(mask, m->d_first + 8 * rep, 8, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "first-writer masks");
        }
        uint8_t *o = order.data() + (size_t)224 * c;
        int n = 0;
        for (int pass = 0; pass < 2; pass++)
            for (int ee = 0; ee < 8; ee++)
                for (int pa = 0, p = 0; pa < 8; pa++)
                    for (int pb = pa + 1; pb < 8; pb++, p++) {
                        const bool first = (mask[pa] >> pb) & 1;
                        if (first == (pass == 0)) o[n++] = (uint8_t)(28 * ee + p);
                    }
    }
    e = cudaMemcpy(m->d_item_order, order.data(), order.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "tangent item order");
    return JETSCI_OK;
}

}  // namespace jetsci

using namespace jetsci;

extern "C" jetsci_status jetsci_mesh_create(const double *coords_host, int64_t n_nodes,
                                            const int32_t *conn_host, int64_t n_elem,
                                            const int32_t *phase_host, const jetsci_material *mats,
                                            int32_t n_mats, void *stream, jetsci_mesh *out) {
    if (!out) return fail(JETSCI_ERR_ARG, "out is NULL");
    *out = nullptr;
    jetsci_mesh m = new (std::nothrow) jetsci_mesh_s();
    if (!m) return fail(JETSCI_ERR_OOM, "host allocation failed");
    jetsci_status st;
    try {
        cudaError_t e = cudaGetDevice(&m->device);
        if (e != cudaSuccess) {
            delete m;
            return cuda_fail(e, "cudaGetDevice");
        }
        st = create_impl(coords_host, n_nodes, conn_host, n_elem, phase_host, mats, n_mats,
                         (cudaStream_t)stream, m);
    } catch (const std::bad_alloc &) {
        st = fail(JETSCI_ERR_OOM, "host allocation failed");
    } catch (...) {
        st = fail(JETSCI_ERR_ARG, "unexpected host exception");
    }
    if (st != JETSCI_OK) {
        free_mesh(m);
        return st;
    }
    m->last_stream = (cudaStream_t)stream;
    *out = m;
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_mesh_destroy(jetsci_mesh m) {
    if (!m) return JETSCI_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != m->device) cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    free_mesh(m);
    if (cur >= 0 && cur != m->device) cudaSetDevice(cur);
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_mesh_info(jetsci_mesh m, int64_t *n_dof, int64_t *nnz,
                                          const int64_t **rowptr_dev, const int32_t **col_dev,
                                          int32_t *n_colours) {
    if (!m) return fail(JETSCI_ERR_ARG, "mesh is NULL");
    if (n_dof) *n_dof = m->n_dof;
    if (nnz) *nnz = m->nnz;
    if (rowptr_dev) *rowptr_dev = m->d_rowptr;
    if (col_dev) *col_dev = m->d_col;
    if (n_colours) *n_colours = m->n_colours;
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_mesh_copy_pattern(jetsci_mesh m, int64_t *rowptr, int32_t *col,
                                                  void *stream) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (!rowptr || (m->nnz > 0 && !col)) return fail(JETSCI_ERR_ARG, "rowptr or col is NULL");
    JETSCI_CUDA_TRY(cudaMemcpyAsync(rowptr, m->d_rowptr, (m->n_dof + 1) * sizeof(int64_t), cudaMemcpyDefault, s));
    if (m->nnz > 0)
        JETSCI_CUDA_TRY(cudaMemcpyAsync(col, m->d_col, m->nnz * sizeof(int32_t), cudaMemcpyDefault, s));
    JETSCI_CUDA_TRY(cudaStreamSynchronize(s));
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_mesh_check(jetsci_mesh m, uint32_t *flags_host) {
    cudaStream_t s;
    jetsci_status st = enter(m, m ? (void *)m->last_stream : nullptr, &s);
    if (st) return st;
    if (!flags_host) return fail(JETSCI_ERR_ARG, "flags_host is NULL");
    uint32_t f = 0;
    JETSCI_CUDA_TRY(cudaStreamSynchronize(s));
    JETSCI_CUDA_TRY(cudaMemcpy(&f, m->d_flags, sizeof(f), cudaMemcpyDeviceToHost));
    JETSCI_CUDA_TRY(cudaMemset(m->d_flags, 0, sizeof(uint32_t)));
    *flags_host = f;
    if (f) return fail(JETSCI_ERR_NONFINITE, "kernel flags 0x" + std::to_string(f));
    return JETSCI_OK;
}

extern "C" jetsci_status jetsci_mesh_surrogate_fallbacks(jetsci_mesh m, uint32_t *count_host) {
    cudaStream_t s;
    jetsci_status st = enter(m, m ? (void *)m->last_stream : nullptr, &s);
    if (st) return st;
    if (!count_host) return fail(JETSCI_ERR_ARG, "count_host is NULL");
    JETSCI_CUDA_TRY(cudaStreamSynchronize(s));
    JETSCI_CUDA_TRY(cudaMemcpy(count_host, m->d_fallback, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return JETSCI_OK;
}

extern "C" const char *jetsci_last_error(void) { return jetsci::g_last_error.c_str(); }

extern "C" const char *jetsci_version(void) { return "jetsci-b300 0.1 (sm_103a)"; }
