// Structural check of a mesh's assembly data (jetsci_mesh_validate), on the device: the facts
// the coloured scatters, the slot map and the first-writer stores rely on.  No memory checker
// runs on this GPU, so these checks stand in for one: they read only the mesh's own arrays and
// count violations (atomics are fine here: this is a debugging aid, not an assembly path).
#include <cuda_runtime.h>

#include <string>

#include "jetsci_internal.h"

namespace jetsci {
namespace {

enum { kBadNode = 0, kBadColour = 1, kBadSlot = 2, kBadFirst = 3, kNumChecks = 4 };

// Thread = (element e, local node a).  Node id in range; for every local node b the slot lies in
// node a's neighbour list and all three rows of node a hold node b's DOF columns 3nb, 3nb+1, 3nb+2
// there; first-writer bits are counted per CSR node-pair block (block id = the number of blocks
// of the nodes before a, rowptr[3a] / 9, plus the slot).
__global__ void k_validate_slots(int64_t n_elem, int64_t n_nodes, int64_t nnz, const int32_t *__restrict__ conn,
                                 const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                 const uint8_t *__restrict__ slot, const uint8_t *__restrict__ first,
                                 uint32_t *__restrict__ block_writers, unsigned long long *__restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * n_elem) return;
    const int64_t e = t >> 3;
    const int32_t na = conn[t];
    if (na < 0 || na >= n_nodes) {
        atomicAdd(&bad[kBadNode], 1ull);
        return;
    }
    const int64_t r0 = rowptr[3 * (int64_t)na];
    const int64_t nnb = (rowptr[3 * (int64_t)na + 1] - r0) / 3;
    const uint32_t fb = first[t];
    for (int b = 0; b < 8; b++) {
        const int32_t nb = conn[8 * e + b];
        if (nb < 0 || nb >= n_nodes) continue;  // counted by the thread of (e, b)
        const int s = slot[8 * t + b];
        bool ok = s < nnb;
        for (int i = 0; i < 3 && ok; i++) {
            const int64_t idx = rowptr[3 * (int64_t)na + i] + 3 * (int64_t)s;
            ok = idx >= 0 && idx + 2 < nnz && col[idx] == 3 * nb && col[idx + 1] == 3 * nb + 1 &&
                 col[idx + 2] == 3 * nb + 2;
        }
        if (!ok) {
            atomicAdd(&bad[kBadSlot], 1ull);
            continue;
        }
        const int64_t blk = r0 / 9 + s;
        if (((fb >> b) & 1u) && blk < nnz / 9) atomicAdd(&block_writers[blk], 1u);
    }
}

// CSR blocks whose number of first writers is not exactly one.
__global__ void k_count_first_writers(int64_t n_blocks, const uint32_t *__restrict__ block_writers,
                                      unsigned long long *__restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_blocks && block_writers[t] != 1u) atomicAdd(&bad[kBadFirst], 1ull);
}

// Thread = (entry of one colour's element list, local node): counts each listed element once and
// each of its nodes once per element.
__global__ void k_colour_hits(const int32_t *__restrict__ elems, int64_t n, int64_t n_elem, int64_t n_nodes,
                              const int32_t *__restrict__ conn, uint32_t *__restrict__ node_hits,
                              uint32_t *__restrict__ elem_hits, unsigned long long *__restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * n) return;
    const int32_t e = elems[t >> 3];
    if (e < 0 || e >= n_elem) {
        if ((t & 7) == 0) atomicAdd(&bad[kBadColour], 1ull);
        return;
    }
    if ((t & 7) == 0) atomicAdd(&elem_hits[e], 1u);
    const int32_t nd = conn[8 * (int64_t)e + (t & 7)];
    if (nd >= 0 && nd < n_nodes) atomicAdd(&node_hits[nd], 1u);
}

// Nodes that two elements of the colour just counted share; clears the counts for the next colour.
__global__ void k_colour_conflicts(int64_t n_nodes, uint32_t *__restrict__ node_hits,
                                   unsigned long long *__restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes) return;
    if (node_hits[t] > 1u) atomicAdd(&bad[kBadColour], 1ull);
    node_hits[t] = 0u;
}

// Elements listed in no colour or in more than one.
__global__ void k_colour_cover(int64_t n_elem, const uint32_t *__restrict__ elem_hits,
                               unsigned long long *__restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_elem && elem_hits[t] != 1u) atomicAdd(&bad[kBadColour], 1ull);
}

unsigned blocks_for(int64_t threads) { return (unsigned)((threads + 255) / 256); }

// Temporary device buffers of one validation, freed on every return path.
struct Scratch {
    unsigned long long *bad = nullptr;
    uint32_t *node_hits = nullptr, *elem_hits = nullptr, *block_writers = nullptr;
    ~Scratch() {
        cudaFree(bad);
        cudaFree(node_hits);
        cudaFree(elem_hits);
        cudaFree(block_writers);
    }
};

}  // namespace
}  // namespace jetsci

using namespace jetsci;

extern "C" jetsci_status jetsci_mesh_validate(jetsci_mesh m, uint64_t *counts_host, void *stream) {
    cudaStream_t s;
    jetsci_status st = enter(m, stream, &s);
    if (st) return st;
    if (!counts_host) return fail(JETSCI_ERR_ARG, "counts_host is NULL");
    for (int i = 0; i < kNumChecks; i++) counts_host[i] = 0;
    if (m->n_elem == 0) return JETSCI_OK;
    const int64_t n_blocks = m->nnz / 9;
    Scratch w;
    JETSCI_CUDA_TRY(cudaStreamSynchronize(s));
    JETSCI_CUDA_TRY(cudaMalloc(&w.bad, kNumChecks * sizeof(unsigned long long)));
    JETSCI_CUDA_TRY(cudaMalloc(&w.node_hits, m->n_nodes * sizeof(uint32_t)));
    JETSCI_CUDA_TRY(cudaMalloc(&w.elem_hits, m->n_elem * sizeof(uint32_t)));
    JETSCI_CUDA_TRY(cudaMalloc(&w.block_writers, (n_blocks > 0 ? n_blocks : 1) * sizeof(uint32_t)));
    JETSCI_CUDA_TRY(cudaMemsetAsync(w.bad, 0, kNumChecks * sizeof(unsigned long long), s));
    JETSCI_CUDA_TRY(cudaMemsetAsync(w.node_hits, 0, m->n_nodes * sizeof(uint32_t), s));
    JETSCI_CUDA_TRY(cudaMemsetAsync(w.elem_hits, 0, m->n_elem * sizeof(uint32_t), s));
    JETSCI_CUDA_TRY(cudaMemsetAsync(w.block_writers, 0, (n_blocks > 0 ? n_blocks : 1) * sizeof(uint32_t), s));
    k_validate_slots<<<blocks_for(8 * m->n_elem), 256, 0, s>>>(m->n_elem, m->n_nodes, m->nnz, m->d_conn, m->d_rowptr,
                                                               m->d_col, m->d_slot, m->d_first, w.block_writers,
                                                               w.bad);
    if (n_blocks > 0) k_count_first_writers<<<blocks_for(n_blocks), 256, 0, s>>>(n_blocks, w.block_writers, w.bad);
    for_each_colour(m, [&](const int32_t *elems, int64_t n) {
        k_colour_hits<<<blocks_for(8 * n), 256, 0, s>>>(elems, n, m->n_elem, m->n_nodes, m->d_conn, w.node_hits,
                                                        w.elem_hits, w.bad);
        k_colour_conflicts<<<blocks_for(m->n_nodes), 256, 0, s>>>(m->n_nodes, w.node_hits, w.bad);
    });
    k_colour_cover<<<blocks_for(m->n_elem), 256, 0, s>>>(m->n_elem, w.elem_hits, w.bad);
    JETSCI_CUDA_TRY(cudaGetLastError());
    unsigned long long c[kNumChecks];
    JETSCI_CUDA_TRY(cudaMemcpyAsync(c, w.bad, sizeof(c), cudaMemcpyDeviceToHost, s));
    JETSCI_CUDA_TRY(cudaStreamSynchronize(s));
    uint64_t total = 0;
    for (int i = 0; i < kNumChecks; i++) {
        counts_host[i] = c[i];
        total += c[i];
    }
    if (total)
        return fail(JETSCI_ERR_MESH, "mesh validation: " + std::to_string(c[kBadNode]) + " node ids out of range, " +
                                         std::to_string(c[kBadColour]) + " colouring violations, " +
                                         std::to_string(c[kBadSlot]) + " slot-map entries off their CSR columns, " +
                                         std::to_string(c[kBadFirst]) + " CSR blocks without exactly one first writer");
    return JETSCI_OK;
}
