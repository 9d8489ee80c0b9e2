// Node-row pass of the row-gather assembly: every CSR row block (the three rows of one node)
// is formed from the element blocks of the elements around its node and written once.
//
// K_ab = sum over the elements e holding both a and b of K_e(a, b) (the assembly of Section
// III-B, K = sum_e P_e^T K_e P_e), summed in ascending element order, so the values are
// deterministic and independent of launch shapes; R_a = sum_e R_e(a) likewise.  The pass needs
// no clearing of the outputs, no atomics and no colouring: node a reads the element rows
// 3a..3a+2 of its elements (each element row is read once, by its own node) and writes each
// CSR value once, contiguously.
#include <cuda_runtime.h>

#include "blocks.cuh"
#include "jetsci_internal.h"

namespace jetsci {

namespace {

constexpr int kGroupLanes = 8;  // lanes per node (lane = column node lb of the element)
constexpr int kNodesPerWarp = 32 / kGroupLanes;
constexpr int kRowWarps = 4;    // warps per block
constexpr int kSlots = 28;      // neighbour slots per accumulation pass (more take further passes)
constexpr int kAccStride = 12;  // accumulator values per slot (3 x 3 block, 16-byte aligned)

// elements whose blocks a lane loads at once (in flight together); measured at 128^3: 2 is
// faster than 4 and 8, whose registers cost more occupancy than the deeper prefetch gains, and
// than staging whole element rows in shared memory by asynchronous copies (2.14 and 2.59 ms
// against 2.07 ms)
constexpr int kChunk = 2;

// Block K_e(la, lb) (rows at node la) of the rows layout [e][24][24] into y[3 i + k].
template <typename VT>
__device__ __forceinline__ void load_block(const VT *__restrict__ blocks, int64_t e, int la, int lb, VT y[9]) {
    const VT *p = blocks + 576 * e + 72 * la + 3 * lb;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) y[3 * i + k] = __ldg(p + 24 * i + k);
}

// Brings element e's rows into L2 in whole lines (the blocks of the node rows that follow then
// hit L2 instead of fetching short pieces from DRAM one node at a time).
template <typename VT>
__device__ __forceinline__ void prefetch_element(const VT *__restrict__ blocks, int64_t e) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(blocks + 576 * e), "r"(576u * (unsigned)sizeof(VT))
                 : "memory");
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Eight lanes per node a, four nodes per warp.  The node's rows are accumulated in shared
// memory, one 3 x 3 block per neighbour slot; at each element step (elements in ascending
// order) lane lb adds the element's block K_e(a, b) of its column node b at b's slot (the slot
// map).  The eight blocks of one element go to eight distinct slots, so the lanes never
// collide, and every contribution to an entry arrives in element order.  A lane loads the
// blocks of several elements before adding any (they are in flight together).  Nodes with more
// than 32 neighbours take one pass per 32 slots.
template <typename VT>
__global__ void __launch_bounds__(32 * kRowWarps) k_gather_rows(int64_t n_nodes, const int64_t *__restrict__ ne_ptr,
                                                                const uint32_t *__restrict__ ne,
                                                                const uint8_t *__restrict__ slot,
                                                                const int64_t *__restrict__ rowptr,
                                                                const VT *__restrict__ blocks,
                                                                const double *__restrict__ Re,
                                                                VT *__restrict__ vals, double *__restrict__ R) {
    constexpr int kV16 = 16 / (int)sizeof(VT);
    __shared__ __align__(16) VT acc_s[kRowWarps * kNodesPerWarp][kSlots * kAccStride];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = lane / kGroupLanes, lb = lane % kGroupLanes, gl0 = kGroupLanes * grp;
    const int64_t a = ((int64_t)blockIdx.x * kRowWarps + w) * kNodesPerWarp + grp;
    const bool valid = a < n_nodes;
    int64_t j0 = 0, base = 0;
    int cnt = 0, nnb = 0;
    if (valid) {
        j0 = ne_ptr[a];
        cnt = (int)(ne_ptr[a + 1] - j0);
        base = rowptr[3 * a];
        nnb = (int)((rowptr[3 * a + 1] - base) / 3);
    }
    const int n_sc = (nnb + kSlots - 1) / kSlots;
    const int n_sc_max = warp_max(n_sc), cnt_max = warp_max(cnt);
    VT *acc = acc_s[w * kNodesPerWarp + grp];
    double racc = 0.0;
    for (int sc = 0; sc < (n_sc_max > 0 ? n_sc_max : 1); sc++) {
        if (sc < n_sc)
            for (int c = lb; c < kSlots * kAccStride / kV16; c += kGroupLanes)
                reinterpret_cast<uint4 *>(acc)[c] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        for (int ec = 0; ec < cnt_max; ec += kChunk) {
            const int nc = cnt - ec < 0 ? 0 : (cnt - ec < kChunk ? cnt - ec : kChunk);
            // lane lb (< kChunk) holds element ec + lb of its node: entry 8e + la and the slot
            // bytes of la's row
            uint32_t tm = 0;
            uint2 sw = make_uint2(0u, 0u);
            if (lb < nc) {
                tm = ne[j0 + ec + lb];
                sw = __ldg(reinterpret_cast<const uint2 *>(slot + 64 * (int64_t)(tm >> 3) + 8 * (tm & 7)));
                // the element's first node (local node 0, the lowest id on ordered meshes) pulls
                // the whole element into L2 (measured 4-5% faster at 128^3)
                if ((tm & 7) == 0 && sc == 0) prefetch_element<VT>(blocks, tm >> 3);
            }
            VT y[kChunk][9];
#pragma unroll
            for (int j = 0; j < kChunk; j++) {
                const uint32_t t = __shfl_sync(0xffffffffu, tm, gl0 + j);
                if (j < nc && sc < n_sc) load_block<VT>(blocks, t >> 3, (int)(t & 7), lb, y[j]);
            }
#pragma unroll
            for (int j = 0; j < kChunk; j++) {
                const uint32_t t = __shfl_sync(0xffffffffu, tm, gl0 + j);
                const uint32_t wx = __shfl_sync(0xffffffffu, sw.x, gl0 + j), wy = __shfl_sync(0xffffffffu, sw.y, gl0 + j);
                if (j < nc) {
                    const int sl = (int)(((lb < 4 ? wx : wy) >> (8 * (lb & 3))) & 0xffu);
                    const int rel = sl - kSlots * sc;  // the slot within this pass
                    if (sc < n_sc && (unsigned)rel < (unsigned)kSlots) {
                        VT *d = acc + kAccStride * rel;
                        VT z[kAccStride];
#pragma unroll
                        for (int c = 0; c < kAccStride / kV16; c++)
                            reinterpret_cast<uint4 *>(z)[c] = reinterpret_cast<const uint4 *>(d)[c];
#pragma unroll
                        for (int c = 0; c < 9; c++) z[c] += y[j][c];
#pragma unroll
                        for (int c = 0; c < kAccStride / kV16; c++)
                            reinterpret_cast<uint4 *>(d)[c] = reinterpret_cast<const uint4 *>(z)[c];
                    }
                    if (R && sc == 0 && lb < 3) racc += Re[3 * (int64_t)t + lb];
                }
                __syncwarp();
            }
        }
        if (sc < n_sc) {
            // rows 3a, 3a+1, 3a+2 (3 nnb values each, contiguous); value 3 s + k of row i is
            // entry (i, k) of slot s's block
            const int ns = nnb - kSlots * sc < kSlots ? nnb - kSlots * sc : kSlots;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                VT *row = vals + base + (int64_t)i * 3 * nnb + 3 * kSlots * sc;
                for (int c = lb; c < 3 * ns; c += kGroupLanes) {
                    const int s3 = c / 3;
                    row[c] = acc[kAccStride * s3 + 3 * i + (c - 3 * s3)];
                }
            }
        }
        __syncwarp();
    }
    if (R && valid && lb < 3) R[3 * a + lb] = racc;
}

}  // namespace

jetsci_status ensure_block_workspace(jetsci_mesh m, size_t values_bytes, cudaStream_t s, void **blocks, double **Re) {
    const size_t need = values_bytes + blk_residual_bytes(m->n_elem);
    if (!m->d_blocks || m->blocks_bytes < need) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        JETSCI_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return fail(JETSCI_ERR_ARG, "the element-block workspace (" + std::to_string(need) +
                                            " bytes) is allocated by the first call of this precision on a mesh; "
                                            "make one call before capturing the stream");
        JETSCI_CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(m->d_blocks);
        m->d_blocks = nullptr;
        m->blocks_bytes = 0;
        JETSCI_CUDA_TRY(cudaMalloc(&m->d_blocks, need));
        m->blocks_bytes = need;
    }
    *blocks = m->d_blocks;
    *Re = reinterpret_cast<double *>(reinterpret_cast<char *>(m->d_blocks) + values_bytes);
    return JETSCI_OK;
}

template <typename VT>
jetsci_status launch_gather_rows(jetsci_mesh m, const VT *blocks, const double *Re, VT *vals, double *R,
                                 cudaStream_t s) {
    if (m->n_nodes == 0) return JETSCI_OK;
    constexpr int kNodes = kRowWarps * kNodesPerWarp;
    const unsigned grid = (unsigned)((m->n_nodes + kNodes - 1) / kNodes);
    // several blocks per SM need more shared memory than the default carveout gives
    if (jetsci_status st = kernel_attrs_once<k_gather_rows<VT>>(0, true)) return st;
    k_gather_rows<VT><<<grid, 32 * kRowWarps, 0, s>>>(m->n_nodes, m->d_ne_ptr, m->d_ne, m->d_slot, m->d_rowptr,
                                                      blocks, Re, vals, R);
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

template jetsci_status launch_gather_rows<float>(jetsci_mesh, const float *, const double *, float *, double *,
                                                 cudaStream_t);
template jetsci_status launch_gather_rows<double>(jetsci_mesh, const double *, const double *, double *, double *,
                                                  cudaStream_t);

}  // namespace jetsci
