// Node-row pass of the row-gather assembly: every CSR row block (the three rows of one node)
// is formed from the element blocks of the elements around its node and written once.
//
// K_ab = sum over the elements e holding both a and b of K_e(a, b) (the assembly of Section
// III-B, K = sum_e P_e^T K_e P_e), summed in ascending element order, so the values are
// deterministic and independent of launch shapes; R_a = sum_e R_e(a) likewise.  The pass needs
// no clearing of the outputs, no atomics and no colouring: it reads each element block about
// twice (once per node of the pair) and writes each value once, contiguously.
#include <cuda_runtime.h>

#include "blocks.cuh"
#include "jetsci_internal.h"

namespace jetsci {

namespace {

constexpr int kChunk = 8;  // elements staged per step

// nodes (warps) per block of the row pass: shared memory stays under 48 KB
template <typename VT>
constexpr int row_warps() { return sizeof(VT) == 4 ? 8 : 4; }

template <typename VT>
struct RowSmem {
    // per warp: the staged blocks of a chunk -- compact layout: [element j][lb][kBlkStride],
    // block (min(la,lb), max(la,lb)) as stored; caller layout: [element j][72], node la's three
    // rows as stored -- reused to stage the output rows (3 x 96 values)
    VT blk[row_warps<VT>()][kChunk * 8 * kBlkStride];
    uint2 slots[row_warps<VT>()][kChunk];  // slot bytes of node a's row in each element
    double re[row_warps<VT>()][kChunk][3]; // residual vectors R_e(a)
};

// Asynchronous global -> shared copy of N (8 or 16) bytes; completed by cp.async.wait_group.
template <int N>
__device__ __forceinline__ void cp_async(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    if constexpr (N == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(N) : "memory");
}

// One warp per node a.  For each element around the node (eight at a time, ascending), the
// warp copies the eight blocks K_e(a, b) of node a's rows into shared memory with 16-byte
// asynchronous copies (compact layout: lane = (element, lb), whole blocks; caller layout: the 72
// contiguous values of node a's rows); lane s then sums, over the staged elements in order, the
// block whose column node has rank s in node a's neighbour list (the slot map), for s = lane,
// lane + 32, ...  Blocks stored as (lb, la) with lb < la are read transposed.
template <typename VT, bool kFull>
__global__ void __launch_bounds__(32 * row_warps<VT>()) k_gather_rows(int64_t n_nodes, const int64_t *__restrict__ ne_ptr,
                                                                      const uint32_t *__restrict__ ne,
                                                                      const uint8_t *__restrict__ slot,
                                                                      const int64_t *__restrict__ rowptr,
                                                                      const VT *__restrict__ blocks,
                                                                      const double *__restrict__ Re,
                                                                      VT *__restrict__ vals, double *__restrict__ R) {
    constexpr int kV16 = 16 / (int)sizeof(VT);  // values per 16-byte copy
    __shared__ __align__(16) RowSmem<VT> sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t a = (int64_t)blockIdx.x * row_warps<VT>() + w;
    if (a >= n_nodes) return;  // warp-uniform
    const int64_t j0 = ne_ptr[a], cnt = ne_ptr[a + 1] - j0;
    const int64_t base = rowptr[3 * a];
    const int nnb = (int)((rowptr[3 * a + 1] - base) / 3);
    const int n_sc = (nnb + 31) / 32;
    VT *const blk = sm.blk[w];
    double racc = 0.0;
    for (int sc = 0; sc < (n_sc > 0 ? n_sc : 1); sc++) {
        const int s = 32 * sc + lane;
        VT acc[9];
#pragma unroll
        for (int c = 0; c < 9; c++) acc[c] = VT(0);
        for (int64_t ec = 0; ec < cnt; ec += kChunk) {
            const int nc = (int)(cnt - ec < kChunk ? cnt - ec : kChunk);
            const uint32_t tl = lane < nc ? ne[j0 + ec + lane] : 0u;
            uint32_t la_pack = 0;  // 3 bits per element of the chunk
#pragma unroll
            for (int j = 0; j < kChunk; j++) la_pack |= (__shfl_sync(0xffffffffu, tl, j) & 7u) << (3 * j);
            if (n_sc > 0) {
                if constexpr (kFull) {
                    constexpr int kPer = 72 / kV16;  // 16-byte pieces of one element's rows
                    for (int q0 = 0; q0 < nc * kPer; q0 += 32) {  // warp-uniform trip count
                        const int q = q0 + lane;
                        const int j = q / kPer < kChunk ? q / kPer : kChunk - 1, part = q - kPer * j;
                        const uint32_t t = __shfl_sync(0xffffffffu, tl, j);
                        if (q < nc * kPer)
                            cp_async<16>(blk + 72 * j + kV16 * part,
                                         blocks + 576 * (int64_t)(t >> 3) + 72 * (t & 7) + kV16 * part);
                    }
                } else {
                    const int lb = lane & 7;
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int j = (lane >> 3) + 4 * h;
                        const uint32_t t = __shfl_sync(0xffffffffu, tl, j);
                        if (j < nc) {
                            const int64_t e = t >> 3;
                            const int la = (int)(t & 7);
                            const VT *src = blocks + kBlkStride * blk_index(e, la < lb ? la : lb, la < lb ? lb : la);
                            VT *dst = blk + kBlkStride * (8 * j + lb);
#pragma unroll
                            for (int c = 0; c < kBlkStride / kV16; c++) cp_async<16>(dst + kV16 * c, src + kV16 * c);
                        }
                    }
                }
                if (lane < nc) cp_async<8>(&sm.slots[w][lane], slot + 64 * (int64_t)(tl >> 3) + 8 * (tl & 7));
            }
            if (R && sc == 0) {  // lane 3 j + c copies R_e(a)_c of element j
                const uint32_t t = __shfl_sync(0xffffffffu, tl, lane / 3 < kChunk ? lane / 3 : kChunk - 1);
                if (lane < 3 * nc) cp_async<8>(&sm.re[w][0][0] + lane, Re + 3 * (int64_t)t + lane % 3);
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
            __syncwarp();
            if (s < nnb) {
                const uint32_t rep = 0x01010101u * (uint32_t)s;
                for (int j = 0; j < nc; j++) {
                    const uint2 sw = sm.slots[w][j];
                    const uint32_t mlo = __vcmpeq4(sw.x, rep), mhi = __vcmpeq4(sw.y, rep);
                    if (mlo | mhi) {
                        const int lb = mlo ? (__ffs(mlo) - 1) >> 3 : 4 + ((__ffs(mhi) - 1) >> 3);
                        if constexpr (kFull) {
                            const VT *x = blk + 72 * j + 3 * lb;
#pragma unroll
                            for (int i = 0; i < 3; i++)
#pragma unroll
                                for (int k = 0; k < 3; k++) acc[3 * i + k] += x[24 * i + k];
                        } else {
                            VT y[kBlkStride];
#pragma unroll
                            for (int c = 0; c < kBlkStride / kV16; c++)
                                reinterpret_cast<uint4 *>(y)[c] =
                                    reinterpret_cast<const uint4 *>(blk + kBlkStride * (8 * j + lb))[c];
                            const bool tr = (int)((la_pack >> (3 * j)) & 7u) > lb;
#pragma unroll
                            for (int i = 0; i < 3; i++)
#pragma unroll
                                for (int k = 0; k < 3; k++) acc[3 * i + k] += tr ? y[3 * k + i] : y[3 * i + k];
                        }
                    }
                }
            }
            if (R && sc == 0) {
                // lane 3 j + c holds R_e(a)_c of element j; a fixed tree over j (8 -> 4 -> 2 -> 1)
                double r = lane < 3 * nc ? (&sm.re[w][0][0])[lane] : 0.0;
                r += __shfl_down_sync(0xffffffffu, r, 12);
                r += __shfl_down_sync(0xffffffffu, r, 6);
                r += __shfl_down_sync(0xffffffffu, r, 3);
                racc += r;
            }
            __syncwarp();
        }
        if (n_sc == 0) break;
        // rows 3a, 3a+1, 3a+2 are contiguous (3 nnb values each): stage, then write coalesced
        const int ns = nnb - 32 * sc < 32 ? nnb - 32 * sc : 32;
        if (lane < ns)
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int k = 0; k < 3; k++) blk[96 * i + 3 * lane + k] = acc[3 * i + k];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 3; i++) {
            VT *row = vals + base + (int64_t)i * 3 * nnb + 96 * sc;
            for (int c = lane; c < 3 * ns; c += 32) row[c] = blk[96 * i + c];
        }
        __syncwarp();
    }
    if (R && lane < 3) R[3 * a + lane] = racc;
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
jetsci_status launch_gather_rows(jetsci_mesh m, const VT *blocks, bool full, const double *Re, VT *vals,
                                 double *R, cudaStream_t s) {
    if (m->n_nodes == 0) return JETSCI_OK;
    constexpr int kW = row_warps<VT>();
    const unsigned grid = (unsigned)((m->n_nodes + kW - 1) / kW);
    // several blocks per SM need more shared memory than the default carveout gives
    JETSCI_CUDA_TRY(cudaFuncSetAttribute(full ? k_gather_rows<VT, true> : k_gather_rows<VT, false>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared));
    if (full)
        k_gather_rows<VT, true><<<grid, 32 * kW, 0, s>>>(m->n_nodes, m->d_ne_ptr, m->d_ne, m->d_slot,
                                                                m->d_rowptr, blocks, Re, vals, R);
    else
        k_gather_rows<VT, false><<<grid, 32 * kW, 0, s>>>(m->n_nodes, m->d_ne_ptr, m->d_ne, m->d_slot,
                                                                 m->d_rowptr, blocks, Re, vals, R);
    JETSCI_CUDA_TRY(cudaGetLastError());
    return JETSCI_OK;
}

template jetsci_status launch_gather_rows<float>(jetsci_mesh, const float *, bool, const double *, float *,
                                                 double *, cudaStream_t);
template jetsci_status launch_gather_rows<double>(jetsci_mesh, const double *, bool, const double *, double *,
                                                  double *, cudaStream_t);

}  // namespace jetsci
