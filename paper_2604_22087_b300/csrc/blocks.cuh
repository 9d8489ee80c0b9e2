// Element-block workspace of the row-gather assembly (element pass -> node-row pass).
//
// The element pass writes, per element, the 36 node-pair blocks a <= b of its (symmetric)
// tangent, each 3x3 row-major (row = displacement component at node a) in a slot of 12 values
// (the last 3 unused, so that every block starts on a 16-byte boundary), and its 8 nodal
// residual vectors; the row pass (gather.cu) forms every CSR row from the blocks of the
// elements around the row's node.  Elements are grouped by 8 (element e is position e % 8 of
// group e / 8); a group stores its 288 blocks in the element pass's work-item order, so that a
// warp's 32 consecutive items land in 32 consecutive blocks:
//   blocks 0..223:   position * 28 + p(a, b), the pairs a < b of each element, p row by row
//   blocks 224..287: 224 + position * 8 + a, the pairs a == b
// The residual part is [element][local node][3] doubles.
#pragma once

#include <stdint.h>

namespace jetsci {

constexpr int kBlkGroup = 8;      // elements per group
constexpr int kBlkPerGroup = 288; // 8 * 36 blocks
constexpr int kBlkOff = 224;      // 8 * 28 off-diagonal blocks first
constexpr int kBlkVals = 9;
constexpr int kBlkStride = 12;    // values per stored block
constexpr int kBlkPad = 16;       // element count padding (element passes run 8 or 16 per block)

// rank of the pair (a, b), a < b, among the 28 pairs ordered row by row
__host__ __device__ __forceinline__ int blk_pair(int a, int b) { return 7 * a - (a * (a - 1)) / 2 + (b - a - 1); }

// block index of the pair (a, b), a <= b, of element e
__host__ __device__ __forceinline__ int64_t blk_index(int64_t e, int a, int b) {
    const int64_t g = e / kBlkGroup;
    const int pos = (int)(e - kBlkGroup * g);
    const int r = a < b ? pos * 28 + blk_pair(a, b) : kBlkOff + pos * 8 + a;
    return g * kBlkPerGroup + r;
}

inline int64_t blk_padded_elems(int64_t n_elem) { return (n_elem + kBlkPad - 1) / kBlkPad * kBlkPad; }

// bytes of the block part of the workspace for value type size vs: compact symmetric layout,
// and the full layout [element][24][24] (element rows as a caller would pass them)
inline size_t blk_values_bytes(int64_t n_elem, size_t vs) {
    return (size_t)blk_padded_elems(n_elem) * 36 * kBlkStride * vs;
}
inline size_t blk_full_bytes(int64_t n_elem, size_t vs) { return (size_t)blk_padded_elems(n_elem) * 576 * vs; }
// bytes of the residual part ([element][local node][3] doubles), which follows the blocks
inline size_t blk_residual_bytes(int64_t n_elem) { return (size_t)blk_padded_elems(n_elem) * 24 * sizeof(double); }

}  // namespace jetsci
