// Element-block workspace of the row-gather assembly (element pass -> node-row pass).
//
// The element pass writes, per element, the 24 x 24 stiffness rows (row 3a + i, column 3b + k:
// local node a, component i; 2,304 bytes in FP32, each row 96 contiguous bytes) and the 8 nodal
// residual vectors; the row pass (gather.cu) forms every CSR row from the rows of the elements
// around the row's node.  The same layout is the one callers of
// jetsci_assemble_element_blocks pass.  Element counts are padded to a multiple of 16.
#pragma once

#include <stdint.h>

namespace jetsci {

constexpr int kBlkPad = 16;  // element count padding (element passes run 8 or 16 per block)

inline int64_t blk_padded_elems(int64_t n_elem) { return (n_elem + kBlkPad - 1) / kBlkPad * kBlkPad; }

// bytes of the rows part of the workspace for value type size vs
inline size_t blk_full_bytes(int64_t n_elem, size_t vs) { return (size_t)blk_padded_elems(n_elem) * 576 * vs; }
// bytes of the residual part ([element][local node][3] doubles), which follows the rows
inline size_t blk_residual_bytes(int64_t n_elem) { return (size_t)blk_padded_elems(n_elem) * 24 * sizeof(double); }

}  // namespace jetsci
