// Index helpers of the grid hierarchy shared by the kernels: coarse node k
// of an axis with n fine nodes sits at fine position min(2k, n - 1) (every
// even node is kept, and for even n the last node too); the other nodes are
// the coefficient nodes of the axis.
#pragma once

namespace mgb {

__device__ __forceinline__ int cpos(int k, int n) { return min(2 * k, n - 1); }
__device__ __forceinline__ bool is_coef(int j, int n) { return (j & 1) && (j != n - 1); }
__device__ __forceinline__ int nodal_k(int j, int n, int nc) { return j == n - 1 ? nc - 1 : (j >> 1); }

}  // namespace mgb
