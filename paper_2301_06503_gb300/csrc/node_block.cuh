// Device helpers shared by the assembly and multigrid translation units: the
// node-block inverse of the block-Jacobi preconditioner and the member search
// of the batched kernels.
#pragma once
#include "lgdm_internal.cuh"

namespace lgdm {

// Inverse of each node's nd x nd diagonal block (Gauss-Jordan, partial
// pivoting, in double), or of its diagonal only (point Jacobi).
template <int ND, typename TT>
__device__ __forceinline__ void precond_node(const PatternView &p, const TT *__restrict__ vals, int kind,
                                             TT *__restrict__ minv, int32_t a) {
  if (a >= p.nnode) return;
  const int32_t pb = p.nbr_ptr[a], deg = p.nbr_ptr[a + 1] - pb;
  const int32_t s = p.diag_pair[a] - pb;
  const int64_t vbase = (int64_t)ND * ND * pb + (int64_t)ND * s;
  double M[ND][2 * ND];
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const double v = (double)vals[vbase + (int64_t)i * ND * deg + j];
      M[i][j] = (kind == LGDM_PRECOND_NODE_BLOCK || i == j) ? v : 0.0;
      M[i][ND + j] = (i == j) ? 1.0 : 0.0;
    }
#pragma unroll
  for (int c = 0; c < ND; ++c) {
    int piv = c;
    double best = fabs(M[c][c]);
#pragma unroll
    for (int r = c + 1; r < ND; ++r)
      if (fabs(M[r][c]) > best) { best = fabs(M[r][c]); piv = r; }
#pragma unroll
    for (int r = 0; r < ND; ++r)
      if (r == piv && piv != c) {
#pragma unroll
        for (int k = 0; k < 2 * ND; ++k) { const double t = M[c][k]; M[c][k] = M[r][k]; M[r][k] = t; }
      }
    const double inv = (M[c][c] != 0.0) ? 1.0 / M[c][c] : 0.0;
#pragma unroll
    for (int k = 0; k < 2 * ND; ++k) M[c][k] *= inv;
#pragma unroll
    for (int r = 0; r < ND; ++r)
      if (r != c) {
        const double f = M[r][c];
#pragma unroll
        for (int k = 0; k < 2 * ND; ++k) M[r][k] -= f * M[c][k];
      }
  }
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) minv[((int64_t)a * ND + i) * ND + j] = (TT)M[i][ND + j];
}

// Many simulations of one element type in one launch.  The members' element
// tiles (pairs, nodes) are numbered consecutively; a block finds its member
// by binary search in the prefix array.  Inactive members are skipped.
__device__ __forceinline__ int find_member(const int64_t *__restrict__ start, int n, int64_t k) {
  int lo = 0, hi = n;                          // start[lo] <= k < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= k) lo = mid;
    else hi = mid;
  }
  return lo;
}


}  // namespace lgdm
