// Aggregation multigrid for the node-block systems of the coupled tangent
// (Eq. 11a-d): the hierarchy of node graphs, built once per mesh on the host,
// and the per-assembly set-up of its level matrices on the device.
//
// Aggregation (host): nodes are visited in index order; a node whose
// neighbours are all still free forms an aggregate with them; every node
// left over joins the aggregate most frequent among its neighbours (the
// lowest index on ties), or forms one alone.  On the structured meshes of
// the benchmark this gives 3 x 3 (quads) and 3 x 3 x 3 (hexahedra) node
// aggregates.  The prolongation copies an aggregate's nd values to each of
// its nodes; the restriction is its transpose (sum over the aggregate).
//
// Set-up (device, after each assembly): the level-(l+1) matrix is the
// Galerkin product R A_l P.  Each of its nd x nd blocks (aggregate pair I, J)
// is the sum of the level-l blocks of the node pairs (a, b) with a in I and b
// in J, taken in increasing pair order from a map built on the host: no
// float atomics, the same result on every run.  Then the block-Jacobi
// inverses of each level, and the dense inverse of the coarsest matrix
// (Gauss-Jordan with partial pivoting in shared memory).
#include "lgdm_internal.cuh"
#include "node_block.cuh"

#include <algorithm>

namespace lgdm {

bool amg_build(int32_t n0, const std::vector<int32_t> &ptr0, const std::vector<int32_t> &nbr0, AmgHost &h) {
  h.lev.clear();
  h.lev.emplace_back();
  h.lev[0].nnode = n0;
  auto gptr = [&](size_t l) -> const std::vector<int32_t> & { return l == 0 ? ptr0 : h.lev[l].nbr_ptr; };
  auto gnbr = [&](size_t l) -> const std::vector<int32_t> & { return l == 0 ? nbr0 : h.lev[l].nbr; };
  while (h.lev.back().nnode > AMG_COARSE_MAX && (int)h.lev.size() < AMG_MAX_LEVELS) {
    const size_t l = h.lev.size() - 1;
    const int32_t n = h.lev[l].nnode;
    const std::vector<int32_t> &ptr = gptr(l), &nb = gnbr(l);
    std::vector<int32_t> agg(n, -1);
    int32_t na = 0;
    for (int32_t a = 0; a < n; ++a) {
      if (agg[a] >= 0) continue;
      bool free_all = true;
      for (int32_t k = ptr[a]; k < ptr[a + 1] && free_all; ++k) free_all = agg[nb[k]] < 0;
      if (!free_all) continue;
      for (int32_t k = ptr[a]; k < ptr[a + 1]; ++k) agg[nb[k]] = na;
      agg[a] = na;
      ++na;
    }
    std::vector<int32_t> cand;
    for (int32_t a = 0; a < n; ++a) {
      if (agg[a] >= 0) continue;
      cand.clear();
      for (int32_t k = ptr[a]; k < ptr[a + 1]; ++k)
        if (agg[nb[k]] >= 0) cand.push_back(agg[nb[k]]);
      if (cand.empty()) {
        agg[a] = na++;
        continue;
      }
      std::sort(cand.begin(), cand.end());
      int32_t best = cand[0], bestc = 0;
      for (size_t i = 0; i < cand.size();) {
        size_t j = i;
        while (j < cand.size() && cand[j] == cand[i]) ++j;
        if ((int32_t)(j - i) > bestc) { bestc = (int32_t)(j - i); best = cand[i]; }
        i = j;
      }
      agg[a] = best;
    }
    if (na > (int64_t)n * 4 / 5) break;                  // the graph does not coarsen
    AmgHost::Lev nx;
    nx.nnode = na;
    // members of each aggregate, in node order
    nx.mem_ptr.assign(na + 1, 0);
    for (int32_t a = 0; a < n; ++a) nx.mem_ptr[agg[a] + 1]++;
    for (int32_t i = 0; i < na; ++i) nx.mem_ptr[i + 1] += nx.mem_ptr[i];
    nx.mem.resize(n);
    {
      std::vector<int32_t> pos(nx.mem_ptr.begin(), nx.mem_ptr.end() - 1);
      for (int32_t a = 0; a < n; ++a) nx.mem[pos[agg[a]]++] = a;
    }
    // aggregate graph: I ~ J when a node of I neighbours a node of J
    nx.nbr_ptr.assign(na + 1, 0);
    std::vector<int32_t> tmp;
    for (int32_t I = 0; I < na; ++I) {
      tmp.clear();
      for (int32_t m = nx.mem_ptr[I]; m < nx.mem_ptr[I + 1]; ++m) {
        const int32_t a = nx.mem[m];
        for (int32_t k = ptr[a]; k < ptr[a + 1]; ++k) tmp.push_back(agg[nb[k]]);
      }
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      nx.nbr.insert(nx.nbr.end(), tmp.begin(), tmp.end());
      nx.nbr_ptr[I + 1] = (int32_t)nx.nbr.size();
    }
    const int32_t ncp = nx.nbr_ptr[na];
    nx.pair_node.resize(ncp);
    nx.diag_pair.resize(na);
    for (int32_t I = 0; I < na; ++I)
      for (int32_t k = nx.nbr_ptr[I]; k < nx.nbr_ptr[I + 1]; ++k) {
        nx.pair_node[k] = I;
        if (nx.nbr[k] == I) nx.diag_pair[I] = k;
      }
    // Galerkin map: level-l pairs grouped by the aggregate pair they sum into
    const int32_t nfp = ptr[n];
    std::vector<int32_t> target(nfp);
    nx.cmap_ptr.assign(ncp + 1, 0);
    for (int32_t a = 0; a < n; ++a)
      for (int32_t k = ptr[a]; k < ptr[a + 1]; ++k) {
        const int32_t I = agg[a], J = agg[nb[k]];
        const int32_t *lo = nx.nbr.data() + nx.nbr_ptr[I], *hi = nx.nbr.data() + nx.nbr_ptr[I + 1];
        const int32_t cp = (int32_t)(std::lower_bound(lo, hi, J) - nx.nbr.data());
        target[k] = cp;
        nx.cmap_ptr[cp + 1]++;
      }
    for (int32_t c = 0; c < ncp; ++c) nx.cmap_ptr[c + 1] += nx.cmap_ptr[c];
    nx.cmap.resize(nfp);
    {
      std::vector<int32_t> pos(nx.cmap_ptr.begin(), nx.cmap_ptr.end() - 1);
      for (int32_t k = 0; k < nfp; ++k) nx.cmap[pos[target[k]]++] = k;
    }
    h.lev[l].agg = std::move(agg);
    h.lev.push_back(std::move(nx));
  }
  return h.lev.size() >= 2 || n0 <= AMG_COARSE_MAX;
}

}  // namespace lgdm

namespace lgdm {

// Galerkin values of coarse pair cp of level l: the fixed-order sum of the
// level-(l-1) blocks listed for it.  Accumulated in double, stored as TT.
template <int ND, typename TT>
__device__ __forceinline__ void galerkin_pair(const AmgLevel &F, const AmgLevel &C, int64_t cp) {
  if (cp >= C.npairs) return;
  const int32_t I = C.pair_node[cp], pbI = C.nbr_ptr[I], degI = C.nbr_ptr[I + 1] - pbI;
  const int32_t sI = (int32_t)(cp - pbI);
  double acc[ND][ND];
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) acc[i][j] = 0.0;
  const TT *fv = static_cast<const TT *>(F.vals);
  const int32_t c1 = C.cmap_ptr[cp + 1];
  for (int32_t c = C.cmap_ptr[cp]; c < c1; ++c) {
    const int32_t fp = C.cmap[c];
    const int32_t a = F.pair_node[fp], pb = F.nbr_ptr[a], deg = F.nbr_ptr[a + 1] - pb;
    const TT *blk = fv + (int64_t)ND * ND * pb + (int64_t)ND * (fp - pb);
    if (F.held) {                              // held dofs of the finer level are not prolongated
      const int64_t ra = (int64_t)ND * a, cb = (int64_t)ND * F.nbr[fp];
#pragma unroll
      for (int i = 0; i < ND; ++i)
#pragma unroll
        for (int j = 0; j < ND; ++j)
          if (!F.held[ra + i] && !F.held[cb + j]) acc[i][j] += (double)blk[(int64_t)i * ND * deg + j];
    } else {
#pragma unroll
      for (int i = 0; i < ND; ++i)
#pragma unroll
        for (int j = 0; j < ND; ++j) acc[i][j] += (double)blk[(int64_t)i * ND * deg + j];
    }
  }
  TT *out = static_cast<TT *>(C.vals) + (int64_t)ND * ND * pbI + (int64_t)ND * sI;
#pragma unroll
  for (int i = 0; i < ND; ++i)
#pragma unroll
    for (int j = 0; j < ND; ++j) out[(int64_t)i * ND * degI + j] = (TT)acc[i][j];
}

template <int ND, typename TT>
__global__ void __launch_bounds__(256)
batch_amg_galerkin_kernel(const BatchSim *__restrict__ sims, const int32_t *__restrict__ members,
                          const int64_t *__restrict__ block_start, int nm, const int32_t *__restrict__ active,
                          int level) {
  const int j = find_member(block_start, nm, blockIdx.x);
  const int sm = members[j];
  if (!active[sm]) return;
  const AmgLevel *lev = sims[sm].amg.lev;
  galerkin_pair<ND, TT>(lev[level - 1], lev[level], (blockIdx.x - block_start[j]) * 256 + threadIdx.x);
}

template <int ND, typename TT>
__global__ void __launch_bounds__(128)
batch_amg_precond_kernel(const BatchSim *__restrict__ sims, const int32_t *__restrict__ members,
                         const int64_t *__restrict__ block_start, int nm, const int32_t *__restrict__ active,
                         int level) {
  const int j = find_member(block_start, nm, blockIdx.x);
  const int sm = members[j];
  if (!active[sm]) return;
  const AmgLevel &L = sims[sm].amg.lev[level];
  PatternView p{};
  p.nnode = L.nnode;
  p.nbr_ptr = L.nbr_ptr;
  p.diag_pair = L.diag_pair;
  precond_node<ND, TT>(p, static_cast<const TT *>(L.vals), LGDM_PRECOND_NODE_BLOCK, static_cast<TT *>(L.minv),
                       (int32_t)((blockIdx.x - block_start[j]) * 128 + threadIdx.x));
}

// Dense inverse of the coarsest matrix (N = nd * nc <= nd * AMG_COARSE_MAX
// rows): Gauss-Jordan with partial pivoting on [A | I] in shared memory, one
// block per member.  A zero pivot leaves its row of the inverse zero.
template <int ND, typename TT>
__global__ void __launch_bounds__(256)
batch_amg_coarse_kernel(const BatchSim *__restrict__ sims, const int32_t *__restrict__ members,
                        const int32_t *__restrict__ active) {
  extern __shared__ __align__(16) double M[];                // [N][2N]
  __shared__ double fcol[ND * AMG_COARSE_MAX];
  __shared__ int s_piv;
  __shared__ double s_inv;
  const int sm = members[blockIdx.x];
  if (!active[sm]) return;
  const AmgInfo &info = sims[sm].amg;
  if (info.cinv == nullptr) return;
  const AmgLevel &C = info.lev[info.nlev - 1];
  const int nc = C.nnode, N = ND * nc, W = 2 * N;
  for (int k = threadIdx.x; k < N * W; k += blockDim.x) {
    const int r = k / W, c = k % W;
    M[k] = (c >= N) ? ((c - N == r) ? 1.0 : 0.0) : 0.0;
  }
  __syncthreads();
  const TT *cv = static_cast<const TT *>(C.vals);
  for (int k = threadIdx.x; k < C.npairs; k += blockDim.x) {
    const int32_t I = C.pair_node[k], J = C.nbr[k], pb = C.nbr_ptr[I], deg = C.nbr_ptr[I + 1] - pb;
    const TT *blk = cv + (int64_t)ND * ND * pb + (int64_t)ND * (k - pb);
#pragma unroll
    for (int i = 0; i < ND; ++i)
#pragma unroll
      for (int j = 0; j < ND; ++j) M[(ND * I + i) * W + ND * J + j] = (double)blk[(int64_t)i * ND * deg + j];
  }
  __syncthreads();
  for (int c = 0; c < N; ++c) {
    if (threadIdx.x == 0) {
      int piv = c;
      double best = fabs(M[c * W + c]);
      for (int r = c + 1; r < N; ++r)
        if (fabs(M[r * W + c]) > best) { best = fabs(M[r * W + c]); piv = r; }
      s_piv = piv;
      s_inv = (M[piv * W + c] != 0.0) ? 1.0 / M[piv * W + c] : 0.0;
    }
    __syncthreads();
    const int piv = s_piv;
    const double inv = s_inv;
    for (int k = threadIdx.x; k < W; k += blockDim.x) {      // swap rows c and piv, scale row c
      const double a = M[c * W + k], b = M[piv * W + k];
      M[piv * W + k] = (piv != c) ? a : b;
      M[c * W + k] = b * inv;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x) fcol[r] = (r == c) ? 0.0 : M[r * W + c];
    __syncthreads();
    for (int k = threadIdx.x; k < N * W; k += blockDim.x) {
      const int r = k / W, col = k % W;
      if (r != c) M[k] -= fcol[r] * M[c * W + col];
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) info.cinv[k] = M[(k / N) * W + N + (k % N)];
}

template <typename TT>
cudaError_t launch_batch_amg_level(int nd, int level, const BatchSim *sims, const int32_t *members,
                                   const int64_t *pair_blocks, const int64_t *node_blocks, int nm, int64_t total_pb,
                                   int64_t total_nb, const int32_t *active, cudaStream_t s) {
  if (total_pb <= 0) return cudaSuccess;
#define LGDM_AL(ND)                                                                                                   \
  batch_amg_galerkin_kernel<ND, TT><<<(unsigned)total_pb, 256, 0, s>>>(sims, members, pair_blocks, nm, active, level); \
  batch_amg_precond_kernel<ND, TT><<<(unsigned)total_nb, 128, 0, s>>>(sims, members, node_blocks, nm, active, level);  \
  break
  switch (nd) {
    case 2: LGDM_AL(2);
    case 3: LGDM_AL(3);
    case 4: LGDM_AL(4);
    default: return cudaErrorInvalidValue;
  }
#undef LGDM_AL
  return cudaGetLastError();
}
template cudaError_t launch_batch_amg_level<double>(int, int, const BatchSim *, const int32_t *, const int64_t *,
                                                    const int64_t *, int, int64_t, int64_t, const int32_t *,
                                                    cudaStream_t);
template cudaError_t launch_batch_amg_level<float>(int, int, const BatchSim *, const int32_t *, const int64_t *,
                                                   const int64_t *, int, int64_t, int64_t, const int32_t *,
                                                   cudaStream_t);

template <typename TT>
cudaError_t launch_batch_amg_coarse(int nd, const BatchSim *sims, const int32_t *members, int nm,
                                    const int32_t *active, cudaStream_t s) {
  if (nm <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * (size_t)(nd * AMG_COARSE_MAX) * (2 * nd * AMG_COARSE_MAX);
  const void *fn = nullptr;
  switch (nd) {
    case 2: fn = (const void *)batch_amg_coarse_kernel<2, TT>; break;
    case 3: fn = (const void *)batch_amg_coarse_kernel<3, TT>; break;
    case 4: fn = (const void *)batch_amg_coarse_kernel<4, TT>; break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  switch (nd) {
    case 2: batch_amg_coarse_kernel<2, TT><<<nm, 256, smem, s>>>(sims, members, active); break;
    case 3: batch_amg_coarse_kernel<3, TT><<<nm, 256, smem, s>>>(sims, members, active); break;
    case 4: batch_amg_coarse_kernel<4, TT><<<nm, 256, smem, s>>>(sims, members, active); break;
  }
  return cudaGetLastError();
}
template cudaError_t launch_batch_amg_coarse<double>(int, const BatchSim *, const int32_t *, int, const int32_t *,
                                                     cudaStream_t);
template cudaError_t launch_batch_amg_coarse<float>(int, const BatchSim *, const int32_t *, int, const int32_t *,
                                                    cudaStream_t);

}  // namespace lgdm
