// Preconditioned BiCGSTAB for the nonsymmetric coupled tangent (Eq. 11),
// one persistent cooperative launch per solve.
//
// Each block owns a contiguous range of nodes (so the node-block Jacobi
// preconditioner is block-local) and the rows of those nodes.  The CSR
// values are stored node-block by node-block: the columns of node pair
// (a, b) are contiguous, so the SpMV reads the node neighbour list instead
// of a column index per value.  Inner products are summed over fixed node
// tiles (see krylov_tile), published per tile, and after a grid barrier
// every block adds the tile sums in the same fixed order: all blocks see
// bit-identical scalars, and the result depends neither on timing nor on
// the number of blocks.  The grid barrier spins with a time limit and
// reports a timeout instead of hanging.
//
// mode 1 ends the launch with the Newton update u += delta and the
// convergence test ||du|| <= tol ||u||, ||de|| <= tol ||e|| (Algorithm 2);
// mode 2 does only that update; mode 0 only solves.
#include "lgdm_internal.cuh"
#include <cuda/atomic>

namespace lgdm {

constexpr int KT = KRYLOV_THREADS;
constexpr int KRYLOV_MAX_RESTARTS = 8;

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false when the wait timed out (another block never arrived within
// limit_ns nanoseconds of this block's arrival).
__device__ bool grid_barrier(unsigned int *count, unsigned int *gen, unsigned int nblocks,
                             unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> c(*count), g(*gen);
    // the block's writes reach thread 0 through __syncthreads; its release
    // (cumulative) publishes them, the acquire below receives the others'
    const unsigned int my_gen = g.load(cuda::memory_order_acquire);
    int ok = 1;
    if (c.fetch_add(1u, cuda::memory_order_acq_rel) == nblocks - 1) {
      c.store(0u, cuda::memory_order_relaxed);
      g.fetch_add(1u, cuda::memory_order_release);
    } else {
      const unsigned long long t0 = globaltimer();
      unsigned int spins = 0;
      while (g.load(cuda::memory_order_acquire) == my_gen) {
        if ((++spins & 255u) == 0 && globaltimer() - t0 > limit_ns) { ok = 0; break; }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Deterministic block sum of one value per thread (fixed shuffle tree).
__device__ double block_sum(double v) {
  __shared__ double ws[KT / 32];
  __shared__ double total;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < KT / 32; ++w) s += ws[w];
    total = s;
  }
  __syncthreads();
  const double r = total;
  __syncthreads();
  return r;
}

// Sum of the nb published partials (tile sums), same order in every block.
__device__ double grid_sum(const double *part, int nb) {
  double v = 0.0;
  for (int k = threadIdx.x; k < nb; k += KT) v += __ldcg(part + k);
  return block_sum(v);
}

// One row of y = K x.  The matrix may be float (FP32 tangent), but x is
// read and the products are accumulated in double: the smooth, low-energy
// vectors BiCGSTAB must resolve have |Kx| far below |K||x|, and a float
// accumulation would lose them.  x is written by other blocks during the
// launch, so it is read through L2 (__ldcg), never through a stale L1 line.
template <int ND, typename TT>
__device__ __forceinline__ double spmv_row(const PatternView &p, const TT *__restrict__ vals, const double *x,
                                           int64_t row) {
  const int32_t a = (int32_t)(row / ND), i = (int32_t)(row % ND);
  const int32_t pb = p.nbr_ptr[a], deg = p.nbr_ptr[a + 1] - pb;
  const TT *v = vals + (int64_t)ND * ND * pb + (int64_t)i * ND * deg;
  double acc = 0.0;
  for (int32_t s = 0; s < deg; ++s) {
    const double *xb = x + (int64_t)ND * p.nbr[pb + s];
#pragma unroll
    for (int j = 0; j < ND; ++j) acc += (double)v[ND * s + j] * __ldcg(xb + j);
  }
  return acc;
}

template <int ND, typename TT>
__device__ __forceinline__ void precond_rows(const TT *__restrict__ minv, const double *in, double *out,
                                             int64_t r0, int64_t r1) {
  for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
    const int64_t a = row / ND;
    const int i = (int)(row % ND);
    const TT *m = minv + (a * ND + i) * ND;
    const double *x = in + a * ND;
    double s = 0.0;                 // stored in TT, applied in double: a linear preconditioner
#pragma unroll
    for (int j = 0; j < ND; ++j) s += (double)m[j] * x[j];
    out[row] = s;
  }
}

// y = K x for the nd rows of node a.  One neighbour index and nd values of
// x feed nd*nd products, accumulated in double.  x is written by other
// blocks during the launch, so it is read through L2 (__ldcg).
template <int ND, typename TT>
__device__ __forceinline__ void spmv_node(const PatternView &p, const TT *__restrict__ vals, const double *x,
                                          int64_t a, double *y) {
  const int32_t pb = p.nbr_ptr[a], deg = p.nbr_ptr[a + 1] - pb;
  const TT *v = vals + (int64_t)ND * ND * pb;
  const int64_t rs = (int64_t)ND * deg;           // stride between the node's rows
#pragma unroll
  for (int i = 0; i < ND; ++i) y[i] = 0.0;
#pragma unroll 3
  for (int32_t s = 0; s < deg; ++s) {
    const double *xb = x + (int64_t)ND * p.nbr[pb + s];
    double xv[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) xv[j] = __ldcg(xb + j);
#pragma unroll
    for (int i = 0; i < ND; ++i)
#pragma unroll
      for (int j = 0; j < ND; ++j) y[i] += (double)v[i * rs + ND * s + j] * xv[j];
  }
}

// FP32-pipe products for the FP32 tangent.  A double x is carried as a float
// pair hi + lo (hi = x rounded to float, lo = the rest rounded to float:
// |x - hi - lo| <= 2^-48 |x|), written once by the vector's producer.  Each
// product m * hi is split exactly into p + e (p rounded, e = fma(m, hi, -p));
// the p are summed with a two-sum that keeps every rounding error, and the
// errors, the e and the m * lo are summed in a second float.  The row value
// (double)S + (double)C is within a few 2^-48 of sum |m x| of the exact
// double-product row: FP64-grade for the Krylov iteration, on the FP32 pipe.
__device__ __forceinline__ float2 split_hl(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

template <bool CG>
__device__ __forceinline__ float2 vld2(const float2 *p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// y = K x for the nd rows of node a, K float, x as float pairs.
template <int ND, bool CG>
__device__ __forceinline__ void spmv_node_hl(const int32_t *__restrict__ nbr_ptr, const int32_t *__restrict__ nbr,
                                             const float *__restrict__ vals, const float2 *x, int64_t a,
                                             double *y) {
  const int32_t pb = nbr_ptr[a], deg = nbr_ptr[a + 1] - pb;
  const float *v = vals + (int64_t)ND * ND * pb;
  const int64_t rs = (int64_t)ND * deg;
  float S[ND], Cs[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) S[i] = Cs[i] = 0.0f;
#pragma unroll 3
  for (int32_t s = 0; s < deg; ++s) {
    const float2 *xb = x + (int64_t)ND * nbr[pb + s];
    float2 xv[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) xv[j] = vld2<CG>(xb + j);
#pragma unroll
    for (int i = 0; i < ND; ++i)
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const float m = v[i * rs + ND * s + j];
        const float p = __fmul_rn(m, xv[j].x);
        const float e = __fmaf_rn(m, xv[j].x, -p);           // m * hi = p + e exactly
        const float t = __fadd_rn(S[i], p);                  // two-sum: S + p = t + es exactly
        const float bp = __fsub_rn(t, S[i]);
        const float es = __fadd_rn(__fsub_rn(S[i], __fsub_rn(t, bp)), __fsub_rn(p, bp));
        S[i] = t;
        Cs[i] += es + __fmaf_rn(m, xv[j].y, e);
      }
  }
#pragma unroll
  for (int i = 0; i < ND; ++i) y[i] = (double)S[i] + (double)Cs[i];
}

// out = M^-1 in for node a (stored in TT, applied in double).
template <int ND, typename TT>
__device__ __forceinline__ void precond_apply(const TT *__restrict__ minv, int64_t a, const double *in, double *out) {
  const TT *m = minv + a * ND * ND;
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < ND; ++j) s += (double)m[i * ND + j] * in[j];
    out[i] = s;
  }
}

// Tile sums of NV per-node quantities over the block's nodes [n0, n1)
// (tiles [t0, t1) of T nodes): f(a, v) adds node a's terms to v[0..NV).
// Warp w of chunk c sums nodes n0 + c*KT + 32w .. +31 in a fixed shuffle
// tree; the tile sum adds its T/32 warp sums in order; tile k's sum of value
// j goes to out[j * stride + t0 + k].  ws holds 4 * KRYLOV_MAXW doubles.
template <int NV, typename F>
__device__ __forceinline__ void reduce_tiles(int64_t n0, int64_t n1, int64_t t0, int64_t t1, int T, double *ws,
                                             double *out, int64_t stride, F &&f) {
  __syncthreads();                               // ws may still be read by the previous call
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t len = n1 - n0;
  const int64_t nch = (len + KT - 1) / KT;
  const int nwc = (int)((len + 31) / 32);
  for (int64_t c = 0; c < nch; ++c) {
    const int64_t a = n0 + c * KT + threadIdx.x;
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    if (a < n1) f(a, v);
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int64_t wc = c * (KT / 32) + w;
    if (lane == 0 && wc < nwc) {
#pragma unroll
      for (int k = 0; k < NV; ++k) ws[k * KRYLOV_MAXW + wc] = v[k];
    }
  }
  __syncthreads();
  const int wpt = T / 32;
  const int ntl = (int)(t1 - t0);
  for (int i = threadIdx.x; i < ntl * NV; i += KT) {
    const int k = i / ntl, tt = i - k * ntl;
    const int j0 = tt * wpt, j1 = min(j0 + wpt, nwc);
    double sum = 0.0;
    for (int j = j0; j < j1; ++j) sum += ws[k * KRYLOV_MAXW + j];
    __stcg(out + k * stride + t0 + tt, sum);
  }
}

// ---------------------------------------------------------------- multigrid V-cycle
// Loads of the V-cycle vectors.  Grid-wide levels read values other blocks
// wrote during the launch: through L2 (CG).  The single-block levels read
// only what their own block wrote since the last __syncthreads: through L1.
template <bool CG>
__device__ __forceinline__ double vld(const double *p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// y = (A_l x~) for node a of level l, with x~[b] = x[b] + zc[agg[b]] when zc
// is given (the prolonged coarse correction added on the fly).
template <int ND, typename TT, bool CG>
__device__ __forceinline__ void lev_spmv(const AmgLevel &L, int64_t a, const double *x, const double *zc,
                                         double *y) {
  const int32_t pb = L.nbr_ptr[a], deg = L.nbr_ptr[a + 1] - pb;
  const TT *v = static_cast<const TT *>(L.vals) + (int64_t)ND * ND * pb;
  const int64_t rs = (int64_t)ND * deg;
  const int32_t *nbr = L.nbr, *agg = L.agg;
  const uint8_t *held = L.held;
#pragma unroll
  for (int i = 0; i < ND; ++i) y[i] = 0.0;
#pragma unroll 3
  for (int32_t s = 0; s < deg; ++s) {
    const int32_t b = nbr[pb + s];
    double xv[ND];
#pragma unroll
    for (int j = 0; j < ND; ++j) xv[j] = vld<CG>(x + (int64_t)ND * b + j);
    if (zc) {
      const double *zb = zc + (int64_t)ND * agg[b];
      if (held) {
#pragma unroll
        for (int j = 0; j < ND; ++j)
          if (!held[(int64_t)ND * b + j]) xv[j] += vld<CG>(zb + j);
      } else {
#pragma unroll
        for (int j = 0; j < ND; ++j) xv[j] += vld<CG>(zb + j);
      }
    }
#pragma unroll
    for (int i = 0; i < ND; ++i)
#pragma unroll
      for (int j = 0; j < ND; ++j) y[i] += (double)v[i * rs + ND * s + j] * xv[j];
  }
}

// X[a] = omega M_l^-1 v[a]  (v read through L2: it may come from another block)
template <int ND, typename TT>
__device__ __forceinline__ void lev_presmooth(const AmgLevel &L, int64_t a, const double *v, double *X) {
  double in[ND], out[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) in[i] = __ldcg(v + ND * a + i);
  precond_apply<ND, TT>(static_cast<const TT *>(L.minv), a, in, out);
  float2 *Xhl = L.Xhl;
#pragma unroll
  for (int i = 0; i < ND; ++i) X[ND * a + i] = AMG_OMEGA * out[i];
  if (Xhl) {
#pragma unroll
    for (int i = 0; i < ND; ++i) Xhl[ND * a + i] = split_hl(AMG_OMEGA * out[i]);
  }
}

// R[a] = v[a] - (A_l X)[a]
template <int ND, typename TT, bool CG>
__device__ __forceinline__ void lev_residual(const AmgLevel &L, int64_t a, const double *v, const double *X,
                                             double *R) {
  double y[ND];
  if constexpr (sizeof(TT) == 4) {
    if (L.Xhl) spmv_node_hl<ND, CG>(L.nbr_ptr, L.nbr, static_cast<const float *>(L.vals), L.Xhl, a, y);
    else lev_spmv<ND, TT, CG>(L, a, X, nullptr, y);
  } else {
    lev_spmv<ND, TT, CG>(L, a, X, nullptr, y);
  }
#pragma unroll
  for (int i = 0; i < ND; ++i) R[ND * a + i] = __ldcg(v + ND * a + i) - y[i];
}

// v_c[I] = sum of R over the members of aggregate I (fixed order; dofs the
// finer level holds are left out); with Xc given also Xc[I] = omega M_c^-1 v_c[I].
template <int ND, typename TT, bool CG>
__device__ __forceinline__ void lev_restrict(const AmgLevel &C, int64_t I, const double *R, double *vc, double *Xc,
                                             const uint8_t *fheld) {
  double acc[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) acc[i] = 0.0;
  const int32_t m1 = C.mem_ptr[I + 1];
  if (fheld) {
    for (int32_t m = C.mem_ptr[I]; m < m1; ++m) {
      const int64_t f = (int64_t)ND * C.mem[m];
#pragma unroll
      for (int i = 0; i < ND; ++i)
        if (!fheld[f + i]) acc[i] += vld<CG>(R + f + i);
    }
  } else {
    for (int32_t m = C.mem_ptr[I]; m < m1; ++m) {
      const double *r = R + (int64_t)ND * C.mem[m];
#pragma unroll
      for (int i = 0; i < ND; ++i) acc[i] += vld<CG>(r + i);
    }
  }
#pragma unroll
  for (int i = 0; i < ND; ++i) vc[ND * I + i] = acc[i];
  if (Xc) {
    double out[ND];
    precond_apply<ND, TT>(static_cast<const TT *>(C.minv), I, acc, out);
#pragma unroll
    for (int i = 0; i < ND; ++i) Xc[ND * I + i] = AMG_OMEGA * out[i];
  }
}

// Coarse correction and post-smoothing of node a: with x~ = X + P zc,
// z[a] = x~[a] + omega M_l^-1 (v[a] - (A_l x~)[a]).
template <int ND, typename TT, bool CG>
__device__ __forceinline__ void lev_postsmooth(const AmgLevel &L, int64_t a, const double *v, const double *X,
                                               const double *zc, double *z, float2 *zhl = nullptr) {
  double y[ND], r[ND], out[ND], zv[ND];
  const uint8_t *held = L.held;
  lev_spmv<ND, TT, CG>(L, a, X, zc, y);
  const double *za = zc + (int64_t)ND * L.agg[a];
#pragma unroll
  for (int i = 0; i < ND; ++i) r[i] = __ldcg(v + ND * a + i) - y[i];
  precond_apply<ND, TT>(static_cast<const TT *>(L.minv), a, r, out);
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    const double c = (held && held[ND * a + i]) ? 0.0 : vld<CG>(za + i);
    zv[i] = vld<CG>(X + ND * a + i) + c + AMG_OMEGA * out[i];
  }
#pragma unroll
  for (int i = 0; i < ND; ++i) z[ND * a + i] = zv[i];
  if (zhl) {
#pragma unroll
    for (int i = 0; i < ND; ++i) zhl[ND * a + i] = split_hl(zv[i]);
  }
}

// The V-cycle below level k run by one block: vk in, zk out (levels k ..
// nlev-1, __syncthreads between the steps).  The coarsest level is solved with
// its dense inverse, or, without one, by four damped block-Jacobi sweeps.
template <int ND, typename TT>
__device__ void amg_single_block(const AmgInfo &M, int k, const double *vk, double *zk, float2 *zkhl = nullptr) {
  const AmgLevel *lev = M.lev;
  const int L = M.nlev;
  if (k < L - 1)
    for (int64_t a = threadIdx.x; a < lev[k].nnode; a += KT) lev_presmooth<ND, TT>(lev[k], a, vk, lev[k].X);
  __syncthreads();
  for (int l = k; l < L - 1; ++l) {
    const AmgLevel &F = lev[l], &C = lev[l + 1];
    const double *v = (l == k) ? vk : F.v;
    for (int64_t a = threadIdx.x; a < F.nnode; a += KT) lev_residual<ND, TT, false>(F, a, v, F.X, F.R);
    __syncthreads();
    for (int64_t I = threadIdx.x; I < C.nnode; I += KT)
      lev_restrict<ND, TT, false>(C, I, F.R, C.v, (l + 1 < L - 1) ? C.X : nullptr, F.held);
    __syncthreads();
  }
  {
    const AmgLevel &C = lev[L - 1];
    const double *v = (L - 1 == k) ? vk : C.v;
    double *z = (L - 1 == k) ? zk : C.z;
    const int64_t N = (int64_t)ND * C.nnode;
    if (M.cinv) {
      for (int64_t i = threadIdx.x; i < N; i += KT) {
        double acc = 0.0;
        const double *row = M.cinv + i * N;
        for (int64_t j = 0; j < N; ++j) acc += row[j] * __ldcg(v + j);
        z[i] = acc;
      }
      __syncthreads();
    } else {
      for (int64_t a = threadIdx.x; a < C.nnode; a += KT) lev_presmooth<ND, TT>(C, a, v, C.X);
      __syncthreads();
      for (int sweep = 0; sweep < 4; ++sweep) {
        for (int64_t a = threadIdx.x; a < C.nnode; a += KT) {
          double y[ND], r[ND], out[ND];
          lev_spmv<ND, TT, false>(C, a, C.X, nullptr, y);
#pragma unroll
          for (int i = 0; i < ND; ++i) r[i] = __ldcg(v + ND * a + i) - y[i];
          precond_apply<ND, TT>(static_cast<const TT *>(C.minv), a, r, out);
#pragma unroll
          for (int i = 0; i < ND; ++i) z[ND * a + i] = C.X[ND * a + i] + AMG_OMEGA * out[i];
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < N; i += KT) C.X[i] = z[i];
        __syncthreads();
      }
    }
    if (L - 1 == k && zkhl) {                  // a one-level hierarchy: z is the output
      for (int64_t i = threadIdx.x; i < N; i += KT) zkhl[i] = split_hl(z[i]);
      __syncthreads();
    }
  }
  for (int l = L - 2; l >= k; --l) {
    const AmgLevel &F = lev[l];
    const double *v = (l == k) ? vk : F.v;
    double *z = (l == k) ? zk : F.z;
    for (int64_t a = threadIdx.x; a < F.nnode; a += KT)
      lev_postsmooth<ND, TT, false>(F, a, v, F.X, lev[l + 1].z, z, (l == k) ? zkhl : nullptr);
    __syncthreads();
  }
}

// z = M^-1 vin with M one multigrid V-cycle (one pre- and one post-smoothing
// sweep of damped block Jacobi per level), for the system of a group of nb
// blocks.  Level-0 nodes [n0, n1) are this block's; coarse levels above the
// single-block size are split evenly over the group; the levels from
// sb_level down are run by the group's first block.  Every value is a per-node
// fixed-order sum, so z does not depend on the group size.  Returns false if a
// grid barrier timed out.  On return z is complete for this block's level-0
// nodes only: the caller's next grid barrier publishes it.
template <int ND, typename TT>
__device__ bool amg_apply(const KrylovArgs &A, const double *vin, double *zout, float2 *zhl, int nb, int bid,
                          unsigned int nbar, int64_t n0, int64_t n1) {
  const AmgInfo &M = A.amg;
  const AmgLevel *lev = M.lev;
  const int S = M.sb_level;
  if (S == 0) {
    if (!grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns)) return false;
    if (bid == 0) amg_single_block<ND, TT>(M, 0, vin, zout, zhl);
    return true;
  }
  for (int64_t a = n0 + threadIdx.x; a < n1; a += KT) lev_presmooth<ND, TT>(lev[0], a, vin, lev[0].X);
  for (int l = 0; l < S; ++l) {
    const AmgLevel &F = lev[l], &C = lev[l + 1];
    const double *v = (l == 0) ? vin : F.v;
    const int64_t a0 = (l == 0) ? n0 : (int64_t)bid * F.nnode / nb, a1 = (l == 0) ? n1 : (int64_t)(bid + 1) * F.nnode / nb;
    if (!grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns)) return false;     // X_l published
    for (int64_t a = a0 + threadIdx.x; a < a1; a += KT) lev_residual<ND, TT, true>(F, a, v, F.X, F.R);
    if (!grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns)) return false;     // R_l published
    const int64_t c0 = (int64_t)bid * C.nnode / nb, c1 = (int64_t)(bid + 1) * C.nnode / nb;
    for (int64_t I = c0 + threadIdx.x; I < c1; I += KT)
      lev_restrict<ND, TT, true>(C, I, F.R, C.v, (l + 1 < S) ? C.X : nullptr, F.held);
  }
  if (!grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns)) return false;       // v_S published
  if (bid == 0) amg_single_block<ND, TT>(M, S, lev[S].v, lev[S].z);
  if (!grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns)) return false;       // z_S published
  for (int l = S - 1; l >= 0; --l) {
    const AmgLevel &F = lev[l];
    const double *v = (l == 0) ? vin : F.v;
    double *z = (l == 0) ? zout : F.z;
    const int64_t a0 = (l == 0) ? n0 : (int64_t)bid * F.nnode / nb, a1 = (l == 0) ? n1 : (int64_t)(bid + 1) * F.nnode / nb;
    for (int64_t a = a0 + threadIdx.x; a < a1; a += KT)
      lev_postsmooth<ND, TT, true>(F, a, v, F.X, lev[l + 1].z, z, (l == 0) ? zhl : nullptr);
    if (l > 0 && !grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns)) return false;   // z_l published
  }
  return true;
}

// The BiCGSTAB product K x for node a: on the FP32 pipe from the float-pair
// copy when the system has one (FP32 tangent), else with double products.
template <int ND, typename TT>
__device__ __forceinline__ void spmv_main(const KrylovArgs &A, const TT *vals, const double *x, const float2 *xhl,
                                          int64_t a, double *y) {
  if constexpr (sizeof(TT) == 4) {
    if (xhl) {
      spmv_node_hl<ND, true>(A.p.nbr_ptr, A.p.nbr, vals, xhl, a, y);
      return;
    }
  }
  spmv_node<ND, TT>(A.p, vals, x, a, y);
}

// The solver for one system on a group of nb blocks (bid = rank in the group).
// A thread owns whole nodes: their nd rows in every vector, the node-block
// preconditioner and the SpMV rows.
template <int ND, typename TT>
__device__ __forceinline__ void bicgstab_body(const KrylovArgs &A, const int nb, const int bid, const int mode) {
  __shared__ double ws[4 * KRYLOV_MAXW];
  const int T = A.tile;
  const int64_t NT = A.ntiles;
  const unsigned int nbar = (unsigned int)(nb + A.barrier_extra);   // blocks each grid barrier waits for
  const int64_t t0 = (int64_t)bid * NT / nb, t1 = (int64_t)(bid + 1) * NT / nb;
  const int64_t n0 = min(t0 * T, (int64_t)A.nnode), n1 = min(t1 * T, (int64_t)A.nnode);
  const TT *vals = static_cast<const TT *>(A.vals);
  const TT *minv = static_cast<const TT *>(A.minv);
  const bool mg = A.amg.nlev > 0;             // preconditioner: multigrid V-cycle, else block Jacobi
  double *P = A.partial;                      // [3 slots][4 values][ntiles]
  auto part = [&](int slot, int k) { return P + ((int64_t)slot * 4 + k) * NT; };
#define LGDM_NODES for (int64_t a = n0 + threadIdx.x; a < n1; a += KT)
#define LGDM_REDUCE(NV, slot, k0) reduce_tiles<NV>(n0, n1, t0, t1, T, ws, part(slot, k0), NT, [&](int64_t a, double *lv)
  int status = 1, it = 0;
  double rel = 0.0, bnorm = 0.0;
  double rho = 0.0, alpha = 1.0, omega = 1.0, rho_old = 1.0;
  double best = 1.0;                           // best relative residual seen; xb holds its iterate
  bool ok = true;

  if (mode != 2) {
    // bnorm = ||b||; x = 0
    LGDM_REDUCE(1, 2, 0) {
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        const int64_t row = ND * a + i;
        const double b = A.rhs[row];
        A.x[row] = 0.0;
        A.xb[row] = 0.0;
        lv[0] += b * b;
      }
    });
    ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns);
    if (ok) {
      bnorm = sqrt(grid_sum(part(2, 0), NT));
      if (!(bnorm > 0.0)) status = isfinite(bnorm) ? 0 : 3;
    }
    bool fresh = true, verify = false, first = true;
    int restarts = 0, since_best = 0;
    while (ok && bnorm > 0.0 && isfinite(bnorm)) {
      if (fresh) {
        // (re)start: r = b - K x (the true residual), shadow residual r0 = r
        if (restarts > 0) {
          LGDM_NODES {
#pragma unroll
            for (int i = 0; i < ND; ++i) A.ph[ND * a + i] = A.x[ND * a + i];
          }
          if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
        }
        LGDM_REDUCE(1, 2, 0) {
          double y[ND];
          if (restarts > 0) spmv_node<ND, TT>(A.p, vals, A.ph, a, y);
#pragma unroll
          for (int i = 0; i < ND; ++i) {
            const int64_t row = ND * a + i;
            const double rn = A.rhs[row] - (restarts > 0 ? y[i] : 0.0);
            A.r[row] = rn;
            A.r0[row] = rn;
            A.pv[row] = 0.0;
            A.v[row] = 0.0;
            lv[0] += rn * rn;
          }
        });
        if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
        rho = grid_sum(part(2, 0), NT);
        rel = sqrt(rho) / bnorm;
        if (!isfinite(rho)) { status = 3; break; }
        if (rel < best) {                       // the true residual of x: keep x as the best iterate
          best = rel;
          LGDM_NODES {
#pragma unroll
            for (int i = 0; i < ND; ++i) A.xb[ND * a + i] = A.x[ND * a + i];
          }
        }
        if (rel <= A.rtol) { status = 0; break; }
        if (verify && restarts >= KRYLOV_MAX_RESTARTS) { status = 1; break; }
        alpha = omega = rho_old = 1.0;
        fresh = false;
        verify = false;
        first = true;
      }
      if (it >= A.max_iter) { status = 1; break; }
      ++it;
      const double beta = first ? 0.0 : (rho / rho_old) * (alpha / omega);
      first = false;
      // p = r + beta (p - omega v); phat = M^-1 p
      LGDM_NODES {
        double pv[ND], ph[ND];
#pragma unroll
        for (int i = 0; i < ND; ++i) {
          const int64_t row = ND * a + i;
          pv[i] = A.r[row] + beta * (A.pv[row] - omega * A.v[row]);
          A.pv[row] = pv[i];
        }
        if (!mg) {
          precond_apply<ND, TT>(minv, a, pv, ph);
#pragma unroll
          for (int i = 0; i < ND; ++i) {
            A.ph[ND * a + i] = ph[i];
            if (A.ph_hl) A.ph_hl[ND * a + i] = split_hl(ph[i]);
          }
        }
      }
      if (mg && !(ok = amg_apply<ND, TT>(A, A.pv, A.ph, A.ph_hl, nb, bid, nbar, n0, n1))) break;
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      LGDM_REDUCE(1, 0, 0) {
        double y[ND];
        spmv_main<ND, TT>(A, vals, A.ph, A.ph_hl, a, y);
#pragma unroll
        for (int i = 0; i < ND; ++i) {
          A.v[ND * a + i] = y[i];
          lv[0] += A.r0[ND * a + i] * y[i];
        }
      });
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      const double r0v = grid_sum(part(0, 0), NT);
      if (!isfinite(r0v)) { status = 3; break; }
      if (r0v == 0.0) {                         // breakdown: restart from x
        if (restarts >= KRYLOV_MAX_RESTARTS) { status = 2; break; }
        ++restarts;
        fresh = true;
        continue;
      }
      alpha = rho / r0v;
      // s = r - alpha v; shat = M^-1 s
      LGDM_NODES {
        double sv[ND], sh[ND];
#pragma unroll
        for (int i = 0; i < ND; ++i) {
          const int64_t row = ND * a + i;
          sv[i] = A.r[row] - alpha * A.v[row];
          A.sv[row] = sv[i];
        }
        if (!mg) {
          precond_apply<ND, TT>(minv, a, sv, sh);
#pragma unroll
          for (int i = 0; i < ND; ++i) {
            A.sh[ND * a + i] = sh[i];
            if (A.sh_hl) A.sh_hl[ND * a + i] = split_hl(sh[i]);
          }
        }
      }
      if (mg && !(ok = amg_apply<ND, TT>(A, A.sv, A.sh, A.sh_hl, nb, bid, nbar, n0, n1))) break;
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      LGDM_REDUCE(2, 1, 0) {
        double y[ND];
        spmv_main<ND, TT>(A, vals, A.sh, A.sh_hl, a, y);
#pragma unroll
        for (int i = 0; i < ND; ++i) {
          A.t[ND * a + i] = y[i];
          lv[0] += y[i] * A.sv[ND * a + i];
          lv[1] += y[i] * y[i];
        }
      });
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      const double ts = grid_sum(part(1, 0), NT), tt = grid_sum(part(1, 1), NT);
      omega = (tt > 0.0) ? ts / tt : 0.0;
      LGDM_REDUCE(2, 2, 0) {
#pragma unroll
        for (int i = 0; i < ND; ++i) {
          const int64_t row = ND * a + i;
          A.x[row] += alpha * A.ph[row] + omega * A.sh[row];
          const double rn = A.sv[row] - omega * A.t[row];
          A.r[row] = rn;
          lv[0] += rn * rn;
          lv[1] += A.r0[row] * rn;
        }
      });
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      const double rr = grid_sum(part(2, 0), NT);
      rho_old = rho;
      rho = grid_sum(part(2, 1), NT);
      rel = sqrt(rr) / bnorm;
      if (!isfinite(rr)) { status = 3; break; }
      if (rel < best) {
        best = rel;
        since_best = 0;
        LGDM_NODES {
#pragma unroll
          for (int i = 0; i < ND; ++i) A.xb[ND * a + i] = A.x[ND * a + i];
        }
      } else if (++since_best > A.stall_iters) {   // no progress: stop with the best iterate
        status = 1;
        break;
      }
      if (rel <= A.rtol || omega == 0.0 || rho == 0.0) {
        // recursive residual small, or breakdown: check the true residual
        // and restart from x when it is not small enough
        if (restarts >= KRYLOV_MAX_RESTARTS && rel > A.rtol) { status = 2; break; }
        ++restarts;
        fresh = true;
        verify = rel <= A.rtol;
      }
    }
  }
  if (ok && mode != 2 && status != 0 && status != 3 && bnorm > 0.0) {
    // not converged: return the best iterate
    LGDM_NODES {
#pragma unroll
      for (int i = 0; i < ND; ++i) A.x[ND * a + i] = A.xb[ND * a + i];
    }
    rel = best;
  }
  if (ok && mode != 0 && status != 3) {
    LGDM_REDUCE(4, 0, 0) {
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        const int64_t row = ND * a + i;
        const double d = A.x[row];
        const double un = A.u[row] + d;
        A.u[row] = un;
        if (i == ND - 1) {
          lv[2] += d * d;
          lv[3] += un * un;
        } else {
          lv[0] += d * d;
          lv[1] += un * un;
        }
      }
    });
    ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns);
    if (ok) {
      double nrm[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) nrm[k] = sqrt(grid_sum(part(0, k), NT));
      if (bid == 0 && threadIdx.x == 0) {
        const bool cu = nrm[1] > 0.0 ? nrm[0] <= A.newton_tol * nrm[1] : nrm[0] <= 1e-30;
        const bool ce = nrm[3] > 0.0 ? nrm[2] <= A.newton_tol * nrm[3] : nrm[2] <= 1e-30;
        // a stalled or broken-down solve can return a tiny increment: never
        // accept it as convergence
        const bool solved = (mode == 2) ? (A.res->rel_res <= KRYLOV_NEWTON_ETA)
                                        : (status == 0 || rel <= KRYLOV_NEWTON_ETA);
        A.res->converged = (cu && ce && solved) ? 1 : 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) A.res->norms[k] = nrm[k];
        if (!(isfinite(nrm[0]) && isfinite(nrm[1]) && isfinite(nrm[2]) && isfinite(nrm[3]))) status = 3;
      }
    }
  }
#undef LGDM_NODES
#undef LGDM_REDUCE
  if (!ok) {
    if (threadIdx.x == 0) atomicMax(&A.res->status, 4);
    return;
  }
  if (bid == 0 && threadIdx.x == 0) {
    if (mode != 2) {
      A.res->iters = it;
      A.res->rel_res = rel;
      A.res->bnorm = bnorm;
    }
    atomicMax(&A.res->status, status);
  }
}

template <int ND, typename TT>
__global__ void __launch_bounds__(KT) bicgstab_kernel(KrylovArgs A, int mode) {
  bicgstab_body<ND, TT>(A, gridDim.x, blockIdx.x, mode);
}

// Several independent systems in one cooperative launch: block b belongs to
// the system s with group_start[s] <= b < group_start[s+1]; every system has
// its own barrier words and tile sums, so its arithmetic and its result are
// those of the system solved alone, whatever its group size.
template <int ND, typename TT>
__global__ void __launch_bounds__(KT) bicgstab_grouped_kernel(const KrylovArgs *__restrict__ args,
                                                              const int32_t *__restrict__ members,
                                                              const int32_t *__restrict__ group_start,
                                                              const int32_t *__restrict__ active, int nsys,
                                                              int mode) {
  int lo = 0, hi = nsys;                       // group_start[lo] <= b < group_start[hi]
  const int b = blockIdx.x;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (group_start[mid] <= b) lo = mid;
    else hi = mid;
  }
  const int sm = members[lo];
  if (!active[sm]) return;
  const KrylovArgs A = args[sm];
  bicgstab_body<ND, TT>(A, group_start[lo + 1] - group_start[lo], b - group_start[lo], mode);
}

// Zero the barrier words and the status of every active member before a
// grouped launch; a solve (mode != 2) also clears the previous result, which
// the update launch (mode 2) still reads.
__global__ void reset_members_kernel(const KrylovArgs *__restrict__ args, const int32_t *__restrict__ members,
                                     const int32_t *__restrict__ active, int n, int mode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sm = members[i];
  if (!active[sm]) return;
  args[sm].bar_count[0] = 0u;
  args[sm].bar_gen[0] = 0u;
  args[sm].res->status = 0;
  if (mode != 2) {
    args[sm].res->iters = 0;
    args[sm].res->rel_res = 0.0;
    args[sm].res->bnorm = 0.0;
  }
}

// Copy every member's result block into one array (one copy to the host).
__global__ void collect_results_kernel(const KrylovArgs *__restrict__ args, int n, SolveResult *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = *args[i].res;
}

cudaError_t launch_collect_results(const KrylovArgs *d_args, int n, SolveResult *d_out, cudaStream_t s) {
  collect_results_kernel<<<(n + 127) / 128, 128, 0, s>>>(d_args, n, d_out);
  return cudaGetLastError();
}

template <typename TT>
cudaError_t launch_bicgstab_grouped(int nd, const KrylovArgs *d_args, const int32_t *d_members,
                                    const int32_t *d_group_start, const int32_t *d_active, int nsys,
                                    int total_blocks, int mode, cudaStream_t s) {
  reset_members_kernel<<<(nsys + 127) / 128, 128, 0, s>>>(d_args, d_members, d_active, nsys, mode);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int ns = nsys;
  void *params[] = {(void *)&d_args, (void *)&d_members, (void *)&d_group_start, (void *)&d_active, &ns, &mode};
  const void *fn = nullptr;
  switch (nd) {
    case 2: fn = (const void *)bicgstab_grouped_kernel<2, TT>; break;
    case 3: fn = (const void *)bicgstab_grouped_kernel<3, TT>; break;
    case 4: fn = (const void *)bicgstab_grouped_kernel<4, TT>; break;
    default: return cudaErrorInvalidValue;
  }
  return cudaLaunchCooperativeKernel(fn, dim3(total_blocks), dim3(KT), params, 0, s);
}
template cudaError_t launch_bicgstab_grouped<double>(int, const KrylovArgs *, const int32_t *, const int32_t *,
                                                     const int32_t *, int, int, int, cudaStream_t);
template cudaError_t launch_bicgstab_grouped<float>(int, const KrylovArgs *, const int32_t *, const int32_t *,
                                                    const int32_t *, int, int, int, cudaStream_t);

template <typename TT>
int bicgstab_grouped_max_blocks() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int p2 = 0, p3 = 0, p4 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, bicgstab_grouped_kernel<2, TT>, KT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p3, bicgstab_grouped_kernel<3, TT>, KT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, bicgstab_grouped_kernel<4, TT>, KT, 0);
  int per = p2 < p3 ? p2 : p3;
  per = per < p4 ? per : p4;
  return per * sms;
}
template int bicgstab_grouped_max_blocks<double>();
template int bicgstab_grouped_max_blocks<float>();

template <typename TT>
int bicgstab_max_blocks() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per = 1 << 30;
  int p2 = 0, p3 = 0, p4 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, bicgstab_kernel<2, TT>, KT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p3, bicgstab_kernel<3, TT>, KT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, bicgstab_kernel<4, TT>, KT, 0);
  per = p2 < p3 ? p2 : p3;
  per = per < p4 ? per : p4;
  return per * sms;
}
template int bicgstab_max_blocks<double>();
template int bicgstab_max_blocks<float>();

template <typename TT>
cudaError_t launch_bicgstab(const KrylovArgs &a, int nblocks, int mode, cudaStream_t s) {
  KrylovArgs args = a;
  void *params[] = {&args, &mode};
  const void *fn = nullptr;
  switch (a.nd) {
    case 2: fn = (const void *)bicgstab_kernel<2, TT>; break;
    case 3: fn = (const void *)bicgstab_kernel<3, TT>; break;
    case 4: fn = (const void *)bicgstab_kernel<4, TT>; break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaMemsetAsync(a.bar_count, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&a.res->status, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(KT), params, 0, s);
}
template cudaError_t launch_bicgstab<double>(const KrylovArgs &, int, int, cudaStream_t);
template cudaError_t launch_bicgstab<float>(const KrylovArgs &, int, int, cudaStream_t);

// ====================================================================== GMRES
// Restarted GMRES(m), right-preconditioned by the node-block Jacobi inverse,
// classical Gram-Schmidt with one re-orthogonalisation pass.  It is the
// fallback when BiCGSTAB stagnates or diverges on an indefinite tangent:
// GMRES never increases the residual within a cycle.  Warm start from the
// x already in A.x.  Inner products against the basis are computed
// warp-per-vector over each block's rows, published per block, reduced by
// one block per value, then read by all: every block sees the same numbers.
namespace {

template <int ND, typename TT>
__device__ void gm_residual(const KrylovArgs &A, const GmresArgs &G, int64_t r0, int64_t r1, double *rout,
                            double *lsq) {
  // rout = b - K x (x copied to the scratch vector first: other blocks read it)
  double l = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
    const double rn = A.rhs[row] - spmv_row<ND, TT>(A.p, static_cast<const TT *>(A.vals), G.xs, row);
    rout[row] = rn;
    l += rn * rn;
  }
  *lsq = l;
}

}  // namespace

template <int ND, typename TT>
__global__ void __launch_bounds__(KT) gmres_kernel(KrylovArgs A, GmresArgs G) {
  const int nb = gridDim.x, bid = blockIdx.x;
  const unsigned int nbar = (unsigned int)(nb + A.barrier_extra);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = KT / 32;
  const int64_t n0 = (int64_t)bid * A.nnode / nb, n1 = (int64_t)(bid + 1) * A.nnode / nb;
  const int64_t r0 = ND * n0, r1 = ND * n1;
  const int64_t ld = G.ld;
  const int m = G.m;
  const TT *minv = static_cast<const TT *>(A.minv);
  double *V = G.V;
  __shared__ double s_h[GMRES_MAX_M + 2], s_h2[GMRES_MAX_M + 2];
  __shared__ double s_cs[GMRES_MAX_M], s_sn[GMRES_MAX_M], s_g[GMRES_MAX_M + 1];
  __shared__ int s_k;
  auto part = [&](int i) { return G.dots + (int64_t)i * nb; };
  // block-sum of one value per thread, published as partial i
  auto publish = [&](int i, double v) {
    const double s = block_sum(v);
    if (threadIdx.x == 0) __stcg(part(i) + bid, s);
  };
  // one block per value sums the nb partials of values 0..cnt-1 into G.final
  auto reduce = [&](int cnt) {
    for (int i = bid; i < cnt; i += nb) {
      const double s = grid_sum(part(i), nb);
      if (threadIdx.x == 0) __stcg(G.final + i, s);
    }
  };
  bool ok = true;
  int status = 1, it = 0;
  double bnorm = 0.0, rel = 1.0;
  // ||b||
  {
    double l = 0.0;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) l += A.rhs[row] * A.rhs[row];
    publish(0, l);
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) G.xs[row] = A.x[row];
    ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns);
    if (ok) bnorm = sqrt(grid_sum(part(0), nb));
  }
  if (ok && !(bnorm > 0.0)) status = isfinite(bnorm) ? 0 : 3;
  double prev_cycle = 1e300;
  for (int cycle = 0; ok && bnorm > 0.0 && isfinite(bnorm); ++cycle) {
    // true residual of the current x
    double l;
    gm_residual<ND, TT>(A, G, r0, r1, V, &l);            // V_0 <- r (unnormalised)
    publish(0, l);
    if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
    const double beta = sqrt(grid_sum(part(0), nb));
    rel = beta / bnorm;
    if (!isfinite(beta)) { status = 3; break; }
    if (rel <= A.rtol) { status = 0; break; }
    if (rel >= prev_cycle) {
      // the cycle made the true residual worse (rounding in an ill-conditioned
      // least-squares update): return the previous iterate
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) A.x[row] = A.xb[row];
      rel = prev_cycle;
      status = 1;
      break;
    }
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) A.xb[row] = A.x[row];
    if (it >= A.max_iter) { status = 1; break; }
    if (rel > 0.999 * prev_cycle) { status = 1; break; }    // a whole cycle without progress
    prev_cycle = rel;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) V[row] /= beta;
    if (threadIdx.x == 0) {
      s_g[0] = beta;
      for (int i = 1; i <= m; ++i) s_g[i] = 0.0;
    }
    __syncthreads();              // the preconditioner reads whole nodes: rows of other threads
    int k = 0;
    for (int j = 0; j < m && it < A.max_iter; ++j) {
      ++it;
      const double *Vj = V + j * ld;
      double *W = V + (j + 1) * ld;
      // z = M^-1 V_j (node-local), into the scratch vector read by the SpMV
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
        const int64_t a = row / ND;
        const int i = (int)(row % ND);
        const TT *mm = minv + (a * ND + i) * ND;
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < ND; ++q) s += (double)mm[q] * Vj[a * ND + q];
        G.xs[row] = s;
      }
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT)
        W[row] = spmv_row<ND, TT>(A.p, static_cast<const TT *>(A.vals), G.xs, row);
      __syncthreads();
      // pass 1: h_i = (V_i, w)
      for (int i = warp; i <= j; i += NW) {
        const double *Vi = V + i * ld;
        double s = 0.0;
        for (int64_t row = r0 + lane; row < r1; row += 32) s += Vi[row] * W[row];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) __stcg(part(i) + bid, s);
      }
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      reduce(j + 1);
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      for (int i = threadIdx.x; i <= j; i += KT) s_h[i] = __ldcg(G.final + i);
      __syncthreads();
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
        double s = 0.0;
        for (int i = 0; i <= j; ++i) s += s_h[i] * V[i * ld + row];
        W[row] -= s;
      }
      __syncthreads();
      // pass 2 (re-orthogonalisation)
      for (int i = warp; i <= j; i += NW) {
        const double *Vi = V + i * ld;
        double s = 0.0;
        for (int64_t row = r0 + lane; row < r1; row += 32) s += Vi[row] * W[row];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) __stcg(part(i) + bid, s);
      }
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      reduce(j + 1);
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      for (int i = threadIdx.x; i <= j; i += KT) s_h2[i] = __ldcg(G.final + i);
      __syncthreads();
      // ||w|| after both passes, computed directly (a Pythagorean update
      // cancels when the new direction is nearly in the span)
      double lw = 0.0;
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
        double s = 0.0;
        for (int i = 0; i <= j; ++i) s += s_h2[i] * V[i * ld + row];
        const double wn = W[row] - s;
        W[row] = wn;
        lw += wn * wn;
      }
      publish(GMRES_MAX_M + 1, lw);
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
      const double hnext = sqrt(grid_sum(part(GMRES_MAX_M + 1), nb));
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) W[row] = (hnext > 0.0) ? W[row] / hnext : 0.0;
      // Hessenberg column, previous rotations, new rotation (same in every block)
      if (threadIdx.x == 0) {
        double col[GMRES_MAX_M + 1];
        for (int i = 0; i <= j; ++i) col[i] = s_h[i] + s_h2[i];
        col[j + 1] = hnext;
        for (int i = 0; i < j; ++i) {
          const double t = s_cs[i] * col[i] + s_sn[i] * col[i + 1];
          col[i + 1] = -s_sn[i] * col[i] + s_cs[i] * col[i + 1];
          col[i] = t;
        }
        const double den = sqrt(col[j] * col[j] + col[j + 1] * col[j + 1]);
        const double c = den > 0.0 ? col[j] / den : 1.0, sn = den > 0.0 ? col[j + 1] / den : 0.0;
        s_cs[j] = c;
        s_sn[j] = sn;
        col[j] = den;
        s_g[j + 1] = -sn * s_g[j];
        s_g[j] = c * s_g[j];
        if (bid == 0)
          for (int i = 0; i <= j; ++i) G.R[(int64_t)j * (m + 1) + i] = col[i];
        s_k = j + 1;
      }
      __syncthreads();
      k = s_k;
      rel = fabs(s_g[k]) / bnorm;
      if (!isfinite(rel)) { status = 3; break; }
      if (rel <= A.rtol || hnext == 0.0) break;
    }
    if (!ok || status == 3) break;
    // x += M^-1 V_k y with R y = g (back substitution in block 0)
    if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
    if (bid == 0 && threadIdx.x == 0) {
      for (int i = k - 1; i >= 0; --i) {
        double s = s_g[i];
        for (int q = i + 1; q < k; ++q) s -= __ldcg(G.R + (int64_t)q * (m + 1) + i) * G.y[q];
        const double d = __ldcg(G.R + (int64_t)i * (m + 1) + i);
        G.y[i] = (d != 0.0) ? s / d : 0.0;
      }
    }
    if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += __ldcg(G.y + i) * V[i * ld + row];
      A.t[row] = s;
    }
    __syncthreads();
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
      const int64_t a = row / ND;
      const int i = (int)(row % ND);
      const TT *mm = minv + (a * ND + i) * ND;
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < ND; ++q) s += (double)mm[q] * A.t[a * ND + q];
      A.x[row] += s;
      G.xs[row] = A.x[row];
    }
    if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nbar, A.wait_ns))) break;
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicMax(&A.res->status, 4);
    return;
  }
  if (bid == 0 && threadIdx.x == 0) {
    A.res->iters = it;
    A.res->rel_res = rel;
    A.res->bnorm = bnorm;
    atomicMax(&A.res->status, status);
  }
}

template <typename TT>
int gmres_max_blocks() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int p2 = 0, p3 = 0, p4 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, gmres_kernel<2, TT>, KT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p3, gmres_kernel<3, TT>, KT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, gmres_kernel<4, TT>, KT, 0);
  int per = p2 < p3 ? p2 : p3;
  per = per < p4 ? per : p4;
  return per * sms;
}
template int gmres_max_blocks<double>();
template int gmres_max_blocks<float>();

template <typename TT>
cudaError_t launch_gmres(const KrylovArgs &a, const GmresArgs &g, int nblocks, cudaStream_t s) {
  if (g.m < 1 || g.m > GMRES_MAX_M) return cudaErrorInvalidValue;
  KrylovArgs args = a;
  GmresArgs gg = g;
  void *params[] = {&args, &gg};
  const void *fn = nullptr;
  switch (a.nd) {
    case 2: fn = (const void *)gmres_kernel<2, TT>; break;
    case 3: fn = (const void *)gmres_kernel<3, TT>; break;
    case 4: fn = (const void *)gmres_kernel<4, TT>; break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaMemsetAsync(a.bar_count, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&a.res->status, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(KT), params, 0, s);
}
template cudaError_t launch_gmres<double>(const KrylovArgs &, const GmresArgs &, int, cudaStream_t);
template cudaError_t launch_gmres<float>(const KrylovArgs &, const GmresArgs &, int, cudaStream_t);

}  // namespace lgdm
