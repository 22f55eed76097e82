// Preconditioned BiCGSTAB for the nonsymmetric coupled tangent (Eq. 11),
// one persistent cooperative launch per solve.
//
// Each block owns a contiguous range of nodes (so the node-block Jacobi
// preconditioner is block-local) and the rows of those nodes.  The CSR
// values are stored node-block by node-block: the columns of node pair
// (a, b) are contiguous, so the SpMV reads the node neighbour list instead
// of a column index per value.  Inner products are summed per block in a
// fixed tree, published, and after a grid barrier every block adds the
// per-block partials in the same fixed order: all blocks see bit-identical
// scalars and the result does not depend on timing.  The grid barrier spins
// with a time limit and reports a timeout instead of hanging.
//
// mode 1 ends the launch with the Newton update u += delta and the
// convergence test ||du|| <= tol ||u||, ||de|| <= tol ||e|| (Algorithm 2,
// lines 9 and 18); mode 2 does only that update; mode 0 only solves.
#include "lgdm_internal.cuh"
#include <cuda/atomic>

namespace lgdm {

constexpr int KT = KRYLOV_THREADS;
constexpr unsigned long long BARRIER_NS = 2000000000ull;   // 2 s
constexpr int KRYLOV_MAX_RESTARTS = 8;

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false when the wait timed out (another block never arrived).
__device__ bool grid_barrier(unsigned int *count, unsigned int *gen, unsigned int nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> c(*count), g(*gen);
    const unsigned int my_gen = g.load(cuda::memory_order_acquire);
    int ok = 1;
    __threadfence();
    if (c.fetch_add(1u, cuda::memory_order_acq_rel) == nblocks - 1) {
      c.store(0u, cuda::memory_order_relaxed);
      g.fetch_add(1u, cuda::memory_order_release);
    } else {
      const unsigned long long t0 = globaltimer();
      unsigned int spins = 0;
      while (g.load(cuda::memory_order_acquire) == my_gen) {
        if ((++spins & 255u) == 0 && globaltimer() - t0 > BARRIER_NS) { ok = 0; break; }
        __nanosleep(32);
      }
    }
    __threadfence();
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

// Sum of the nb published partials, same order in every block.
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
    TT s = (TT)0;
#pragma unroll
    for (int j = 0; j < ND; ++j) s += m[j] * (TT)x[j];
    out[row] = (double)s;
  }
}

template <int ND, typename TT>
__global__ void __launch_bounds__(KT) bicgstab_kernel(KrylovArgs A, int mode) {
  const int nb = gridDim.x, bid = blockIdx.x;
  const int64_t n0 = (int64_t)bid * A.nnode / nb, n1 = (int64_t)(bid + 1) * A.nnode / nb;
  const int64_t r0 = ND * n0, r1 = ND * n1;
  const TT *vals = static_cast<const TT *>(A.vals);
  const TT *minv = static_cast<const TT *>(A.minv);
  double *P = A.partial;                      // [3 slots][4 values][nb]
  auto part = [&](int slot, int k) { return P + ((int64_t)slot * 4 + k) * nb; };
  auto publish = [&](int slot, int k, double v) {
    const double s = block_sum(v);
    if (threadIdx.x == 0) __stcg(part(slot, k) + bid, s);
  };
  int status = 1, it = 0;
  double rel = 0.0, bnorm = 0.0;
  double rho = 0.0, alpha = 1.0, omega = 1.0, rho_old = 1.0;
  double best = 1.0;                           // best relative residual seen; xb holds its iterate
  bool ok = true;

  if (mode != 2) {
    // bnorm = ||b||; x = 0
    double l = 0.0;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
      const double b = A.rhs[row];
      A.x[row] = 0.0;
      A.xb[row] = 0.0;
      l += b * b;
    }
    publish(2, 0, l);
    ok = grid_barrier(A.bar_count, A.bar_gen, nb);
    if (ok) {
      bnorm = sqrt(grid_sum(part(2, 0), nb));
      if (!(bnorm > 0.0)) status = isfinite(bnorm) ? 0 : 3;
    }
    bool fresh = true, verify = false, first = true;
    int restarts = 0, since_best = 0;
    while (ok && bnorm > 0.0 && isfinite(bnorm)) {
      if (fresh) {
        // (re)start: r = b - K x (the true residual), shadow residual r0 = r
        if (restarts > 0) {
          for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) A.ph[row] = A.x[row];
          if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nb))) break;
        }
        double lrr = 0.0;
        for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
          const double rn = A.rhs[row] - (restarts > 0 ? spmv_row<ND, TT>(A.p, vals, A.ph, row) : 0.0);
          A.r[row] = rn;
          A.r0[row] = rn;
          A.pv[row] = 0.0;
          A.v[row] = 0.0;
          lrr += rn * rn;
        }
        publish(2, 0, lrr);
        if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nb))) break;
        rho = grid_sum(part(2, 0), nb);
        rel = sqrt(rho) / bnorm;
        if (!isfinite(rho)) { status = 3; break; }
        if (rel < best) {                       // the true residual of x: keep x as the best iterate
          best = rel;
          for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) A.xb[row] = A.x[row];
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
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT)
        A.pv[row] = A.r[row] + beta * (A.pv[row] - omega * A.v[row]);
      __syncthreads();
      precond_rows<ND, TT>(minv, A.pv, A.ph, r0, r1);
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nb))) break;
      double l1 = 0.0;
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
        const double vv = spmv_row<ND, TT>(A.p, vals, A.ph, row);
        A.v[row] = vv;
        l1 += A.r0[row] * vv;
      }
      publish(0, 0, l1);
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nb))) break;
      const double r0v = grid_sum(part(0, 0), nb);
      if (!isfinite(r0v)) { status = 3; break; }
      if (r0v == 0.0) {                         // breakdown: restart from x
        if (restarts >= KRYLOV_MAX_RESTARTS) { status = 2; break; }
        ++restarts;
        fresh = true;
        continue;
      }
      alpha = rho / r0v;
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) A.sv[row] = A.r[row] - alpha * A.v[row];
      __syncthreads();
      precond_rows<ND, TT>(minv, A.sv, A.sh, r0, r1);
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nb))) break;
      double lts = 0.0, ltt = 0.0;
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
        const double tv = spmv_row<ND, TT>(A.p, vals, A.sh, row);
        A.t[row] = tv;
        lts += tv * A.sv[row];
        ltt += tv * tv;
      }
      publish(1, 0, lts);
      publish(1, 1, ltt);
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nb))) break;
      const double ts = grid_sum(part(1, 0), nb), tt = grid_sum(part(1, 1), nb);
      omega = (tt > 0.0) ? ts / tt : 0.0;
      double lrr = 0.0, lrho = 0.0;
      for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
        A.x[row] += alpha * A.ph[row] + omega * A.sh[row];
        const double rn = A.sv[row] - omega * A.t[row];
        A.r[row] = rn;
        lrr += rn * rn;
        lrho += A.r0[row] * rn;
      }
      publish(2, 0, lrr);
      publish(2, 1, lrho);
      if (!(ok = grid_barrier(A.bar_count, A.bar_gen, nb))) break;
      const double rr = grid_sum(part(2, 0), nb);
      rho_old = rho;
      rho = grid_sum(part(2, 1), nb);
      rel = sqrt(rr) / bnorm;
      if (!isfinite(rr)) { status = 3; break; }
      if (rel < best) {
        best = rel;
        since_best = 0;
        for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) A.xb[row] = A.x[row];
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
    // not converged: return the best iterate (its recursive residual may be
    // an underestimate of the true one by the drift BiCGSTAB accumulates)
    __syncthreads();
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) A.x[row] = A.xb[row];
    rel = best;
  }
  if (ok && mode != 0 && status != 3) {
    double ldu = 0.0, lu = 0.0, lde = 0.0, le = 0.0;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
      const double d = A.x[row];
      const double un = A.u[row] + d;
      A.u[row] = un;
      if (row % ND == ND - 1) {
        lde += d * d;
        le += un * un;
      } else {
        ldu += d * d;
        lu += un * un;
      }
    }
    publish(0, 0, ldu);
    publish(0, 1, lu);
    publish(0, 2, lde);
    publish(0, 3, le);
    ok = grid_barrier(A.bar_count, A.bar_gen, nb);
    if (ok) {
      double nrm[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) nrm[k] = sqrt(grid_sum(part(0, k), nb));
      if (bid == 0 && threadIdx.x == 0) {
        const bool cu = nrm[1] > 0.0 ? nrm[0] <= A.newton_tol * nrm[1] : nrm[0] <= 1e-30;
        const bool ce = nrm[3] > 0.0 ? nrm[2] <= A.newton_tol * nrm[3] : nrm[2] <= 1e-30;
        // a stalled or broken-down solve can return a tiny increment: never
        // accept it as convergence
        const bool solved = (mode == 2) || status == 0 || rel <= 100.0 * A.rtol;
        A.res->converged = (cu && ce && solved) ? 1 : 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) A.res->norms[k] = nrm[k];
        if (!(isfinite(nrm[0]) && isfinite(nrm[1]) && isfinite(nrm[2]) && isfinite(nrm[3]))) status = 3;
      }
    }
  }
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

}  // namespace lgdm
