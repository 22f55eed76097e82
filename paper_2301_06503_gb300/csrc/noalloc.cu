// Allocation-free BiCGSTAB solve of a node-block CSR system.
//
// Some callers cannot allocate device memory at all: code that runs inside
// a host framework whose memory is fully pre-reserved, callers holding a
// captured-allocation budget, or plugins that must not touch the CUDA
// allocator.  For them lgdm_solve_noalloc takes its working storage from one
// file-scope __device__ array instead of a workspace: the caller passes only
// the system (inputs) and the solution buffer (output).
//
// CUDA loads the library's device code lazily, and this file's module holds
// only the array: the array is reserved on a device by the first call there,
// when its address is fetched with cudaGetSymbolAddress (with that device
// current; the address is cached per device), and it stays reserved until
// the process exits.  A call with nnode == 0 does only this set-up, so a
// caller can make it before reserving the rest of the device memory.  Host
// code cannot use the array's name as a device address: it only ever passes
// the fetched address to the kernels.
#include "lgdm_internal.cuh"

#include <algorithm>
#include <mutex>
#include <string>

namespace lgdm {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};
size_t up256(size_t n) { return (n + 255) & ~size_t(255); }

lgdm_status err(lgdm_status s, const std::string &m) {
  set_global_error(m);
  return s;
}

}  // namespace
}  // namespace lgdm

using namespace lgdm;

extern "C" lgdm_status lgdm_solve_noalloc(int32_t nd, int32_t nnode, const int32_t *nbr_ptr, const int32_t *nbr,
                                          const double *vals, const double *rhs, double *x, double rtol,
                                          int32_t max_iter, void *stream, int32_t *iters, double *rel_res) {
  if (nnode < 0 || (nnode > 0 && (nd < 2 || nd > 4 || !nbr_ptr || !nbr || !vals || !rhs || !x || !(rtol > 0.0) ||
                                   max_iter < 1)))
    return err(LGDM_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
    return err(LGDM_ERR_CUDA, "no current CUDA device");
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return err(LGDM_ERR_OOM, "the 64 MiB static scratch array could not be reserved on device " +
                                     std::to_string(dev) + " (device memory exhausted): make a first call "
                                     "(nnode = 0 suffices) before reserving the device memory");
      }
      if (e != cudaSuccess) return err(LGDM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  if (nnode == 0) return LGDM_OK;                  // set-up only
  const int nblocks_max = bicgstab_max_blocks<double>();
  const int64_t ndof = (int64_t)nd * nnode;
  const int64_t ntiles = krylov_ntiles(nnode);
  // layout inside the static array
  const size_t vec = up256(sizeof(double) * ndof);
  const size_t need = 9 * vec + up256(sizeof(double) * nnode * nd * nd) + up256(sizeof(double) * 12 * ntiles) +
                      up256(2 * sizeof(unsigned int)) + up256(sizeof(SolveResult)) + up256(sizeof(int32_t) * nnode);
  if (need > NOALLOC_SCRATCH_BYTES)
    return err(LGDM_ERR_OOM, "system needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
                                 std::to_string(NOALLOC_SCRATCH_BYTES));
  int64_t nb64 = std::min<int64_t>((ndof + 2 * KRYLOV_THREADS - 1) / (2 * KRYLOV_THREADS), ntiles);
  nb64 = std::min<int64_t>(std::max<int64_t>(nb64, krylov_min_blocks(nnode)), nblocks_max);
  if (krylov_min_blocks(nnode) < 1 || nb64 < krylov_min_blocks(nnode))
    return err(LGDM_ERR_INVALID_ARG, "system too large for one Krylov launch");
  const int nb = (int)std::max<int64_t>(nb64, 1);
  char *c = static_cast<char *>(base);
  double *v[9];
  for (int k = 0; k < 9; ++k, c += vec) v[k] = reinterpret_cast<double *>(c);
  double *minv = reinterpret_cast<double *>(c);
  c += up256(sizeof(double) * nnode * nd * nd);
  double *partial = reinterpret_cast<double *>(c);
  c += up256(sizeof(double) * 12 * ntiles);
  unsigned int *bar = reinterpret_cast<unsigned int *>(c);
  c += up256(2 * sizeof(unsigned int));
  SolveResult *res = reinterpret_cast<SolveResult *>(c);
  c += up256(sizeof(SolveResult));
  int32_t *diag = reinterpret_cast<int32_t *>(c);

  PatternView p{};
  p.nnode = nnode;
  p.nbr_ptr = nbr_ptr;
  p.nbr = nbr;
  p.diag_pair = diag;
  cudaError_t e = launch_diag_pairs(p, diag, s);
  if (e == cudaSuccess) e = launch_precond<double>(nd, p, vals, LGDM_PRECOND_NODE_BLOCK, minv, s);
  if (e != cudaSuccess) return err(LGDM_ERR_CUDA, std::string("set-up: ") + cudaGetErrorString(e));
  KrylovArgs a{};
  a.nd = nd;
  a.nnode = nnode;
  a.max_iter = max_iter;
  a.stall_iters = std::max(500, max_iter / 4);
  a.tile = krylov_tile(nnode);
  a.ntiles = (int32_t)ntiles;
  a.rtol = rtol;
  a.newton_tol = 0.0;
  a.p = p;
  a.vals = vals;
  a.minv = minv;
  a.rhs = rhs;
  a.x = x;
  a.r = v[0];
  a.r0 = v[1];
  a.pv = v[2];
  a.v = v[3];
  a.sv = v[4];
  a.t = v[5];
  a.ph = v[6];
  a.sh = v[7];
  a.xb = v[8];
  a.u = nullptr;
  a.partial = partial;
  a.bar_count = bar;
  a.bar_gen = bar + 1;
  a.res = res;
  a.wait_ns = 2000000000ull;                       // 2 s per grid-barrier wait
  a.barrier_extra = 0;
  e = cudaMemsetAsync(res, 0, sizeof(SolveResult), s);   // no stale result survives a timed-out launch
  if (e == cudaSuccess) e = launch_bicgstab<double>(a, nb, 0, s);
  if (e != cudaSuccess) return err(LGDM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  SolveResult out{};
  e = cudaMemcpyAsync(&out, res, sizeof(SolveResult), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return err(LGDM_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
  if (out.status == 4) return err(LGDM_ERR_TIMEOUT, "grid barrier timed out");
  if (iters) *iters = out.iters;
  if (rel_res) *rel_res = out.rel_res;
  if (out.status == 3) return err(LGDM_ERR_NONFINITE, "non-finite value in the solve");
  return LGDM_OK;
}
