// Host side of the LGDM C ABI: input checks, the node-block CSR pattern and
// element-to-nonzero map, workspace layout, and the incremental-iterative
// driver (Algorithm 2) built from the device kernels.
#include "lgdm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace lgdm;

namespace {

thread_local std::string g_last_error;   // errors raised before a handle exists

int nen_of(int elem) { return elem_nen(elem); }
int dim_of(int elem) {
  return (elem == LGDM_L2 || elem == LGDM_L3) ? 1 : (elem == LGDM_Q4 || elem == LGDM_Q9) ? 2 : elem == LGDM_H8 ? 3 : 0;
}
// leading local nodes that carry the micro-equivalent strain
int nve_of(int elem) { return elem == LGDM_L3 ? 2 : elem == LGDM_Q9 ? 4 : nen_of(elem); }
// bits per local node in a packed element-pair contribution (element << 2 LB | a << LB | b)
int pack_bits(int nen) { return nen > 8 ? 4 : 3; }

// Node adjacency (nodes sharing an element, self included, sorted) and the
// element-to-node-pair contribution lists.
struct Pattern {
  std::vector<int32_t> nbr_ptr, nbr, pair_node, pc_ptr, pc, diag_pair;
  int64_t npairs = 0;
};

lgdm_status build_pattern(const lgdm_mesh &m, Pattern &P, bool with_contrib, std::string &err) {
  const int nen = nen_of(m.elem);
  const int32_t nn = m.nnode, ne = m.nelem;
  // incident elements per node
  std::vector<int32_t> inc_ptr(nn + 1, 0);
  for (int64_t k = 0; k < (int64_t)ne * nen; ++k) {
    const int32_t n = m.conn[k];
    if (n < 0 || n >= nn) {
      err = "connectivity entry " + std::to_string(k) + " out of range";
      return LGDM_ERR_INVALID_ARG;
    }
    inc_ptr[n + 1]++;
  }
  for (int32_t n = 0; n < nn; ++n)
    if (inc_ptr[n + 1] == 0) {                 // its rows would be empty: a singular system
      err = "node " + std::to_string(n) + " belongs to no element";
      return LGDM_ERR_INVALID_ARG;
    }
  for (int32_t n = 0; n < nn; ++n) inc_ptr[n + 1] += inc_ptr[n];
  std::vector<int32_t> inc(inc_ptr[nn]), fill(inc_ptr.begin(), inc_ptr.end() - 1);
  for (int32_t e = 0; e < ne; ++e)
    for (int a = 0; a < nen; ++a) inc[fill[m.conn[(int64_t)e * nen + a]]++] = e;
  // neighbour lists
  P.nbr_ptr.assign(nn + 1, 0);
  std::vector<int32_t> tmp;
  tmp.reserve(64 * 8);
  P.nbr.clear();
  P.nbr.reserve((size_t)nn * (nen == 8 ? 27 : nen == 4 ? 9 : 3));
  for (int32_t n = 0; n < nn; ++n) {
    tmp.clear();
    tmp.push_back(n);
    for (int32_t k = inc_ptr[n]; k < inc_ptr[n + 1]; ++k) {
      const int32_t e = inc[k];
      for (int b = 0; b < nen; ++b) tmp.push_back(m.conn[(int64_t)e * nen + b]);
    }
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    P.nbr.insert(P.nbr.end(), tmp.begin(), tmp.end());
    P.nbr_ptr[n + 1] = (int32_t)P.nbr.size();
    if ((int64_t)P.nbr.size() > INT32_MAX / 16) {
      err = "mesh too large for 32-bit pair indices";
      return LGDM_ERR_INVALID_ARG;
    }
  }
  P.npairs = (int64_t)P.nbr.size();
  if (!with_contrib) return LGDM_OK;
  const int LB = pack_bits(nen);
  if (((int64_t)ne << (2 * LB)) > INT32_MAX) {
    err = "too many elements for the packed contribution map";
    return LGDM_ERR_INVALID_ARG;
  }
  P.pair_node.resize(P.npairs);
  P.diag_pair.resize(nn);
  for (int32_t n = 0; n < nn; ++n)
    for (int32_t k = P.nbr_ptr[n]; k < P.nbr_ptr[n + 1]; ++k) {
      P.pair_node[k] = n;
      if (P.nbr[k] == n) P.diag_pair[n] = k;
    }
  auto pair_of = [&](int32_t a, int32_t b) {
    const int32_t *lo = P.nbr.data() + P.nbr_ptr[a], *hi = P.nbr.data() + P.nbr_ptr[a + 1];
    return (int32_t)(std::lower_bound(lo, hi, b) - P.nbr.data());
  };
  // contributions grouped by pair, in increasing element order
  P.pc_ptr.assign(P.npairs + 1, 0);
  std::vector<int32_t> epair((size_t)ne * nen * nen);
  for (int32_t e = 0; e < ne; ++e)
    for (int a = 0; a < nen; ++a)
      for (int b = 0; b < nen; ++b) {
        const int32_t p = pair_of(m.conn[(int64_t)e * nen + a], m.conn[(int64_t)e * nen + b]);
        epair[((int64_t)e * nen + a) * nen + b] = p;
        P.pc_ptr[p + 1]++;
      }
  for (int64_t p = 0; p < P.npairs; ++p) P.pc_ptr[p + 1] += P.pc_ptr[p];
  P.pc.resize(P.pc_ptr[P.npairs]);
  std::vector<int32_t> pos(P.pc_ptr.begin(), P.pc_ptr.end() - 1);
  for (int32_t e = 0; e < ne; ++e)
    for (int a = 0; a < nen; ++a)
      for (int b = 0; b < nen; ++b) {
        const int32_t p = epair[((int64_t)e * nen + a) * nen + b];
        P.pc[pos[p]++] = (e << (2 * LB)) | (a << LB) | b;
      }
  return LGDM_OK;
}

int64_t nd_sq(int nd) { return (int64_t)nd * nd; }

// Bump allocator over the caller's workspace; with base == nullptr it only counts.
struct Carver {
  char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

}  // namespace

struct lgdm_sim;
namespace {
void resolve_timers(lgdm_sim *s);
}

struct lgdm_sim {
  int elem = 0, dim = 0, nen = 0, ngp = 0, nd = 0;
  int32_t nnode = 0, nel = 0;
  int64_t ndof = 0, nnz = 0, npairs = 0, ncontrib = 0;
  lgdm_options opt{};
  lgdm_material mat{};
  MatConst mc{};
  cudaStream_t stream = nullptr;
  char *ws = nullptr;
  size_t ws_bytes = 0, ws_needed = 0;
  size_t tsize = 8;           // bytes of a tangent value
  // device arrays
  double *x = nullptr, *y = nullptr, *z = nullptr, *e_scale = nullptr, *vol_scale = nullptr;
  int32_t *conn = nullptr;
  int32_t *nbr_ptr = nullptr, *nbr = nullptr, *pair_node = nullptr, *pc_ptr = nullptr, *pc = nullptr,
          *diag_pair = nullptr;
  uint8_t *isdir = nullptr;
  int32_t *dir_dof = nullptr;
  double *dir_scale = nullptr;
  int32_t ndir = 0;
  int32_t *reac_elems = nullptr, *reac_idx = nullptr;
  double *reac_w = nullptr, *reac_re = nullptr;
  int32_t n_reac_elems = 0, n_reac = 0;
  double *u = nullptr, *u_commit = nullptr, *kappa_hist = nullptr;
  void *Ke = nullptr, *vals = nullptr, *minv = nullptr;
  void *Kcor = nullptr, *vals_sec = nullptr;     // multigrid: loading-indicator terms, secant matrix
  double *re = nullptr, *rraw = nullptr, *rhs = nullptr;
  double *kv[11] = {};
  float2 *khl = nullptr;     // FP32 tangent: float-pair copies of ph, sh and the multigrid's level-0 X
  double *gm_V = nullptr, *gm_R = nullptr, *gm_y = nullptr, *gm_dots = nullptr, *gm_final = nullptr;
  int64_t gm_ld = 0;
  int gmres_blocks = 1;
  double *partial = nullptr, *field_tmp = nullptr;
  // committed-state scalars on the device: [0] reaction, [1] external work
  // (trapezoid rule over the committed load-reaction points), [2] reaction
  // of the commit before
  double *reaction = nullptr;
  unsigned int *bar = nullptr;
  SolveResult *res = nullptr;
  int krylov_blocks = 1;
  SolveResult last{};
  // the simulation as a batch of one: the single path runs the batched
  // kernels, so a member computes bitwise the same alone and in a batch
  BatchSim *d_self = nullptr;
  KrylovArgs *d_kself = nullptr;
  KrylovArgs *d_kjac = nullptr;    // with the multigrid: the same system with the block-Jacobi preconditioner
  int32_t *d_one = nullptr;            // [0] = 0 (member index), [1] = 1 (active)
  int64_t *d_prefix = nullptr;         // tiles [0, t], gather blocks [0, g], precond blocks [0, p]
  int32_t *d_gstart = nullptr;         // [0, krylov_blocks]
  int64_t self_tiles = 0, self_gblocks = 0, self_pblocks = 0;
  // phase timers and counters
  bool timers_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double phase_ms[LGDM_NPHASES] = {};
  int64_t phase_n[LGDM_NPHASES] = {};
  int64_t counters[7] = {};
  // secant-tangent fallback: current mode, the value last written to the
  // device descriptor, whether this load step used it, consecutive steps
  int secant = 0, secant_dev = 0;
  bool step_secant = false;
  int secant_streak = 0;
  // aggregation multigrid: host hierarchy, device level descriptors and
  // arrays, launch prefixes of the set-up ([level][0..3]: pair blocks {0,
  // n}, node blocks {0, n})
  AmgHost amgh;
  int amg_levels = 0, amg_sb = 0;
  std::vector<AmgLevel> h_lev;
  AmgLevel *d_lev = nullptr;
  double *amg_cinv = nullptr;
  int64_t *d_amg_prefix = nullptr;
  std::vector<int64_t> amg_pblocks, amg_nblocks;   // per level: set-up blocks
  // host copies
  std::vector<int32_t> h_nbr_ptr, h_nbr;
  std::string err;
  double load_commit = 0.0, load_trial = 0.0;
  // external work: the load of the last point of the load-reaction curve it
  // covers, and whether commits are internal sub-steps of a halved load step
  // (not points of the curve)
  double load_point = 0.0;
  bool substep_commits = false;
  bool assembled = false;
  int fault = 0;                       // pending failure injection (lgdm_inject_fault)

  ~lgdm_sim() {
    for (auto &p : ev_pending) {
      cudaEventDestroy(p.second.first);
      cudaEventDestroy(p.second.second);
    }
    for (auto e : ev_pool) cudaEventDestroy(e);
  }

  MeshView mesh_view() const {
    return MeshView{x, y, z, conn, e_scale, vol_scale, nel, nnode};
  }
  PatternView pattern_view() const {
    return PatternView{nnode, npairs, nbr_ptr, nbr, pair_node, pc_ptr, pc, diag_pair, isdir};
  }
};

namespace {

}  // namespace

void lgdm::set_global_error(const std::string &msg) { g_last_error = msg; }

namespace {

lgdm_status fail(lgdm_sim *s, lgdm_status st, const std::string &msg) {
  if (s) s->err = msg;
  else g_last_error = msg;
  return st;
}

cudaEvent_t take_event(lgdm_sim *s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Times one phase with an event pair when timers are on.
struct PhaseTimer {
  lgdm_sim *s;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseTimer(lgdm_sim *s_, int ph) : s(s_), phase(ph) {
    if (s->timers_on && (a = take_event(s))) cudaEventRecord(a, s->stream);
  }
  ~PhaseTimer() {
    if (!a) return;
    cudaEvent_t b = take_event(s);
    if (!b) {
      s->ev_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, s->stream);
    s->ev_pending.push_back({phase, {a, b}});
  }
};

void resolve_timers(lgdm_sim *s) {
  for (auto &p : s->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
      s->phase_ms[p.first] += ms;
      s->phase_n[p.first] += 1;
    }
    s->ev_pool.push_back(p.second.first);
    s->ev_pool.push_back(p.second.second);
  }
  s->ev_pending.clear();
}

#define LGDM_CUDA(sim, call)                                                                  \
  do {                                                                                        \
    cudaError_t _e = (call);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return fail(sim, LGDM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e));    \
  } while (0)

lgdm_status check_mesh(const lgdm_mesh *m) {
  if (!m) return fail(nullptr, LGDM_ERR_INVALID_ARG, "mesh is NULL");
  const int d = dim_of(m->elem);
  if (!d) return fail(nullptr, LGDM_ERR_INVALID_ARG, "unknown element type");
  if (m->nnode <= 0 || m->nelem <= 0 || !m->x || !m->conn)
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "empty mesh or missing coordinates / connectivity");
  if ((d >= 2 && !m->y) || (d >= 3 && !m->z))
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "missing y or z coordinates");
  return LGDM_OK;
}

// Lay out (or only size) the workspace.
void carve(lgdm_sim &s, Carver &c) {
  s.x = c.take<double>(s.nnode);
  if (s.dim > 1) s.y = c.take<double>(s.nnode);
  if (s.dim > 2) s.z = c.take<double>(s.nnode);
  s.conn = c.take<int32_t>((size_t)s.nel * s.nen);
  s.e_scale = c.take<double>(s.nel);
  s.vol_scale = c.take<double>(s.nel);
  s.nbr_ptr = c.take<int32_t>(s.nnode + 1);
  s.nbr = c.take<int32_t>(s.npairs);
  s.pair_node = c.take<int32_t>(s.npairs);
  s.pc_ptr = c.take<int32_t>(s.npairs + 1);
  s.pc = c.take<int32_t>(s.ncontrib);
  s.diag_pair = c.take<int32_t>(s.nnode);
  s.isdir = c.take<uint8_t>(s.ndof);
  s.dir_dof = c.take<int32_t>(std::max(s.ndir, 1));
  s.dir_scale = c.take<double>(std::max(s.ndir, 1));
  s.reac_elems = c.take<int32_t>(std::max(s.n_reac_elems, 1));
  s.reac_idx = c.take<int32_t>(std::max(s.n_reac, 1));
  s.reac_w = c.take<double>(std::max(s.n_reac, 1));
  s.reac_re = c.take<double>((size_t)std::max(s.n_reac_elems, 1) * s.nen * s.nd);
  s.u = c.take<double>(s.ndof);
  s.u_commit = c.take<double>(s.ndof);
  s.kappa_hist = c.take<double>((size_t)s.nel * s.ngp);
  const size_t ke = (size_t)s.nel * s.nen * s.nd * s.nen * s.nd;
  s.Ke = c.take<char>(ke * s.tsize);
  s.re = c.take<double>((size_t)s.nel * s.nen * s.nd);
  s.vals = c.take<char>((size_t)s.nnz * s.tsize);
  s.minv = c.take<char>((size_t)s.nnode * s.nd * s.nd * s.tsize);
  s.rraw = c.take<double>(s.ndof);
  s.rhs = c.take<double>(s.ndof);
  for (int k = 0; k < 11; ++k) s.kv[k] = c.take<double>(s.ndof);
  s.khl = (s.opt.precision == LGDM_PREC_FP32_TANGENT) ? c.take<float2>((size_t)3 * s.ndof) : nullptr;
  if (s.opt.gmres_m > 0) {
    const int m = s.opt.gmres_m;
    s.gm_ld = (s.ndof + 31) & ~int64_t(31);
    s.gm_V = c.take<double>((size_t)(m + 1) * s.gm_ld);
    s.gm_R = c.take<double>((size_t)m * (m + 1));
    s.gm_y = c.take<double>(m);
    s.gm_dots = c.take<double>((size_t)(GMRES_MAX_M + 2) * std::max(s.gmres_blocks, 1));
    s.gm_final = c.take<double>(m + 2);
  }
  s.partial = c.take<double>((size_t)3 * 4 * krylov_ntiles(s.nnode));
  s.field_tmp = c.take<double>(std::max((size_t)s.nel * s.ngp, (size_t)s.ndof) + 64);   // + energy block sums
  s.reaction = c.take<double>(3);
  s.bar = c.take<unsigned int>(2);
  s.res = c.take<SolveResult>(1);
  s.d_self = c.take<BatchSim>(1);
  s.d_kself = c.take<KrylovArgs>(1);
  s.d_one = c.take<int32_t>(2);
  s.d_prefix = c.take<int64_t>(6);
  s.d_gstart = c.take<int32_t>(2);
  const int L = s.amg_levels;
  s.h_lev.assign(L, AmgLevel{});
  s.Kcor = s.vals_sec = nullptr;
  if (L > 0) {
    s.d_kjac = c.take<KrylovArgs>(1);
    s.Kcor = c.take<char>((size_t)s.nel * s.nen * s.nen * s.nd * s.tsize);
    s.vals_sec = c.take<char>((size_t)s.nnz * s.tsize);
    s.d_lev = c.take<AmgLevel>(L);
    s.d_amg_prefix = c.take<int64_t>((size_t)4 * L);
    const size_t ts = s.tsize, nd = (size_t)s.nd;
    for (int l = 0; l < L; ++l) {
      const AmgHost::Lev &H = s.amgh.lev[l];
      AmgLevel &V = s.h_lev[l];
      V.nnode = H.nnode;
      const size_t n = (size_t)H.nnode;
      if (l == 0) {
        V.npairs = (int32_t)s.npairs;
      } else {
        V.npairs = H.nbr_ptr.empty() ? 0 : H.nbr_ptr.back();
        const size_t np = (size_t)V.npairs, nprev = (size_t)s.amgh.lev[l - 1].nnode;
        const size_t npprev = (l == 1) ? (size_t)s.npairs : (size_t)s.h_lev[l - 1].npairs;
        V.nbr_ptr = c.take<int32_t>(n + 1);
        V.nbr = c.take<int32_t>(np);
        V.pair_node = c.take<int32_t>(np);
        V.diag_pair = c.take<int32_t>(n);
        V.mem_ptr = c.take<int32_t>(n + 1);
        V.mem = c.take<int32_t>(nprev);
        V.cmap_ptr = c.take<int32_t>(np + 1);
        V.cmap = c.take<int32_t>(npprev);
        V.vals = c.take<char>(nd * nd * np * ts);
        V.minv = c.take<char>(nd * nd * n * ts);
        V.v = c.take<double>(nd * n);
        V.z = c.take<double>(nd * n);
      }
      if (l + 1 < L) V.agg = c.take<int32_t>(n);
      V.X = c.take<double>(nd * n);
      V.R = c.take<double>(nd * n);
    }
    const int64_t nc = s.amgh.lev[L - 1].nnode;
    s.amg_cinv = (nc <= AMG_COARSE_MAX) ? c.take<double>((size_t)(nd_sq(s.nd) * nc * nc)) : nullptr;
    AmgLevel &V0 = s.h_lev[0];                 // level 0: the system's pattern, secant values
    V0.nbr_ptr = s.nbr_ptr;
    V0.nbr = s.nbr;
    V0.pair_node = s.pair_node;
    V0.diag_pair = s.diag_pair;
    V0.vals = s.vals_sec;
    V0.minv = s.minv;
    V0.held = (nve_of(s.elem) < s.nen) ? s.isdir : nullptr;
    V0.Xhl = s.khl ? s.khl + 2 * s.ndof : nullptr;
  }
  s.ws_needed = c.off + 256;
}

int max_krylov_blocks(bool fp32) {
  static int cache[2] = {-1, -1};
  int &v = cache[fp32 ? 1 : 0];
  if (v < 0) v = fp32 ? std::min(bicgstab_max_blocks<float>(), bicgstab_grouped_max_blocks<float>())
                      : std::min(bicgstab_max_blocks<double>(), bicgstab_grouped_max_blocks<double>());
  return v;
}

// Krylov grid: one node per thread, and as many co-resident blocks as keep
// at least 16 nodes each -- the FP64 pipe of an SM (2 FMA per clock on this
// part) must not carry a small system alone.  A block owns whole reduction
// tiles (at most one block per tile) and at most 32 * KRYLOV_MAXW nodes.
int choose_krylov_blocks(const lgdm_sim &s, bool query_device) {
  int cap = 152 * 2;
  if (query_device) {
    const int m = max_krylov_blocks(s.opt.precision == LGDM_PREC_FP32_TANGENT);
    if (m > 0) cap = m;
  }
  int64_t want = std::max<int64_t>((s.nnode + KRYLOV_THREADS - 1) / KRYLOV_THREADS,
                                   std::min<int64_t>(cap, (s.nnode + 15) / 16));
  if (s.opt.krylov_blocks > 0) want = s.opt.krylov_blocks;
  want = std::min<int64_t>(want, krylov_ntiles(s.nnode));
  want = std::max<int64_t>(want, krylov_min_blocks(s.nnode));
  if (want < 1) want = 1;
  return (int)std::min<int64_t>(want, cap);
}

lgdm_status plan(lgdm_sim &s, const lgdm_mesh &m, const lgdm_options &o, const lgdm_bcs *bcs, Pattern *P,
                 bool query_device) {
  s.elem = m.elem;
  s.dim = dim_of(m.elem);
  s.nen = nen_of(m.elem);
  s.ngp = s.nen;
  s.nd = s.dim + 1;
  s.nnode = m.nnode;
  s.nel = m.nelem;
  s.ndof = (int64_t)s.nd * m.nnode;
  s.opt = o;
  s.tsize = (o.precision == LGDM_PREC_FP32_TANGENT) ? sizeof(float) : sizeof(double);
  Pattern local;
  Pattern &pat = P ? *P : local;
  std::string err;
  lgdm_status st = build_pattern(m, pat, P != nullptr, err);
  if (st != LGDM_OK) return fail(nullptr, st, err);
  s.npairs = pat.npairs;
  s.nnz = pat.npairs * s.nd * s.nd;
  s.amg_levels = 0;
  if (o.precond == LGDM_PRECOND_MULTIGRID) {
    if (!amg_build(s.nnode, pat.nbr_ptr, pat.nbr, s.amgh))
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "the mesh's node graph does not coarsen for the multigrid");
    s.amg_levels = (int)s.amgh.lev.size();
    int sb = s.amg_levels - 1;
    for (int l = 0; l < s.amg_levels; ++l)
      if (s.amgh.lev[l].nnode <= AMG_SINGLE_BLOCK) { sb = l; break; }
    s.amg_sb = sb;
  }
  s.ncontrib = (int64_t)s.nel * s.nen * s.nen;
  s.ndir = bcs ? bcs->n_dir : 0;
  if (krylov_min_blocks(s.nnode) < 1 || krylov_min_blocks(s.nnode) > (query_device ? max_krylov_blocks(
          o.precision == LGDM_PREC_FP32_TANGENT) : 152 * 16))
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "mesh too large for one Krylov launch (nodes per block limit)");
  s.krylov_blocks = choose_krylov_blocks(s, query_device);
  s.gmres_blocks = s.krylov_blocks;
  if (query_device && o.gmres_m > 0) {
    const int cap = (o.precision == LGDM_PREC_FP32_TANGENT) ? gmres_max_blocks<float>() : gmres_max_blocks<double>();
    if (cap > 0) s.gmres_blocks = std::min(s.gmres_blocks, cap);
  }
  return LGDM_OK;
}

}  // namespace

namespace {

KrylovArgs krylov_args(lgdm_sim *s);

// Multigrid set-up of a simulation after its assembly and fine block-Jacobi
// inverses: Galerkin values and inverses level by level, then the dense
// inverse of the coarsest level.
template <typename TT>
cudaError_t multigrid_setup(lgdm_sim *s) {
  const int32_t *mem = s->d_one, *act = s->d_one + 1;
  for (int l = 1; l < s->amg_levels; ++l) {
    const cudaError_t e = launch_batch_amg_level<TT>(s->nd, l, s->d_self, mem, s->d_amg_prefix + 4 * l,
                                                     s->d_amg_prefix + 4 * l + 2, 1, s->amg_pblocks[l],
                                                     s->amg_nblocks[l], act, s->stream);
    if (e != cudaSuccess) return e;
  }
  if (s->amg_levels > 0 && s->amg_cinv) return launch_batch_amg_coarse<TT>(s->nd, s->d_self, mem, 1, act, s->stream);
  return cudaSuccess;
}

AmgInfo amg_info(const lgdm_sim *s) {
  AmgInfo m{};
  m.lev = s->d_lev;
  m.nlev = s->amg_levels;
  m.sb_level = s->amg_sb;
  m.cinv = s->amg_cinv;
  m.nc = s->amg_levels > 0 ? s->h_lev[s->amg_levels - 1].nnode : 0;
  return m;
}

BatchSim self_desc(lgdm_sim *s) {
  BatchSim d{};
  d.m = s->mesh_view();
  d.mc = s->mc;
  d.u = s->u;
  d.kh = s->kappa_hist;
  d.Ke = s->Ke;
  d.re = s->re;
  d.p = s->pattern_view();
  d.vals = s->vals;
  d.rraw = s->rraw;
  d.rhs = s->rhs;
  d.minv = s->minv;
  d.precond = (s->opt.precond == LGDM_PRECOND_JACOBI) ? LGDM_PRECOND_JACOBI : LGDM_PRECOND_NODE_BLOCK;
  d.amg = amg_info(s);
  d.Kcor = s->Kcor;
  d.vals_sec = s->vals_sec;
  return d;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int32_t lgdm_abi_version(void) { return LGDM_ABI_VERSION; }

const char *lgdm_status_string(lgdm_status s) {
  switch (s) {
    case LGDM_OK: return "ok";
    case LGDM_ERR_INVALID_ARG: return "invalid argument";
    case LGDM_ERR_OOM: return "workspace too small";
    case LGDM_ERR_CUDA: return "CUDA error";
    case LGDM_ERR_NOT_CONVERGED: return "Newton did not converge";
    case LGDM_ERR_NONFINITE: return "non-finite value";
    case LGDM_ERR_TIMEOUT: return "device wait timed out";
    case LGDM_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

lgdm_status lgdm_default_options(lgdm_options *o) {
  if (!o) return fail(nullptr, LGDM_ERR_INVALID_ARG, "options is NULL");
  o->precision = LGDM_PREC_FP64;
  o->precond = LGDM_PRECOND_MULTIGRID;
  o->newton_tol = 1e-8;
  o->krylov_rtol = 1e-8;
  o->max_newton = 50;
  o->max_krylov = 5000;
  o->max_halvings = 6;
  o->krylov_blocks = 0;
  o->gmres_m = 64;
  o->krylov_method = 0;
  o->wait_limit_s = 2.0;
  return LGDM_OK;
}

lgdm_status lgdm_workspace_size(const lgdm_mesh *m, const lgdm_options *o, size_t *bytes) {
  try {
    if (!bytes || !o) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL argument");
    lgdm_status st = check_mesh(m);
    if (st != LGDM_OK) return st;
    lgdm_sim s;
    st = plan(s, *m, *o, nullptr, nullptr, false);
    if (st != LGDM_OK) return st;
    // the Dirichlet count is unknown here: size the Dirichlet and reaction
    // lists for every dof / element (small next to the matrix)
    s.ndir = (int32_t)std::min<int64_t>(s.ndof, INT32_MAX);
    s.n_reac_elems = s.nel;
    s.n_reac = (int32_t)std::min<int64_t>((int64_t)s.nel * s.nen * s.nd, INT32_MAX);
    s.krylov_blocks = 152 * 16;
    s.gmres_blocks = 152 * 16;
    Carver c{nullptr};
    carve(s, c);
    *bytes = s.ws_needed;
    return LGDM_OK;
  } catch (const std::bad_alloc &) {
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "host out of memory while sizing the pattern");
  } catch (...) {
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "unexpected host exception");
  }
}

lgdm_status lgdm_pattern_counts(const lgdm_mesh *m, int64_t *npairs, int64_t *nnz) {
  try {
    if (!npairs || !nnz) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL argument");
    lgdm_status st = check_mesh(m);
    if (st != LGDM_OK) return st;
    Pattern P;
    std::string err;
    st = build_pattern(*m, P, false, err);
    if (st != LGDM_OK) return fail(nullptr, st, err);
    const int64_t nd = dim_of(m->elem) + 1;
    *npairs = P.npairs;
    *nnz = P.npairs * nd * nd;
    return LGDM_OK;
  } catch (const std::bad_alloc &) {
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "host out of memory while counting the pattern");
  } catch (...) {
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "unexpected host exception");
  }
}

lgdm_status lgdm_create(const lgdm_mesh *m, const lgdm_material *mat, const lgdm_bcs *bcs,
                        const lgdm_options *o, void *ws, size_t ws_bytes, void *stream, lgdm_sim **out) {
  lgdm_sim *s = nullptr;
  try {
    if (!out || !mat || !o) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    lgdm_status st = check_mesh(m);
    if (st != LGDM_OK) return st;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
    if (o->precision != LGDM_PREC_FP64 && o->precision != LGDM_PREC_FP32_TANGENT)
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "unknown precision");
    if (o->precond < LGDM_PRECOND_JACOBI || o->precond > LGDM_PRECOND_MULTIGRID)
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "unknown preconditioner");
    if (o->max_newton < 1 || o->max_krylov < 1 || o->max_halvings < 0 || !(o->newton_tol > 0.0))
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "bad iteration limits or tolerance");
    if (o->gmres_m < 0 || o->gmres_m > GMRES_MAX_M)
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "gmres_m must be in 0..128");
    if (o->krylov_method != 0 && !(o->krylov_method == 1 && o->gmres_m > 0))
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "krylov_method 1 (GMRES) needs gmres_m > 0");
    if (!(o->wait_limit_s >= 1e-6 && o->wait_limit_s <= 60.0))
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "wait_limit_s must be in 1e-6 .. 60 s");
    if (bcs && bcs->n_dir > 0 && (!bcs->dir_dof || !bcs->dir_scale))
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "Dirichlet arrays missing");
    s = new lgdm_sim();
    s->stream = static_cast<cudaStream_t>(stream);
    s->mat = *mat;
    Pattern P;
    st = plan(*s, *m, *o, bcs, &P, true);
    if (st != LGDM_OK) { delete s; return st; }
    s->mc = make_matconst(*mat, s->dim);
    // Dirichlet flags and the reaction contributions
    std::vector<uint8_t> isdir(s->ndof, 0);
    std::vector<double> dscale(s->ndof, 0.0);
    for (int32_t i = 0; i < s->ndir; ++i) {
      const int32_t d = bcs->dir_dof[i];
      if (d < 0 || d >= s->ndof || isdir[d]) {
        delete s;
        return fail(nullptr, LGDM_ERR_INVALID_ARG, "Dirichlet dof out of range or repeated");
      }
      isdir[d] = 1;
      dscale[d] = bcs->dir_scale[i];
    }
    // mixed order: the micro-equivalent strain of a node that is no element's
    // vertex is in no equation; it is held at zero like an unloaded Dirichlet dof
    if (nve_of(m->elem) < s->nen) {
      std::vector<uint8_t> vertex(s->nnode, 0);
      for (int32_t e = 0; e < s->nel; ++e)
        for (int a = 0; a < nve_of(m->elem); ++a) vertex[m->conn[(int64_t)e * s->nen + a]] = 1;
      for (int32_t n = 0; n < s->nnode; ++n)
        if (!vertex[n]) isdir[(int64_t)s->nd * n + s->dim] = 1;
    }
    std::vector<int32_t> reac_elems, reac_idx;
    std::vector<double> reac_w;
    for (int32_t e = 0; e < s->nel; ++e) {
      bool any = false;
      for (int a = 0; a < s->nen; ++a)
        for (int i = 0; i < s->nd; ++i) {
          const int64_t d = (int64_t)s->nd * m->conn[(int64_t)e * s->nen + a] + i;
          if (isdir[d] && dscale[d] != 0.0) {
            if (!any) { reac_elems.push_back(e); any = true; }
            reac_idx.push_back((int32_t)(((int64_t)(reac_elems.size() - 1) * s->nen + a) * s->nd + i));
            reac_w.push_back(dscale[d]);
          }
        }
    }
    s->n_reac_elems = (int32_t)reac_elems.size();
    s->n_reac = (int32_t)reac_idx.size();
    s->ws = static_cast<char *>(ws);
    s->ws_bytes = ws_bytes;
    Carver c{s->ws};
    carve(*s, c);
    if (s->ws_needed > ws_bytes) {
      const std::string msg = "workspace " + std::to_string(ws_bytes) + " < needed " + std::to_string(s->ws_needed);
      delete s;
      return fail(nullptr, LGDM_ERR_OOM, msg);
    }
    cudaStream_t st_ = s->stream;
    auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
      if (!bytes) return cudaSuccess;
      return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st_);
    };
    cudaError_t e = cudaSuccess;
    std::vector<double> ones(s->nel, 1.0);
    e = e ? e : up(s->x, m->x, sizeof(double) * s->nnode);
    if (s->dim > 1) e = e ? e : up(s->y, m->y, sizeof(double) * s->nnode);
    if (s->dim > 2) e = e ? e : up(s->z, m->z, sizeof(double) * s->nnode);
    e = e ? e : up(s->conn, m->conn, sizeof(int32_t) * s->nel * s->nen);
    e = e ? e : up(s->e_scale, m->e_scale ? m->e_scale : ones.data(), sizeof(double) * s->nel);
    e = e ? e : up(s->vol_scale, m->vol_scale ? m->vol_scale : ones.data(), sizeof(double) * s->nel);
    e = e ? e : up(s->nbr_ptr, P.nbr_ptr.data(), sizeof(int32_t) * (s->nnode + 1));
    e = e ? e : up(s->nbr, P.nbr.data(), sizeof(int32_t) * s->npairs);
    e = e ? e : up(s->pair_node, P.pair_node.data(), sizeof(int32_t) * s->npairs);
    e = e ? e : up(s->pc_ptr, P.pc_ptr.data(), sizeof(int32_t) * (s->npairs + 1));
    e = e ? e : up(s->pc, P.pc.data(), sizeof(int32_t) * s->ncontrib);
    e = e ? e : up(s->diag_pair, P.diag_pair.data(), sizeof(int32_t) * s->nnode);
    e = e ? e : up(s->isdir, isdir.data(), s->ndof);
    if (s->ndir > 0) {
      e = e ? e : up(s->dir_dof, bcs->dir_dof, sizeof(int32_t) * s->ndir);
      e = e ? e : up(s->dir_scale, bcs->dir_scale, sizeof(double) * s->ndir);
    }
    if (s->n_reac > 0) {
      e = e ? e : up(s->reac_elems, reac_elems.data(), sizeof(int32_t) * s->n_reac_elems);
      e = e ? e : up(s->reac_idx, reac_idx.data(), sizeof(int32_t) * s->n_reac);
      e = e ? e : up(s->reac_w, reac_w.data(), sizeof(double) * s->n_reac);
    }
    std::vector<double> kh((size_t)s->nel * s->ngp, mat->kappa0);
    e = e ? e : up(s->kappa_hist, kh.data(), sizeof(double) * kh.size());
    e = e ? e : cudaMemsetAsync(s->u, 0, sizeof(double) * s->ndof, st_);
    e = e ? e : cudaMemsetAsync(s->u_commit, 0, sizeof(double) * s->ndof, st_);
    e = e ? e : cudaMemsetAsync(s->reaction, 0, 3 * sizeof(double), st_);
    e = e ? e : cudaMemsetAsync(s->res, 0, sizeof(SolveResult), st_);
    // multigrid levels: pattern, maps, descriptors and set-up prefixes
    std::vector<int64_t> amg_prefix;
    if (s->amg_levels > 0) {
      const int L = s->amg_levels;
      s->amg_pblocks.assign(L, 0);
      s->amg_nblocks.assign(L, 0);
      amg_prefix.assign((size_t)4 * L, 0);
      for (int l = 0; l < L; ++l) {
        const AmgHost::Lev &H = s->amgh.lev[l];
        AmgLevel &V = s->h_lev[l];
        auto upv = [&](const int32_t *dst, const std::vector<int32_t> &v) {
          if (e == cudaSuccess && !v.empty()) e = up(const_cast<int32_t *>(dst), v.data(), sizeof(int32_t) * v.size());
        };
        if (l > 0) {
          upv(V.nbr_ptr, H.nbr_ptr);
          upv(V.nbr, H.nbr);
          upv(V.pair_node, H.pair_node);
          upv(V.diag_pair, H.diag_pair);
          upv(V.mem_ptr, H.mem_ptr);
          upv(V.mem, H.mem);
          upv(V.cmap_ptr, H.cmap_ptr);
          upv(V.cmap, H.cmap);
          s->amg_pblocks[l] = (V.npairs + 255) / 256;
          s->amg_nblocks[l] = (V.nnode + 127) / 128;
          amg_prefix[4 * l + 1] = s->amg_pblocks[l];
          amg_prefix[4 * l + 3] = s->amg_nblocks[l];
        }
        if (l + 1 < L) upv(V.agg, H.agg);
      }
      e = e ? e : up(s->d_lev, s->h_lev.data(), sizeof(AmgLevel) * L);
      e = e ? e : up(s->d_amg_prefix, amg_prefix.data(), sizeof(int64_t) * amg_prefix.size());
    }
    BatchSim self{};
    KrylovArgs kself{}, kjac{};
    int32_t one[2] = {0, 1};
    int64_t prefix[6] = {0, 0, 0, 0, 0, 0};
    int32_t gstart[2] = {0, 0};
    if (e == cudaSuccess) {
      self = self_desc(s);
      kself = krylov_args(s);
      const int epb_self = batch_tile_elements(s->elem, s->opt.precision == LGDM_PREC_FP32_TANGENT, s->mc.hterm != 0, 128);
      s->self_tiles = (s->nel + epb_self - 1) / epb_self;
      s->self_gblocks = (s->npairs + 255) / 256;
      s->self_pblocks = (s->nnode + 127) / 128;
      prefix[1] = s->self_tiles;
      prefix[3] = s->self_gblocks;
      prefix[5] = s->self_pblocks;
      gstart[1] = s->krylov_blocks;
      e = up(s->d_self, &self, sizeof(BatchSim));
      e = e ? e : up(s->d_kself, &kself, sizeof(KrylovArgs));
      if (s->d_kjac) {
        kjac = kself;
        kjac.amg = AmgInfo{};
        kjac.stall_iters = std::max(500, s->opt.max_krylov / 4);
        e = e ? e : up(s->d_kjac, &kjac, sizeof(KrylovArgs));
      }
      e = e ? e : up(s->d_one, one, sizeof(one));
      e = e ? e : up(s->d_prefix, prefix, sizeof(prefix));
      e = e ? e : up(s->d_gstart, gstart, sizeof(gstart));
    }
    e = e ? e : cudaStreamSynchronize(st_);   // host staging vectors die at return
    s->amgh = AmgHost();                      // the device holds the hierarchy now
    if (e != cudaSuccess) {
      const std::string msg = std::string("upload failed: ") + cudaGetErrorString(e);
      delete s;
      return fail(nullptr, LGDM_ERR_CUDA, msg);
    }
    s->h_nbr_ptr = std::move(P.nbr_ptr);
    s->h_nbr = std::move(P.nbr);
    *out = s;
    return LGDM_OK;
  } catch (const std::bad_alloc &) {
    delete s;
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "host out of memory while building the pattern");
  } catch (...) {
    delete s;
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "unexpected host exception");
  }
}

void lgdm_destroy(lgdm_sim *s) { delete s; }

const char *lgdm_last_error(const lgdm_sim *s) { return s ? s->err.c_str() : g_last_error.c_str(); }

lgdm_status lgdm_get_sizes(const lgdm_sim *s, lgdm_sizes *o) {
  if (!s || !o) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL argument");
  o->dim = s->dim;
  o->nen = s->nen;
  o->ngp = s->ngp;
  o->nd = s->nd;
  o->nnode = s->nnode;
  o->nelem = s->nel;
  o->ndof = s->ndof;
  o->nnz = s->nnz;
  o->npairs = s->npairs;
  o->workspace_bytes = s->ws_needed;
  o->mg_levels = s->amg_levels;
  for (int l = 0; l < LGDM_MG_MAX_LEVELS; ++l) {
    o->mg_nnode[l] = l < s->amg_levels ? s->h_lev[l].nnode : 0;
    o->mg_npairs[l] = l < s->amg_levels ? s->h_lev[l].npairs : 0;
  }
  return LGDM_OK;
}

lgdm_status lgdm_set_state(lgdm_sim *s, const double *u, const double *kh) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  if (u)
    for (int64_t k = 0; k < s->ndof; ++k)
      if (!std::isfinite(u[k])) return fail(s, LGDM_ERR_NONFINITE, "u[" + std::to_string(k) + "] is not finite");
  if (kh)
    for (int64_t k = 0; k < (int64_t)s->nel * s->ngp; ++k)
      if (!std::isfinite(kh[k]))
        return fail(s, LGDM_ERR_NONFINITE, "kappa_hist[" + std::to_string(k) + "] is not finite");
  if (u) {
    LGDM_CUDA(s, cudaMemcpyAsync(s->u, u, sizeof(double) * s->ndof, cudaMemcpyHostToDevice, s->stream));
    LGDM_CUDA(s, cudaMemcpyAsync(s->u_commit, s->u, sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
  }
  if (kh)
    LGDM_CUDA(s, cudaMemcpyAsync(s->kappa_hist, kh, sizeof(double) * s->nel * s->ngp, cudaMemcpyHostToDevice,
                                 s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  s->assembled = false;
  s->secant = 0;
  s->secant_streak = 0;
  s->step_secant = false;
  return LGDM_OK;
}

lgdm_status lgdm_reset_state(lgdm_sim *s) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  LGDM_CUDA(s, cudaMemsetAsync(s->u, 0, sizeof(double) * s->ndof, s->stream));
  LGDM_CUDA(s, cudaMemsetAsync(s->u_commit, 0, sizeof(double) * s->ndof, s->stream));
  LGDM_CUDA(s, launch_fill(s->kappa_hist, (int64_t)s->nel * s->ngp, s->mat.kappa0, s->stream));
  LGDM_CUDA(s, cudaMemsetAsync(s->reaction, 0, 3 * sizeof(double), s->stream));
  s->counters[0] += 1;
  s->load_commit = s->load_trial = s->load_point = 0.0;
  s->assembled = false;
  s->secant = 0;
  s->secant_streak = 0;
  s->step_secant = false;
  return LGDM_OK;
}

lgdm_status lgdm_get_field(lgdm_sim *s, int32_t which, double *dst, size_t n) {
  if (!s || !dst) return fail(s, LGDM_ERR_INVALID_ARG, "NULL argument");
  const size_t ngpt = (size_t)s->nel * s->ngp;
  const double *src = nullptr;
  size_t need = (size_t)s->ndof;
  switch (which) {
    case LGDM_FIELD_U: src = s->u; break;
    case LGDM_FIELD_KAPPA_HIST: src = s->kappa_hist; need = ngpt; break;
    case LGDM_FIELD_DAMAGE:
      need = ngpt;
      LGDM_CUDA(s, launch_damage_field(s->mc, s->kappa_hist, (int64_t)ngpt, s->field_tmp, s->stream));
      src = s->field_tmp;
      break;
    case LGDM_FIELD_DELTA: src = s->kv[0]; break;
    case LGDM_FIELD_RESIDUAL: src = s->rraw; break;
    case LGDM_FIELD_RHS: src = s->rhs; break;
    default: return fail(s, LGDM_ERR_INVALID_ARG, "unknown field");
  }
  if (n != need) return fail(s, LGDM_ERR_INVALID_ARG, "field length mismatch: expected " + std::to_string(need));
  LGDM_CUDA(s, cudaMemcpyAsync(dst, src, sizeof(double) * need, cudaMemcpyDeviceToHost, s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  return LGDM_OK;
}

lgdm_status lgdm_begin_step(lgdm_sim *s, double load) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  PhaseTimer pt(s, 5);
  // a load step starts with the consistent tangent, unless the previous
  // steps needed the secant one (then every 8th step tries it again)
  s->secant = (s->secant_streak > 0 && s->secant_streak % 8 != 0) ? 1 : 0;
  s->step_secant = false;
  s->load_trial = load;
  LGDM_CUDA(s, cudaMemcpyAsync(s->u, s->u_commit, sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
  LGDM_CUDA(s, launch_set_dirichlet(s->u, s->dir_dof, s->dir_scale, s->ndir, load, s->stream));
  s->counters[0] += 1;
  s->assembled = false;
  return LGDM_OK;
}

lgdm_status lgdm_assemble(lgdm_sim *s) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  if (s->fault == 2) {                         // injected: a NaN in the current dofs
    static const double nan_value = std::nan("");
    s->fault = 0;
    LGDM_CUDA(s, cudaMemcpyAsync(s->u + (int64_t)s->nd * (s->nnode / 2), &nan_value, sizeof(double),
                                 cudaMemcpyHostToDevice, s->stream));
  }
  if (s->secant != s->secant_dev) {            // the tangent mode lives in the device descriptor
    s->secant_dev = s->secant;
    char *dst = reinterpret_cast<char *>(s->d_self) + offsetof(BatchSim, mc) + offsetof(MatConst, secant);
    LGDM_CUDA(s, cudaMemcpyAsync(dst, &s->secant_dev, sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
  }
  const MeshView mv = s->mesh_view();
  const PatternView pv = s->pattern_view();
  const int32_t *mem = s->d_one, *act = s->d_one + 1;
  const int64_t *tiles = s->d_prefix, *gb = s->d_prefix + 2, *pb = s->d_prefix + 4;
  const int grid = (int)std::min<int64_t>(s->self_tiles, 2 * 152);
  if (s->opt.precision == LGDM_PREC_FP32_TANGENT) {
    {
      PhaseTimer pt(s, 0);
      LGDM_CUDA(s, launch_batch_element<float>(s->elem, 128, s->mc.hterm != 0, s->d_self, mem, tiles, 1, s->self_tiles,
                                               act, grid, s->stream));
    }
    {
      PhaseTimer pt(s, 1);
      LGDM_CUDA(s, launch_batch_gather<float>(s->elem, s->d_self, mem, gb, 1, s->self_gblocks, act, s->stream));
    }
    {
      PhaseTimer pt(s, 2);
      LGDM_CUDA(s, launch_batch_precond<float>(s->nd, s->d_self, mem, pb, 1, s->self_pblocks, act, s->stream));
      LGDM_CUDA(s, multigrid_setup<float>(s));
    }
  } else {
    {
      PhaseTimer pt(s, 0);
      LGDM_CUDA(s, launch_batch_element<double>(s->elem, 128, s->mc.hterm != 0, s->d_self, mem, tiles, 1, s->self_tiles,
                                                act, grid, s->stream));
    }
    {
      PhaseTimer pt(s, 1);
      LGDM_CUDA(s, launch_batch_gather<double>(s->elem, s->d_self, mem, gb, 1, s->self_gblocks, act, s->stream));
    }
    {
      PhaseTimer pt(s, 2);
      LGDM_CUDA(s, launch_batch_precond<double>(s->nd, s->d_self, mem, pb, 1, s->self_pblocks, act, s->stream));
      LGDM_CUDA(s, multigrid_setup<double>(s));
    }
  }
  s->counters[0] += 3 + (s->amg_levels > 0 ? 2 * (s->amg_levels - 1) + (s->amg_cinv ? 1 : 0) : 0);
  s->counters[1] += 1;
  s->assembled = true;
  return LGDM_OK;
}

lgdm_status lgdm_get_system(lgdm_sim *s, int32_t *rowptr, int32_t *col, double *vals, double *rhs) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  if (!s->assembled) return fail(s, LGDM_ERR_STATE, "no assembled system");
  const int nd = s->nd;
  if (rowptr || col) {
    for (int32_t a = 0; a < s->nnode; ++a) {
      const int32_t pb = s->h_nbr_ptr[a], deg = s->h_nbr_ptr[a + 1] - pb;
      for (int i = 0; i < nd; ++i) {
        const int64_t row = (int64_t)nd * a + i;
        const int64_t start = (int64_t)nd * nd * pb + (int64_t)i * nd * deg;
        if (rowptr) rowptr[row] = (int32_t)start;
        if (col)
          for (int32_t k = 0; k < deg; ++k)
            for (int j = 0; j < nd; ++j) col[start + (int64_t)nd * k + j] = nd * s->h_nbr[pb + k] + j;
      }
    }
    if (rowptr) rowptr[s->ndof] = (int32_t)s->nnz;
  }
  if (vals) {
    if (s->tsize == sizeof(double)) {
      LGDM_CUDA(s, cudaMemcpyAsync(vals, s->vals, sizeof(double) * s->nnz, cudaMemcpyDeviceToHost, s->stream));
      LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
    } else {
      std::vector<float> tmp(s->nnz);
      LGDM_CUDA(s, cudaMemcpyAsync(tmp.data(), s->vals, sizeof(float) * s->nnz, cudaMemcpyDeviceToHost, s->stream));
      LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
      for (int64_t k = 0; k < s->nnz; ++k) vals[k] = (double)tmp[k];
    }
  }
  if (rhs) {
    LGDM_CUDA(s, cudaMemcpyAsync(rhs, s->rhs, sizeof(double) * s->ndof, cudaMemcpyDeviceToHost, s->stream));
    LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  }
  return LGDM_OK;
}

}  // extern "C"

namespace {

KrylovArgs krylov_args(lgdm_sim *s) {
  KrylovArgs a{};
  a.nd = s->nd;
  a.nnode = s->nnode;
  a.max_iter = s->opt.max_krylov;
  a.rtol = s->opt.krylov_rtol;
  a.newton_tol = s->opt.newton_tol;
  a.p = s->pattern_view();
  a.vals = s->vals;
  a.minv = s->minv;
  a.rhs = s->rhs;
  a.x = s->kv[0];
  a.r = s->kv[1];
  a.r0 = s->kv[2];
  a.pv = s->kv[3];
  a.v = s->kv[4];
  a.sv = s->kv[5];
  a.t = s->kv[6];
  a.ph = s->kv[7];
  a.sh = s->kv[8];
  a.xb = s->kv[9];
  a.ph_hl = s->khl;
  a.sh_hl = s->khl ? s->khl + s->ndof : nullptr;
  // stop a solve that stopped improving: a multigrid-preconditioned solve
  // converges in at most a few hundred iterations when it converges at all
  a.stall_iters = (s->amg_levels > 0) ? std::max(100, s->opt.max_krylov / 20) : std::max(500, s->opt.max_krylov / 4);
  a.tile = krylov_tile(s->nnode);
  a.ntiles = (int32_t)krylov_ntiles(s->nnode);
  a.u = s->u;
  a.partial = s->partial;
  a.bar_count = s->bar;
  a.bar_gen = s->bar + 1;
  a.res = s->res;
  a.wait_ns = (unsigned long long)(s->opt.wait_limit_s * 1e9);
  a.barrier_extra = 0;
  a.amg = amg_info(s);
  return a;
}

lgdm_status finish_launch(lgdm_sim *s, int mode, SolveResult *out) {
  s->counters[0] += 1;
  LGDM_CUDA(s, cudaMemcpyAsync(out, s->res, sizeof(SolveResult), cudaMemcpyDeviceToHost, s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  if (s->timers_on) resolve_timers(s);
  if (out->status == 4) {
    s->last.status = 4;
    return fail(s, LGDM_ERR_TIMEOUT, "grid barrier timed out in the Krylov launch");
  }
  if (mode != 2) s->counters[2] += out->iters;
  if (mode == 2) {
    s->last.converged = out->converged;
    for (int k = 0; k < 4; ++k) s->last.norms[k] = out->norms[k];
  } else {
    s->last = *out;
  }
  if (out->status == 3) return fail(s, LGDM_ERR_NONFINITE, "non-finite value in the Krylov solve or update");
  return LGDM_OK;
}

// Writes the barrier_extra word of the simulation's Krylov descriptor.
cudaError_t set_barrier_extra(lgdm_sim *s, int v) {
  static const int32_t values[2] = {0, 1};
  char *dst = reinterpret_cast<char *>(s->d_kself) + offsetof(KrylovArgs, barrier_extra);
  return cudaMemcpyAsync(dst, &values[v ? 1 : 0], sizeof(int32_t), cudaMemcpyHostToDevice, s->stream);
}

lgdm_status run_krylov(lgdm_sim *s, int mode, SolveResult *out, bool jacobi = false) {
  KrylovArgs *args = (jacobi && s->d_kjac) ? s->d_kjac : s->d_kself;
  const bool inject = s->fault == 1;
  if (inject) {                                // injected: the barrier waits for a block that never comes
    s->fault = 0;
    LGDM_CUDA(s, set_barrier_extra(s, 1));
  }
  {
    PhaseTimer pt(s, 3);
    if (s->opt.precision == LGDM_PREC_FP32_TANGENT)
      LGDM_CUDA(s, launch_bicgstab_grouped<float>(s->nd, args, s->d_one, s->d_gstart, s->d_one + 1, 1,
                                                  s->krylov_blocks, mode, s->stream));
    else
      LGDM_CUDA(s, launch_bicgstab_grouped<double>(s->nd, args, s->d_one, s->d_gstart, s->d_one + 1, 1,
                                                   s->krylov_blocks, mode, s->stream));
  }
  if (inject) LGDM_CUDA(s, set_barrier_extra(s, 0));
  return finish_launch(s, mode, out);
}

// GMRES from the x left by the previous solve.
lgdm_status run_gmres(lgdm_sim *s, SolveResult *out) {
  const KrylovArgs a = krylov_args(s);
  GmresArgs g{};
  g.m = s->opt.gmres_m;
  g.ld = s->gm_ld;
  g.V = s->gm_V;
  g.R = s->gm_R;
  g.y = s->gm_y;
  g.dots = s->gm_dots;
  g.final = s->gm_final;
  g.xs = s->kv[10];
  {
    PhaseTimer pt(s, 3);
    if (s->opt.precision == LGDM_PREC_FP32_TANGENT)
      LGDM_CUDA(s, launch_gmres<float>(a, g, s->gmres_blocks, s->stream));
    else
      LGDM_CUDA(s, launch_gmres<double>(a, g, s->gmres_blocks, s->stream));
  }
  return finish_launch(s, 0, out);
}

// A solve whose increment Newton may use.
bool solve_acceptable(lgdm_status st, const SolveResult &r) {
  return st == LGDM_OK && (r.status == 0 || r.rel_res <= KRYLOV_NEWTON_ETA);
}

// GMRES continues a BiCGSTAB solve that ended far from krylov_rtol -- unless
// the result is not even usable and the secant tangent is still to be tried
// (with_secant_left): a new tangent is then the better next step.
bool wants_gmres(const lgdm_sim *s, lgdm_status st, const SolveResult &r, bool with_secant_left) {
  const bool short_of = (st == LGDM_ERR_NONFINITE) || (r.status != 0 && r.rel_res > 1e3 * s->opt.krylov_rtol);
  if (!short_of || s->opt.gmres_m <= 0) return false;
  return !(with_secant_left && !solve_acceptable(st, r));
}

// Solve with BiCGSTAB, continue with GMRES when it falls short of krylov_rtol.
lgdm_status solve_robust(lgdm_sim *s, SolveResult *out, bool with_secant_left = false) {
  if (s->opt.krylov_method == 1) {
    LGDM_CUDA(s, cudaMemsetAsync(s->kv[0], 0, sizeof(double) * s->ndof, s->stream));
    return run_gmres(s, out);
  }
  lgdm_status st = run_krylov(s, 0, out);
  if (st != LGDM_OK && st != LGDM_ERR_NONFINITE) return st;
  if (s->d_kjac && st == LGDM_OK && out->status != 0 && out->rel_res > 1e3 * s->opt.krylov_rtol) {
    // the multigrid V-cycle did not carry the solve (its piecewise-constant
    // aggregates can miss soft modes, e.g. the plate bending of a thin 3D
    // specimen): BiCGSTAB again from zero with the node-block Jacobi
    // preconditioner of the same (secant) blocks
    const int32_t mg_iters = out->iters;
    st = run_krylov(s, 0, out, true);
    out->iters += mg_iters;
    s->last.iters = out->iters;
    if (st != LGDM_OK && st != LGDM_ERR_NONFINITE) return st;
  }
  if (!wants_gmres(s, st, *out, with_secant_left)) return st;
  const int32_t bicg_iters = out->iters;
  if (st == LGDM_ERR_NONFINITE)
    LGDM_CUDA(s, cudaMemsetAsync(s->kv[0], 0, sizeof(double) * s->ndof, s->stream));
  else
    LGDM_CUDA(s, cudaMemcpyAsync(s->kv[0], s->kv[9], sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice,
                                 s->stream));   // best BiCGSTAB iterate
  st = run_gmres(s, out);
  out->iters += bicg_iters;
  s->last.iters = out->iters;
  return st;
}

}  // namespace

extern "C" {

lgdm_status lgdm_solve(lgdm_sim *s, int32_t *iters, double *rel_res) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  if (!s->assembled) return fail(s, LGDM_ERR_STATE, "solve before assemble");
  SolveResult r{};
  lgdm_status st = solve_robust(s, &r);
  if (iters) *iters = r.iters;
  if (rel_res) *rel_res = r.rel_res;
  return st;
}

lgdm_status lgdm_update(lgdm_sim *s, int32_t *converged) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  SolveResult r{};
  lgdm_status st = run_krylov(s, 2, &r);
  if (converged) *converged = r.converged;
  s->assembled = false;
  return st;
}

lgdm_status lgdm_newton_step(lgdm_sim *s, int32_t *converged, int32_t *krylov_iters) {
  lgdm_status st = lgdm_assemble(s);
  if (st != LGDM_OK) return st;
  SolveResult r{};
  st = solve_robust(s, &r, !s->secant);
  int32_t its = r.iters;
  if (!solve_acceptable(st, r) && !s->secant && (st == LGDM_OK || st == LGDM_ERR_NONFINITE)) {
    // the consistent tangent defeated the Krylov solver: secant tangent for
    // the rest of this load step
    s->secant = 1;
    st = lgdm_assemble(s);
    if (st != LGDM_OK) return st;
    st = solve_robust(s, &r);
    its += r.iters;
    s->last.iters = its;
  }
  if (st != LGDM_OK) return st;
  if (s->secant) {
    s->step_secant = true;
    s->counters[6] += 1;
  }
  SolveResult u{};
  st = run_krylov(s, 2, &u);
  s->assembled = false;
  if (converged) *converged = u.converged;
  if (krylov_iters) *krylov_iters = its;
  return st;
}

lgdm_status lgdm_commit(lgdm_sim *s) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  PhaseTimer pt(s, 4);
  s->counters[0] += (s->n_reac > 0) ? 3 : 1;
  s->counters[4] += 1;
  s->secant_streak = s->step_secant ? s->secant_streak + 1 : 0;
  s->step_secant = false;
  LGDM_CUDA(s, launch_commit(s->elem, s->mesh_view(), s->u, s->kappa_hist, s->stream));
  LGDM_CUDA(s, cudaMemcpyAsync(s->u_commit, s->u, sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
  if (s->n_reac > 0) {
    // residual at the converged state on the elements touching loaded dofs
    if (s->opt.precision == LGDM_PREC_FP32_TANGENT)
      LGDM_CUDA(s, launch_element<float>(s->elem, s->mesh_view(), s->mc, s->u, s->kappa_hist, s->reac_elems,
                                         s->n_reac_elems, nullptr, s->reac_re, true, s->stream));
    else
      LGDM_CUDA(s, launch_element<double>(s->elem, s->mesh_view(), s->mc, s->u, s->kappa_hist, s->reac_elems,
                                          s->n_reac_elems, nullptr, s->reac_re, true, s->stream));
    LGDM_CUDA(s, launch_reaction_sum(s->reac_re, s->reac_idx, s->reac_w, s->n_reac, s->reaction, s->stream));
  } else {
    LGDM_CUDA(s, cudaMemsetAsync(s->reaction, 0, sizeof(double), s->stream));
  }
  s->load_commit = s->load_trial;
  if (!s->substep_commits) {
    // external work (R17): trapezoid rule from the previous point of the curve
    LGDM_CUDA(s, launch_external_work(s->reaction, s->load_commit - s->load_point, s->stream));
    s->counters[0] += 1;
    s->load_point = s->load_commit;
  }
  return LGDM_OK;
}

lgdm_status lgdm_get_committed(lgdm_sim *s, double *load, double *external_work, double *reaction) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  double v[3] = {0.0, 0.0, 0.0};
  LGDM_CUDA(s, cudaMemcpyAsync(v, s->reaction, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  if (load) *load = s->load_commit;
  if (external_work) *external_work = v[1];
  if (reaction) *reaction = v[0];
  return LGDM_OK;
}

lgdm_status lgdm_set_committed(lgdm_sim *s, double load, double external_work, double reaction) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  if (!std::isfinite(load) || !std::isfinite(external_work) || !std::isfinite(reaction))
    return fail(s, LGDM_ERR_NONFINITE, "committed scalars must be finite");
  const double v[3] = {reaction, external_work, reaction};
  LGDM_CUDA(s, cudaMemcpyAsync(s->reaction, v, 3 * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  s->load_commit = s->load_trial = s->load_point = load;
  return LGDM_OK;
}

lgdm_status lgdm_inject_fault(lgdm_sim *s, int32_t kind) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  if (kind < 0 || kind > 2) return fail(s, LGDM_ERR_INVALID_ARG, "unknown fault kind");
  s->fault = kind;
  return LGDM_OK;
}

lgdm_status lgdm_last_solve(lgdm_sim *s, int32_t *iters, int32_t *status, double *rel_res, double *norms4) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  if (iters) *iters = s->last.iters;
  if (status) *status = s->last.status;
  if (rel_res) *rel_res = s->last.rel_res;
  if (norms4)
    for (int k = 0; k < 4; ++k) norms4[k] = s->last.norms[k];
  return LGDM_OK;
}

lgdm_status lgdm_enable_timers(lgdm_sim *s, int32_t on) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  s->timers_on = on != 0;
  return LGDM_OK;
}

lgdm_status lgdm_get_timers(lgdm_sim *s, double *ms, int64_t *launches) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  resolve_timers(s);
  for (int k = 0; k < LGDM_NPHASES; ++k) {
    if (ms) ms[k] = s->phase_ms[k];
    if (launches) launches[k] = s->phase_n[k];
  }
  return LGDM_OK;
}

lgdm_status lgdm_reset_timers(lgdm_sim *s) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  resolve_timers(s);
  for (int k = 0; k < LGDM_NPHASES; ++k) {
    s->phase_ms[k] = 0.0;
    s->phase_n[k] = 0;
  }
  return LGDM_OK;
}

lgdm_status lgdm_get_counters(const lgdm_sim *s, int64_t *c, int32_t n) {
  if (!s || !c || n < 0 || n > 7) return fail(nullptr, LGDM_ERR_INVALID_ARG, "bad counters request");
  for (int k = 0; k < n; ++k) c[k] = s->counters[k];
  return LGDM_OK;
}

lgdm_status lgdm_get_energy(lgdm_sim *s, double *psi) {
  if (!s || !psi) return fail(s, LGDM_ERR_INVALID_ARG, "NULL argument");
  // per-Gauss-point values in the element residual scratch, block sums in field_tmp
  LGDM_CUDA(s, launch_energy(s->elem, s->mesh_view(), s->mc, s->u, s->kappa_hist, s->re, s->field_tmp,
                             s->field_tmp + ((int64_t)s->nel * s->ngp + 4095) / 4096 + 1, s->stream));
  double v = 0.0;
  LGDM_CUDA(s, cudaMemcpyAsync(&v, s->field_tmp + ((int64_t)s->nel * s->ngp + 4095) / 4096 + 1, sizeof(double),
                               cudaMemcpyDeviceToHost, s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  s->counters[0] += 3;
  s->assembled = false;
  *psi = v;
  return LGDM_OK;
}

lgdm_status lgdm_get_dissipated_energy(lgdm_sim *s, double *dissipated, double *psi) {
  if (!s || !dissipated) return fail(s, LGDM_ERR_INVALID_ARG, "NULL argument");
  double e = 0.0, w = 0.0;
  lgdm_status st = lgdm_get_energy(s, &e);
  if (st != LGDM_OK) return st;
  st = lgdm_get_committed(s, nullptr, &w, nullptr);
  if (st != LGDM_OK) return st;
  *dissipated = w - e;
  if (psi) *psi = e;
  return LGDM_OK;
}

lgdm_status lgdm_get_damaged_volume(lgdm_sim *s, double threshold, double *volume) {
  if (!s || !volume) return fail(s, LGDM_ERR_INVALID_ARG, "NULL argument");
  if (!std::isfinite(threshold)) return fail(s, LGDM_ERR_INVALID_ARG, "threshold must be finite");
  const int64_t nblk = ((int64_t)s->nel * s->ngp + 4095) / 4096;
  LGDM_CUDA(s, launch_damaged_volume(s->elem, s->mesh_view(), s->mc, s->kappa_hist, threshold, s->re, s->field_tmp,
                                     s->field_tmp + nblk + 1, s->stream));
  double v = 0.0;
  LGDM_CUDA(s, cudaMemcpyAsync(&v, s->field_tmp + nblk + 1, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  s->counters[0] += 3;
  s->assembled = false;
  *volume = v;
  return LGDM_OK;
}

lgdm_status lgdm_get_reaction(lgdm_sim *s, double *reaction) {
  if (!s || !reaction) return fail(s, LGDM_ERR_INVALID_ARG, "NULL argument");
  LGDM_CUDA(s, cudaMemcpyAsync(reaction, s->reaction, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  return LGDM_OK;
}

}  // extern "C"

namespace {

// Newton iterations at `load` from the committed state; *done = converged.
lgdm_status attempt(lgdm_sim *s, double load, bool *done, int32_t *iters) {
  lgdm_status st = lgdm_begin_step(s, load);
  if (st != LGDM_OK) return st;
  *done = false;
  for (int k = 1; k <= s->opt.max_newton; ++k) {
    int32_t conv = 0;
    st = lgdm_newton_step(s, &conv, nullptr);
    ++*iters;
    s->counters[3] += 1;
    if (st == LGDM_ERR_NONFINITE) return LGDM_OK;   // treated like divergence: halve
    if (st != LGDM_OK) return st;
    if (conv) {
      *done = true;
      return LGDM_OK;
    }
  }
  return LGDM_OK;
}

lgdm_status advance(lgdm_sim *s, double from, double to, int depth, int32_t *iters) {
  bool done = false;
  lgdm_status st = attempt(s, to, &done, iters);
  if (st != LGDM_OK) return st;
  if (done) return lgdm_commit(s);
  if (depth >= s->opt.max_halvings) {
    LGDM_CUDA(s, cudaMemcpyAsync(s->u, s->u_commit, sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
    return fail(s, LGDM_ERR_NOT_CONVERGED,
                "Newton did not converge at load " + std::to_string(to) + " after " + std::to_string(depth) +
                    " halvings");
  }
  const double mid = 0.5 * (from + to);
  s->counters[5] += 1;
  st = advance(s, from, mid, depth + 1, iters);
  if (st != LGDM_OK) return st;
  return advance(s, mid, to, depth + 1, iters);
}

// A load step driven by the library, halvings included, is one point of the
// load-reaction curve: the commits of its sub-steps add no external work, the
// end point adds the trapezoid from the previous point.
lgdm_status advance_step(lgdm_sim *s, double from, double to, int depth, int32_t *iters) {
  s->substep_commits = true;
  lgdm_status st = advance(s, from, to, depth, iters);
  s->substep_commits = false;
  if (st != LGDM_OK) return st;
  LGDM_CUDA(s, launch_external_work(s->reaction, s->load_commit - s->load_point, s->stream));
  s->counters[0] += 1;
  s->load_point = s->load_commit;
  return LGDM_OK;
}

}  // namespace

extern "C" lgdm_status lgdm_run_step(lgdm_sim *s, double load, int32_t *newton_iters) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  int32_t its = 0;
  lgdm_status st = advance_step(s, s->load_commit, load, 0, &its);
  if (newton_iters) *newton_iters = its;
  return st;
}

// ====================================================================== batch
// Several simulations advanced together: one persistent element launch per
// element type over all members' tiles, batched gather and preconditioner
// set-up, one cooperative BiCGSTAB launch per wave of members (each member on
// its own block group and barrier; the tile sums make its result independent
// of the group size), a second batched pass with the secant tangent for the
// members whose solve failed, the batched update, and a CUDA graph of the
// launches of a Newton step.
struct lgdm_batch {
  std::vector<lgdm_sim *> sims;
  int n = 0;
  cudaStream_t stream = nullptr;
  bool fp32 = false;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  BatchSim *d_sims = nullptr;
  KrylovArgs *d_kargs = nullptr;
  int32_t *d_active = nullptr;
  SolveResult *d_res = nullptr;
  struct AmgLaunch {                   // multigrid set-up of one level for the members that have it
    int level = 0;
    int nm = 0;
    int32_t *d_members = nullptr;
    int64_t *d_pb = nullptr, *d_nb = nullptr;
    int64_t tot_pb = 0, tot_nb = 0;
  };
  struct Group {                       // members of one element type and stress variant
    int elem = 0, nd = 0;
    bool hterm = false;
    std::vector<int32_t> members;
    int32_t *d_members = nullptr;
    int64_t *d_tile = nullptr, *d_gblock = nullptr, *d_pblock = nullptr;
    int64_t tiles = 0, gblocks = 0, pblocks = 0;
    std::vector<AmgLaunch> amg;
    int n_coarse = 0;
    int32_t *d_coarse = nullptr;       // members with a dense coarsest inverse
  };
  std::vector<Group> groups;
  struct Wave {                        // members whose block groups fit one co-resident launch
    int nd = 0;
    std::vector<int32_t> members;
    int32_t *d_members = nullptr, *d_start = nullptr;
    int blocks = 0;
  };
  std::vector<Wave> waves;
  int32_t *d_wave_members = nullptr;   // [n] members of all waves, wave after wave
  int32_t *d_wave_start = nullptr;     // [2n] block-group starts of all waves
  int nodes_per_block = 4096;          // solve tuning: target nodes per Krylov block
  int64_t launches = 0;                // kernels issued by batched passes (directly or by the graph)
  std::vector<int32_t> h_wave_members, h_wave_start;
  int bt = 128, grid_factor = 2, sms = 152;
  bool graph_on = true, graph_ok = false, graph_tried = false;
  int graph_mode = 0;                  // 0 none, 1 assembly launches, 2 assembly and solve
  int direct_issues = 0;
  std::string graph_note;
  cudaGraphExec_t graph = nullptr;
  std::vector<int32_t> h_active;
  std::vector<int32_t> h_secant;       // tangent mode written into each member's descriptor
  std::vector<SolveResult> h_res;
  std::string err;
  // host sources of asynchronous uploads at creation (kept until the stream has synchronised)
  std::vector<std::vector<int32_t>> amg_staging;
  std::vector<std::vector<int64_t>> amg_staging64;
  // phase timers: events before the element launches, after them, after the
  // gathers, after the preconditioner set-ups and after the first solve
  bool timers_on = false;
  cudaEvent_t tev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double t_ms[4] = {0, 0, 0, 0};
  int64_t t_n[4] = {0, 0, 0, 0};
  ~lgdm_batch() {
    if (graph) cudaGraphExecDestroy(graph);
    for (auto e : tev)
      if (e) cudaEventDestroy(e);
  }
};

namespace {

size_t batch_bytes(int n) {
  // descriptors, flags, results and prefix arrays; a generous bound per member
  const size_t amg = (size_t)6 * AMG_MAX_LEVELS * ((size_t)n * 4 + 2 * (size_t)(n + 1) * 8 + 3 * 256) +
                     (size_t)6 * ((size_t)n * 4 + 256);
  return (size_t)n * (sizeof(BatchSim) + sizeof(KrylovArgs) + sizeof(SolveResult) + 4 * 64 + 10 * 8) +
         (size_t)(n + 8) * 8 * 24 + amg + (1 << 16);
}

lgdm_status bfail(lgdm_batch *b, lgdm_status st, const std::string &m) {
  if (b) b->err = m;
  g_last_error = m;
  return st;
}

#define LGDM_BCUDA(b, call)                                                                          \
  do {                                                                                               \
    cudaError_t _e = (call);                                                                         \
    if (_e != cudaSuccess) return bfail(b, LGDM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

#define LGDM_BMARK(b, k)                                                  \
  do {                                                                    \
    if ((b)->timers_on) LGDM_BCUDA(b, cudaEventRecord((b)->tev[k], (b)->stream)); \
  } while (0)

// Solve waves: the members of one nd are given block groups of about
// nodes_per_block nodes per block (at least their fewest, at most one block
// per reduction tile), then packed, largest first, into co-resident
// cooperative launches (first fit); the blocks a wave has left over are
// shared out in proportion to node counts.  The waves run one after the
// other.  A member's result does not depend on its group size (tile-ordered
// inner products, per-node multigrid arithmetic).
lgdm_status build_waves(lgdm_batch *b, int nodes_per_block) {
  const int cap = b->fp32 ? bicgstab_grouped_max_blocks<float>() : bicgstab_grouped_max_blocks<double>();
  const int n = b->n;
  b->waves.clear();
  b->h_wave_start.clear();
  for (int nd = 2; nd <= 4; ++nd) {
    std::vector<int32_t> ms;
    for (int i = 0; i < n; ++i)
      if (b->sims[i]->nd == nd) ms.push_back(i);
    std::stable_sort(ms.begin(), ms.end(), [&](int32_t x, int32_t y) { return b->sims[x]->nnode > b->sims[y]->nnode; });
    std::vector<std::vector<int32_t>> wm;
    std::vector<std::vector<int64_t>> wb;
    std::vector<int64_t> used;
    for (int32_t i : ms) {
      lgdm_sim *s = b->sims[i];
      const int64_t lo = std::max<int64_t>(1, krylov_min_blocks(s->nnode));
      if (lo > cap) return bfail(b, LGDM_ERR_INVALID_ARG, "member Krylov grid too large");
      const int64_t hi = std::max<int64_t>(lo, std::min<int64_t>(krylov_ntiles(s->nnode), cap));
      const int64_t want = std::min(hi, std::max(lo, ((int64_t)s->nnode + nodes_per_block - 1) / nodes_per_block));
      size_t w = 0;
      while (w < used.size() && used[w] + want > cap) ++w;
      if (w == used.size()) {
        wm.emplace_back();
        wb.emplace_back();
        used.push_back(0);
      }
      wm[w].push_back(i);
      wb[w].push_back(want);
      used[w] += want;
    }
    for (size_t w = 0; w < wm.size(); ++w) {
      // share the left-over blocks in proportion to node counts, up to each member's maximum
      int64_t nodes = 0;
      for (int32_t i : wm[w]) nodes += b->sims[i]->nnode;
      int64_t spare = cap - used[w];
      for (size_t j = 0; j < wm[w].size() && spare > 0; ++j) {
        lgdm_sim *s = b->sims[wm[w][j]];
        const int64_t hi = std::min<int64_t>(krylov_ntiles(s->nnode), cap);
        const int64_t add = std::min<int64_t>(
            {spare, std::max<int64_t>(0, hi - wb[w][j]),
             (int64_t)((double)(cap - used[w]) * (double)s->nnode / (double)std::max<int64_t>(nodes, 1))});
        wb[w][j] += add;
        spare -= add;
      }
      lgdm_batch::Wave wv;
      wv.nd = nd;
      // members in index order inside the wave
      std::vector<size_t> ord(wm[w].size());
      for (size_t j = 0; j < ord.size(); ++j) ord[j] = j;
      std::sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return wm[w][x] < wm[w][y]; });
      std::vector<int32_t> st(1, 0);
      for (size_t j : ord) {
        wv.members.push_back(wm[w][j]);
        st.push_back(st.back() + (int32_t)wb[w][j]);
      }
      wv.blocks = st.back();
      b->waves.push_back(std::move(wv));
      b->waves.back().d_start = nullptr;
      b->h_wave_start.insert(b->h_wave_start.end(), st.begin(), st.end());
    }
  }
  // device copies: members wave after wave, block starts wave after wave
  b->h_wave_members.clear();
  size_t mo = 0, so = 0;
  for (auto &w : b->waves) {
    w.d_members = b->d_wave_members + mo;
    w.d_start = b->d_wave_start + so;
    b->h_wave_members.insert(b->h_wave_members.end(), w.members.begin(), w.members.end());
    mo += w.members.size();
    so += w.members.size() + 1;
  }
  LGDM_BCUDA(b, cudaMemcpyAsync(b->d_wave_members, b->h_wave_members.data(), sizeof(int32_t) * mo,
                                cudaMemcpyHostToDevice, b->stream));
  LGDM_BCUDA(b, cudaMemcpyAsync(b->d_wave_start, b->h_wave_start.data(), sizeof(int32_t) * so, cudaMemcpyHostToDevice,
                                b->stream));
  LGDM_BCUDA(b, cudaStreamSynchronize(b->stream));
  return LGDM_OK;
}

// The launches of one batched Newton step up to the solve (mode 0): the
// element launches of every element-type group, then the gathers, then the
// preconditioner set-ups.
int64_t assembly_launches(const lgdm_batch *b) {
  int64_t k = 0;
  for (const auto &g : b->groups) k += 3 + 2 * (int64_t)g.amg.size() + (g.n_coarse > 0 ? 1 : 0);
  return k;
}

lgdm_status batch_issue_assembly(lgdm_batch *b) {
  const int grid_cap = b->grid_factor * b->sms;
  LGDM_BMARK(b, 0);
  for (auto &g : b->groups) {
    const int grid = (int)std::min<int64_t>(g.tiles, grid_cap);
    if (b->fp32)
      LGDM_BCUDA(b, launch_batch_element<float>(g.elem, b->bt, g.hterm, b->d_sims, g.d_members, g.d_tile, (int)g.members.size(),
                                                g.tiles, b->d_active, grid, b->stream));
    else
      LGDM_BCUDA(b, launch_batch_element<double>(g.elem, b->bt, g.hterm, b->d_sims, g.d_members, g.d_tile, (int)g.members.size(),
                                                 g.tiles, b->d_active, grid, b->stream));
  }
  LGDM_BMARK(b, 1);
  for (auto &g : b->groups) {
    if (b->fp32)
      LGDM_BCUDA(b, launch_batch_gather<float>(g.elem, b->d_sims, g.d_members, g.d_gblock, (int)g.members.size(),
                                               g.gblocks, b->d_active, b->stream));
    else
      LGDM_BCUDA(b, launch_batch_gather<double>(g.elem, b->d_sims, g.d_members, g.d_gblock, (int)g.members.size(),
                                                g.gblocks, b->d_active, b->stream));
  }
  LGDM_BMARK(b, 2);
  for (auto &g : b->groups) {
    if (b->fp32)
      LGDM_BCUDA(b, launch_batch_precond<float>(g.nd, b->d_sims, g.d_members, g.d_pblock, (int)g.members.size(),
                                                g.pblocks, b->d_active, b->stream));
    else
      LGDM_BCUDA(b, launch_batch_precond<double>(g.nd, b->d_sims, g.d_members, g.d_pblock, (int)g.members.size(),
                                                 g.pblocks, b->d_active, b->stream));
    for (const auto &al : g.amg) {
      if (b->fp32)
        LGDM_BCUDA(b, launch_batch_amg_level<float>(g.nd, al.level, b->d_sims, al.d_members, al.d_pb, al.d_nb, al.nm,
                                                    al.tot_pb, al.tot_nb, b->d_active, b->stream));
      else
        LGDM_BCUDA(b, launch_batch_amg_level<double>(g.nd, al.level, b->d_sims, al.d_members, al.d_pb, al.d_nb, al.nm,
                                                     al.tot_pb, al.tot_nb, b->d_active, b->stream));
    }
    if (b->fp32)
      LGDM_BCUDA(b, launch_batch_amg_coarse<float>(g.nd, b->d_sims, g.d_coarse, g.n_coarse, b->d_active, b->stream));
    else
      LGDM_BCUDA(b, launch_batch_amg_coarse<double>(g.nd, b->d_sims, g.d_coarse, g.n_coarse, b->d_active, b->stream));
  }
  LGDM_BMARK(b, 3);
  return LGDM_OK;
}

// Adds the phase times of the last Newton step (its events have completed).
void batch_resolve_timers(lgdm_batch *b) {
  if (!b->timers_on) return;
  for (int k = 0; k < 4; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->tev[k], b->tev[k + 1]) == cudaSuccess) {
      b->t_ms[k] += ms;
      b->t_n[k] += 1;
    }
  }
  cudaGetLastError();
}

lgdm_status batch_issue_solve(lgdm_batch *b, int mode) {
  b->launches += 2 * (int64_t)b->waves.size();          // reset + grouped solve per wave
  for (auto &w : b->waves) {
    if (b->fp32)
      LGDM_BCUDA(b, launch_bicgstab_grouped<float>(w.nd, b->d_kargs, w.d_members, w.d_start, b->d_active,
                                                   (int)w.members.size(), w.blocks, mode, b->stream));
    else
      LGDM_BCUDA(b, launch_bicgstab_grouped<double>(w.nd, b->d_kargs, w.d_members, w.d_start, b->d_active,
                                                    (int)w.members.size(), w.blocks, mode, b->stream));
  }
  if (mode == 0) LGDM_BMARK(b, 4);
  return LGDM_OK;
}

// Capture the given launches into an executable graph; false if refused.
bool batch_capture(lgdm_batch *b, bool with_solve) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    b->graph_note = std::string("begin capture: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return false;
  }
  const int64_t counted = b->launches;         // capture records launches without running them
  lgdm_status st = batch_issue_assembly(b);
  if (st == LGDM_OK && with_solve) st = batch_issue_solve(b, 0);
  b->launches = counted;
  e = cudaStreamEndCapture(b->stream, &g);
  bool ok = false;
  if (st == LGDM_OK && e == cudaSuccess && g) {
    e = cudaGraphInstantiate(&b->graph, g, 0);
    ok = e == cudaSuccess;
  }
  if (!ok) b->graph_note = (st != LGDM_OK) ? b->err : std::string(cudaGetErrorString(e));
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return ok;
}

lgdm_status batch_assemble_and_solve(lgdm_batch *b) {
  // the first step runs directly (kernel attributes get set outside any
  // capture); with phase timers on every step runs directly (events recorded
  // by graph nodes give no elapsed times)
  const bool use_graph = b->graph_on && !b->timers_on;
  if (use_graph && !b->graph_tried && b->direct_issues > 0) {
    b->graph_tried = true;
    if (batch_capture(b, true)) b->graph_mode = 2;
    else if (batch_capture(b, false)) b->graph_mode = 1;
    b->graph_ok = b->graph_mode > 0;
  }
  if (use_graph && b->graph_ok) {
    LGDM_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
    b->launches += assembly_launches(b) + (b->graph_mode == 2 ? 2 * (int64_t)b->waves.size() : 0);
    if (b->graph_mode == 1) return batch_issue_solve(b, 0);
    return LGDM_OK;
  }
  ++b->direct_issues;
  b->launches += assembly_launches(b);
  lgdm_status st = batch_issue_assembly(b);
  if (st != LGDM_OK) return st;
  return batch_issue_solve(b, 0);
}

}  // namespace

extern "C" {

lgdm_status lgdm_batch_workspace_size(int32_t n, size_t *bytes) {
  if (n <= 0 || !bytes) return fail(nullptr, LGDM_ERR_INVALID_ARG, "bad batch size");
  *bytes = batch_bytes(n);
  return LGDM_OK;
}

lgdm_status lgdm_batch_create(lgdm_sim *const *sims, int32_t n, void *ws, size_t ws_bytes, void *stream,
                              lgdm_batch **out) {
  if (!sims || n <= 0 || !out || !ws) return fail(nullptr, LGDM_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  if (ws_bytes < batch_bytes(n)) return fail(nullptr, LGDM_ERR_OOM, "batch workspace too small");
  lgdm_batch *b = nullptr;
  try {
    b = new lgdm_batch();
    b->n = n;
    b->stream = static_cast<cudaStream_t>(stream);
    b->ws = static_cast<char *>(ws);
    b->ws_bytes = ws_bytes;
    for (int i = 0; i < n; ++i) {
      lgdm_sim *s = sims[i];
      if (!s) { delete b; return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL member"); }
      if (s->stream != b->stream) { delete b; return fail(nullptr, LGDM_ERR_INVALID_ARG, "members must use the batch stream"); }
      const bool f = s->opt.precision == LGDM_PREC_FP32_TANGENT;
      if (i == 0) b->fp32 = f;
      else if (f != b->fp32) { delete b; return fail(nullptr, LGDM_ERR_INVALID_ARG, "members must share the precision"); }
      b->sims.push_back(s);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    Carver c{b->ws};
    b->d_sims = c.take<BatchSim>(n);
    b->d_kargs = c.take<KrylovArgs>(n);
    b->d_active = c.take<int32_t>(n);
    b->d_res = c.take<SolveResult>(n);
    std::vector<BatchSim> hs(n);
    std::vector<KrylovArgs> hk(n);
    for (int i = 0; i < n; ++i) {
      lgdm_sim *s = b->sims[i];
      BatchSim &d = hs[i];
      d.m = s->mesh_view();
      d.mc = s->mc;
      d.u = s->u;
      d.kh = s->kappa_hist;
      d.Ke = s->Ke;
      d.re = s->re;
      d.p = s->pattern_view();
      d.vals = s->vals;
      d.rraw = s->rraw;
      d.rhs = s->rhs;
      d.minv = s->minv;
      d.precond = (s->opt.precond == LGDM_PRECOND_JACOBI) ? LGDM_PRECOND_JACOBI : LGDM_PRECOND_NODE_BLOCK;
      d.amg = amg_info(s);
      d.Kcor = s->Kcor;
      d.vals_sec = s->vals_sec;
      hk[i] = krylov_args(s);
    }
    // groups of one element type and stress variant (one element kernel each)
    for (int elem : {LGDM_L2, LGDM_Q4, LGDM_H8, LGDM_L3, LGDM_Q9})
      for (int ht = 0; ht < 2; ++ht) {
        lgdm_batch::Group g;
        g.elem = elem;
        g.nd = dim_of(elem) + 1;
        g.hterm = ht != 0;
        for (int i = 0; i < n; ++i)
          if (b->sims[i]->elem == elem && (b->sims[i]->mc.hterm != 0) == g.hterm) g.members.push_back(i);
        if (!g.members.empty()) b->groups.push_back(g);
      }
    const int epb = 1;   // prefixes are in tiles of the tuned block size: rebuilt by set_tiles
    (void)epb;
    const size_t nm_max = n;
    for (auto &g : b->groups) {
      const int m = (int)g.members.size();
      g.d_members = c.take<int32_t>(nm_max);
      g.d_tile = c.take<int64_t>(m + 1);
      g.d_gblock = c.take<int64_t>(m + 1);
      g.d_pblock = c.take<int64_t>(m + 1);
      std::vector<int64_t> gb(m + 1, 0), pbk(m + 1, 0);
      for (int j = 0; j < m; ++j) {
        lgdm_sim *s = b->sims[g.members[j]];
        gb[j + 1] = gb[j] + (s->npairs + 255) / 256;
        pbk[j + 1] = pbk[j] + (s->nnode + 127) / 128;
      }
      g.gblocks = gb[m];
      g.pblocks = pbk[m];
      // multigrid set-up launches: per level, the members that have it
      int maxl = 0;
      for (int j = 0; j < m; ++j) maxl = std::max(maxl, b->sims[g.members[j]]->amg_levels);
      for (int l = 1; l < maxl; ++l) {
        lgdm_batch::AmgLaunch al;
        al.level = l;
        std::vector<int32_t> mm;
        std::vector<int64_t> pbv(1, 0), nbv(1, 0);
        for (int j = 0; j < m; ++j) {
          lgdm_sim *s = b->sims[g.members[j]];
          if (s->amg_levels <= l) continue;
          mm.push_back(g.members[j]);
          pbv.push_back(pbv.back() + s->amg_pblocks[l]);
          nbv.push_back(nbv.back() + s->amg_nblocks[l]);
        }
        al.nm = (int)mm.size();
        al.tot_pb = pbv.back();
        al.tot_nb = nbv.back();
        al.d_members = c.take<int32_t>(al.nm);
        al.d_pb = c.take<int64_t>(al.nm + 1);
        al.d_nb = c.take<int64_t>(al.nm + 1);
        LGDM_BCUDA(b, cudaMemcpyAsync(al.d_members, mm.data(), sizeof(int32_t) * al.nm, cudaMemcpyHostToDevice, b->stream));
        LGDM_BCUDA(b, cudaMemcpyAsync(al.d_pb, pbv.data(), sizeof(int64_t) * (al.nm + 1), cudaMemcpyHostToDevice, b->stream));
        LGDM_BCUDA(b, cudaMemcpyAsync(al.d_nb, nbv.data(), sizeof(int64_t) * (al.nm + 1), cudaMemcpyHostToDevice, b->stream));
        g.amg.push_back(std::move(al));
        b->amg_staging.push_back(std::move(mm));
        b->amg_staging64.push_back(std::move(pbv));
        b->amg_staging64.push_back(std::move(nbv));
      }
      std::vector<int32_t> cm;
      for (int j = 0; j < m; ++j)
        if (b->sims[g.members[j]]->amg_cinv) cm.push_back(g.members[j]);
      g.n_coarse = (int)cm.size();
      g.d_coarse = c.take<int32_t>(std::max(g.n_coarse, 1));
      if (g.n_coarse > 0)
        LGDM_BCUDA(b, cudaMemcpyAsync(g.d_coarse, cm.data(), sizeof(int32_t) * g.n_coarse, cudaMemcpyHostToDevice,
                                      b->stream));
      b->amg_staging.push_back(std::move(cm));
      LGDM_BCUDA(b, cudaMemcpyAsync(g.d_members, g.members.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, b->stream));
      LGDM_BCUDA(b, cudaMemcpyAsync(g.d_gblock, gb.data(), sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, b->stream));
      LGDM_BCUDA(b, cudaMemcpyAsync(g.d_pblock, pbk.data(), sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, b->stream));
    }
    b->d_wave_members = c.take<int32_t>(n);
    b->d_wave_start = c.take<int32_t>(2 * (size_t)n);
    {
      const lgdm_status wst = build_waves(b, b->nodes_per_block);
      if (wst != LGDM_OK) { const std::string m = b->err; delete b; return fail(nullptr, wst, m); }
    }
    if (c.off > ws_bytes) { delete b; return fail(nullptr, LGDM_ERR_OOM, "batch workspace too small"); }
    LGDM_BCUDA(b, cudaMemcpyAsync(b->d_sims, hs.data(), sizeof(BatchSim) * n, cudaMemcpyHostToDevice, b->stream));
    LGDM_BCUDA(b, cudaMemcpyAsync(b->d_kargs, hk.data(), sizeof(KrylovArgs) * n, cudaMemcpyHostToDevice, b->stream));
    b->h_active.assign(n, 0);
    b->h_secant.assign(n, 0);
    b->h_res.resize(n);
    // tile prefixes for the default block size
    for (auto &g : b->groups) {
      const int m = (int)g.members.size();
      std::vector<int64_t> tl(m + 1, 0);
      const int epb_ = batch_tile_elements(g.elem, b->fp32, g.hterm, b->bt);
      for (int j = 0; j < m; ++j) tl[j + 1] = tl[j] + (b->sims[g.members[j]]->nel + epb_ - 1) / epb_;
      g.tiles = tl[m];
      LGDM_BCUDA(b, cudaMemcpyAsync(g.d_tile, tl.data(), sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, b->stream));
    }
    LGDM_BCUDA(b, cudaStreamSynchronize(b->stream));
    b->amg_staging.clear();
    b->amg_staging64.clear();
    *out = b;
    return LGDM_OK;
  } catch (...) {
    delete b;
    return fail(nullptr, LGDM_ERR_INVALID_ARG, "host exception while creating the batch");
  }
}

void lgdm_batch_destroy(lgdm_batch *b) { delete b; }

const char *lgdm_batch_last_error(const lgdm_batch *b) { return b ? b->err.c_str() : g_last_error.c_str(); }

lgdm_status lgdm_batch_set_tuning(lgdm_batch *b, int32_t block_threads, int32_t grid_factor, int32_t use_graph) {
  if (!b || (block_threads != 64 && block_threads != 128 && block_threads != 256) || grid_factor < 1 || grid_factor > 32)
    return bfail(b, LGDM_ERR_INVALID_ARG, "block_threads must be 64, 128 or 256; grid_factor 1..32");
  b->bt = block_threads;
  b->grid_factor = grid_factor;
  b->graph_on = use_graph != 0;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_ok = b->graph_tried = false;
  b->graph_mode = 0;
  b->direct_issues = 0;
  for (auto &g : b->groups) {
    const int m = (int)g.members.size();
    std::vector<int64_t> tl(m + 1, 0);
    const int epb = batch_tile_elements(g.elem, b->fp32, g.hterm, b->bt);
    for (int j = 0; j < m; ++j) tl[j + 1] = tl[j] + (b->sims[g.members[j]]->nel + epb - 1) / epb;
    g.tiles = tl[m];
    LGDM_BCUDA(b, cudaMemcpyAsync(g.d_tile, tl.data(), sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, b->stream));
  }
  LGDM_BCUDA(b, cudaStreamSynchronize(b->stream));
  return LGDM_OK;
}

lgdm_status lgdm_batch_set_solve_tuning(lgdm_batch *b, int32_t nodes_per_block) {
  if (!b || nodes_per_block < 32 || nodes_per_block > (1 << 20))
    return bfail(b, LGDM_ERR_INVALID_ARG, "nodes_per_block must be in 32 .. 2^20");
  b->nodes_per_block = nodes_per_block;
  if (b->graph) cudaGraphExecDestroy(b->graph);       // the waves are baked into the captured graph
  b->graph = nullptr;
  b->graph_ok = b->graph_tried = false;
  b->graph_mode = 0;
  b->direct_issues = 0;
  return build_waves(b, nodes_per_block);
}

lgdm_status lgdm_batch_get_launches(const lgdm_batch *b, int64_t *launches) {
  if (!b || !launches) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL argument");
  *launches = b->launches;
  return LGDM_OK;
}

lgdm_status lgdm_batch_get_solve_tuning(const lgdm_batch *b, int32_t *nodes_per_block, int32_t *waves) {
  if (!b) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL batch");
  if (nodes_per_block) *nodes_per_block = b->nodes_per_block;
  if (waves) *waves = (int32_t)b->waves.size();
  return LGDM_OK;
}

lgdm_status lgdm_batch_get_tuning(const lgdm_batch *b, int32_t *block_threads, int32_t *grid_factor, int32_t *graph) {
  if (!b) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL batch");
  if (block_threads) *block_threads = b->bt;
  if (grid_factor) *grid_factor = b->grid_factor;
  if (graph) *graph = (b->graph_on && b->graph_ok) ? b->graph_mode : 0;
  if (b->graph_tried && !b->graph_ok) const_cast<lgdm_batch *>(b)->err = "graph capture refused: " + b->graph_note;
  return LGDM_OK;
}

lgdm_status lgdm_batch_enable_timers(lgdm_batch *b, int32_t on) {
  if (!b) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL batch");
  if (on)
    for (auto &e : b->tev)
      if (!e) LGDM_BCUDA(b, cudaEventCreate(&e));
  if ((on != 0) != b->timers_on) {               // capture the graph again after a change
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_ok = b->graph_tried = false;
    b->graph_mode = 0;
    b->direct_issues = 0;
  }
  b->timers_on = on != 0;
  return LGDM_OK;
}

lgdm_status lgdm_batch_get_timers(lgdm_batch *b, double *ms, int64_t *count, int32_t reset) {
  if (!b) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL batch");
  for (int k = 0; k < 4; ++k) {
    if (ms) ms[k] = b->t_ms[k];
    if (count) count[k] = b->t_n[k];
    if (reset) {
      b->t_ms[k] = 0.0;
      b->t_n[k] = 0;
    }
  }
  return LGDM_OK;
}

// One batched assembly and solve of the members flagged in b->h_active,
// each with its own tangent mode; members the first solve left far from
// its tolerance continue with GMRES, one by one.  kit accumulates the Krylov
// iterations, res receives each member's final solve.
lgdm_status batch_solve_pass(lgdm_batch *b, std::vector<int32_t> &kit, std::vector<SolveResult> &res,
                             std::vector<lgdm_status> &mst) {
  for (int i = 0; i < b->n; ++i) {
    lgdm_sim *s = b->sims[i];
    if (!b->h_active[i] || b->h_secant[i] == s->secant) continue;
    b->h_secant[i] = s->secant;                       // the tangent mode lives in the batch descriptor
    char *dst = reinterpret_cast<char *>(b->d_sims + i) + offsetof(BatchSim, mc) + offsetof(MatConst, secant);
    LGDM_BCUDA(b, cudaMemcpyAsync(dst, &b->h_secant[i], sizeof(int32_t), cudaMemcpyHostToDevice, b->stream));
  }
  LGDM_BCUDA(b, cudaMemcpyAsync(b->d_active, b->h_active.data(), sizeof(int32_t) * b->n, cudaMemcpyHostToDevice, b->stream));
  lgdm_status st = batch_assemble_and_solve(b);
  if (st != LGDM_OK) return st;
  LGDM_BCUDA(b, launch_collect_results(b->d_kargs, b->n, b->d_res, b->stream));
  b->launches += 1;
  LGDM_BCUDA(b, cudaMemcpyAsync(b->h_res.data(), b->d_res, sizeof(SolveResult) * b->n, cudaMemcpyDeviceToHost, b->stream));
  LGDM_BCUDA(b, cudaStreamSynchronize(b->stream));
  batch_resolve_timers(b);
  for (int i = 0; i < b->n; ++i) {
    if (!b->h_active[i]) continue;
    lgdm_sim *s = b->sims[i];
    SolveResult r = b->h_res[i];
    s->counters[1] += 1;
    s->counters[2] += r.iters;
    s->last = r;
    if (r.status == 4) return bfail(b, LGDM_ERR_TIMEOUT, "grid barrier timed out in a grouped Krylov launch");
    const bool nonfinite = r.status == 3;
    lgdm_status ms = nonfinite ? LGDM_ERR_NONFINITE : LGDM_OK;
    if (wants_gmres(s, ms, r, !s->secant)) {
      if (nonfinite)
        LGDM_BCUDA(b, cudaMemsetAsync(s->kv[0], 0, sizeof(double) * s->ndof, s->stream));
      else
        LGDM_BCUDA(b, cudaMemcpyAsync(s->kv[0], s->kv[9], sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
      SolveResult g{};
      const int32_t bi = r.iters;
      ms = run_gmres(s, &g);
      if (ms != LGDM_OK && ms != LGDM_ERR_NONFINITE) return bfail(b, ms, s->err);
      g.iters += bi;
      s->last.iters = g.iters;
      r = g;
    }
    kit[i] += r.iters;
    res[i] = r;
    mst[i] = ms;
  }
  return LGDM_OK;
}

lgdm_status lgdm_batch_newton_step(lgdm_batch *b, const int32_t *active, int32_t *converged, int32_t *krylov_iters) {
  if (!b || !active) return bfail(b, LGDM_ERR_INVALID_ARG, "NULL argument");
  int nact = 0;
  std::vector<int32_t> act(b->n);
  for (int i = 0; i < b->n; ++i) {
    act[i] = active[i] ? 1 : 0;
    nact += act[i];
  }
  if (nact == 0) return LGDM_OK;
  std::vector<int32_t> kit(b->n, 0);
  std::vector<SolveResult> res(b->n);
  std::vector<lgdm_status> mst(b->n, LGDM_OK);
  b->h_active = act;
  lgdm_status st = batch_solve_pass(b, kit, res, mst);
  if (st != LGDM_OK) return st;
  // members whose consistent tangent defeated the Krylov solver: again with
  // the secant tangent, for the rest of their load step
  int nretry = 0;
  for (int i = 0; i < b->n; ++i) {
    lgdm_sim *s = b->sims[i];
    const bool retry = act[i] && !s->secant && !solve_acceptable(mst[i], res[i]);
    b->h_active[i] = retry ? 1 : 0;
    if (retry) {
      s->secant = 1;
      ++nretry;
    }
  }
  if (nretry > 0) {
    st = batch_solve_pass(b, kit, res, mst);
    if (st != LGDM_OK) return st;
  }
  b->h_active = act;
  LGDM_BCUDA(b, cudaMemcpyAsync(b->d_active, b->h_active.data(), sizeof(int32_t) * b->n, cudaMemcpyHostToDevice, b->stream));
  for (int i = 0; i < b->n; ++i) {
    if (!act[i]) continue;
    lgdm_sim *s = b->sims[i];
    s->last.iters = kit[i];
    if (krylov_iters) krylov_iters[i] = kit[i];
    if (s->secant) {
      s->step_secant = true;
      s->counters[6] += 1;
    }
  }
  // batched update and Newton test (mode 2), same block groups
  st = batch_issue_solve(b, 2);
  if (st != LGDM_OK) return st;
  LGDM_BCUDA(b, launch_collect_results(b->d_kargs, b->n, b->d_res, b->stream));
  b->launches += 1;
  LGDM_BCUDA(b, cudaMemcpyAsync(b->h_res.data(), b->d_res, sizeof(SolveResult) * b->n, cudaMemcpyDeviceToHost, b->stream));
  LGDM_BCUDA(b, cudaStreamSynchronize(b->stream));
  for (int i = 0; i < b->n; ++i) {
    if (!b->h_active[i]) continue;
    lgdm_sim *s = b->sims[i];
    const SolveResult &r = b->h_res[i];
    s->last.converged = r.converged;
    for (int k = 0; k < 4; ++k) s->last.norms[k] = r.norms[k];
    s->assembled = false;
    if (r.status == 4) return bfail(b, LGDM_ERR_TIMEOUT, "grid barrier timed out in the batched update");
    if (converged) converged[i] = (r.status == 3) ? -1 : r.converged;
  }
  return LGDM_OK;
}

lgdm_status lgdm_batch_run_step(lgdm_batch *b, const double *loads, int32_t *newton_iters, int32_t *status) {
  if (!b || !loads) return bfail(b, LGDM_ERR_INVALID_ARG, "NULL argument");
  const int n = b->n;
  std::vector<int32_t> act(n, 0), conv(n, 0), its(n, 0);
  int max_newton = 0;
  for (int i = 0; i < n; ++i) {
    if (newton_iters) newton_iters[i] = 0;
    if (status) status[i] = LGDM_OK;
    if (loads[i] != loads[i]) continue;          // NaN: member sits this step out
    lgdm_status st = lgdm_begin_step(b->sims[i], loads[i]);
    if (st != LGDM_OK) return bfail(b, st, b->sims[i]->err);
    act[i] = 1;
    max_newton = std::max(max_newton, b->sims[i]->opt.max_newton);
  }
  std::vector<int32_t> todo(act);
  for (int k = 1; k <= max_newton; ++k) {
    bool any = false;
    for (int i = 0; i < n; ++i)
      if (act[i] && k > b->sims[i]->opt.max_newton) act[i] = 0;
    for (int i = 0; i < n; ++i) any = any || act[i];
    if (!any) break;
    lgdm_status st = lgdm_batch_newton_step(b, act.data(), conv.data(), nullptr);
    if (st != LGDM_OK) return st;
    for (int i = 0; i < n; ++i) {
      if (!act[i]) continue;
      its[i] = k;
      b->sims[i]->counters[3] += 1;
      if (conv[i] == 1) {
        st = lgdm_commit(b->sims[i]);
        if (st != LGDM_OK) return bfail(b, st, b->sims[i]->err);
        act[i] = 0;
        todo[i] = 0;
      } else if (conv[i] == -1) {
        act[i] = 0;                                // diverged: halve below
      }
    }
  }
  // members that did not converge: increment halving from the committed state, alone
  for (int i = 0; i < n; ++i) {
    if (!todo[i]) continue;
    lgdm_sim *s = b->sims[i];
    LGDM_BCUDA(b, cudaMemcpyAsync(s->u, s->u_commit, sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
    int32_t extra = 0;
    lgdm_status st = LGDM_ERR_NOT_CONVERGED;
    if (s->opt.max_halvings > 0) {
      const double from = s->load_commit, mid = 0.5 * (from + loads[i]);
      s->counters[5] += 1;
      s->substep_commits = true;
      st = advance(s, from, mid, 1, &extra);
      if (st == LGDM_OK) st = advance(s, mid, loads[i], 1, &extra);
      s->substep_commits = false;
      if (st == LGDM_OK) {                          // the halved step is one point of the curve
        LGDM_BCUDA(b, launch_external_work(s->reaction, s->load_commit - s->load_point, s->stream));
        s->load_point = s->load_commit;
      }
    }
    its[i] += extra;
    if (status) status[i] = st;
    else if (st != LGDM_OK) return bfail(b, st, s->err);
  }
  if (newton_iters)
    for (int i = 0; i < n; ++i) newton_iters[i] = its[i];
  return LGDM_OK;
}

}  // extern "C"

namespace {

lgdm_status batch_assemble_only(lgdm_batch *b) {
  b->launches += assembly_launches(b);
  return batch_issue_assembly(b);
}

}  // namespace

extern "C" {

lgdm_status lgdm_batch_assemble(lgdm_batch *b, const int32_t *active) {
  if (!b || !active) return bfail(b, LGDM_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < b->n; ++i) b->h_active[i] = active[i] ? 1 : 0;
  LGDM_BCUDA(b, cudaMemcpyAsync(b->d_active, b->h_active.data(), sizeof(int32_t) * b->n, cudaMemcpyHostToDevice, b->stream));
  lgdm_status st = batch_assemble_only(b);
  for (int i = 0; i < b->n; ++i)
    if (b->h_active[i]) {
      b->sims[i]->assembled = true;
      b->sims[i]->counters[1] += 1;
    }
  return st;
}

lgdm_status lgdm_batch_autotune(lgdm_batch *b, int32_t *block_threads, int32_t *grid_factor, double *best_ms) {
  if (!b) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL batch");
  std::vector<int32_t> all(b->n, 1);
  cudaEvent_t e0, e1;
  LGDM_BCUDA(b, cudaEventCreate(&e0));
  LGDM_BCUDA(b, cudaEventCreate(&e1));
  double best = 1e300;
  int bbt = b->bt, bgf = b->grid_factor;
  const bool g = b->graph_on;
  for (int bt : {64, 128, 256})
    for (int gf : {1, 2, 4, 8}) {
      lgdm_status st = lgdm_batch_set_tuning(b, bt, gf, g);
      if (st != LGDM_OK) return st;
      st = lgdm_batch_assemble(b, all.data());            // warm-up (and attribute set-up)
      if (st != LGDM_OK) return st;
      LGDM_BCUDA(b, cudaEventRecord(e0, b->stream));
      for (int r = 0; r < 3; ++r) {
        st = batch_assemble_only(b);
        if (st != LGDM_OK) return st;
      }
      LGDM_BCUDA(b, cudaEventRecord(e1, b->stream));
      LGDM_BCUDA(b, cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 3.0 < best) {
        best = ms / 3.0;
        bbt = bt;
        bgf = gf;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lgdm_status st = lgdm_batch_set_tuning(b, bbt, bgf, g);
  if (block_threads) *block_threads = bbt;
  if (grid_factor) *grid_factor = bgf;
  if (best_ms) *best_ms = best;
  return st;
}

}  // extern "C"
