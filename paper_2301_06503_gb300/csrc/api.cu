// Host side of the LGDM C ABI: input checks, the node-block CSR pattern and
// element-to-nonzero map, workspace layout, and the incremental-iterative
// driver (Algorithm 2) built from the device kernels.
#include "lgdm_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace lgdm;

namespace {

thread_local std::string g_last_error;   // errors raised before a handle exists

int nen_of(int elem) { return elem == LGDM_L2 ? 2 : elem == LGDM_Q4 ? 4 : elem == LGDM_H8 ? 8 : 0; }
int dim_of(int elem) { return elem == LGDM_L2 ? 1 : elem == LGDM_Q4 ? 2 : elem == LGDM_H8 ? 3 : 0; }

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
  if ((int64_t)ne * 64 > INT32_MAX) {
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
        P.pc[pos[p]++] = e * 64 + a * 8 + b;
      }
  return LGDM_OK;
}

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
  double *re = nullptr, *rraw = nullptr, *rhs = nullptr;
  double *kv[11] = {};
  double *gm_V = nullptr, *gm_R = nullptr, *gm_y = nullptr, *gm_dots = nullptr, *gm_final = nullptr;
  int64_t gm_ld = 0;
  int gmres_blocks = 1;
  double *partial = nullptr, *field_tmp = nullptr, *reaction = nullptr;
  unsigned int *bar = nullptr;
  SolveResult *res = nullptr;
  int krylov_blocks = 1;
  SolveResult last{};
  // phase timers and counters
  bool timers_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double phase_ms[LGDM_NPHASES] = {};
  int64_t phase_n[LGDM_NPHASES] = {};
  int64_t counters[6] = {};
  // host copies
  std::vector<int32_t> h_nbr_ptr, h_nbr;
  std::string err;
  double load_commit = 0.0;
  bool assembled = false;

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
  if (s.opt.gmres_m > 0) {
    const int m = s.opt.gmres_m;
    s.gm_ld = (s.ndof + 31) & ~int64_t(31);
    s.gm_V = c.take<double>((size_t)(m + 1) * s.gm_ld);
    s.gm_R = c.take<double>((size_t)m * (m + 1));
    s.gm_y = c.take<double>(m);
    s.gm_dots = c.take<double>((size_t)(GMRES_MAX_M + 2) * std::max(s.gmres_blocks, 1));
    s.gm_final = c.take<double>(m + 2);
  }
  s.partial = c.take<double>((size_t)3 * 4 * std::max(s.krylov_blocks, 1));
  s.field_tmp = c.take<double>(std::max((size_t)s.nel * s.ngp, (size_t)s.ndof));
  s.reaction = c.take<double>(1);
  s.bar = c.take<unsigned int>(2);
  s.res = c.take<SolveResult>(1);
  s.ws_needed = c.off + 256;
}

int max_krylov_blocks(bool fp32) {
  static int cache[2] = {-1, -1};
  int &v = cache[fp32 ? 1 : 0];
  if (v < 0) v = fp32 ? bicgstab_max_blocks<float>() : bicgstab_max_blocks<double>();
  return v;
}

// Krylov grid: co-resident blocks, about two nodes' rows per thread at most.
int choose_krylov_blocks(const lgdm_sim &s, bool query_device) {
  int want = (int)((s.ndof + 2 * KRYLOV_THREADS - 1) / (2 * KRYLOV_THREADS));
  if (want < 1) want = 1;
  int cap = 152 * 4;
  if (query_device) {
    const int m = max_krylov_blocks(s.opt.precision == LGDM_PREC_FP32_TANGENT);
    if (m > 0) cap = m;
  }
  if (s.opt.krylov_blocks > 0) want = s.opt.krylov_blocks;
  return std::min(want, cap);
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
  s.ncontrib = (int64_t)s.nel * s.nen * s.nen;
  s.ndir = bcs ? bcs->n_dir : 0;
  s.krylov_blocks = choose_krylov_blocks(s, query_device);
  s.gmres_blocks = s.krylov_blocks;
  if (query_device && o.gmres_m > 0) {
    const int cap = (o.precision == LGDM_PREC_FP32_TANGENT) ? gmres_max_blocks<float>() : gmres_max_blocks<double>();
    if (cap > 0) s.gmres_blocks = std::min(s.gmres_blocks, cap);
  }
  return LGDM_OK;
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
  o->precond = LGDM_PRECOND_NODE_BLOCK;
  o->newton_tol = 1e-8;
  o->krylov_rtol = 1e-8;
  o->max_newton = 50;
  o->max_krylov = 5000;
  o->max_halvings = 6;
  o->krylov_blocks = 0;
  o->gmres_m = 64;
  o->krylov_method = 0;
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
    if (o->max_newton < 1 || o->max_krylov < 1 || o->max_halvings < 0 || !(o->newton_tol > 0.0))
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "bad iteration limits or tolerance");
    if (o->gmres_m < 0 || o->gmres_m > GMRES_MAX_M)
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "gmres_m must be in 0..128");
    if (o->krylov_method != 0 && !(o->krylov_method == 1 && o->gmres_m > 0))
      return fail(nullptr, LGDM_ERR_INVALID_ARG, "krylov_method 1 (GMRES) needs gmres_m > 0");
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
    e = e ? e : cudaMemsetAsync(s->reaction, 0, sizeof(double), st_);
    e = e ? e : cudaMemsetAsync(s->res, 0, sizeof(SolveResult), st_);
    e = e ? e : cudaStreamSynchronize(st_);   // host staging vectors die at return
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
  return LGDM_OK;
}

lgdm_status lgdm_set_state(lgdm_sim *s, const double *u, const double *kh) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  if (u) {
    LGDM_CUDA(s, cudaMemcpyAsync(s->u, u, sizeof(double) * s->ndof, cudaMemcpyHostToDevice, s->stream));
    LGDM_CUDA(s, cudaMemcpyAsync(s->u_commit, s->u, sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
  }
  if (kh)
    LGDM_CUDA(s, cudaMemcpyAsync(s->kappa_hist, kh, sizeof(double) * s->nel * s->ngp, cudaMemcpyHostToDevice,
                                 s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  s->assembled = false;
  return LGDM_OK;
}

lgdm_status lgdm_reset_state(lgdm_sim *s) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  LGDM_CUDA(s, cudaMemsetAsync(s->u, 0, sizeof(double) * s->ndof, s->stream));
  LGDM_CUDA(s, cudaMemsetAsync(s->u_commit, 0, sizeof(double) * s->ndof, s->stream));
  LGDM_CUDA(s, launch_fill(s->kappa_hist, (int64_t)s->nel * s->ngp, s->mat.kappa0, s->stream));
  LGDM_CUDA(s, cudaMemsetAsync(s->reaction, 0, sizeof(double), s->stream));
  s->counters[0] += 1;
  s->load_commit = 0.0;
  s->assembled = false;
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
  LGDM_CUDA(s, cudaMemcpyAsync(s->u, s->u_commit, sizeof(double) * s->ndof, cudaMemcpyDeviceToDevice, s->stream));
  LGDM_CUDA(s, launch_set_dirichlet(s->u, s->dir_dof, s->dir_scale, s->ndir, load, s->stream));
  s->counters[0] += 1;
  s->assembled = false;
  return LGDM_OK;
}

lgdm_status lgdm_assemble(lgdm_sim *s) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  const MeshView mv = s->mesh_view();
  const PatternView pv = s->pattern_view();
  if (s->opt.precision == LGDM_PREC_FP32_TANGENT) {
    {
      PhaseTimer pt(s, 0);
      LGDM_CUDA(s, launch_element<float>(s->elem, mv, s->mc, s->u, s->kappa_hist, nullptr, s->nel,
                                         static_cast<float *>(s->Ke), s->re, false, s->stream));
    }
    {
      PhaseTimer pt(s, 1);
      LGDM_CUDA(s, launch_gather<float>(s->elem, pv, static_cast<float *>(s->Ke), s->re,
                                        static_cast<float *>(s->vals), s->rraw, s->rhs, s->stream));
    }
    {
      PhaseTimer pt(s, 2);
      LGDM_CUDA(s, launch_precond<float>(s->nd, pv, static_cast<float *>(s->vals), s->opt.precond,
                                         static_cast<float *>(s->minv), s->stream));
    }
  } else {
    {
      PhaseTimer pt(s, 0);
      LGDM_CUDA(s, launch_element<double>(s->elem, mv, s->mc, s->u, s->kappa_hist, nullptr, s->nel,
                                          static_cast<double *>(s->Ke), s->re, false, s->stream));
    }
    {
      PhaseTimer pt(s, 1);
      LGDM_CUDA(s, launch_gather<double>(s->elem, pv, static_cast<double *>(s->Ke), s->re,
                                         static_cast<double *>(s->vals), s->rraw, s->rhs, s->stream));
    }
    {
      PhaseTimer pt(s, 2);
      LGDM_CUDA(s, launch_precond<double>(s->nd, pv, static_cast<double *>(s->vals), s->opt.precond,
                                          static_cast<double *>(s->minv), s->stream));
    }
  }
  s->counters[0] += 3;
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
  a.prior_rel = s->last.rel_res;
  a.stall_iters = std::max(500, s->opt.max_krylov / 4);
  a.u = s->u;
  a.partial = s->partial;
  a.bar_count = s->bar;
  a.bar_gen = s->bar + 1;
  a.res = s->res;
  return a;
}

lgdm_status finish_launch(lgdm_sim *s, int mode, SolveResult *out) {
  s->counters[0] += 1;
  LGDM_CUDA(s, cudaMemcpyAsync(out, s->res, sizeof(SolveResult), cudaMemcpyDeviceToHost, s->stream));
  LGDM_CUDA(s, cudaStreamSynchronize(s->stream));
  if (mode != 2) s->counters[2] += out->iters;
  if (s->timers_on) resolve_timers(s);
  if (mode == 2) {
    s->last.converged = out->converged;
    for (int k = 0; k < 4; ++k) s->last.norms[k] = out->norms[k];
  } else {
    s->last = *out;
  }
  if (out->status == 4) return fail(s, LGDM_ERR_TIMEOUT, "grid barrier timed out in the Krylov launch");
  if (out->status == 3) return fail(s, LGDM_ERR_NONFINITE, "non-finite value in the Krylov solve or update");
  return LGDM_OK;
}

lgdm_status run_krylov(lgdm_sim *s, int mode, SolveResult *out) {
  const KrylovArgs a = krylov_args(s);
  {
    PhaseTimer pt(s, 3);
    if (s->opt.precision == LGDM_PREC_FP32_TANGENT)
      LGDM_CUDA(s, launch_bicgstab<float>(a, s->krylov_blocks, mode, s->stream));
    else
      LGDM_CUDA(s, launch_bicgstab<double>(a, s->krylov_blocks, mode, s->stream));
  }
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

// Solve with BiCGSTAB, continue with GMRES when it falls short of krylov_rtol.
lgdm_status solve_robust(lgdm_sim *s, SolveResult *out) {
  if (s->opt.krylov_method == 1) {
    LGDM_CUDA(s, cudaMemsetAsync(s->kv[0], 0, sizeof(double) * s->ndof, s->stream));
    return run_gmres(s, out);
  }
  lgdm_status st = run_krylov(s, 0, out);
  if (st != LGDM_OK && st != LGDM_ERR_NONFINITE) return st;
  // hand over to GMRES only when BiCGSTAB ended far from its tolerance
  const bool short_of = (st == LGDM_ERR_NONFINITE) || (out->status != 0 && out->rel_res > 1e3 * s->opt.krylov_rtol);
  if (!short_of || s->opt.gmres_m <= 0) return st;
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
  st = solve_robust(s, &r);
  if (st != LGDM_OK) return st;
  const int32_t its = r.iters;
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
  if (!s || !c || n < 0 || n > 6) return fail(nullptr, LGDM_ERR_INVALID_ARG, "bad counters request");
  for (int k = 0; k < n; ++k) c[k] = s->counters[k];
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
  if (done) {
    st = lgdm_commit(s);
    if (st == LGDM_OK) s->load_commit = to;
    return st;
  }
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

}  // namespace

extern "C" lgdm_status lgdm_run_step(lgdm_sim *s, double load, int32_t *newton_iters) {
  if (!s) return fail(nullptr, LGDM_ERR_INVALID_ARG, "NULL handle");
  int32_t its = 0;
  lgdm_status st = advance(s, s->load_commit, load, 0, &its);
  if (newton_iters) *newton_iters = its;
  return st;
}
