// Internal declarations of the LGDM CUDA library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include "lgdm.h"

namespace lgdm {

// ---------------------------------------------------------------- element traits
// NEN: displacement nodes (= Gauss points); NVE: the leading local nodes that
// carry the micro-equivalent strain; MIXED: quadratic u with linear NVE-node
// micro-equivalent strain and the 3-point rule (Sec. 2.2), else equal order
// with the 2-point rule.
template <int ELEM> struct Elem;
template <> struct Elem<LGDM_L2> { static constexpr int DIM = 1, NEN = 2, NV = 1, NVE = 2; static constexpr bool MIXED = false; };
template <> struct Elem<LGDM_Q4> { static constexpr int DIM = 2, NEN = 4, NV = 3, NVE = 4; static constexpr bool MIXED = false; };
template <> struct Elem<LGDM_H8> { static constexpr int DIM = 3, NEN = 8, NV = 6, NVE = 8; static constexpr bool MIXED = false; };
template <> struct Elem<LGDM_L3> { static constexpr int DIM = 1, NEN = 3, NV = 1, NVE = 2; static constexpr bool MIXED = true; };
template <> struct Elem<LGDM_Q9> { static constexpr int DIM = 2, NEN = 9, NV = 3, NVE = 4; static constexpr bool MIXED = true; };

// Reference node signs; the first 2 rows serve the bar, the first 4 the quad.
__host__ __device__ constexpr int ref_sign(int a, int i) {
  return ((i == 0) ? ((a & 3) == 1 || (a & 3) == 2) : (i == 1) ? ((a & 3) >= 2) : (a >= 4)) ? 1 : -1;
}
// 2-point Gauss rule: factor (1 + xi_q xi_a)/2 with xi_q = +-1/sqrt(3).
constexpr double INV_SQRT3 = 0.57735026918962576451;
constexpr double GP_P = 0.5 + 0.5 * INV_SQRT3;   // signs agree
constexpr double GP_M = 0.5 - 0.5 * INV_SQRT3;   // signs differ

template <int DIM>
__host__ __device__ constexpr double shape_N(int q, int a) {
  double v = 1.0;
  for (int i = 0; i < DIM; ++i) v *= (ref_sign(q, i) == ref_sign(a, i)) ? GP_P : GP_M;
  return v;
}
// dN_a / dxi_j at Gauss point q.
template <int DIM>
__host__ __device__ constexpr double shape_dN(int q, int a, int j) {
  double v = 0.5 * ref_sign(a, j);
  for (int i = 0; i < DIM; ++i)
    if (i != j) v *= (ref_sign(q, i) == ref_sign(a, i)) ? GP_P : GP_M;
  return v;
}

// Quadratic elements: reference coordinate (-1, 0, 1) of local node a in
// direction i (the 3-node bar, dim 1: ends, then middle; the 9-node quad:
// corners as the 4-node quad, mid-sides of the edges xi2=-1, xi1=1, xi2=1,
// xi1=-1, then the centre).
__host__ __device__ constexpr int quad_ref(int dim, int a, int i) {
  return (dim == 1) ? ((a < 2) ? ref_sign(a, 0) : 0)
       : (a < 4) ? ref_sign(a, i)
       : (a == 8) ? 0
       : (i == 0) ? ((a == 5) ? 1 : (a == 7) ? -1 : 0)
                  : ((a == 4) ? -1 : (a == 6) ? 1 : 0);
}
// 3-point rule: Gauss point q at sqrt(3/5) times the position of node q.
constexpr double SQRT_3_5 = 0.77459666924148337704;
// 1D Lagrange polynomial of node r in {-1, 0, 1} at t, and its derivative.
__host__ __device__ constexpr double lagrange2(int r, double t) {
  return (r == 0) ? 1.0 - t * t : 0.5 * t * (t + r);
}
__host__ __device__ constexpr double lagrange2_d(int r, double t) {
  return (r == 0) ? -2.0 * t : t + 0.5 * r;
}

// Element-generic shape data at Gauss point q: u shape functions (and
// geometry), micro-equivalent-strain shape functions (node a < NVE), the
// Gauss weight.  The equal-order elements keep the closed forms above.
template <int ELEM>
__host__ __device__ constexpr double shapeU_N(int q, int a) {
  constexpr int DIM = Elem<ELEM>::DIM;
  if constexpr (!Elem<ELEM>::MIXED) {
    return shape_N<DIM>(q, a);
  } else {
    double v = 1.0;
    for (int i = 0; i < DIM; ++i) v *= lagrange2(quad_ref(DIM, a, i), SQRT_3_5 * quad_ref(DIM, q, i));
    return v;
  }
}
template <int ELEM>
__host__ __device__ constexpr double shapeU_dN(int q, int a, int j) {
  constexpr int DIM = Elem<ELEM>::DIM;
  if constexpr (!Elem<ELEM>::MIXED) {
    return shape_dN<DIM>(q, a, j);
  } else {
    double v = 1.0;
    for (int i = 0; i < DIM; ++i) {
      const double t = SQRT_3_5 * quad_ref(DIM, q, i);
      v *= (i == j) ? lagrange2_d(quad_ref(DIM, a, i), t) : lagrange2(quad_ref(DIM, a, i), t);
    }
    return v;
  }
}
template <int ELEM>
__host__ __device__ constexpr double shapeE_N(int q, int a) {
  constexpr int DIM = Elem<ELEM>::DIM;
  if constexpr (!Elem<ELEM>::MIXED) {
    return shape_N<DIM>(q, a);
  } else {
    double v = 1.0;
    for (int i = 0; i < DIM; ++i) v *= 0.5 * (1.0 + ref_sign(a, i) * SQRT_3_5 * quad_ref(DIM, q, i));
    return v;
  }
}
template <int ELEM>
__host__ __device__ constexpr double shapeE_dN(int q, int a, int j) {
  constexpr int DIM = Elem<ELEM>::DIM;
  if constexpr (!Elem<ELEM>::MIXED) {
    return shape_dN<DIM>(q, a, j);
  } else {
    double v = 1.0;
    for (int i = 0; i < DIM; ++i)
      v *= (i == j) ? 0.5 * ref_sign(a, i) : 0.5 * (1.0 + ref_sign(a, i) * SQRT_3_5 * quad_ref(DIM, q, i));
    return v;
  }
}
template <int ELEM>
__host__ __device__ constexpr double gp_weight(int q) {
  if constexpr (!Elem<ELEM>::MIXED) {
    return 1.0;
  } else {
    double w = 1.0;
    for (int i = 0; i < Elem<ELEM>::DIM; ++i) w *= (quad_ref(Elem<ELEM>::DIM, q, i) == 0) ? 8.0 / 9.0 : 5.0 / 9.0;
    return w;
  }
}

// ---------------------------------------------------------------- material
struct MatConst {
  double lam, mu;             // Lame constants (2D plane strain / 3D); 1D: lam = E, mu = 0
  double evm_a, evm_b2, evm_cJ, inv2k;   // Eq. A.3 coefficients
  double kappa0, alpha, beta;            // Eq. A.1
  double g_a, g_b, eta;                  // g = g_a e^{-eta D} + g_b  (Eq. A.4)
  double h, c;
  // 1: assemble the secant tangent -- the loading indicator chi of Eq. 11b
  // and 11d is taken as 0, which drops the D'(kappa) terms; the residual
  // and the damage are unchanged
  int32_t secant;
  int32_t hterm;                         // 1: Eq. 2-literal stress (h-term in sigma)
};

MatConst make_matconst(const lgdm_material &m, int dim);

// Largest relative linear residual with which a Newton increment may still be
// accepted (an inexact-Newton forcing term); a solve that ends above it with
// the consistent tangent is repeated with the secant tangent.
constexpr double KRYLOV_NEWTON_ETA = 1e-3;

// ---------------------------------------------------------------- device views
struct MeshView {
  const double *x, *y, *z;
  const int32_t *conn;        // [nel*nen]
  const double *e_scale, *vol_scale;
  int32_t nel, nnode;
};

struct PatternView {
  int32_t nnode;
  int64_t npairs;
  const int32_t *nbr_ptr;     // [nnode+1]
  const int32_t *nbr;         // [npairs] neighbour node of each pair (sorted per node)
  const int32_t *pair_node;   // [npairs] owning node of each pair
  const int32_t *pc_ptr;      // [npairs+1] contributions of each pair
  const int32_t *pc;          // [ncontrib] packed (element*64 + a_loc*8 + b_loc)
  const int32_t *diag_pair;   // [nnode] pair index of (a, a)
  const uint8_t *isdir;       // [ndof]
};

// Result block written by the persistent Krylov kernel.
struct SolveResult {
  int32_t iters;
  int32_t status;             // 0 ok, 1 max iterations, 2 breakdown, 3 nonfinite, 4 barrier timeout (max wins)
  int32_t converged;          // Newton test after the fused update
  int32_t pad;
  double rel_res;
  double bnorm;
  double norms[4];            // ||du||, ||u||, ||de||, ||e||
};

// ---------------------------------------------------------------- launchers
template <typename TT>
cudaError_t launch_element(int elem, const MeshView &m, const MatConst &mc, const double *u,
                           const double *kappa_hist, const int32_t *elem_list, int32_t n_elem,
                           TT *Ke, double *re, bool residual_only, cudaStream_t s);   // mc.hterm selects the variant
template <typename TT>
cudaError_t launch_gather(int elem, const PatternView &p, const TT *Ke, const double *re,
                          TT *vals, double *rraw, double *rhs, cudaStream_t s);
template <typename TT>
cudaError_t launch_precond(int nd, const PatternView &p, const TT *vals, int kind, TT *minv,
                           cudaStream_t s);
cudaError_t launch_set_dirichlet(double *u, const int32_t *dof, const double *scale, int32_t n,
                                 double load, cudaStream_t s);
cudaError_t launch_commit(int elem, const MeshView &m, const double *u, double *kappa_hist,
                          cudaStream_t s);
cudaError_t launch_fill(double *p, int64_t n, double v, cudaStream_t s);
// stored energy (Eq. 1): per-Gauss-point values into psi [nel*ngp], their sum into *out
cudaError_t launch_energy(int elem, const MeshView &m, const MatConst &mc, const double *u, const double *kh,
                          double *psi, double *part, double *out, cudaStream_t s);
// diag[a] = position of node a in its own neighbour list
cudaError_t launch_diag_pairs(const PatternView &p, int32_t *diag, cudaStream_t s);
// message for lgdm_last_error(NULL)
void set_global_error(const std::string &msg);
cudaError_t launch_damage_field(const MatConst &mc, const double *kappa_hist, int64_t n, double *out,
                                cudaStream_t s);
cudaError_t launch_reaction_sum(const double *re, const int32_t *idx, const double *w, int32_t n,
                                double *out, cudaStream_t s);
// committed scalars c[0] reaction, c[1] external work, c[2] previous reaction:
// c[1] += (c[0] + c[2]) dload / 2; c[2] = c[0]
cudaError_t launch_external_work(double *c, double dload, cudaStream_t s);
// volume of the Gauss points whose damage D(kappa_hist) exceeds threshold:
// per-point dV (or 0) into vol [nel*ngp], fixed-order sum into *out
cudaError_t launch_damaged_volume(int elem, const MeshView &m, const MatConst &mc, const double *kh,
                                  double threshold, double *vol, double *part, double *out, cudaStream_t s);

// ---------------------------------------------------------------- aggregation multigrid
// Levels of the aggregation multigrid preconditioner.  Level 0 is the
// system's own node-block CSR; level l+1 has one node per aggregate of level
// l (a node and its neighbours, chosen greedily), the prolongation copies an
// aggregate's nd values to each of its nodes, the restriction sums them, and
// the level-(l+1) matrix is the Galerkin product R A_l P: every block of it is
// the fixed-order sum of the level-l blocks of the node pairs that map to it.
constexpr int AMG_MAX_LEVELS = LGDM_MG_MAX_LEVELS;
constexpr int AMG_COARSE_MAX = 24;        // nodes of the coarsest level (dense inverse)
constexpr int AMG_SINGLE_BLOCK = 2048;    // levels with at most this many nodes run in one block
constexpr double AMG_OMEGA = 0.7;         // damping of the block-Jacobi smoother

struct AmgLevel {
  int32_t nnode;
  int32_t npairs;
  const int32_t *nbr_ptr, *nbr, *pair_node, *diag_pair;   // pattern (level 0: the system's)
  void *vals, *minv;                       // TT node-block values and block-Jacobi inverses
  const int32_t *mem_ptr, *mem;            // members of each node (level >= 1): [nnode+1], [n_{l-1}]
  const int32_t *cmap_ptr, *cmap;          // Galerkin map (level >= 1): [npairs+1], [npairs_{l-1}]
  const int32_t *agg;                      // node -> node of the next level (all but the coarsest)
  double *v, *X, *R, *z;                   // [nd*nnode] V-cycle vectors (level 0: X, R only)
  // level 0 of mixed-order meshes: per-dof flag of the held (Dirichlet and
  // uninterpolated micro-strain) dofs, which the prolongation, restriction and
  // Galerkin product leave out; NULL elsewhere
  const uint8_t *held;
  // level 0 with the FP32 tangent: X as float pairs for the FP32-pipe
  // residual SpMV; NULL elsewhere
  float2 *Xhl;
};

struct AmgInfo {
  const AmgLevel *lev;                     // [nlev] device array
  int32_t nlev;                            // 0: no multigrid (block Jacobi)
  int32_t sb_level;                        // first level run by a single block
  double *cinv;                            // [(nd n_c)^2] inverse of the coarsest matrix
  int32_t nc;                              // nodes of the coarsest level
};

// Host-built hierarchy (pattern only; values are set up per assembly).
struct AmgHost {
  struct Lev {
    int32_t nnode = 0;
    std::vector<int32_t> nbr_ptr, nbr, pair_node, diag_pair, mem_ptr, mem, cmap_ptr, cmap, agg;
  };
  std::vector<Lev> lev;                    // lev[0] holds only agg (the pattern is the system's)
};
// Builds the coarse levels from the fine node graph (nbr_ptr, nbr); false if
// the graph does not coarsen.
bool amg_build(int32_t nnode, const std::vector<int32_t> &nbr_ptr, const std::vector<int32_t> &nbr, AmgHost &h);

// One member of a batch, as the batched kernels see it.
struct BatchSim {
  MeshView m;
  MatConst mc;
  const double *u, *kh;
  void *Ke;
  double *re;
  PatternView p;
  void *vals;
  double *rraw, *rhs;
  void *minv;
  int32_t precond;
  AmgInfo amg;
  // multigrid preconditioning of the consistent tangent by the secant one:
  // per-element loading-indicator terms [nel][nen][nen][nd] and the secant
  // matrix (the consistent values minus them); both NULL without multigrid
  void *Kcor, *vals_sec;
};
// elements per tile of the batched element launch at block size bt (after
// element_block's shared-memory fit)
int batch_tile_elements(int elem, bool fp32, bool hterm, int bt);
int element_block(int elem, bool fp32, bool hterm, int bt);
int elem_nen(int elem);          // displacement nodes (= Gauss points) of an element type, 0 if unknown
template <typename TT>
cudaError_t launch_batch_element(int elem, int bt, bool hterm, const BatchSim *sims, const int32_t *members,
                                 const int64_t *tile_start, int nm, int64_t total, const int32_t *active, int grid,
                                 cudaStream_t s);
template <typename TT>
cudaError_t launch_batch_gather(int elem, const BatchSim *sims, const int32_t *members, const int64_t *block_start,
                                int nm, int64_t total_blocks, const int32_t *active, cudaStream_t s);
template <typename TT>
cudaError_t launch_batch_precond(int nd, const BatchSim *sims, const int32_t *members, const int64_t *block_start,
                                 int nm, int64_t total_blocks, const int32_t *active, cudaStream_t s);
// Multigrid set-up of level l (>= 1) for the members listed: Galerkin values
// (256 coarse pairs per block, prefix pair_blocks) then block-Jacobi inverses
// (128 nodes per block, prefix node_blocks).
template <typename TT>
cudaError_t launch_batch_amg_level(int nd, int level, const BatchSim *sims, const int32_t *members,
                                   const int64_t *pair_blocks, const int64_t *node_blocks, int nm, int64_t total_pb,
                                   int64_t total_nb, const int32_t *active, cudaStream_t s);
// Dense inverse of each listed member's coarsest level, one block per member.
template <typename TT>
cudaError_t launch_batch_amg_coarse(int nd, const BatchSim *sims, const int32_t *members, int nm,
                                    const int32_t *active, cudaStream_t s);

constexpr int KRYLOV_THREADS = 256;

// Inner products of the Krylov solvers are summed over fixed tiles of nodes
// (tile = 32 * 2^k nodes, at most KRYLOV_MAX_TILES tiles per system): a warp
// sums 32 consecutive nodes in a fixed shuffle tree, a tile adds its warp
// sums in order, and the tile sums are added in tile order.  The tiles
// depend on the node count only, so the result of a solve does not depend
// on how many blocks share the system (alone or in a batch).  A block owns
// a contiguous range of tiles and at most 32 * KRYLOV_MAXW nodes.
constexpr int KRYLOV_MAXW = 512;
constexpr int64_t KRYLOV_MAX_TILES = 2048;
inline int krylov_tile(int64_t nnode) {
  int t = 32;
  while ((nnode + t - 1) / t > KRYLOV_MAX_TILES) t *= 2;
  return t;
}
inline int64_t krylov_ntiles(int64_t nnode) {
  const int t = krylov_tile(nnode);
  return nnode > 0 ? (nnode + t - 1) / t : 1;
}
// fewest blocks that keep every block within 32 * KRYLOV_MAXW nodes (0: too large)
inline int64_t krylov_min_blocks(int64_t nnode) {
  const int t = krylov_tile(nnode);
  const int64_t per = (int64_t)32 * KRYLOV_MAXW / t;
  if (per < 1) return 0;
  return (krylov_ntiles(nnode) + per - 1) / per;
}

struct KrylovArgs {
  int32_t nd, nnode;
  int32_t max_iter;
  int32_t stall_iters;        // stop after this many iterations without a new best residual
  int32_t tile, ntiles;       // reduction tiles (krylov_tile, krylov_ntiles)
  double rtol, newton_tol;
  PatternView p;
  const void *vals;           // TT [nnz]
  const void *minv;           // TT [nnode*nd*nd]
  const double *rhs;          // [ndof]
  double *x, *r, *r0, *pv, *v, *sv, *t, *ph, *sh, *xb;   // [ndof] each; xb = best iterate
  // FP32 tangent: ph and sh also as float pairs (hi + lo = the double to
  // 2^-48), the input of the FP32-pipe SpMV; NULL otherwise (FP64 products)
  float2 *ph_hl, *sh_hl;
  double *u;                  // [ndof] state (modes 1 and 2)
  double *partial;            // [3 slots][4 values][ntiles]
  unsigned int *bar_count, *bar_gen;
  SolveResult *res;
  unsigned long long wait_ns;  // limit of each grid-barrier wait
  int32_t barrier_extra;       // blocks the barrier waits for beyond those launched (failure injection; 0)
  AmgInfo amg;                 // nlev > 0: the preconditioner is one multigrid V-cycle
};
// mode 0: solve; 1: solve, u += delta, Newton test; 2: update and test only.
template <typename TT>
cudaError_t launch_bicgstab(const KrylovArgs &a, int nblocks, int mode, cudaStream_t s);
template <typename TT>
int bicgstab_max_blocks();
// one cooperative launch over several systems (block groups, see krylov.cu)
template <typename TT>
cudaError_t launch_bicgstab_grouped(int nd, const KrylovArgs *d_args, const int32_t *d_members,
                                    const int32_t *d_group_start, const int32_t *d_active, int nsys,
                                    int total_blocks, int mode, cudaStream_t s);
cudaError_t launch_collect_results(const KrylovArgs *d_args, int n, SolveResult *d_out, cudaStream_t s);
template <typename TT>
int bicgstab_grouped_max_blocks();

constexpr int GMRES_MAX_M = 128;
struct GmresArgs {
  int32_t m;                  // restart length (<= GMRES_MAX_M)
  int64_t ld;                 // leading dimension of the basis
  double *V;                  // [(m+1) * ld] Krylov basis
  double *R;                  // [m * (m+1)] rotated Hessenberg columns (block 0 writes)
  double *y;                  // [m]
  double *dots;               // [(GMRES_MAX_M+2) * gridDim] per-block partials
  double *final;              // [m+2] reduced inner products
  double *xs;                 // [ndof] scratch vector read by the SpMV
};
template <typename TT>
cudaError_t launch_gmres(const KrylovArgs &a, const GmresArgs &g, int nblocks, cudaStream_t s);
template <typename TT>
int gmres_max_blocks();

}  // namespace lgdm
