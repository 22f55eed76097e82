/*
 * lgdm.h - C ABI of the GB300 library for the localizing gradient damage
 * method (LGDM): per-Newton-iteration integration of the coupled
 * displacement / micro-equivalent-strain system over all elements and Gauss
 * points, deterministic assembly into a fixed CSR pattern, a preconditioned
 * Krylov solve, the Newton update and the history commit.
 *
 * The calls follow the paper's statement of the problem (Algorithm 1 and 2
 * take the geometry, the material, the loads and the boundary conditions and
 * return the damage field and the structural response): a mesh, a material
 * and a set of displacement-controlled Dirichlet conditions go in; load-step,
 * Newton-step, assemble, solve and commit calls drive the
 * incremental-iterative procedure.
 *
 * Conventions used by every call
 *   - Units: mm, N, MPa.  Scalars are double unless stated.
 *   - Dofs are interleaved per node: dof nd*a + i with nd = dim + 1; i < dim
 *     are displacement components, i == dim is the micro-equivalent strain.
 *   - Gauss point q of an element sits at the reference position of its local
 *     node q scaled by 1/sqrt(3); per-Gauss-point arrays are [nelem][ngp].
 *   - Host pointers passed in are read during the call only (copied); the
 *     caller keeps ownership.  Device memory is never allocated by the
 *     library: the caller passes one device workspace (sized by
 *     lgdm_workspace_size) and a CUDA stream, both caller-owned and required
 *     to outlive the simulation handle.
 *   - Kernels run on the caller's stream.  Calls that return host scalars
 *     synchronise that stream only; the others are asynchronous.
 *   - Every call returns an lgdm_status; on failure a message is available
 *     from lgdm_last_error().  No C++ exception crosses this boundary.
 *   - A handle is not thread-safe: one host thread drives one handle at a time.
 */
#ifndef LGDM_H
#define LGDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LGDM_ABI_VERSION 2

typedef enum {
  LGDM_OK = 0,
  LGDM_ERR_INVALID_ARG = 1,   /* bad pointer, size or option                   */
  LGDM_ERR_OOM = 2,           /* workspace smaller than lgdm_workspace_size()  */
  LGDM_ERR_CUDA = 3,          /* a CUDA runtime call failed                    */
  LGDM_ERR_NOT_CONVERGED = 4, /* Newton failed after all increment halvings    */
  LGDM_ERR_NONFINITE = 5,     /* NaN/Inf met in the solve or the update        */
  LGDM_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up            */
  LGDM_ERR_STATE = 7          /* call out of order                             */
} lgdm_status;

typedef enum { LGDM_L2 = 1, LGDM_Q4 = 2, LGDM_H8 = 3, LGDM_L3 = 4, LGDM_Q9 = 5 } lgdm_elem;

/* Arithmetic of the tangent.  FP64: everything in double.  FP32_TANGENT: the
 * element tangent is computed in float and the CSR values and node-block
 * inverses are stored in float (an inexact-Newton matrix); the SpMV and the
 * preconditioner multiply those floats into double accumulators, and the
 * residual, Krylov vectors, inner products, the update and the convergence
 * test stay double. */
typedef enum { LGDM_PREC_FP64 = 0, LGDM_PREC_FP32_TANGENT = 1 } lgdm_precision;

/* Preconditioner of the BiCGSTAB solve.  JACOBI: the diagonal; NODE_BLOCK:
 * the inverse of each node's nd x nd diagonal block; MULTIGRID: one V-cycle
 * of aggregation multigrid -- node aggregates of a node and its neighbours
 * (coarsened to at most 24 nodes, at most 10 levels), piecewise-constant
 * prolongation, Galerkin coarse matrices (fixed-order sums of the finer
 * level's node blocks, no atomics), one damped (0.7) node-block Jacobi sweep
 * before and after each coarse correction, and a dense inverse of the
 * coarsest matrix.  The hierarchy is built from the secant tangent (the
 * tangent of Eq. 11a-d with the loading indicator chi taken as 0; its
 * diagonal blocks are positive definite), while BiCGSTAB iterates on the
 * consistent tangent: a damaged, indefinite consistent tangent keeps a
 * well-behaved preconditioner and Newton keeps its quadratic convergence.
 * The assembly writes both matrices; the multigrid set-up runs after every
 * assembly.  The GMRES fallback uses the node blocks (of the secant matrix
 * with the multigrid). */
typedef enum { LGDM_PRECOND_JACOBI = 0, LGDM_PRECOND_NODE_BLOCK = 1, LGDM_PRECOND_MULTIGRID = 2 } lgdm_precond;

typedef enum {
  LGDM_FIELD_U = 0,          /* [ndof]  current nodal dofs (interleaved)         */
  LGDM_FIELD_KAPPA_HIST = 1, /* [nelem*ngp] committed history (Eq. A.2)          */
  LGDM_FIELD_DAMAGE = 2,     /* [nelem*ngp] D(kappa_hist) (Eq. A.1)              */
  LGDM_FIELD_DELTA = 3,      /* [ndof]  last Newton increment from lgdm_solve    */
  LGDM_FIELD_RESIDUAL = 4,   /* [ndof]  last assembled r = -F before Dirichlet rows */
  LGDM_FIELD_RHS = 5         /* [ndof]  -r with zeros on Dirichlet dofs          */
} lgdm_field;

/* Mesh (Sec. 2.2).  Equal order (L2, Q4, H8): both fields on every node,
 * 2 / 2x2 / 2x2x2 Gauss points at +-1/sqrt(3), unit weights.  Mixed order
 * (L3, Q9; the paper's 1D and 2D discretisation): quadratic / biquadratic u
 * on 3 / 9 nodes, linear / bilinear micro-equivalent strain on the leading
 * 2 / 4 (vertex) nodes, 3 / 3x3 Gauss points at 0, +-sqrt(3/5) with weights
 * 8/9, 5/9; the geometry is interpolated like u.  Local node order: bar
 * left->right (L3: ends, then middle); quad counter-clockwise from (-1,-1)
 * (Q9: the four corners so, then the mid-sides of the edges xi2=-1, xi1=+1,
 * xi2=+1, xi1=-1, then the centre); hex bottom face counter-clockwise then
 * top face.  Gauss point q sits at the rule's abscissa times the reference
 * position of local node q (ngp = nen).  Every node carries dim+1 dofs; the
 * micro-equivalent-strain dof of a node that is no element's vertex (mixed
 * order) is in no equation: the library holds it at zero like a Dirichlet
 * dof with no load and no reaction. */
typedef struct {
  int32_t elem;               /* lgdm_elem                                        */
  int32_t nnode, nelem;
  const double *x, *y, *z;    /* [nnode] coordinates; y, z NULL when unused       */
  const int32_t *conn;        /* [nelem*nen] element-major connectivity           */
  const double *e_scale;      /* [nelem] multiplies the elasticity only; NULL = 1 */
  const double *vol_scale;    /* [nelem] multiplies dV (bar area); NULL = 1       */
} lgdm_mesh;

/* Material (Sec. 2.1, Appendix A).  eta is the exponent "n" of Eq. A.4.
 * evm_variant 0 uses 12k/(1+nu)^2 in front of J2 = dev(eps):dev(eps)/2 in
 * Eq. A.3 (uniaxial stress gives eps_eq = axial strain); 1 uses the printed
 * 2k/(1-nu)^2.  In 1D eps_eq is the axial strain and nu, k are ignored.
 * h_stress 0: sigma = (1 - D) C eps (the paper's element code); 1: Eq. 2 as
 * printed, sigma = (1 - D) C eps + h (eps_eq - ebar) d eps_eq/d eps, with the
 * full consistent tangent (K_uu gains B^T [h d (x) d + h (eps_eq - ebar)
 * d2 eps_eq/d eps2] B dV, K_ue gains -B^T h d N^T dV; Eq. 11a-b). */
typedef struct {
  double E, nu, k, kappa0, alpha, beta, R, eta, c, h;
  int32_t evm_variant;
  int32_t h_stress;
} lgdm_material;

/* Displacement control: u[dir_dof[i]] = dir_scale[i] * load at each load
 * step.  The reaction is sum_i dir_scale[i] * r[dir_dof[i]]. */
typedef struct {
  int32_t n_dir;
  const int32_t *dir_dof;
  const double *dir_scale;
} lgdm_bcs;

typedef struct {
  int32_t precision;          /* lgdm_precision                                   */
  int32_t precond;            /* lgdm_precond                                     */
  double newton_tol;          /* ||du|| <= tol ||u|| and ||de|| <= tol ||e||      */
  double krylov_rtol;         /* BiCGSTAB stop: ||r|| <= rtol ||b||               */
  int32_t max_newton;         /* Newton iterations per attempt                    */
  int32_t max_krylov;         /* BiCGSTAB iterations per solve                    */
  int32_t max_halvings;       /* load-increment halvings before giving up         */
  int32_t krylov_blocks;      /* 0 = as many co-resident blocks as fit            */
  int32_t gmres_m;            /* restart of GMRES (1..128); 0 = no GMRES          */
  int32_t krylov_method;      /* 0 BiCGSTAB, GMRES when it falls short; 1 GMRES    */
  double wait_limit_s;        /* limit of every device-side wait (the Krylov grid
                                 barrier): a wait that runs longer gives up, the
                                 launch returns and the call reports
                                 LGDM_ERR_TIMEOUT; 1e-6 .. 60 s, default 2 s      */
} lgdm_options;

typedef struct lgdm_sim lgdm_sim;

/* Sizes of a created simulation.  mg_levels: levels of the multigrid
 * preconditioner (0 without it); mg_nnode / mg_npairs: nodes and node pairs
 * of each level (level 0 is the system itself). */
#define LGDM_MG_MAX_LEVELS 10
typedef struct {
  int32_t dim, nen, ngp, nd;
  int32_t nnode, nelem;
  int64_t ndof, nnz, npairs;  /* npairs: node pairs sharing an element */
  size_t workspace_bytes;
  int32_t mg_levels;
  int32_t mg_nnode[LGDM_MG_MAX_LEVELS];
  int64_t mg_npairs[LGDM_MG_MAX_LEVELS];
} lgdm_sizes;

int32_t lgdm_abi_version(void);
const char *lgdm_status_string(lgdm_status s);

/* Fill *opt with the defaults (FP64, multigrid preconditioner, tol 1e-8, rtol 1e-8,
 * 50 Newton iterations, 5000 Krylov iterations, 6 halvings, GMRES(64)
 * fallback, 2 s device wait limit). */
lgdm_status lgdm_default_options(lgdm_options *opt);

/* Device workspace bytes the simulation of this mesh needs.  Builds the node
 * adjacency on the host to count the CSR pattern exactly. */
lgdm_status lgdm_workspace_size(const lgdm_mesh *mesh, const lgdm_options *opt, size_t *bytes);

/* Size of the fixed CSR pattern of this mesh, host only (no device call):
 * npairs = node pairs (a, b) that share an element, a == b included; the
 * node-block CSR holds nnz = nd * nd * npairs values (Sec. 2.2 assembles into
 * this pattern).  Errors: LGDM_ERR_INVALID_ARG for a bad mesh (unknown
 * element type, missing arrays, connectivity out of range, a node that
 * belongs to no element); lgdm_workspace_size and lgdm_create refuse the
 * same meshes. */
lgdm_status lgdm_pattern_counts(const lgdm_mesh *mesh, int64_t *npairs, int64_t *nnz);

/* Create a simulation.  Copies the mesh, material and conditions, builds the
 * node-block CSR pattern and the element-to-nonzero map on the host, uploads
 * them into dev_workspace (>= lgdm_workspace_size bytes, 256-byte aligned)
 * on `stream` (a cudaStream_t; NULL = the default stream), and sets the
 * initial state u = 0, kappa_hist = kappa0 (Eq. A.1-A.2). */
lgdm_status lgdm_create(const lgdm_mesh *mesh, const lgdm_material *mat, const lgdm_bcs *bcs,
                        const lgdm_options *opt, void *dev_workspace, size_t workspace_bytes,
                        void *stream, lgdm_sim **out);
void lgdm_destroy(lgdm_sim *sim);
const char *lgdm_last_error(const lgdm_sim *sim);
lgdm_status lgdm_get_sizes(const lgdm_sim *sim, lgdm_sizes *out);

/* Replace the state from host arrays u [ndof] and kappa_hist [nelem*ngp]
 * (either may be NULL to keep it).  The result is also the committed state.
 * Both arrays are checked on the host first: a NaN or an infinity returns
 * LGDM_ERR_NONFINITE and leaves the state unchanged.  The committed load,
 * external work and reaction are kept (see lgdm_set_committed). */
lgdm_status lgdm_set_state(lgdm_sim *sim, const double *u, const double *kappa_hist);

/* Scalars of the committed state: the load parameter of the last committed
 * load step, the external work W_ext accumulated by the trapezoid rule over
 * the committed load-reaction points (R17: W_ext(n) = W_ext(n-1) + (R(n) +
 * R(n-1)) (load(n) - load(n-1)) / 2, starting from 0 at the initial state),
 * and the reaction at the committed state.  The points of that curve are
 * the end points of the load steps (one per lgdm_run_step, or per
 * lgdm_commit called by the caller); the committed midpoints of halved
 * increments inside lgdm_run_step are not points of it.  Together with the U and
 * KAPPA_HIST fields they are a checkpoint: lgdm_set_state followed by
 * lgdm_set_committed resumes a simulation exactly.  get synchronises; any
 * pointer may be NULL. */
lgdm_status lgdm_get_committed(lgdm_sim *sim, double *load, double *external_work, double *reaction);
lgdm_status lgdm_set_committed(lgdm_sim *sim, double load, double external_work, double reaction);

/* Return to the initial state on the device (u = 0, kappa_hist = kappa0,
 * committed load 0) without re-creating the simulation.  Asynchronous. */
lgdm_status lgdm_reset_state(lgdm_sim *sim);

/* Copy a field (lgdm_field) into host memory of n doubles (n must match). */
lgdm_status lgdm_get_field(lgdm_sim *sim, int32_t which, double *host_dst, size_t n);

/* Start a load step (Algorithm 2): set the Dirichlet dofs of the
 * committed state to dir_scale * load. */
lgdm_status lgdm_begin_step(lgdm_sim *sim, double load);

/* Compute and assemble K and F at the current state (Algorithm 2, lines
 * 6-7; Eq. 11a-f): element integration over every Gauss point, deterministic
 * summation into the CSR values and the residual (no float atomics; the
 * summation order is fixed by the mesh alone), identity rows and zero
 * columns on Dirichlet dofs.  Asynchronous. */
lgdm_status lgdm_assemble(lgdm_sim *sim);

/* Copy the assembled system to the host: rowptr [ndof+1], col [nnz],
 * vals [nnz] (as double in either precision), rhs [ndof] (= F with zeros on
 * Dirichlet dofs).  Any pointer may be NULL to skip it. */
lgdm_status lgdm_get_system(lgdm_sim *sim, int32_t *rowptr, int32_t *col, double *vals, double *rhs);

/* Solve K delta = F (Algorithm 2) with BiCGSTAB preconditioned by the
 * chosen Jacobi variant, one persistent launch; delta is kept on the device
 * (LGDM_FIELD_DELTA).  Synchronises; iters / rel_res may be NULL. */
lgdm_status lgdm_solve(lgdm_sim *sim, int32_t *iters, double *rel_res);

/* u += delta and the convergence test of Algorithm 2.  Synchronises. */
lgdm_status lgdm_update(lgdm_sim *sim, int32_t *converged);

/* One Newton iteration: assemble, solve (BiCGSTAB; when it does not reach
 * krylov_rtol, restarted GMRES continues from its best iterate), then the
 * update and the convergence test.  The increment is accepted as converged
 * only if its linear solve reached a relative residual of 1e-3 or less.
 * When the solve with the consistent tangent (Eq. 11a-d) ends above that
 * bound, the system is assembled again with the secant tangent (the loading
 * indicator chi taken as 0, which drops the D'(kappa) terms of Eq. 11b and
 * 11d; residual and damage unchanged) and solved; the load step continues
 * with the secant tangent (a quasi-Newton iteration on the same residual,
 * so the converged state is the same).  The next load step starts with the
 * consistent tangent again, unless the previous steps all needed the
 * secant one (then every 8th step tries the consistent tangent). */
lgdm_status lgdm_newton_step(lgdm_sim *sim, int32_t *converged, int32_t *krylov_iters);

/* One load step to `load`: begin_step, Newton iterations until convergence,
 * commit; on non-convergence the increment is halved and retried from the
 * committed state, up to max_halvings times.  newton_iters (may be NULL)
 * receives the total number of Newton iterations spent. */
lgdm_status lgdm_run_step(lgdm_sim *sim, double load, int32_t *newton_iters);

/* History commit after convergence (Eq. A.2): kappa_hist <- max(kappa_hist,
 * ebar at every Gauss point); the current u becomes the committed state and
 * the reaction at this converged state is evaluated on the device. */
lgdm_status lgdm_commit(lgdm_sim *sim);

/* Statistics of the last Krylov launch (lgdm_solve, lgdm_update or
 * lgdm_newton_step): iterations, status (0 converged, 1 iteration limit,
 * 2 breakdown, 3 non-finite, 4 barrier timeout), relative residual, and the
 * norms ||du||, ||u||, ||de||, ||e|| of the last update (norms4 may be NULL). */
lgdm_status lgdm_last_solve(lgdm_sim *sim, int32_t *iters, int32_t *status, double *rel_res, double *norms4);

/* Phase timers (CUDA events recorded on the simulation's stream around each
 * launch).  Phases: 0 element integration, 1 CSR gather + Dirichlet rows,
 * 2 preconditioner set-up, 3 Krylov solve + update, 4 commit + reaction,
 * 5 begin_step.  lgdm_get_timers synchronises the stream and returns, per
 * phase, the summed milliseconds and the number of launches timed since the
 * last reset (arrays of LGDM_NPHASES entries; either may be NULL). */
#define LGDM_NPHASES 6
lgdm_status lgdm_enable_timers(lgdm_sim *sim, int32_t on);
lgdm_status lgdm_get_timers(lgdm_sim *sim, double *ms, int64_t *launches);
lgdm_status lgdm_reset_timers(lgdm_sim *sim);

/* Counters since creation: [0] kernel launches made for this simulation
 * (the batched passes of a batch are counted by the batch,
 * lgdm_batch_get_launches), [1] assemblies,
 * [2] Krylov iterations, [3] Newton iterations, [4] committed load steps,
 * [5] increment halvings, [6] Newton iterations taken with the secant
 * tangent (see lgdm_newton_step).  n entries are written (n <= 7). */
lgdm_status lgdm_get_counters(const lgdm_sim *sim, int64_t *counters, int32_t n);

/* Stored energy Psi (Eq. 1) integrated over the mesh at the current state,
 * with the trial history max(kappa_hist, ebar) (at a committed state this is
 * kappa_hist).  Uses the assembly scratch: call it between load steps.
 * Synchronises. */
lgdm_status lgdm_get_energy(lgdm_sim *sim, double *psi);

/* Reaction at the last committed state.  Synchronises. */
lgdm_status lgdm_get_reaction(lgdm_sim *sim, double *reaction);

/* Dissipated energy at the committed state (R17): the external work of
 * lgdm_get_committed minus the stored energy Psi of Eq. 1 (lgdm_get_energy).
 * Uses the assembly scratch: call it between load steps.  Synchronises;
 * psi (may be NULL) receives the stored energy. */
lgdm_status lgdm_get_dissipated_energy(lgdm_sim *sim, double *dissipated, double *psi);

/* Volume of the region whose committed damage D(kappa_hist) (Eq. A.1)
 * exceeds `threshold` (e.g. 0.9, the localised zone of Sec. 3.3): the sum of
 * the integration weights dV = w det(J) vol_scale over those Gauss points,
 * in fixed order.  Synchronises. */
lgdm_status lgdm_get_damaged_volume(lgdm_sim *sim, double threshold, double *volume);

/* Failure injection for tests of the failure paths; nothing here faults the
 * GPU.  kind:
 *   1  the next Krylov launch of this simulation waits at its grid barrier
 *      for one block more than it launched: no block passes, every wait
 *      gives up after wait_limit_s, the launch returns and the call reports
 *      LGDM_ERR_TIMEOUT (the device context stays usable);
 *   2  the next assembly sees a NaN in the current dofs (written into the
 *      device state by the library): the solve reports a non-finite right-
 *      hand side, lgdm_newton_step returns LGDM_ERR_NONFINITE, and
 *      lgdm_run_step treats it like a diverged Newton iteration (the
 *      increment is halved from the clean committed state);
 *   0  clears a pending injection. */
lgdm_status lgdm_inject_fault(lgdm_sim *sim, int32_t kind);

/* ---------------------------------------------------------------- batches
 * Several simulations advanced together on one stream.  Per element type,
 * one persistent launch integrates every member's elements (tiles of a tuned
 * block size, walked by a tuned number of resident blocks); batched launches
 * gather the CSR values and set up the preconditioners; one cooperative
 * launch per wave solves the members' systems, each member on its own block
 * group (sized in proportion to its node count) with its own grid barrier.
 * Inner products are summed over fixed node tiles, so a member's results do
 * not depend on its group size: they are bitwise those of the member run
 * alone.  A member whose consistent tangent defeats the Krylov solvers is
 * assembled and solved again with the secant tangent in a second batched
 * pass, exactly as lgdm_newton_step does alone.  The launches of a Newton
 * step up to the solve are captured once into a CUDA graph.  Members
 * must have been created on the batch's stream with the same precision and
 * must not be driven individually while a batch call runs.  The batch
 * workspace (device, caller-owned, lgdm_batch_workspace_size bytes) holds
 * the member descriptors and work lists. */
typedef struct lgdm_batch lgdm_batch;
lgdm_status lgdm_batch_workspace_size(int32_t n, size_t *bytes);
lgdm_status lgdm_batch_create(lgdm_sim *const *sims, int32_t n, void *dev_workspace, size_t workspace_bytes,
                              void *stream, lgdm_batch **out);
void lgdm_batch_destroy(lgdm_batch *batch);
const char *lgdm_batch_last_error(const lgdm_batch *batch);
/* Element block size (64, 128 or 256 threads), resident blocks per SM of the
 * persistent element launch (1..32) and CUDA-graph use.  graph_in_use: 0 no
 * graph, 1 the assembly launches are a graph, 2 assembly and solve are.
 * Graphs need a created stream: on the legacy default stream capture is not
 * permitted and the launches are issued directly (lgdm_batch_last_error
 * then holds the reason). */
lgdm_status lgdm_batch_set_tuning(lgdm_batch *batch, int32_t block_threads, int32_t grid_factor, int32_t use_graph);
lgdm_status lgdm_batch_get_tuning(const lgdm_batch *batch, int32_t *block_threads, int32_t *grid_factor,
                                  int32_t *graph_in_use);
/* Solve tuning: each member's Krylov launch group gets about
 * nodes_per_block nodes per block (default 4096; at least the blocks its
 * reduction tiles need, at most one per tile); members of the same nd are
 * packed, largest first, into co-resident cooperative launches ("waves")
 * that run one after the other.  Results do not depend on this setting.
 * get returns the setting and the number of waves. */
lgdm_status lgdm_batch_set_solve_tuning(lgdm_batch *batch, int32_t nodes_per_block);
lgdm_status lgdm_batch_get_solve_tuning(const lgdm_batch *batch, int32_t *nodes_per_block, int32_t *waves);
/* Kernels issued by the batch's own batched passes since creation (directly
 * or as nodes of its CUDA graph).  Launches made for one member alone (its
 * begin_step, commit, GMRES fallback) are in that member's counters. */
lgdm_status lgdm_batch_get_launches(const lgdm_batch *batch, int64_t *launches);
/* Autotuner: times the batched assembly for every block size and grid factor
 * with CUDA events on the current states and keeps the fastest. */
lgdm_status lgdm_batch_autotune(lgdm_batch *batch, int32_t *block_threads, int32_t *grid_factor, double *ms);
/* Batched assembly of the members with active[i] != 0 (host array of n). */
lgdm_status lgdm_batch_assemble(lgdm_batch *batch, const int32_t *active);
/* Phase timers of a batch: CUDA events on the batch stream around the
 * element launches, the gathers, the preconditioner set-ups and the grouped
 * solve of every batched assembly-and-solve pass, in that order.  While
 * timers are on the passes are launched directly, not through the captured
 * graph.  get_timers returns the summed milliseconds and the number of timed
 * passes per phase {element, gather, precond, krylov}; reset != 0 zeroes
 * them. */
lgdm_status lgdm_batch_enable_timers(lgdm_batch *batch, int32_t on);
lgdm_status lgdm_batch_get_timers(lgdm_batch *batch, double *ms4, int64_t *count4, int32_t reset);

/* One Newton iteration (Algorithm 2) for the active members;
 * converged[i] = 1 converged, 0 not yet, -1 non-finite (host arrays of n,
 * krylov_iters may be NULL).  Synchronises. */
lgdm_status lgdm_batch_newton_step(lgdm_batch *batch, const int32_t *active, int32_t *converged,
                                   int32_t *krylov_iters);
/* One load step for every member to loads[i] (NaN: the member sits out):
 * batched Newton iterations, the commit of each member at its convergence,
 * and increment halving, member by member, for those that do not converge.
 * newton_iters[i] and status[i] (lgdm_status of the member) may be NULL;
 * with status NULL the first member failure is returned. */
lgdm_status lgdm_batch_run_step(lgdm_batch *batch, const double *loads, int32_t *newton_iters, int32_t *status);

/* Solve K x = b by BiCGSTAB with node-block Jacobi, allocating nothing.
 *
 * For callers that cannot allocate device memory (a host framework that has
 * reserved all of it, a plugin that must not touch the CUDA allocator): the
 * working storage -- Krylov vectors, block inverses, partial sums, barrier
 * words, result -- comes from one statically declared 64 MiB device array.
 * The paper has no counterpart; this is the same solver as lgdm_solve on a
 * caller-held system.
 *
 *   nd, nnode  dofs per node (2..4) and nodes; ndof = nd * nnode
 *   nbr_ptr    device int32 [nnode+1]; nbr device int32 [nbr_ptr[nnode]]:
 *              sorted neighbour nodes of every node, the node itself included
 *   vals       device double, node-block CSR: row nd*a+i starts at
 *              nd*nd*nbr_ptr[a] + i*nd*deg(a) and holds, for each neighbour
 *              slot s, the nd columns nd*nbr[nbr_ptr[a]+s] + j (the order of
 *              lgdm_get_system)
 *   rhs, x     device double [ndof]; x receives the solution (x = 0 start)
 *   rtol       stop when ||b - K x|| <= rtol ||b||; max_iter iteration cap
 *   stream     cudaStream_t (NULL = default stream); the call synchronises it
 *   iters, rel_res  may be NULL; written only when the solve ran to an end
 *              (not on LGDM_ERR_TIMEOUT)
 *
 * When the array is reserved: CUDA loads a library's device code lazily, so
 * the 64 MiB are reserved on a device the first time this entry point runs
 * there (it then also looks up the array's device address, once per device,
 * with that device current; make that first call before any stream
 * capture).  A call with nnode == 0 does only this set-up and returns
 * LGDM_OK: a caller that is about to reserve all remaining device memory
 * makes it first.  If the reservation itself fails the call returns
 * LGDM_ERR_OOM.  The array then stays reserved until the process exits.
 *
 * Size limit: the scratch takes 72 + 8 nd + 4 / nd bytes per dof (9 vectors,
 * the nd x nd block inverses, one diagonal index per node) plus 96 bytes per
 * reduction tile, each piece rounded up to 256 bytes: at most about 745 k
 * dofs for nd = 2, 689 k for nd = 3 and 639 k for nd = 4.  Larger systems are
 * rejected with LGDM_ERR_OOM and a message (lgdm_last_error(NULL)) before
 * anything is launched.  All calls share the array and it keeps the previous
 * call's contents (the barrier words and the result block are cleared at
 * each call, every vector is written before it is read): calls that overlap
 * on the GPU, from any thread or stream, race and must be serialised. */
lgdm_status lgdm_solve_noalloc(int32_t nd, int32_t nnode, const int32_t *nbr_ptr, const int32_t *nbr,
                               const double *vals, const double *rhs, double *x, double rtol,
                               int32_t max_iter, void *stream, int32_t *iters, double *rel_res);

#ifdef __cplusplus
}
#endif
#endif /* LGDM_H */
