/*
 * yasps.h -- C ABI of the B300-native IPC Newton hot path.
 *
 * What is computed follows YASPS (arxiv 2605.23088): per-element energy,
 * gradient and PSD-projected Hessian of elastic and contact-barrier terms,
 * scatter into a duplicate-free upper-triangular 3x3 block-sparse Hessian
 * (App. B), block-Jacobi PCG on H p = g with a BSR SpMV (Sec. 8, App. C, D),
 * and the contact-pair broadphase and CCD step bound that feed the line search
 * of the incremental-potential Newton step (Sec. 3, "System Overview").
 *
 * Conventions shared by every entry point
 *  - All entry points are C, take plain pointers and sizes, and never throw.
 *  - Return value: YASPS_OK (0) or a negative yasps_status.  On failure the
 *    system stays valid and yasps_last_error() holds a message.
 *  - "_dev" pointers are CUDA device pointers on the system's device; "_host"
 *    pointers are host memory.  The caller owns every pointer it passes; the
 *    library never frees caller memory and keeps no caller pointer after the
 *    call returns (yasps_build_system copies the scene).
 *  - The DOF vector x is an array of n_nodes nodes, 3 values each (node-major,
 *    x[3*i + k]).  Nodes are: every free vertex (not fixed, not in an affine
 *    body) in increasing vertex order, then 4 nodes per affine body:
 *    t (translation) and the three columns of A, so that a body vertex with
 *    body-relative rest position r sits at p = t + r1 A_1 + r2 A_2 + r3 A_3
 *    (App. A "Gradient Size Computation": 3N + 9 + 3 DOF for one body).
 *  - x, v, gradients and energies are FP64 in both precisions.  Hessian
 *    values and PCG vectors are FP64 (precision 0) or FP32 (precision 1,
 *    "FP32-mixed").
 *  - All work is issued on the stream given at build time.  Calls that
 *    return host scalars synchronise that stream; the others are asynchronous.
 */
#ifndef YASPS_H
#define YASPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct yasps_system yasps_system; /* opaque; owned by the library */
typedef int yasps_status;

#define YASPS_OK 0
#define YASPS_E_INVAL (-1)      /* bad argument or scene */
#define YASPS_E_NOMEM (-2)      /* device allocation failed */
#define YASPS_E_CUDA (-3)       /* a CUDA call failed */
#define YASPS_E_CAPACITY (-4)   /* a bounded buffer overflowed */
#define YASPS_E_NOCONV (-5)     /* PCG or Newton hit its iteration cap */
#define YASPS_E_LINESEARCH (-6) /* no decreasing step within ls_max_iter halvings */
#define YASPS_E_TIMEOUT (-7)    /* a bounded device-side wait gave up */
#define YASPS_E_NAN (-8)        /* a NaN/Inf appeared in the gradient, the solve or the energy */

/* Device allocator used for every library workspace.  alloc returns a device
 * pointer of at least `bytes` (256-byte aligned) or NULL; free releases it.
 * Both are called on the host with the system's stream.  Pass NULL to
 * yasps_build_system to use cudaMallocAsync / cudaFreeAsync on that stream. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* cuda_stream);
  void (*free)(void* ctx, void* ptr, void* cuda_stream);
} yasps_allocator;

/* Solver and step parameters. */
typedef struct {
  int precision;      /* 0: FP64 plain; 1: FP32-mixed (FP32 local Hessians, SpMV and PCG
                         vectors with FP64 residual refinement; FP64 kept for positions,
                         gradients, distances, barrier values, CCD and energies) */
  double dt;          /* time step h (s) */
  double dhat;        /* barrier activation distance (m): pairs with d^2 < dhat^2 are active */
  double kappa;       /* barrier stiffness (multiplies sum b(d^2) in the incremental potential) */
  double gravity[3];  /* m/s^2 */
  double newton_tol;  /* stop when ||p||_inf <= newton_tol (m) */
  double pcg_rel_tol; /* stop PCG when r^T z <= tol^2 r0^T z0 */
  int pcg_max_iter;   /* <= 0: 10 * number of DOF */
  int newton_max_iter;
  int ls_max_iter;    /* maximum halvings in the line search */
  int barrier_form;   /* 0: -(s - sh)^2 ln(s/sh) (IPC); 1: (s - sh)^2 ln^2(s/sh) (the paper's listing) */
  double ccd_gap;     /* additive CCD keeps at least ccd_gap times the starting distance */
  int ccd_max_iter;   /* cap on additive-CCD advancement steps per pair */
  int refine_sweeps;  /* FP32-mixed only: maximum FP64 residual-refinement sweeps */
  int pcg_warm_start; /* yasps_step: start each Newton iteration's PCG from the part of the
                         previous direction the line search did not take, (1 - alpha) p;
                         PCG then stops when r^T z <= tol^2 g^T M^-1 g (the same accuracy
                         relative to the right-hand side g as a cold start) */
  /* Adaptive barrier stiffness (the adaptive stiffness of IPC, Li et al. 2020,
   * restated per time step; single scenes only).  With kappa_adaptive != 0,
   * yasps_step chooses kappa at the start of each step and keeps it for the
   * whole step: the first step that starts with contact pairs takes
   * argmin_k |g_E + k g_B| = -g_E.g_B / g_B.g_B (g_B: barrier gradient at
   * kappa = 1, g_E: gradient of the rest of the potential) clamped to
   * [kappa_min, kappa_max], and kappa_min before that; every later step
   * doubles kappa (at most kappa_max) when the smallest pair distance at its
   * start is below kappa_dmin (<= 0: dhat / 10) and below the previous
   * step's.  kappa_min <= 0
   * derives the lower bound from the scene: the stiffness at which the
   * barrier alone holds an average vertex's weight (total mass / vertex
   * count) at dhat / 2, m h^2 |g| / (2 d |b'(d^2)|) with d = dhat / 2 (|g| = 0:
   * standard gravity); kappa_max <= 0 takes 1e4 times the lower bound.  The
   * kappa of the last step is in yasps_step_stats.kappa and the state can be
   * read and restored with yasps_get_kappa_state / yasps_set_kappa_state. */
  int kappa_adaptive;
  double kappa_min, kappa_max, kappa_dmin;
  double ls_armijo;   /* line search: accept E(x - alpha p) <= E(x) - ls_armijo alpha g^T p
                         (0: any decrease, up to the rounding of the energy sums) */
} yasps_params;

/* Scene, host pointers, copied at build.  Index arrays are int32, 0-based.
 * Elastic elements (tets, cloth triangles, hinges) may reference free or
 * fixed vertices; affine-body vertices take part in contact and inertia. */
typedef struct {
  int n_verts;
  const double* rest_pos;   /* [n_verts][3] undeformed world positions (also the initial state) */
  const int* vert_body;     /* [n_verts] -1 free, an affine body id (>= 0), or -2: embedded in a cage */
  int n_fixed;
  const int* fixed_verts;   /* [n_fixed] vertices with prescribed positions */
  const double* fixed_vel;  /* [n_fixed][3] prescribed velocity, applied at the start of each step */
  int n_tets;
  const int* tet2v;         /* [n_tets][4], positively oriented */
  const double* tet_E;      /* [n_tets] Young's modulus (Pa) */
  const double* tet_nu;     /* [n_tets] Poisson ratio */
  const double* tet_rho;    /* [n_tets] density (kg/m^3) */
  int n_tris;
  const int* tri2v;         /* [n_tris][3] membrane (cloth) triangles */
  const double* tri_E;
  const double* tri_nu;
  const double* tri_thick;
  const double* tri_rho;
  int n_hinges;
  const int* hinge2v;       /* [n_hinges][4] (e0, e1, a, b): triangles (e0,e1,a) and (e1,e0,b) */
  const double* hinge_kb;   /* [n_hinges] bending stiffness */
  int n_bodies;
  const double* body_mass;  /* [n_bodies] kg, lumped uniformly over the body's vertices */
  const double* body_vol;   /* [n_bodies] m^3 */
  const double* body_kappa; /* [n_bodies] orthogonality stiffness (Pa) */
  int n_surf_tris;
  const int* surf_tri2v;    /* [n_surf_tris][3] collision triangles */
  int n_surf_edges;
  const int* surf_edge2v;   /* [n_surf_edges][2] collision edges */
  int n_surf_verts;
  const int* surf_verts;    /* [n_surf_verts] collision vertices, strictly increasing */
  int n_planes;
  const double* planes;     /* [n_planes][4] (n, c): the half-space n.x >= c is free space */
  /* Batching: n_scenes independent scenes in one system (0 or 1 = one scene).
   * vert_scene[v] in [0, n_scenes), non-decreasing in v; every element, body
   * and fixed vertex lies in one scene.  Pairs between scenes are never formed
   * (scenes may overlap in space; planes are shared), and yasps_step runs
   * Newton, the CCD bound, the line search and PCG's alpha / beta / stopping
   * test per scene, so each scene evolves exactly as it would alone.  At most
   * 1024 scenes (YASPS_E_CAPACITY beyond). */
  int n_scenes;
  const int* vert_scene;    /* [n_verts] or NULL when n_scenes <= 1 */
  /* Cloth model of the membrane triangles: 0 StVK (tri_E, tri_nu: Young's
   * modulus and Poisson ratio, plane stress); 1 Baraff-Witkin stretch and
   * shear (Baraff and Witkin 1998 in F-space, the cloth of the paper's
   * benchmarks, Sec. "Cloths on Bunny on Cloth"): with F = [f_u f_v] (3x2)
   * the deformation gradient over the rest (u, v) frame,
   *   Psi = k_st/2 ((|f_u| - 1)^2 + (|f_v| - 1)^2) + k_sh/2 (f_u . f_v)^2,
   * energy = area * thickness * Psi, k_st = tri_E (stretch stiffness, Pa)
   * and k_sh = tri_shear (shear stiffness, Pa); tri_nu is not read.  The
   * Hessian is projected in the 6x6 F-space (Sec. "Eigendecomposition:
   * Manual Optimization").  tri_shear may be NULL for model 0. */
  int cloth_model;
  const double* tri_shear;  /* [n_tris] shear stiffness (Pa), model 1 */
  /* Cage-embedded vertices (the cage parameterisation of Sec. "Caged Bunny"):
   * vertex embed_verts[e] (vert_body -2; strictly increasing) sits at
   * p = sum_k embed_w[e][k] x(embed_cage[e][k]) over the 8 vertices of the
   * cage cell that encloses it (trilinear weights).  Cage vertices must be
   * free (vert_body -1, not fixed, not embedded); embedded vertices carry no
   * DOF, mass or elastic element of their own -- they take part in contact,
   * and their UNION Jacobian (w_k I3 over up to 8 nodes) carries the contact
   * forces to the cage, whose own elements (e.g. 6 tets per cell) hold it
   * together.  A pair of embedded vertices then spans up to 16 nodes, a
   * point-triangle or edge-edge pair up to 32. */
  int n_embedded;
  const int* embed_verts;   /* [n_embedded] */
  const int* embed_cage;    /* [n_embedded][8] cage vertex ids */
  const double* embed_w;    /* [n_embedded][8] weights (sum 1) */
} yasps_scene_desc;

/* Per-call statistics of yasps_step (the paper's counters, Sec. "Simulation
 * Time Comparison": Newton and CG iterations, pair counts by type). */
typedef struct {
  int newton_iters;
  int pcg_iters_total;
  int n_pt, n_ee, n_pg; /* active pairs at the last Newton iteration */
  int status;
  double alpha_last;    /* last accepted line-search step */
  double p_inf;         /* ||p||_inf at exit */
  double t_eval_ms, t_pcg_ms, t_ccd_ms, t_ls_ms; /* stage times (CUDA events) */
  int n_cand_pt, n_cand_ee; /* swept-box candidates of the last line search */
  double kappa;         /* barrier stiffness the step used */
} yasps_step_stats;

/* One record per Newton iteration of the last yasps_step on a single scene
 * (the convergence diagnostics of Sec. "Solver": why a step needed the
 * iterations it did).  Iteration k: the direction p solved at x_k, its
 * infinity norm and the node holding it, the PCG effort, the CCD bound
 * alpha_ccd along x_k - alpha p, the accepted alpha after ls_halvings
 * halvings, the energies E(x_k) and E(x_k - alpha p), and the active pair
 * counts at x_k.  s_min is the smallest squared pair distance at x_k (-1 when
 * yasps_newton_trace_enable was not on, +inf with no pair).  The last record
 * of a converged step has alpha = 0 (no line search ran). */
typedef struct {
  int pcg_iters, ls_halvings;
  int n_pt, n_ee, n_pg, n_cand_pt, n_cand_ee;
  int pinf_node;
  double p_inf, pcg_rel_res, alpha_ccd, alpha, E0, E1, s_min;
  double g_dot_p;     /* g^T p: the decrease the quadratic model predicts for alpha = 1 is g^T p / 2 */
  double p_at_max[3]; /* p at pinf_node */
} yasps_newton_record;

/* Fill *p with defaults (FP64, dt 0.01, dhat 1e-3, kappa 1e4, g = (0,-9.81,0),
 * newton_tol 1e-6, pcg_rel_tol 1e-4, newton_max_iter 100, ls_max_iter 30,
 * barrier_form 0, ccd_gap 0.1, ccd_max_iter 100000, refine_sweeps 4, pcg_warm_start 1,
 * kappa_adaptive 0, kappa_min, kappa_max and kappa_dmin 0 (derived), ls_armijo 0). */
void yasps_default_params(yasps_params* p);

/* Build a system: uploads the scene, computes rest-shape quantities
 * (Dm^-1, volumes, Lame constants, lumped masses, body frames), the DOF layout
 * and the static BSR sparsity of H (App. B: upper blocks of every elastic and
 * inertia contribution, sorted by (row, col), duplicates removed).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * allocator: NULL for cudaMallocAsync/cudaFreeAsync.
 * Errors: E_INVAL (bad sizes/indices, degenerate rest element, elastic element
 * on an affine-body vertex), E_NOMEM, E_CUDA.  *out is NULL on failure and
 * the message is then available from yasps_build_error(). */
yasps_status yasps_build_system(const yasps_scene_desc* scene, const yasps_params* params,
                                const yasps_allocator* allocator, void* cuda_stream, yasps_system** out);
const char* yasps_build_error(void);

/* Release every device buffer (on the system's stream) and the handle. */
void yasps_destroy(yasps_system* sys);

/* Message of the last failing call on this system (never NULL). */
const char* yasps_last_error(const yasps_system* sys);

/* Replace the solver parameters.  Switching precision re-lays out the
 * Hessian storage. */
yasps_status yasps_set_params(yasps_system* sys, const yasps_params* params);

/* Sizes: n_nodes (3 DOF each), n_free (free-vertex nodes), n_verts. */
yasps_status yasps_get_sizes(const yasps_system* sys, int* n_nodes, int* n_free, int* n_verts);

/* Initial node state from the rest pose and per-vertex initial velocities
 * vel0_host [n_verts][3] (may be NULL: zero).  x_dev, v_dev: [n_nodes][3] FP64.
 * A body gets the mean velocity of its vertices as its translation velocity. */
yasps_status yasps_initial_state(yasps_system* sys, const double* vel0_host, double* x_dev, double* v_dev);

/* World positions of all vertices, P_dev [n_verts][3] FP64, from x_dev (the
 * UNION of free, affine and fixed parameterisations, Sec. "UNION"). */
yasps_status yasps_vertex_positions(yasps_system* sys, const double* x_dev, double* P_dev);

/* x_tilde = x_t + h v_t + h^2 M^-1 f_gravity into xtilde_dev [n_nodes][3]. */
yasps_status yasps_xtilde(yasps_system* sys, const double* xt_dev, const double* vt_dev, double* xtilde_dev);

/* Contact detection at x (Sec. "UNION" code example: collision pairs as a
 * dynamic primitive): point-triangle, edge-edge and point-plane pairs with
 * squared distance below dhat^2; exclusions: shared vertex, same affine body,
 * all vertices fixed.  The lists are kept inside the system (they feed
 * yasps_eval_local) and their counts returned (host scalars; synchronises). */
yasps_status yasps_detect_pairs(yasps_system* sys, const double* x_dev, int* n_pt, int* n_ee, int* n_pg);

/* Copy the current pair lists as (a, b, subtype) int32 triples sorted by (a, b):
 * PT: (vertex, surface triangle, closest-feature subtype 0..6);
 * EE: (edge i, edge j > i, subtype 0..12); PG: (vertex, plane, 0).
 * Any output pointer may be NULL.  Host pointers sized by the counts above. */
yasps_status yasps_export_pairs(yasps_system* sys, int* pt_host, int* ee_host, int* pg_host);

/* Terms for term_mask. */
#define YASPS_TERM_INERTIA 1
#define YASPS_TERM_TET 2
#define YASPS_TERM_MEMBRANE 4
#define YASPS_TERM_BEND 8
#define YASPS_TERM_ABD 16
#define YASPS_TERM_BARRIER 32
#define YASPS_TERM_ALL 63

/* Incremental-potential energy E(x) = 1/2 |x - xtilde|_M^2 + h^2 (elastic +
 * ABD) + kappa sum b(s), FP64 with compensated sums on the device, pair set
 * detected at x (the pair lists of the system are not changed).  terms_host
 * (nullable) receives the six term values in YASPS_TERM bit order.
 * Synchronises. */
yasps_status yasps_energy(yasps_system* sys, const double* x_dev, const double* xtilde_dev, double* energy_host,
                          double* terms_host);

/* Local evaluation (Sec. "Hessian Code Generation"): per element / pair
 * gradient and PSD-projected Hessian (project != 0; exact otherwise),
 * scattered into the system's gradient and H = H_static + H_dynamic (Sec.
 * "Index Computation") by atomic addition (App. B "Assembly"), then the
 * block-Jacobi inverse (App. D; only when YASPS_TERM_INERTIA is in the mask,
 * since the inverse needs the mass-regularised full Hessian).  Uses the pair lists of the last
 * yasps_detect_pairs, which must have been called at the same x.  Zeroes g and
 * H first.  Synchronises (reads the device status).  Errors: E_NAN for a
 * non-finite value, or (project != 0) a diagonal block that is not positive
 * definite; with project == 0 such a block is not an error (exact Hessians can
 * be indefinite) but the block-Jacobi preconditioner is then not usable. */
yasps_status yasps_eval_local(yasps_system* sys, const double* x_dev, const double* xtilde_dev, int term_mask,
                              int project);

/* Build the dynamic BSR sparsity of the contact part from the current pair
 * lists (sort + unique of upper block keys, App. B).  yasps_detect_pairs calls
 * it; exposed for timing. */
yasps_status yasps_assemble(yasps_system* sys);

/* Export for tests: which = 0 static / 1 dynamic upper BSR; nnzb (host),
 * row_ptr [n_nodes+1], col [nnzb], vals [nnzb][9] FP64 and (which = 0 only)
 * the diagonal blocks diag [n_nodes][9] FP64, all host.  NULL skips an array. */
yasps_status yasps_export_bsr(yasps_system* sys, int which, int* nnzb, int* row_ptr_host, int* col_host,
                              double* vals_host, double* diag_host);
/* Gradient of the last evaluation, g_dev [n_nodes][3] FP64 (device copy). */
yasps_status yasps_export_gradient(yasps_system* sys, double* g_dev);

/* y = H x with the assembled H (symmetric upper storage, Alg. 7); FP64 in/out
 * (in FP32-mixed the stored FP32 blocks are applied in FP64). */
yasps_status yasps_spmv(yasps_system* sys, const double* x_dev, double* y_dev);

/* Solve H p = rhs by block-Jacobi PCG (Sec. 8 "Solver", App. D), p not negated
 * (Sec. "Solution Extraction").  rhs_dev, p_dev: [n_nodes][3] FP64.  iters and
 * rel_res (host, nullable): iterations and final sqrt(r^T z / r0^T z0).
 * Errors: E_NOCONV when the cap is hit (p holds the last iterate). */
yasps_status yasps_pcg_solve(yasps_system* sys, const double* rhs_dev, double* p_dev, double rel_tol, int* iters,
                             double* rel_res);

/* Largest safe step along x - alpha p, alpha in [0, 1]: additive CCD
 * (Li et al. 2021) for PT/EE candidates from swept boxes, exact for PG.  Host
 * scalar (synchronises). */
yasps_status yasps_ccd_bound(yasps_system* sys, const double* x_dev, const double* p_dev, double* alpha_host);

/* One implicit time step (Sec. 3: CD -> minimise -> CCD/line search -> update):
 * Newton iterations on the incremental potential until ||p||_inf <= newton_tol,
 * then v = (x - x_t)/h.  x_dev, v_dev: [n_nodes][3] FP64, updated in place.
 * stats (host, nullable).  Errors: E_LINESEARCH, E_NOCONV, E_NAN (x, v keep
 * the last accepted iterate). */
yasps_status yasps_step(yasps_system* sys, double* x_dev, double* v_dev, yasps_step_stats* stats);

/* Newton records of the last yasps_step (single scenes; see
 * yasps_newton_record).  capacity: room in out (host); *count receives the
 * number of records of the step (which may exceed capacity; only
 * min(count, capacity) are written).  yasps_newton_trace_enable(sys, 1)
 * adds the smallest pair distance to every record at the cost of one small
 * kernel and a host read per Newton iteration. */
yasps_status yasps_newton_trace(const yasps_system* sys, int capacity, yasps_newton_record* out_host, int* count);
yasps_status yasps_newton_trace_enable(yasps_system* sys, int enable);

/* Adaptive-kappa state (kappa_adaptive): the current kappa, whether it has
 * been initialised by gradient balance, and the smallest pair distance at the
 * start of the previous step (+inf: none); kappa_lo / kappa_hi receive the
 * bounds in force (kappa_min / kappa_max or the derived ones).  Any output
 * pointer may be NULL.  Read the state to checkpoint a rollout, write it to
 * resume one. */
yasps_status yasps_get_kappa_state(yasps_system* sys, double* kappa, int* initialised, double* dmin_prev,
                                   double* kappa_lo, double* kappa_hi);
yasps_status yasps_set_kappa_state(yasps_system* sys, double kappa, int initialised, double dmin_prev);

/* Prescribed positions of fixed vertices (host [n_verts][3]; only fixed rows
 * are read / written). */
yasps_status yasps_set_fixed_positions(yasps_system* sys, const double* P_host);
yasps_status yasps_get_fixed_positions(yasps_system* sys, double* P_host);

/* Autotuning of the PCG kernel's launch configuration (threads per block,
 * upper blocks per thread in a shared-memory tile, blocks per SM), for the
 * batching form and any large system: yasps_autotune_pcg times `iters` PCG
 * iterations (<= 0: 30) of each of the YASPS_PCG_VARIANTS configurations on
 * the system's current assembly, with its current gradient as right-hand side,
 * and keeps the fastest for later solves.  Needs an assembled system (after
 * yasps_eval_local or yasps_step).  variant (nullable) receives the choice,
 * us_per_iter (nullable, [YASPS_PCG_VARIANTS]) each configuration's time per
 * iteration in microseconds.  yasps_set_pcg_variant picks one directly
 * (variant 0 is the default).  Synchronises. */
#define YASPS_PCG_VARIANTS 5
yasps_status yasps_autotune_pcg(yasps_system* sys, int iters, int* variant, double* us_per_iter);
yasps_status yasps_set_pcg_variant(yasps_system* sys, int variant);

/* Bound of the PCG kernel's device-side waits (its grid barriers and tile
 * copies): after `polls` polls a waiting block raises the kernel's abort flag,
 * every block leaves at its next wait (each still waiting for its own copies
 * in flight), and the solve returns YASPS_E_TIMEOUT with the system still
 * usable.  0 restores the default (2^22 polls, a few seconds).
 * unmet_next != 0 is for testing that path: the next PCG launch's grid
 * barriers wait for one arrival more than the grid has (a count nothing
 * completes), so every block runs into the bound; the setting is cleared by
 * that launch. */
yasps_status yasps_set_wait_limit(yasps_system* sys, long long polls, int unmet_next);

/* Per-scene results of the last yasps_step on a batch (host arrays of
 * n_scenes, each nullable): Newton iterations, PCG iterations summed over the
 * step, and status (YASPS_OK, YASPS_E_NOCONV or YASPS_E_LINESEARCH; a scene
 * whose line search fails stops where it is while the others go on, and
 * yasps_step then returns that status). */
yasps_status yasps_scene_stats(const yasps_system* sys, int* newton_iters, int* pcg_iters, int* status);

/* ---- adjoint of the implicit step (differentiation form) ----------------
 * The paper names differentiable simulation as future work (Sec. "Conclusion
 * and Future Work"); the adjoint here follows the implicit-function theorem on
 * the step's optimality condition grad E(x_{t+1}; x_t, v_t, E) = 0 of the
 * incremental potential, with v_{t+1} = (x_{t+1} - x_t) / h.
 *
 * yasps_set_tet_young: per-tet Young's moduli E_dev (device, [n_tets]),
 * Poisson ratios kept; mu and lam are recomputed (standard Lame).  Returns
 * YASPS_E_INVAL for a non-positive or non-finite modulus.
 *
 * yasps_adjoint_step: one reverse step.  Inputs (device, [n_nodes][3] FP64
 * unless noted): the step's start state x_t, v_t, its solution x_next (as
 * yasps_step returned it), and the adjoints xbar = dL/dx_{t+1}, vbar =
 * dL/dv_{t+1}.  It detects the pairs at x_next, assembles the EXACT
 * (unprojected) Hessian H there, solves H lambda = xbar + vbar / h with the
 * same block-Jacobi PCG (relative tolerance pcg_rel_tol; the system's
 * precision), and writes
 *   xbar_prev = dL/dx_t = M lambda - vbar / h,   vbar_prev = dL/dv_t = h M lambda,
 * and ADDS to Ebar (device, [n_tets]) the per-tet dL/dE_e = -h^2 lambda_e .
 * grad(V Psi_e) / E_e (Psi_SNH is linear in E at a fixed Poisson ratio).
 * Fixed vertices must sit where they were at the end of the forward step
 * (yasps_set_fixed_positions).  Errors: YASPS_E_NAN if the exact Hessian has a
 * non-positive diagonal block (the step solution is not a strict minimum),
 * YASPS_E_NOCONV if the PCG hits its cap, YASPS_E_INVAL for null pointers.
 * Output buffers must not alias the inputs.  Synchronises. */
yasps_status yasps_set_tet_young(yasps_system* sys, const double* E_dev);
yasps_status yasps_adjoint_step(yasps_system* sys, const double* x_t, const double* v_t, const double* x_next,
                                const double* xbar, const double* vbar, double* xbar_prev, double* vbar_prev,
                                double* Ebar, double pcg_rel_tol, int* pcg_iters, double* rel_res);

/* Number of kernels this system has launched since it was built (a host
 * counter incremented at every launch). */
long long yasps_kernel_launches(const yasps_system* sys);

/* Stage timing for measurement.  While enabled, the library brackets every
 * instance of a stage with CUDA events recorded on its own stream and keeps,
 * per stage, the count, the summed event time and the algorithmic bytes the
 * stage must move (inputs read once, unique outputs written once):
 *   YASPS_STAGE_SPMV     the H d phase of one PCG iteration (new direction,
 *                        diagonal product, both upper BSR parts, and the
 *                        grid-wide d^T H d), timed with the device's global
 *                        timer inside the PCG kernel (count = iterations;
 *                        bytes: nnzb (9 s + 4) + 4 n + 9 s n + 4 * 3 v n,
 *                        s = bytes per Hessian scalar, v = bytes per vector
 *                        scalar, n = nodes);
 *   YASPS_STAGE_TET      the Neo-Hookean tet gradient / projected-Hessian kernel;
 *   YASPS_STAGE_BARRIER  the contact-barrier evaluation kernels;
 *   YASPS_STAGE_PCG      one whole PCG solve;
 *   YASPS_STAGE_DETECT   contact detection + dynamic BSR layout (in yasps_step);
 *   YASPS_STAGE_EVAL     the whole local evaluation incl. block-Jacobi (in yasps_step);
 *   YASPS_STAGE_CCD      the CCD step bound (in yasps_step);
 *   YASPS_STAGE_LS       the line search's energy evaluations (in yasps_step);
 *   YASPS_STAGE_PCG_KERNEL one launch of the persistent PCG kernel (all the
 *                        iterations of a solve or of one refinement sweep);
 *                        bytes = iterations x (SpMV bytes + 8 * 3 v n + 9 s n).
 * Enabling (enable != 0) resets the counters.  yasps_profile_get synchronises. */
#define YASPS_STAGE_SPMV 0
#define YASPS_STAGE_TET 1
#define YASPS_STAGE_BARRIER 2
#define YASPS_STAGE_PCG 3
#define YASPS_STAGE_DETECT 4
#define YASPS_STAGE_EVAL 5
#define YASPS_STAGE_CCD 6
#define YASPS_STAGE_LS 7
#define YASPS_STAGE_PCG_KERNEL 8
#define YASPS_NUM_STAGES 9
typedef struct {
  long long count;
  double ms;
  double bytes;
} yasps_stage_stats;
yasps_status yasps_profile_enable(yasps_system* sys, int enable);
yasps_status yasps_profile_get(yasps_system* sys, int stage, yasps_stage_stats* out);

/* Where the PCG kernel's time goes, summed over the iterations run while
 * profiling was enabled (ms, read from the device's global timer by the
 * kernel's first block): out[0] the block's own nodes (new direction and
 * diagonal product), out[1] the upper BSR blocks, out[2] the wait for the
 * grid's d^T H d, out[3] the update + preconditioner phase, out[4] the wait
 * for the grid's r^T z; out[5], out[6] the mean and the largest over the
 * grid's blocks of a block's own-node + upper-block time (the load balance of
 * the H d phase); out[7] the wait at the extra grid barrier of the FP64
 * form, after which the upper blocks read d' directly (0 in FP32 and in
 * batches).  Waits include the time the slowest block of the grid needs
 * beyond the first. */
yasps_status yasps_pcg_phase_ms(const yasps_system* sys, double* out);

/* Load balance of the PCG kernel, block by block: for each block of the grid
 * of the last launch profiled since yasps_profile_enable, its own-node +
 * upper-block time in microseconds per iteration (summed over the profiled
 * launches of that grid size, divided by their iterations) and the SM it ran
 * on in that launch.  *n_blocks (host) receives the grid size (0 before any
 * profiled launch); up to `capacity` entries go to us_per_iter and sm_ids
 * (host arrays, each nullable).  For measurement only. */
yasps_status yasps_pcg_block_busy(const yasps_system* sys, int capacity, int* n_blocks, double* us_per_iter,
                                  int* sm_ids);

/* The SpMV layout study (Sec. "Evaluation", the SpMV experiment; App.
 * "SpMV"): y = (D + A_off) x for a symmetric matrix of 3x3 blocks given in
 * one of four layouts, on caller arrays (all device, asynchronous on
 * cuda_stream, no allocation):
 *   YASPS_SPMV_UPPER_BSR   the library's storage: the nnzb upper blocks
 *                          (row < col) sorted by row, each with its row and
 *                          column; rows reduced by a warp-segmented shuffle,
 *                          the transposed products added by atomics;
 *   YASPS_SPMV_FULL_BSR    every off-diagonal block (both triangles) sorted
 *                          by row: the same segmented reduction, no transposes;
 *   YASPS_SPMV_FULL_BCOO   every off-diagonal block in any order, each adding
 *                          its product to y by atomics;
 *   YASPS_SPMV_UPPER_BCOO  the upper blocks in any order, each adding its
 *                          product and its transpose's by atomics.
 * row_dev, col_dev: int [nnzb]; vals_dev: [nnzb][9] row-major blocks;
 * diag_dev [n_nodes][9]; x_dev, y_dev [n_nodes][3] (y overwritten), all FP64
 * (precision 0) or FP32 (precision 1).  flag_dev (device int, caller-zeroed):
 * set to 1 when a block lies outside the layout (index out of range, row >= col
 * for the upper layouts, row == col for the full ones); such blocks are
 * skipped.  Errors: E_INVAL for bad arguments, E_CUDA for a launch failure. */
#define YASPS_SPMV_UPPER_BSR 0
#define YASPS_SPMV_FULL_BSR 1
#define YASPS_SPMV_FULL_BCOO 2
#define YASPS_SPMV_UPPER_BCOO 3
yasps_status yasps_spmv_format(int format, int precision, int n_nodes, int nnzb, const int* row_dev,
                               const int* col_dev, const void* vals_dev, const void* diag_dev, const void* x_dev,
                               void* y_dev, int* flag_dev, void* cuda_stream);

/* PSD projection of count symmetric n x n matrices (row-major, contiguous,
 * FP64 for precision 0, FP32 for 1): out = V max(Lambda, 0) V^T (Sec. "EVD
 * and PSD Projection"), one warp per matrix with the parallel-ordering Jacobi
 * of the barrier kernel; n in {3, 6, 9, 12, 15, 24} -- the sizes of the
 * paper's projection comparison (Sec. "Eigendecomposition: Automatic
 * Optimization": a point-point barrier in node space is 24 x 24 between two
 * affine vertices and 15 x 15 between a free and an affine one, 6 x 6 in
 * position space).  Device pointers, asynchronous on cuda_stream, no
 * allocation.  Errors: E_INVAL (other n, bad arguments), E_CUDA. */
yasps_status yasps_project_batch(int n, int count, int precision, const void* in_dev, void* out_dev,
                                 void* cuda_stream);

/* Measured FMA throughput of the current device's FP64 (precision 0) or FP32
 * (precision 1) pipe in TFLOP/s (2 flops per FMA), from a kernel of
 * independent register FMA chains on every SM, best of three timed launches
 * on the legacy default stream (synchronises the device).  These are the
 * peaks the element and barrier kernels' ALU rooflines are measured against.
 * Errors: E_INVAL, E_CUDA. */
yasps_status yasps_probe_fma_tflops(int precision, double* tflops_host);

/* Block-Jacobi PCG that allocates no device memory (the paper has no
 * counterpart; it is an interface for callers that cannot allocate).
 * Some callers may not call cudaMalloc / cudaFree at solve time -- code inside
 * another framework's fixed memory budget, real-time loops that forbid
 * allocation after start-up, hosts that only lend their own buffers.  This
 * entry point solves H p = rhs for a symmetric positive-definite matrix the
 * caller has assembled in device memory, in the library's layout: n_nodes 3x3
 * diagonal blocks diag_dev [n_nodes][9] and nnzb upper off-diagonal blocks
 * vals_dev [nnzb][9] at (row_dev[k], col_dev[k]) with row < col (repeated
 * coordinates are summed), all FP64, row-major blocks.  rhs_dev, p_dev:
 * [n_nodes][3] FP64 (p is overwritten).  Preconditioner: 3x3 block Jacobi.
 * Stops when r^T z <= rel_tol^2 r0^T z0 or after max_iter iterations
 * (<= 0: 10 * 3 n_nodes).  iters, rel_res (host, nullable) as in
 * yasps_pcg_solve; err (nullable, err_len bytes) receives a message on failure.
 * Every temporary lives in one fixed __device__ array of about 11 MB that each
 * GPU loading the library holds until exit, so n_nodes is limited to 65536:
 * larger problems get YASPS_E_CAPACITY.  All calls share that array: calls
 * whose work overlaps on the GPU race and must be serialised.  The first call
 * on a device looks up the array's device address; make it before any stream
 * capture.  A call cannot itself be captured into a CUDA graph: it reads its
 * convergence scalars back every 8 iterations.  p_dev must not alias rhs_dev
 * or any other input (equal pointers get E_INVAL).  Work runs on cuda_stream;
 * the call returns after synchronising it.
 * Errors: E_INVAL (bad arguments, aliasing, or an upper block outside
 * 0 <= row < col < n_nodes, which is skipped on the device and reported),
 * E_CAPACITY, E_NAN (a diagonal block that is not positive definite by
 * Sylvester's criterion, r^T z < 0 or NaN from a non-finite rhs, or
 * d^T H d <= 0), E_NOCONV (max_iter reached; p holds the last iterate), E_CUDA.
 * A zero rhs returns YASPS_OK with p = 0. */
yasps_status yasps_pcg_solve_static(int n_nodes, int nnzb, const int* row_dev, const int* col_dev,
                                    const double* vals_dev, const double* diag_dev, const double* rhs_dev,
                                    double* p_dev, double rel_tol, int max_iter, void* cuda_stream, int* iters,
                                    double* rel_res, char* err, int err_len);

#ifdef __cplusplus
}
#endif
#endif /* YASPS_H */
