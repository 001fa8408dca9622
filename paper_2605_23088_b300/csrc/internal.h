// internal.h -- host-side state of a yasps_system and the launch wrappers that
// the library's translation units export to each other.  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "yasps.h"

struct yasps_system;
constexpr int kMaxScenes = 1024;  // scenes per batch (per-block scene sums in shared memory)

// a growable device buffer owned by the system (contents are not kept on growth)
struct gbuf {
  void* p = nullptr;
  size_t cap = 0;
};
bool ensure(yasps_system* s, gbuf& b, size_t bytes);
void release(yasps_system* s, gbuf& b);
template <typename T>
T* as(const gbuf& b) { return static_cast<T*>(b.p); }

// Upper off-diagonal BSR part: rows sorted, columns strictly greater than the
// row and increasing inside a row (App. B: unique, upper triangle, sorted).
struct bsr_struct {
  int nnzb = 0;
  gbuf row_ptr;  // int [nn + 1]
  gbuf col;      // int [nnzb]
  gbuf row;      // int [nnzb] row of each block (block-parallel SpMV)
  gbuf vals;     // T [nnzb][9]
};

struct yasps_system {
  yasps_params prm{};
  cudaStream_t stream = nullptr;
  yasps_allocator allocator{};
  bool have_allocator = false;
  std::string err;
  long long launches = 0;

  // sizes
  int nv = 0, nn = 0, nfree = 0, nb = 0, nt = 0, nc = 0, nh = 0, nst = 0, nse = 0, nsv = 0, npl = 0, nfix = 0;
  double bbox_diag = 1.0;
  int nbits = 1;  // bits of a node id in packed (row, col) keys; node 2^nbits - 1 is the sentinel
  int nscene = 1;  // independent scenes in this system (batching)
  int cloth_model = 0;  // membrane triangles: 0 StVK, 1 Baraff-Witkin
  gbuf vscene;     // int [nv] scene of each vertex (batches only)
  gbuf node_scene; // int [nn] scene of each node (batches only)
  double scene_spacing = 0.0;  // lattice spacing of the scenes' broadphase boxes (batches)
  int pcg_variant = 0;         // launch configuration of the PCG kernel (yasps_autotune_pcg)
  long long wait_limit = 0;    // polls of a device-side wait before it gives up (0: default)
  bool wait_unmet = false;     // the next PCG launch's barriers wait for an arrival that never comes (tests)
  // per-scene results of the last yasps_step (batches)
  std::vector<int> scene_newton, scene_status, scene_pcg;
  gbuf scene_buf;  // per-scene device scratch (sums, tolerances, step bounds)

  // scene, device
  gbuf vnode;     // int [nv] free: node; body: first node of its body; fixed: -1
  gbuf vbody;     // int [nv] -1 free, >= 0 affine body, -2 - e cage-embedded (embedding row e)
  int ne = 0;     // cage-embedded vertices
  gbuf emb_node;  // int [ne][8] nodes of an embedded vertex's cage cell
  gbuf emb_w;     // double [ne][8] its trilinear weights
  gbuf vr;        // double [nv][3] body-relative rest position (body vertices)
  gbuf vmass;     // double [nv]
  gbuf rest;      // double [nv][3]
  gbuf xfix;      // double [nv][3] prescribed positions (rows of fixed vertices)
  gbuf fixed;     // int [nfix]
  gbuf fixvel;    // double [nfix][3]
  gbuf nodemass;  // double [nfree] then [nb][16]
  gbuf tet_v;     // int [nt][4] vertex ids
  gbuf tet_n;     // int [nt][4] node ids (-1 fixed)
  gbuf tet_rest;  // double [nt][12]: Dm^-1 (9, row-major), vol, mu, lam
  gbuf tet_E;     // double [nt] current Young's moduli
  gbuf tet_nu;    // double [nt] Poisson ratios
  gbuf tet_slot;  // int [nt][6] static BSR slot of local pairs (01,02,03,12,13,23), -1 none
  gbuf tri_v, tri_n;  // int [nc][3]
  gbuf tri_rest;      // double [nc][8]: Dm^-1 (4), area*thick, mu, lam, 0 (StVK) | k_st, k_sh, 1 (Baraff-Witkin)
  gbuf tri_slot;      // int [nc][3] (01, 02, 12)
  gbuf hinge_v, hinge_n;  // int [nh][4]
  gbuf hinge_rest;        // double [nh][2]: theta0, kb * 3|e|^2 / (A1 + A2)
  gbuf hinge_slot;        // int [nh][6]
  gbuf body_kv;           // double [nb] kappa_a * vol
  gbuf body_slot;         // int [nb][6] (01,02,03,12,13,23) among the body's 4 nodes
  gbuf stri;   // int [nst][3]
  gbuf sedge;  // int [nse][2]
  gbuf svert;  // int [nsv]
  gbuf planes; // double [npl][4]

  // assembled system
  int hess_precision = -1;  // layout of diag / vals / minv (0 FP64, 1 FP32)
  bsr_struct Hs, Hd;        // static (elastic, inertia, ABD) and dynamic (contact) parts
  gbuf diag;                // T [nn][9]
  gbuf grad;                // double [nn][3]
  gbuf minv;                // T [nfree][9] then [nb][144]
  gbuf dsym;                // T [nn][6] D then [nfree][6] M^-1, packed symmetric for the PCG kernel
  gbuf P;                   // double [nv][3] vertex positions at the last evaluation

  // contact pairs, int [n][3] = (a, b, subtype), sorted by (a, b)
  int npt = 0, nee = 0, npg = 0;
  gbuf pt, ee, pg;
  // swept candidates of the current Newton iteration, int [n][2], sorted by (a, b)
  int ncpt = 0, ncee = 0;
  gbuf cpt, cee;
  bool cand_valid = false;
  gbuf pair_key_off;  // int [npt + nee + 1] offsets of each pair's dynamic keys
  gbuf dyn_slot;      // int [nkeys] dynamic BSR slot per key
  gbuf pcg_bt;        // per-block busy time of the PCG kernel's H d' phase (profiling)
  gbuf pf32;          // FP32 copies of vertex arrays for the candidate prefilters
  gbuf bar_k;         // barrier pairs: g_z and K between the derivative and projection kernels
  gbuf bar_prep;      // per PT / EE pair: barrier derivatives (double2) then classification codes (int)
  int nkeys = 0;

  // workspaces
  gbuf status;    // int: latched device error bits
  gbuf scal;      // device scalars (PCG and reductions)
  gbuf red;       // reduction partials
  gbuf scan_tmp;  // scan block sums
  gbuf ws[12];    // scratch (sort keys/values, grid, counts)
  gbuf vec[10];   // PCG vectors
  gbuf stepv[6];  // step vectors
  cudaEvent_t ev[8] = {};

  // stage profiler (yasps_profile_*)
  bool prof_on = false;
  struct pending {
    int stage;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<pending> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  yasps_stage_stats prof_acc[YASPS_NUM_STAGES] = {};
  double pcg_phase_ms[8] = {};  // yasps_pcg_phase_ms
  std::vector<double> pcg_busy_ns;  // yasps_pcg_block_busy: per-block busy ns, summed
  std::vector<int> pcg_busy_sm;     // SM of each block in the last profiled launch
  long long pcg_busy_iters = 0;

  // Newton records of the last yasps_step (yasps_newton_trace)
  std::vector<yasps_newton_record> trace;
  bool trace_smin = false;  // also record the smallest pair distance (one extra kernel per iteration)
  // adaptive barrier stiffness (kappa_adaptive): initialised by gradient
  // balance, and the smallest pair distance at the previous step's start
  bool kappa_init = false;
  double kappa_lo = 0.0, kappa_hi = 0.0;  // resolved bounds (kappa_min / kappa_max, or derived)
  double kappa_dmin_prev = __builtin_huge_val();  // +inf until a step has started
};

// stage profiler: prof_begin returns an event recorded on the stream (or null
// when profiling is off); prof_end records the closing event.
cudaEvent_t prof_begin(yasps_system* s);
void prof_end(yasps_system* s, int stage, cudaEvent_t a, double bytes);
void prof_resolve(yasps_system* s);  // synchronises and folds pending pairs into the counters

#define SYS_FAIL(s, code, msg) \
  do {                         \
    (s)->err = (msg);          \
    return (code);             \
  } while (0)

yasps_status cuda_check(yasps_system* s, cudaError_t e, const char* where);
#define CK(s, call)                                    \
  do {                                                 \
    yasps_status _rc = cuda_check((s), (call), #call); \
    if (_rc != YASPS_OK) return _rc;                   \
  } while (0)
#define RC(call)                       \
  do {                                 \
    yasps_status _rc = (call);         \
    if (_rc != YASPS_OK) return _rc;   \
  } while (0)
// record a launch and check the launch error
#define LAUNCH_CHECK(s, name)                                  \
  do {                                                         \
    (s)->launches++;                                           \
    yasps_status _rc = cuda_check((s), cudaGetLastError(), name); \
    if (_rc != YASPS_OK) return _rc;                           \
  } while (0)
#define ENSURE(s, buf, bytes)                                                   \
  do {                                                                          \
    if (!ensure((s), (buf), (bytes))) SYS_FAIL((s), YASPS_E_NOMEM, "device allocation failed"); \
  } while (0)

// ---------------------------------------------------------------- sort.cu
// exclusive prefix sum of n int32 (in may alias out); *total_host (nullable) synchronises
yasps_status scan_exclusive(yasps_system* s, const int* in, int* out, int n, int* total_host);
// stable LSD radix sort of (uint64 key, int value) pairs on the low `bits` bits,
// in place in keys/vals, using keys_tmp/vals_tmp as the ping-pong buffers
yasps_status radix_sort_pairs(yasps_system* s, uint64_t* keys, int* vals, uint64_t* keys_tmp, int* vals_tmp, int n,
                              int bits);
// Upper BSR structure from n packed keys (row << nbits | col, row < col; the
// sentinel row 2^nbits - 1 is dropped) with contribution ids vals: sorts,
// removes duplicates, fills B.row_ptr / col / row / nnzb and slot_of[contrib]
// (-1 for sentinel keys).  keys/vals are clobbered; tmp buffers from s->ws[6..8].
yasps_status bsr_from_keys(yasps_system* s, uint64_t* keys, int* vals, int n, bsr_struct& B, int* slot_of,
                           int n_contrib);

// ---------------------------------------------------------------- elements.cu
// rest-shape data (Dm^-1, volumes, Lame constants) and free-vertex lumped masses
yasps_status setup_rest(yasps_system* s, const double* tE, const double* tnu, const double* trho, const double* cE,
                        const double* cnu, const double* cth, const double* crho, const double* hkb);
yasps_status static_sparsity(yasps_system* s);
yasps_status launch_positions(yasps_system* s, const double* x, double* P);
yasps_status launch_xtilde(yasps_system* s, const double* xt, const double* vt, double* xtil);
yasps_status launch_eval_static(yasps_system* s, const double* x, const double* xtil, int mask, int project);
// bend.cu: discrete-shell hinges (gradient + projected Hessian), precision by s->hess_precision
yasps_status launch_bend(yasps_system* s, int project);
yasps_status launch_snh_young_adj(yasps_system* s, const double* P, const double* lam, double h2, double* Ebar);
yasps_status launch_set_young(yasps_system* s, const double* E);
// five static terms (inertia, tet, membrane, bend, ABD) into out5 (host); synchronises
// out5: the five static terms (single scene); with sacc (device [nscene],
// batches) every item's energy is added to its scene's entry instead
yasps_status energy_static(yasps_system* s, const double* x, const double* xtil, double* out5, double* sacc = nullptr);

// ---------------------------------------------------------------- contact.cu
yasps_status detect_pairs(yasps_system* s, const double* P);
yasps_status build_dynamic_bsr(yasps_system* s);
yasps_status launch_eval_barrier(yasps_system* s, int project);
yasps_status barrier_energy(yasps_system* s, const double* P, double* E_host);
yasps_status ccd_bound(yasps_system* s, const double* x, const double* p, double* alpha_host);
// candidates of the segment [x, x - p] (positions at x left in s->P, P(x - p) and
// the displacement in s->stepv[4]); CCD, barrier energy and detection on them
yasps_status swept_candidates(yasps_system* s, const double* x, const double* p);
// alpha_host: one bound, or one per scene for batches ([nscene])
yasps_status ccd_candidates(yasps_system* s, double* alpha_host);
// sacc (device [nscene], batches): per-scene sums added there, E_host untouched
yasps_status barrier_energy_candidates(yasps_system* s, const double* P, double* E_host, double* sacc = nullptr);
yasps_status detect_from_candidates(yasps_system* s, const double* P);
// smallest squared distance over the current pair lists at vertex positions P
// (+inf without pairs); synchronises
yasps_status pairs_min_dist2(yasps_system* s, const double* P, double* s_min_host);
// b'(s) of the barrier form (host)
double barrier_db(double s, double sh, int form);

// ---------------------------------------------------------------- solver.cu
yasps_status alloc_hessian(yasps_system* s);
yasps_status zero_system(yasps_system* s);
yasps_status launch_bjacobi(yasps_system* s);
yasps_status spmv64(yasps_system* s, const double* x, double* y);
// x0 (nullable): initial guess; the stopping test is relative to rhs either way
yasps_status pcg_solve(yasps_system* s, const double* rhs, double* p, double tol, int maxit, int* iters,
                       double* rel_res, const double* x0 = nullptr);
// max |x_i| over n values; arg_host (nullable) receives an index i holding it
yasps_status inf_norm(yasps_system* s, const double* x, int n, double* out_host, int* arg_host = nullptr);
// (a.b, b.b) over n FP64 values; synchronises
yasps_status dot2(yasps_system* s, const double* a, const double* b, int n, double* ab_host, double* bb_host);
yasps_status read_status(yasps_system* s, int* bits);  // synchronises, clears the device word
yasps_status autotune_pcg(yasps_system* s, int iters, int* variant, double* us);
