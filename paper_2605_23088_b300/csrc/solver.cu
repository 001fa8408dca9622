// solver.cu -- block-Jacobi preconditioned CG on H p = g (Sec. 8 "Solver";
// App. C "SpMV"; App. D "Preconditioner").
//
// H is stored as its diagonal blocks plus two upper-triangular BSR parts
// (static and dynamic), so y = H x = D x + U x + U^T x.  The SpMV is
// block-parallel like Alg. 7 (one 3x3 block per thread, blocks sorted by row),
// but the row-segment reduction of U x is a segmented warp reduction done with
// shuffles instead of a linear scan through shared memory; the segment head and
// the transpose term U^T x use atomic additions.
//
// All iterations of a solve run inside one persistent cooperative kernel (one
// block per SM).  An iteration is three grid-wide phases separated by a grid
// barrier whose waits are bounded; each phase leaves one partial sum per
// block, and after the barrier every block adds the partials up in block order,
// so alpha, beta and the stopping decision are bit-identical in all blocks and
// independent of scheduling.  In the FP32-mixed form the inner PCG runs on FP32
// vectors and FP32 blocks; an outer loop recomputes the residual g - H p in
// FP64 and solves for the correction (iterative refinement).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int PT_ = 256;           // threads per block for vector kernels
// Launch configurations of the persistent PCG kernel: threads per block,
// upper blocks per thread in a tile, blocks per SM.  Variant 0 is the default;
// yasps_autotune_pcg times them on the system at hand and keeps the fastest.
template <int NTHR_, int BPT_, int MINB_>
struct pcg_cfg {
  static constexpr int NTHR = NTHR_, BPT = BPT_, MINB = MINB_;
};
template <typename T, int V>
struct pcg_variant;
template <> struct pcg_variant<float, 0> { using C = pcg_cfg<1024, 2, 1>; };
template <> struct pcg_variant<float, 1> { using C = pcg_cfg<1024, 1, 1>; };
template <> struct pcg_variant<float, 2> { using C = pcg_cfg<512, 2, 2>; };
template <> struct pcg_variant<float, 3> { using C = pcg_cfg<256, 2, 4>; };
template <> struct pcg_variant<float, 4> { using C = pcg_cfg<512, 4, 2>; };
// FP64 needs more registers per thread
template <> struct pcg_variant<double, 0> { using C = pcg_cfg<640, 2, 1>; };
template <> struct pcg_variant<double, 1> { using C = pcg_cfg<640, 1, 1>; };
template <> struct pcg_variant<double, 2> { using C = pcg_cfg<320, 2, 2>; };
template <> struct pcg_variant<double, 3> { using C = pcg_cfg<320, 1, 2>; };
template <> struct pcg_variant<double, 4> { using C = pcg_cfg<160, 2, 4>; };
constexpr int kPcgVariants = 5;

// result of one persistent PCG launch (written by block 0 at the end)
struct pcg_dev {
  double rz, rz0;
  int done, iters;  // done: 1 converged, 2 breakdown (d^T H d <= 0), 3 barrier timeout
  unsigned long long t_ns[8];  // block 0's time per phase, summed over iterations (see k_pcg_persistent)
};
// grid barrier state, zeroed before every launch: count only grows (barrier k
// of a launch completes when it reaches (k + 1) * gridDim.x); sum[k % 4]
// collects the per-block partials reduced at barrier k
struct pcg_bar {
  unsigned count;
  int abort;
  unsigned pool[2];  // claimed shared tiles of the H d' phase, iteration parity
  double sum[4];
};

// ---------------------------------------------------------------- SpMV
template <typename T, typename V>
__global__ void k_spmv_diag(int nn, const T* __restrict__ D, const V* __restrict__ x, V* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const T* B = D + 9 * (size_t)i;
  const V x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
#pragma unroll
  for (int a = 0; a < 3; ++a) y[3 * i + a] = (V)B[3 * a] * x0 + (V)B[3 * a + 1] * x1 + (V)B[3 * a + 2] * x2;
}

template <typename V>
__device__ __forceinline__ V shfl_down_v(V v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }

// y += U x + U^T x for one upper BSR part (one block per thread)
template <typename T, typename V>
__global__ void __launch_bounds__(256) k_spmv_upper(int nnzb, const int* __restrict__ row, const int* __restrict__ col,
                                                    const T* __restrict__ vals, const V* __restrict__ x,
                                                    V* __restrict__ y, const int* __restrict__ done) {
  if (done && *done) return;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int r = -1;
  V a0 = 0, a1 = 0, a2 = 0;
  if (k < nnzb) {
    r = row[k];
    const int c = col[k];
    const T* B = vals + 9 * (size_t)k;
    T b[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) b[t] = B[t];
    const V xc0 = x[3 * c], xc1 = x[3 * c + 1], xc2 = x[3 * c + 2];
    const V xr0 = x[3 * r], xr1 = x[3 * r + 1], xr2 = x[3 * r + 2];
    a0 = (V)b[0] * xc0 + (V)b[1] * xc1 + (V)b[2] * xc2;
    a1 = (V)b[3] * xc0 + (V)b[4] * xc1 + (V)b[5] * xc2;
    a2 = (V)b[6] * xc0 + (V)b[7] * xc1 + (V)b[8] * xc2;
    // transpose term into y[c]
    atomicAdd(&y[3 * c], (V)b[0] * xr0 + (V)b[3] * xr1 + (V)b[6] * xr2);
    atomicAdd(&y[3 * c + 1], (V)b[1] * xr0 + (V)b[4] * xr1 + (V)b[7] * xr2);
    atomicAdd(&y[3 * c + 2], (V)b[2] * xr0 + (V)b[5] * xr1 + (V)b[8] * xr2);
  }
  // the U x contributions: FP32 by a segmented suffix reduction within the
  // warp; FP64 by one atomic per block and component (in L2, off the FP64 pipe)
  if constexpr (sizeof(V) == 4) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ro = __shfl_down_sync(0xffffffffu, r, o);
      const V b0 = shfl_down_v(a0, o), b1 = shfl_down_v(a1, o), b2 = shfl_down_v(a2, o);
      if (lane + o < 32 && ro == r) { a0 += b0; a1 += b1; a2 += b2; }
    }
    const int rp = __shfl_up_sync(0xffffffffu, r, 1);
    if (!(r >= 0 && (lane == 0 || rp != r))) return;
  }
  if (r >= 0) {
    atomicAdd(&y[3 * r], a0);
    atomicAdd(&y[3 * r + 1], a1);
    atomicAdd(&y[3 * r + 2], a2);
  }
}

// ---------------------------------------------------------------- block-Jacobi
template <typename T>
__global__ void k_bj_free(int nfree, const T* __restrict__ D, T* __restrict__ Mi, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nfree) return;
  double A[9];
  for (int t = 0; t < 9; ++t) A[t] = (double)D[9 * (size_t)i + t];
  const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
  const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  // positive definite by Sylvester's criterion (leading minors A00, the 2x2
  // one and det); otherwise the identity stands in and the block is reported
  if (!(A[0] > 0.0) || !(A[0] * A[4] - A[1] * A[3] > 0.0) || !(det > 0.0) || !isfinite(det)) {
    dev_flag(status, isfinite(det) ? DEV_INDEFINITE : DEV_NAN);
    for (int t = 0; t < 9; ++t) Mi[9 * (size_t)i + t] = (t % 4 == 0) ? T(1) : T(0);
    return;
  }
  const double inv[9] = {c00 / det, (A[2] * A[7] - A[1] * A[8]) / det, (A[1] * A[5] - A[2] * A[4]) / det,
                         c01 / det, (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                         c02 / det, (A[1] * A[6] - A[0] * A[7]) / det, (A[0] * A[4] - A[1] * A[3]) / det};
  for (int t = 0; t < 9; ++t) Mi[9 * (size_t)i + t] = (T)inv[t];
}

__device__ int find_block(const int* row_ptr, const int* col, int r, int c) {
  for (int q = row_ptr[r]; q < row_ptr[r + 1]; ++q)
    if (col[q] == c) return q;
  return -1;
}

// 12x12 block per affine body (its four nodes), gathered from both parts
template <typename T>
__global__ void k_bj_body(int nb, int nfree, const T* __restrict__ D, const int* __restrict__ bslot,
                          const T* __restrict__ vs, const int* __restrict__ drp, const int* __restrict__ dcol,
                          const T* __restrict__ vd, T* __restrict__ Mi, int* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int b0 = nfree + 4 * b;
  double A[144], I[144];
  for (int t = 0; t < 144; ++t) { A[t] = 0.0; I[t] = (t % 13 == 0) ? 1.0 : 0.0; }
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {1, 2, 3, 2, 3, 3};
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[(3 * a + i) * 12 + 3 * a + j] = (double)D[9 * (size_t)(b0 + a) + 3 * i + j];
  for (int q = 0; q < 6; ++q) {
    const int a = pa[q], c = pb[q];
    double B[9];
    for (int t = 0; t < 9; ++t) B[t] = (double)vs[9 * (size_t)bslot[6 * b + q] + t];
    if (drp) {
      const int k = find_block(drp, dcol, b0 + a, b0 + c);
      if (k >= 0)
        for (int t = 0; t < 9; ++t) B[t] += (double)vd[9 * (size_t)k + t];
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        A[(3 * a + i) * 12 + 3 * c + j] = B[3 * i + j];
        A[(3 * c + j) * 12 + 3 * a + i] = B[3 * i + j];
      }
  }
  // Gauss-Jordan with partial pivoting
  for (int c = 0; c < 12; ++c) {
    int piv = c;
    for (int r = c + 1; r < 12; ++r)
      if (fabs(A[r * 12 + c]) > fabs(A[piv * 12 + c])) piv = r;
    if (piv != c)
      for (int j = 0; j < 12; ++j) {
        double t = A[c * 12 + j]; A[c * 12 + j] = A[piv * 12 + j]; A[piv * 12 + j] = t;
        t = I[c * 12 + j]; I[c * 12 + j] = I[piv * 12 + j]; I[piv * 12 + j] = t;
      }
    const double d = A[c * 12 + c];
    if (!(fabs(d) > 0.0)) { dev_flag(status, isfinite(d) ? DEV_INDEFINITE : DEV_NAN); return; }
    for (int j = 0; j < 12; ++j) { A[c * 12 + j] /= d; I[c * 12 + j] /= d; }
    for (int r = 0; r < 12; ++r)
      if (r != c) {
        const double f = A[r * 12 + c];
        if (f != 0.0)
          for (int j = 0; j < 12; ++j) { A[r * 12 + j] -= f * A[c * 12 + j]; I[r * 12 + j] -= f * I[c * 12 + j]; }
      }
  }
  T* M = Mi + 9 * (size_t)nfree + 144 * (size_t)b;
  for (int t = 0; t < 144; ++t) M[t] = (T)I[t];
}

// ---------------------------------------------------------------- reductions
__device__ double block_sum(double v) {
  __shared__ double sh[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}
// block-wide sum in the vector precision (FP64 ALU is scarce on this part:
// keep per-block reductions of FP32 PCG vectors in FP32)
template <typename V>
__device__ V block_sum_v(V v) {
  __shared__ V shv[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) shv[threadIdx.x >> 5] = v;
  __syncthreads();
  V r = 0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? shv[threadIdx.x] : V(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// z = M^-1 r on free nodes (3x3) and bodies (12x12); v_i = z_i, returns r_i . z_i partial
template <typename T, typename V>
__device__ __forceinline__ V precond_row(int i, int nfree, const T* __restrict__ Mi, const V* __restrict__ r,
                                         V* __restrict__ z) {
  if (i < nfree) {
    const T* M = Mi + 9 * (size_t)i;
    const V r0 = r[3 * i], r1 = r[3 * i + 1], r2 = r[3 * i + 2];
    V acc = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const V za = (V)M[3 * a] * r0 + (V)M[3 * a + 1] * r1 + (V)M[3 * a + 2] * r2;
      z[3 * i + a] = za;
      acc += za * r[3 * i + a];
    }
    return acc;
  }
  const int b = i - nfree;
  const T* M = Mi + 9 * (size_t)nfree + 144 * (size_t)b;
  const size_t o = 3 * ((size_t)nfree + 4 * (size_t)b);
  V acc = 0;
  for (int a = 0; a < 12; ++a) {
    V s = 0;
    for (int c = 0; c < 12; ++c) s += (V)M[12 * a + c] * r[o + c];
    z[o + a] = s;
    acc += s * r[o + a];
  }
  return acc;
}

// ---------------------------------------------------------------- persistent PCG
//
// One cooperative launch (one block per SM) runs all iterations of a solve.
// An iteration has two grid-wide phases, each closed by a reducing barrier:
//   B  d' = z + beta d for the block's own nodes, q += D d', and the upper
//      blocks' q += U d' + U^T d' (d' of other nodes is formed on the fly from
//      z and d, which nobody writes during the phase); partial d'^T H d'
//   C  x += alpha d', r -= alpha q, z = M^-1 r, q = 0; partial r^T z
// d and d' swap roles every iteration.
template <typename T, typename V>
struct pcg_args {
  int nn, nfree, nb, n_s, n_d, maxit;
  double tol2;
  const int *row_s, *col_s, *row_d, *col_d;
  const T *val_s, *val_d, *D, *Mi;
  // D (all nodes) and M^-1 (free nodes) packed symmetric, 6 per node:
  // (00, 01, 02, 11, 12, 22), the mean of the two mirrored entries
  const T *Ds, *Ms;
  const double* rhs;
  V *x, *r, *z, *q;  // written and read across blocks: plain (coherent) loads only
  V *d0, *d1;        // the direction, ping-ponged between iterations
  pcg_dev* sc;
  pcg_bar* bar;
  int* status;
  long long spin_limit;
  double rscale;   // r0 = rscale * rhs (the FP32 inner solves work on a normalised residual)
  unsigned long long* bt;  // per-block busy time of the H d' phase (own nodes + upper blocks), or null
  unsigned unmet;  // extra arrivals every grid barrier waits for (0; 1 makes the waits run out, for tests)
  // batches (nscene > 1): per-scene alpha, beta and stopping test
  int nscene;
  const int* node_scene;  // [nn]
  double* ring;           // [8][nscene]: per-scene sums of reducing barrier k in row k % 8
  double* srz0;           // [nscene] r0^T z0 per scene
  const double* stol2;    // [nscene] squared relative tolerance per scene, or null (tol2)
  int* siters;            // [nscene] iterations each scene ran
  int* sflag;             // [nscene] 2 = breakdown (d^T H d <= 0) in that scene
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Reducing grid barrier k for a cooperative launch (all blocks co-resident).
// Thread 0 of each block adds the block's partial into sum[k % 4], then adds 1
// to the arrival count with release semantics (publishing everything the block
// wrote) and polls the count with acquire loads until all blocks arrived; it
// then reads the total and hands it to the block.  Slot (k - 1) % 4 is dead
// once barrier k completes (every block read it before arriving), so block 0
// clears it for barrier k + 3.  The wait is bounded: after spin_limit polls
// the block raises the abort flag, and every waiting block also leaves when it
// sees the flag, so no block waits forever.  Returns false when the grid has
// aborted.  Float addition order in the slot follows arrival order, so totals
// can differ in the last bits from run to run (never between blocks).
struct no_epilogue {
  __device__ void operator()(double) const {}
};
// The block's partial (thread 0's value) joins the grid-wide sum; every block
// gets the total.  epi(total) runs on thread 0 alone before the block is
// released: scalar work on the total (divisions, tests) belongs there, since
// FP64 arithmetic repeated by every thread of the grid is slow on this part.
template <typename P, typename F = no_epilogue>
__device__ __forceinline__ bool grid_reduce(pcg_bar* bar, unsigned& k, P partial, double& total,
                                            long long spin_limit, unsigned unmet, F epi = F{}) {
  __shared__ int ok;
  __shared__ double tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    atomicAdd(&bar->sum[k & 3], (double)partial);
    red_add_release(&bar->count, 1u);
    const unsigned target = (k + 1) * gridDim.x + unmet;  // unmet > 0: a count no grid reaches (tests)
    long long spins = 0;
    while (ld_acquire(&bar->count) < target) {
      if ((++spins & 255) == 0) {
        if (*(volatile int*)&bar->abort) { good = 0; break; }
        if (spins > spin_limit) { atomicExch(&bar->abort, 1); good = 0; break; }
      }
    }
    tot = *(volatile double*)&bar->sum[k & 3];
    if (blockIdx.x == 0 && k > 0) bar->sum[(k - 1) & 3] = 0.0;
    ok = good && !*(volatile int*)&bar->abort;
    if (ok) epi(tot);
  }
  __syncthreads();
  k += 1;
  total = tot;
  return ok != 0;
}

// ---- shared-memory staging of the upper blocks (bulk async copies)
//
// Each block owns an even, 4-aligned share of the first 90% of the upper
// blocks (static, then dynamic; share_cut) and then claims tiles of the rest
// from a shared pool; tiles hold BPT blocks per thread.  A
// tile's values, rows and columns are contiguous, so thread 0 moves them into
// shared memory with three cp.async.bulk copies completing on an mbarrier,
// double-buffered: the next tile travels while the current one is multiplied,
// and the first two travel while the block does its own nodes' diagonal part.
// Only the gathers of z and d stay exposed.
template <typename T, typename CFG>
struct stage_layout {
  static constexpr int NT = CFG::BPT * CFG::NTHR;      // blocks per tile (BPT per thread)
  static constexpr unsigned VB = NT * 9 * sizeof(T);   // values
  static constexpr unsigned IB = NT * sizeof(int);     // rows / columns
  static constexpr unsigned BUF = VB + 2 * IB;         // one buffer (a multiple of 16)
  static constexpr unsigned SMEM = 2 * BUF + 16;       // two buffers + two mbarriers
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(m))
               : "memory");
}
constexpr long long kDrainPolls = 1LL << 24;  // polls allowed for copies in flight at exit
// bounded wait on one buffer's mbarrier; false after spin_limit polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, unsigned parity, long long spin_limit) {
  for (long long k = 0; k < spin_limit; ++k)
    if (mbar_try_wait(m, parity)) return true;
  return false;
}

// this block's share of the upper blocks: static [s0, s1), dynamic [e0, e1)
struct spmv_share {
  int s0, s1, e0, e1, ts, tt;  // own tiles: ts in the static part, tt in all
  int ps, pd, pts, ptt;        // shared pool: dynamic [pd, n_d) in pts tiles, then static [ps, n_s); ptt in all
};
// Block b's upper blocks: an equal share of the static blocks followed by the
// dynamic ones (one sequence of n_s + n_d), cut at multiples of 4 within each
// array so that every tile starts 16-byte aligned.  Only the block whose share
// straddles the end of the static part gets tiles of both arrays.
__device__ __forceinline__ void share_cut(long long n_s, long long n_d, long long b, long long G, long long& cs,
                                          long long& cd) {
  if (b >= G) { cs = n_s; cd = n_d; return; }
  const long long v = b * (n_s + n_d) / G;
  cs = (v < n_s ? v : n_s) & ~3LL;
  cd = (v > n_s ? v - n_s : 0) & ~3LL;
}
// The blocks of a grid do not finish equal shares at the same time (blocks
// sharing an SM are not scheduled evenly, and contact blocks gather from
// farther away), so the last kPoolPct percent of the upper blocks form a pool
// of tiles that the blocks claim from a counter once their own share is done.
// Pool tiles are full tiles (smaller ones leave lanes idle while costing a
// tile's latency), the dynamic ones first (they take longest).
constexpr int kPoolPct = 10;
template <typename T, typename V>
__device__ __forceinline__ spmv_share share_of(const pcg_args<T, V>& a, int NT) {
  const long long G = gridDim.x, b = blockIdx.x;
  const long long n_s = a.n_s, n_d = a.n_d, N = n_s + n_d;
  const long long vp = N - N * kPoolPct / 100;  // the pool starts at this index of the sequence
  spmv_share o;
  const long long ps = vp < n_s ? (vp & ~3LL) : n_s;
  const long long pd = vp < n_s ? 0 : ((vp - n_s) & ~3LL);
  long long s0, d0, s1, d1;
  share_cut(ps, pd, b, G, s0, d0);
  share_cut(ps, pd, b + 1, G, s1, d1);
  o.s0 = (int)s0; o.s1 = (int)s1;
  o.e0 = (int)d0; o.e1 = (int)d1;
  o.ts = (o.s1 - o.s0 + NT - 1) / NT;
  o.tt = o.ts + (o.e1 - o.e0 + NT - 1) / NT;
  o.ps = (int)ps; o.pd = (int)pd;
  o.pts = (int)((n_d - pd + NT - 1) / NT);  // dynamic pool tiles (claimed first)
  o.ptt = o.pts + (int)((n_s - ps + NT - 1) / NT);
  return o;
}
template <typename T, typename V>
struct tile_src {
  const T* vals;
  const int *row, *col;
  int base, cnt;
};
// tile t of the shared pool (t < sh.ptt): dynamic tiles, then static ones
template <typename T, typename V>
__device__ __forceinline__ tile_src<T, V> pool_tile(const pcg_args<T, V>& a, const spmv_share& sh, int t, int NT) {
  tile_src<T, V> o;
  if (t < sh.pts) {
    o.vals = a.val_d; o.row = a.row_d; o.col = a.col_d;
    o.base = sh.pd + t * NT;
    o.cnt = min(NT, a.n_d - o.base);
  } else {
    o.vals = a.val_s; o.row = a.row_s; o.col = a.col_s;
    o.base = sh.ps + (t - sh.pts) * NT;
    o.cnt = min(NT, a.n_s - o.base);
  }
  return o;
}
template <typename T, typename V>
__device__ __forceinline__ tile_src<T, V> tile_of(const pcg_args<T, V>& a, const spmv_share& sh, int j, int NT) {
  tile_src<T, V> o;
  if (j < sh.ts) {
    o.vals = a.val_s; o.row = a.row_s; o.col = a.col_s;
    o.base = sh.s0 + j * NT;
    o.cnt = min(NT, sh.s1 - o.base);
  } else {
    o.vals = a.val_d; o.row = a.row_d; o.col = a.col_d;
    o.base = sh.e0 + (j - sh.ts) * NT;
    o.cnt = min(NT, sh.e1 - o.base);
  }
  return o;
}
// thread 0: request tile j into buffer buf.  Tile starts are multiples of 4
// blocks, so every source address is 16-byte aligned; sizes are rounded up to
// 16 bytes (the arrays carry that much slack).
template <typename L, typename T, typename V>
__device__ __forceinline__ void issue_tile(const tile_src<T, V>& src, unsigned char* buf, uint64_t* m) {
  const unsigned bv = (unsigned)(src.cnt * 9 * (int)sizeof(T) + 15) & ~15u;
  const unsigned bi = (unsigned)(src.cnt * (int)sizeof(int) + 15) & ~15u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(m, bv + 2 * bi);
  bulk_g2s(buf, src.vals + 9 * (size_t)src.base, bv, m);
  bulk_g2s(buf + L::VB, src.row + src.base, bi, m);
  bulk_g2s(buf + L::VB + L::IB, src.col + src.base, bi, m);
}

// the new direction z + beta d, one rounding per component (the same
// expression wherever it is formed, so every thread sees the same d')
YASPS_D float dnew(float z, float beta, float d) { return __fmaf_rn(beta, d, z); }
YASPS_D double dnew(double z, double beta, double d) { return __fma_rn(beta, d, z); }

// the two d' segments one block needs
template <typename V>
struct gath {
  V c0, c1, c2, r0, r1, r2;
};
template <typename V>
__device__ __forceinline__ void gather_d(int r, int c, const V* z, const V* d, V beta, gath<V>& g) {
  if (r >= 0) {
    const V zc0 = z[3 * c], zc1 = z[3 * c + 1], zc2 = z[3 * c + 2];
    const V zr0 = z[3 * r], zr1 = z[3 * r + 1], zr2 = z[3 * r + 2];
    const V dc0 = d[3 * c], dc1 = d[3 * c + 1], dc2 = d[3 * c + 2];
    const V dr0 = d[3 * r], dr1 = d[3 * r + 1], dr2 = d[3 * r + 2];
    g.c0 = dnew(zc0, beta, dc0); g.c1 = dnew(zc1, beta, dc1); g.c2 = dnew(zc2, beta, dc2);
    g.r0 = dnew(zr0, beta, dr0); g.r1 = dnew(zr1, beta, dr1); g.r2 = dnew(zr2, beta, dr2);
  }
}
// the two d' segments read directly (d' of every node written before the tiles)
template <typename V>
__device__ __forceinline__ void gather_dn(int r, int c, const V* dn, gath<V>& g) {
  if (r >= 0) {
    g.c0 = dn[3 * c]; g.c1 = dn[3 * c + 1]; g.c2 = dn[3 * c + 2];
    g.r0 = dn[3 * r]; g.r1 = dn[3 * r + 1]; g.r2 = dn[3 * r + 2];
  }
}
// Layout of the product q = H d inside the PCG kernel: FP32 uses 16 bytes
// per node, so a node's three contributions go in one vector atomic
// (red.global.add.v4.f32); FP64 keeps 3 scalars per node.
template <typename V>
struct qlay { static constexpr int S = 3; };
template <>
struct qlay<float> { static constexpr int S = 4; };
// index in q of entry o3 of a 3-per-node vector
template <typename V>
__device__ __forceinline__ size_t q_idx(size_t o3) {
  return (o3 / 3) * qlay<V>::S + o3 % 3;
}
__device__ __forceinline__ void q_add3(float* q, int node, float a, float b, float c) {
  atomicAdd(reinterpret_cast<float4*>(q) + node, make_float4(a, b, c, 0.0f));
}
__device__ __forceinline__ void q_add3(double* q, int node, double a, double b, double c) {
  atomicAdd(&q[3 * (size_t)node], a);
  atomicAdd(&q[3 * (size_t)node + 1], b);
  atomicAdd(&q[3 * (size_t)node + 2], c);
}
__device__ __forceinline__ void q_take3(float* q, long long node, float* out) {  // read and clear
  float4* p = reinterpret_cast<float4*>(q) + node;
  const float4 v = *p;
  out[0] = v.x; out[1] = v.y; out[2] = v.z;
  *p = make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void q_take3(double* q, long long node, double* out) {
  for (int c = 0; c < 3; ++c) {
    out[c] = q[3 * node + c];
    q[3 * node + c] = 0.0;
  }
}

// q += B d'_c into the row, q += B^T d'_r into the column; returns the
// block's share 2 d'_r^T B d'_c of d'^T U d'.  FP32 reduces the rows over the
// warp (segmented shuffle, one vector atomic per row segment); FP64 adds
// every block's row part with atomics, which execute in L2: the segmented
// reduction's FP64 additions (15 per block) would run on the SM's FP64 pipe,
// which bounds FP64 SpMV on this part.
template <typename T, typename V>
__device__ __forceinline__ V apply_blk(int r, int c, const T* b, const gath<V>& g, V* q, int lane) {
  V a0 = 0, a1 = 0, a2 = 0, part = 0;
  if (r >= 0) {
    const V xc0 = g.c0, xc1 = g.c1, xc2 = g.c2;
    const V xr0 = g.r0, xr1 = g.r1, xr2 = g.r2;
    a0 = (V)b[0] * xc0 + (V)b[1] * xc1 + (V)b[2] * xc2;
    a1 = (V)b[3] * xc0 + (V)b[4] * xc1 + (V)b[5] * xc2;
    a2 = (V)b[6] * xc0 + (V)b[7] * xc1 + (V)b[8] * xc2;
    part = (V)2 * (xr0 * a0 + xr1 * a1 + xr2 * a2);
    q_add3(q, c, (V)b[0] * xr0 + (V)b[3] * xr1 + (V)b[6] * xr2, (V)b[1] * xr0 + (V)b[4] * xr1 + (V)b[7] * xr2,
           (V)b[2] * xr0 + (V)b[5] * xr1 + (V)b[8] * xr2);
    if constexpr (sizeof(V) == 8) q_add3(q, r, a0, a1, a2);
  }
  if constexpr (sizeof(V) == 4) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int ro = __shfl_down_sync(0xffffffffu, r, off);
      const V b0 = shfl_down_v(a0, off), b1 = shfl_down_v(a1, off), b2 = shfl_down_v(a2, off);
      if (lane + off < 32 && ro == r) { a0 += b0; a1 += b1; a2 += b2; }
    }
    const int rp = __shfl_up_sync(0xffffffffu, r, 1);
    if (r >= 0 && (lane == 0 || rp != r)) q_add3(q, r, a0, a1, a2);
  }
  return part;
}

// y = S x for a symmetric 3x3 S packed as (00, 01, 02, 11, 12, 22)
template <typename T, typename V>
__device__ __forceinline__ void sym3_apply(const T* S, V x0, V x1, V x2, V& y0, V& y1, V& y2) {
  T m[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) m[t] = __ldg(S + t);
  y0 = (V)m[0] * x0 + (V)m[1] * x1 + (V)m[2] * x2;
  y1 = (V)m[1] * x0 + (V)m[3] * x1 + (V)m[4] * x2;
  y2 = (V)m[2] * x0 + (V)m[4] * x1 + (V)m[5] * x2;
}

// unit i: a free node (3 DOF) or an affine body (its 4 nodes, 12 DOF)
__device__ __forceinline__ void unit_range(int i, int nfree, int& cnt, size_t& o) {
  cnt = (i < nfree) ? 3 : 12;
  o = (i < nfree) ? 3 * (size_t)i : 3 * ((size_t)nfree + 4 * (size_t)(i - nfree));
}

// own node i in phase B: d'_i = z_i + beta d_i, q_i += D_i d'_i; d'_i^T D_i d'_i.
// DEFER: the previous iteration's x_i += alpha d_i happens here, where d_i is
// read anyway (the owning thread is the one that wrote d_i), instead of in
// phase C; the last one is applied after the loop.
template <typename T, typename V, bool DEFER>
__device__ __forceinline__ V diag_node(const pcg_args<T, V>& a, long long i, V beta, V alpha_prev, const V* d,
                                       V* dn) {
  const T* B = a.Ds + 6 * (size_t)i;
  T m[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) m[t] = __ldg(B + t);
  const V z0 = a.z[3 * i], z1 = a.z[3 * i + 1], z2 = a.z[3 * i + 2];
  const V e0 = d[3 * i], e1 = d[3 * i + 1], e2 = d[3 * i + 2];
  if constexpr (DEFER) {
    if (alpha_prev != V(0)) {
      V* x = a.x + 3 * i;
      const V x0 = x[0], x1 = x[1], x2 = x[2];
      x[0] = x0 + alpha_prev * e0;
      x[1] = x1 + alpha_prev * e1;
      x[2] = x2 + alpha_prev * e2;
    }
  }
  const V d0 = dnew(z0, beta, e0), d1 = dnew(z1, beta, e1), d2 = dnew(z2, beta, e2);
  const V q0 = (V)m[0] * d0 + (V)m[1] * d1 + (V)m[2] * d2;
  const V q1 = (V)m[1] * d0 + (V)m[3] * d1 + (V)m[4] * d2;
  const V q2 = (V)m[2] * d0 + (V)m[4] * d1 + (V)m[5] * d2;
  dn[3 * i] = d0; dn[3 * i + 1] = d1; dn[3 * i + 2] = d2;
  q_add3(a.q, (int)i, q0, q1, q2);
  return d0 * q0 + d1 * q1 + d2 * q2;
}
// phase C for one free node: x += alpha d' (unless DEFER), r -= alpha q,
// z = M^-1 r, q = 0; r^T z
template <typename T, typename V, bool DEFER>
__device__ __forceinline__ V update_free(const pcg_args<T, V>& a, long long i, V alpha, const V* dn) {
  const T* M = a.Ms + 6 * (size_t)i;
  T m[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) m[t] = __ldg(M + t);
  V xv[3], dv[3], rv[3], qv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (!DEFER) {
      xv[c] = a.x[3 * i + c];
      dv[c] = dn[3 * i + c];
    }
    rv[c] = a.r[3 * i + c];
  }
  q_take3(a.q, i, qv);
  V zv[3], acc = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (!DEFER) xv[c] += alpha * dv[c];
    rv[c] -= alpha * qv[c];
  }
  zv[0] = (V)m[0] * rv[0] + (V)m[1] * rv[1] + (V)m[2] * rv[2];
  zv[1] = (V)m[1] * rv[0] + (V)m[3] * rv[1] + (V)m[4] * rv[2];
  zv[2] = (V)m[2] * rv[0] + (V)m[4] * rv[1] + (V)m[5] * rv[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) acc += zv[c] * rv[c];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (!DEFER) a.x[3 * i + c] = xv[c];
    a.r[3 * i + c] = rv[c];
    a.z[3 * i + c] = zv[c];
  }
  return acc;
}

// z = M^-1 r for unit i inside the PCG kernel: free nodes from the packed
// symmetric M^-1, bodies from their 12x12 block
template <typename T, typename V>
__device__ __forceinline__ V precond_unit(const pcg_args<T, V>& a, int i) {
  if (i >= a.nfree) return precond_row<T, V>(i, a.nfree, a.Mi, a.r, a.z);
  V z0, z1, z2;
  const V r0 = a.r[3 * (size_t)i], r1 = a.r[3 * (size_t)i + 1], r2 = a.r[3 * (size_t)i + 2];
  sym3_apply<T, V>(a.Ms + 6 * (size_t)i, r0, r1, r2, z0, z1, z2);
  a.z[3 * (size_t)i] = z0;
  a.z[3 * (size_t)i + 1] = z1;
  a.z[3 * (size_t)i + 2] = z2;
  return z0 * r0 + z1 * r1 + z2 * r2;
}

// ---- batches: per-scene sums
// Warp-segmented sum over runs of equal keys (runs must be contiguous across
// the lanes, as sorted keys are); the head lane of each run adds the run's sum
// into shs[key].  key < 0 contributes nothing.  All 32 lanes must call.
template <typename V>
__device__ __forceinline__ void seg_add_shared(double* shs, int key, V v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int ko = __shfl_down_sync(0xffffffffu, key, off);
    const V vo = shfl_down_v(v, off);
    if (lane + off < 32 && ko == key) v += vo;
  }
  const int kp = __shfl_up_sync(0xffffffffu, key, 1);
  if (key >= 0 && (lane == 0 || kp != key)) atomicAdd(&shs[key], (double)v);
}
// Per-warp running sum for the scene the warp is on (held by lane 0): a warp
// whose 32 items belong to one scene adds into it without touching shared
// memory; the sum goes to shs when the warp moves to another scene or at
// wacc_flush.  Mixed warps fall back to seg_add_shared.  All lanes call.
struct wacc {
  int key = -1;
  double v = 0.0;
};
template <typename V>
__device__ __forceinline__ void wacc_add(wacc& w, double* shs, int key, V val, int lane) {
  const int k0 = __shfl_sync(0xffffffffu, key, 0);
  if (__all_sync(0xffffffffu, key == k0)) {
    if (k0 < 0) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += shfl_down_v(val, o);
    if (lane == 0) {
      if (k0 != w.key) {
        if (w.key >= 0) atomicAdd(&shs[w.key], w.v);
        w.key = k0;
        w.v = 0.0;
      }
      w.v += (double)val;
    }
  } else {
    seg_add_shared(shs, key, val, lane);
  }
}
__device__ __forceinline__ void wacc_flush(wacc& w, double* shs, int lane) {
  if (lane == 0 && w.key >= 0) atomicAdd(&shs[w.key], w.v);
  w.key = -1;
  w.v = 0.0;
}

// the block's per-scene partials into row `row` of the ring; shs is cleared
__device__ __forceinline__ void flush_scene_sums(double* shs, double* ring, int row, int nscene) {
  __syncthreads();
  for (int t = threadIdx.x; t < nscene; t += blockDim.x) {
    const double v = shs[t];
    if (v != 0.0) {
      atomicAdd(&ring[(size_t)row * nscene + t], v);
      shs[t] = 0.0;
    }
  }
}
// per-scene scalars after the barriers of an iteration
template <typename T, typename V>
struct scene_view {
  const pcg_args<T, V>* a;
  int cp, cpp, kb;  // ring rows: last r^T z, the one before, this iteration's d^T H d
  __device__ double rz(int sc) const { return __ldcg(a->ring + (size_t)cp * a->nscene + sc); }
  __device__ double rz_old(int sc) const { return __ldcg(a->ring + (size_t)cpp * a->nscene + sc); }
  __device__ double tol2(int sc, double t) const { return a->stol2 ? a->stol2[sc] : t; }
  __device__ bool finished(int sc, double t) const {
    return __ldcg(a->sflag + sc) != 0 || !(rz(sc) > tol2(sc, t) * __ldcg(a->srz0 + sc));
  }
};

template <typename T, typename V, bool BATCH, typename CFG>
__global__ void __launch_bounds__(CFG::NTHR, CFG::MINB) k_pcg_persistent(pcg_args<T, V> a) {
  using L = stage_layout<T, CFG>;
  constexpr int BPT = CFG::BPT;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * L::BUF);
  double* shs = reinterpret_cast<double*>(smem + 2 * L::BUF + 16);  // batches: per-scene partials
  V* tab = reinterpret_cast<V*>(shs + kMaxScenes);                   // batches: per-scene beta, then alpha
  const int G = gridDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthr = (long long)G * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int nu = a.nfree + a.nb;
  const spmv_share sh = share_of(a, L::NT);
  const long long n0 = (long long)blockIdx.x * a.nn / G, n1 = (long long)(blockIdx.x + 1) * a.nn / G;
  unsigned kbar = 0;  // reducing barriers passed in this launch
  const bool clock0 = blockIdx.x == 0 && threadIdx.x == 0;
  // block 0's clock per iteration: 0 own nodes (d', D d'), 1 upper blocks,
  // 2 wait + d^T H d, 3 update, 4 wait + r^T z
  __shared__ unsigned long long tph[6];
  // d' of every node first, behind one more grid barrier, then the tiles
  // gather d' itself: in FP64 the on-the-fly z + beta d of every gathered
  // node (six FMAs per upper block) costs the FP64 pipe, which bounds FP64
  // SpMV on this part, more than the barrier does.  FP32 forms d' on the fly.
  constexpr bool DPRE = !BATCH && sizeof(V) == 8;
  __shared__ int sh_active;
  __shared__ int s_tcnt[2];  // blocks in the tile requested into each buffer (0: none)
  unsigned long long tlast = 0, tbusy = 0, tbusy0 = 0;
  if (threadIdx.x < 6) tph[threadIdx.x] = 0;
  if constexpr (BATCH)
    for (int t = threadIdx.x; t < a.nscene; t += blockDim.x) shs[t] = 0.0;
  unsigned parity = 0u;    // bit b: phase parity of buffer b's next completion
  unsigned inflight = 0u;  // bit b: buffer b has a request not yet waited for (thread 0's view)
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // batches: per-scene sums live in ring rows; block 0 clears the row of
  // barrier k - 3 once barrier k has completed (nobody reads it any more)
  auto after_barrier = [&](unsigned kdone) {
    if constexpr (BATCH) {
      if (blockIdx.x == 0 && kdone >= 3) {
        double* row = a.ring + (size_t)((kdone - 3) & 7) * a.nscene;
        for (int t = threadIdx.x; t < a.nscene; t += blockDim.x) row[t] = 0.0;
      }
    }
  };
  // batches: number of scenes still iterating (the same value in every block)
  auto count_active = [&](const scene_view<T, V>& sv) -> int {
    int c = 0;
    for (int t = threadIdx.x; t < a.nscene; t += blockDim.x) c += sv.finished(t, a.tol2) ? 0 : 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (threadIdx.x == 0) sh_active = 0;
    __syncthreads();
    if (lane == 0) atomicAdd(&sh_active, c);
    __syncthreads();
    return sh_active;
  };

  // r = rhs, x = 0, d = 0, q = 0, z = M^-1 r ; r^T z
  V acc = 0;
  if constexpr (!BATCH) {
    for (long long i = tid; i < nu; i += nthr) {
      int cnt;
      size_t o;
      unit_range((int)i, a.nfree, cnt, o);
      for (int c = 0; c < cnt; ++c) {
        a.r[o + c] = (V)(a.rhs[o + c] * a.rscale);
        a.x[o + c] = 0;
        a.d0[o + c] = 0;
        a.q[q_idx<V>(o + c)] = 0;
      }
      acc += precond_unit(a, (int)i);
    }
  } else {
    for (long long base = tid & ~31LL; base < nu; base += nthr) {
      const long long i = base + lane;
      int key = -1;
      V v = 0;
      if (i < nu) {
        int cnt;
        size_t o;
        unit_range((int)i, a.nfree, cnt, o);
        for (int c = 0; c < cnt; ++c) {
          a.r[o + c] = (V)(a.rhs[o + c] * a.rscale);
          a.x[o + c] = 0;
          a.d0[o + c] = 0;
          a.q[q_idx<V>(o + c)] = 0;
        }
        v = precond_unit(a, (int)i);
        key = a.node_scene[i < a.nfree ? i : a.nfree + 4 * (i - a.nfree)];
      }
      seg_add_shared(shs, key, v, lane);
    }
    flush_scene_sums(shs, a.ring, 0, a.nscene);
  }
  V bs = block_sum_v<V>(acc);
  int done = 0, it = 0;
  double rz = 0.0;
  // single system: alpha, beta and the stopping test are thread 0's work,
  // handed to the block through shared memory
  __shared__ V s_alpha, s_beta;
  __shared__ int s_done;
  if (threadIdx.x == 0) s_done = 0;
  if (!grid_reduce(a.bar, kbar, bs, rz, a.spin_limit, a.unmet, [&](double t) {
        if (!BATCH && !(t > 0.0)) s_done = 1;
      }))
    done = 3;
  const double rz0 = rz;
  V vb_next = 0;  // single system: beta of the next iteration
  int cp = 0, cpp = 0;  // batches: ring rows of the last and the previous r^T z
  if constexpr (BATCH) {
    if (!done) {
      if (blockIdx.x == 0)
        for (int t = threadIdx.x; t < a.nscene; t += blockDim.x) a.srz0[t] = __ldcg(a.ring + t);
      // the first stopping test uses the sums themselves (srz0 is visible only
      // after the next barrier): a scene with r0^T z0 = 0 is finished
      int c = 0;
      for (int t = threadIdx.x; t < a.nscene; t += blockDim.x) c += (__ldcg(a.ring + t) > 0.0) ? 1 : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if (threadIdx.x == 0) sh_active = 0;
      __syncthreads();
      if (lane == 0) atomicAdd(&sh_active, c);
      __syncthreads();
      if (sh_active == 0) done = 1;
    }
  } else {
    if (!done) done = s_done;
  }

  V apend = 0;            // single system: x += apend * dpend still to do on own nodes
  const V* dpend = a.d0;
  while (!done && it < a.maxit) {
    V* d = (it & 1) ? a.d1 : a.d0;   // previous direction
    V* dn = (it & 1) ? a.d0 : a.d1;  // this iteration's direction
    const V vb = vb_next;
    const scene_view<T, V> sv{&a, cp, cpp, (int)(kbar & 7)};
    // batches: beta of scene sc (0 in the first iteration and once finished)
    auto beta_of = [&](int sc) -> V {
      if (it == 0 || sc < 0) return V(0);
      if (sv.finished(sc, a.tol2)) return V(0);
      return (V)(sv.rz(sc) / sv.rz_old(sc));
    };
    if (clock0) tlast = global_ns();
    if (a.bt && threadIdx.x == 0) tbusy0 = global_ns();
    // the first two tiles travel while the block does its own nodes
    unsigned* pool_ctr = &a.bar->pool[it & 1];
    int nissued = 0, pend = -1;
    bool pool_out = false;
    // thread 0: request the block's next tile into buffer b (its own tiles
    // first, then claims from the pool; the claim for the next pool tile is
    // made one request ahead, so its round trip overlaps a tile's work)
    auto issue_next = [&](int b) {
      tile_src<T, V> src;
      bool have = false;
      if (nissued < sh.tt) {
        src = tile_of(a, sh, nissued, L::NT);
        have = true;
      } else if (!pool_out) {
        const int t = pend >= 0 ? pend : (int)atomicAdd(pool_ctr, 1u);
        pend = -1;
        if (t < sh.ptt) {
          src = pool_tile(a, sh, t, L::NT);
          have = true;
          pend = (int)atomicAdd(pool_ctr, 1u);
        } else {
          pool_out = true;
        }
      }
      ++nissued;
      if (have) {
        issue_tile<L>(src, smem + b * L::BUF, &mbar[b]);
        inflight |= 1u << b;
        s_tcnt[b] = src.cnt;
      } else {
        s_tcnt[b] = 0;
      }
    };
    if (threadIdx.x == 0) {
      issue_next(0);
      issue_next(1);
    }
    acc = 0;
    wacc wa;
    if constexpr (!BATCH) {
      for (long long i = n0 + threadIdx.x; i < n1; i += blockDim.x)
        acc += diag_node<T, V, true>(a, i, vb, apend, d, dn);
      apend = 0;
    } else {
      for (int t = threadIdx.x; t < a.nscene; t += blockDim.x) tab[t] = beta_of(t);
      __syncthreads();
      for (long long base = n0 + (threadIdx.x & ~31); base < n1; base += blockDim.x) {
        const long long i = base + lane;
        int key = -1;
        V v = 0;
        if (i < n1) {
          key = a.node_scene[i];
          v = diag_node<T, V, false>(a, i, tab[key], V(0), d, dn);
        }
        wacc_add(wa, shs, key, v, lane);
      }
    }
    if (clock0) { const unsigned long long t = global_ns(); tph[0] += t - tlast; tlast = t; }
    if constexpr (DPRE) {
      if (a.bt && threadIdx.x == 0) tbusy += global_ns() - tbusy0;
      double unused = 0.0;
      if (!grid_reduce(a.bar, kbar, V(0), unused, a.spin_limit, a.unmet)) {
        done = 3;
        break;
      }
      if (clock0) { const unsigned long long t = global_ns(); tph[5] += t - tlast; tlast = t; }
      if (a.bt && threadIdx.x == 0) tbusy0 = global_ns();
    }
    // upper blocks, tile by tile from shared memory, until a buffer gets none
    bool ok = true;
    __syncthreads();  // s_tcnt of the first two tiles
    for (int j = 0;; ++j) {
      const int b = j & 1;
      const int cnt = s_tcnt[b];
      if (cnt == 0) break;
      // a wait that gives up leaves the buffer's copy marked in flight (and
      // its parity unchanged) so that the drain below still waits for it
      if (mbar_wait_bounded(&mbar[b], (parity >> b) & 1u, a.spin_limit >> 3)) {
        parity ^= 1u << b;
        inflight &= ~(1u << b);
      } else {
        ok = false;
      }
      if (__syncthreads_or(!ok)) { ok = false; break; }
      const unsigned char* buf = smem + b * L::BUF;
      // BPT blocks per thread (k, k + NTHR, ...; each warp on 32 consecutive
      // blocks): all gathers are in flight before any is used
      const int* rows = reinterpret_cast<const int*>(buf + L::VB);
      const int* cols = reinterpret_cast<const int*>(buf + L::VB + L::IB);
      const T* vals = reinterpret_cast<const T*>(buf);
      int rr[BPT], cc[BPT], ss[BPT];
      gath<V> gg[BPT];
#pragma unroll
      for (int u = 0; u < BPT; ++u) {
        const int k = threadIdx.x + u * CFG::NTHR;
        rr[u] = (k < cnt) ? rows[k] : -1;
        cc[u] = (k < cnt) ? cols[k] : 0;
        if constexpr (BATCH) ss[u] = rr[u] >= 0 ? a.node_scene[rr[u]] : -1;
        else ss[u] = 0;
      }
#pragma unroll
      for (int u = 0; u < BPT; ++u) {
        if constexpr (BATCH) gather_d(rr[u], cc[u], a.z, d, ss[u] >= 0 ? tab[ss[u]] : V(0), gg[u]);
        else if constexpr (DPRE) gather_dn(rr[u], cc[u], dn, gg[u]);
        else gather_d(rr[u], cc[u], a.z, d, vb, gg[u]);
      }
#pragma unroll
      for (int u = 0; u < BPT; ++u) {
        const int k = threadIdx.x + u * CFG::NTHR;
        // a block couples two nodes of one scene: the row's scene gives beta
        const V pu = apply_blk<T, V>(rr[u], cc[u], vals + 9 * k, gg[u], a.q, lane);
        if constexpr (BATCH) wacc_add(wa, shs, ss[u], pu, lane);
        else acc += pu;
      }
      __syncthreads();  // every thread is done with buffer b
      if (threadIdx.x == 0) issue_next(b);
    }
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(&a.bar->abort, 1);
      done = 3;
      break;
    }
    if constexpr (BATCH) {
      wacc_flush(wa, shs, lane);
      flush_scene_sums(shs, a.ring, (int)(kbar & 7), a.nscene);
    }
    bs = block_sum_v<V>(acc);
    if (clock0) { const unsigned long long t = global_ns(); tph[1] += t - tlast; tlast = t; }
    if (a.bt && threadIdx.x == 0) tbusy += global_ns() - tbusy0;
    double dHd = 0.0;
    const int kb = (int)(kbar & 7);
    if (!grid_reduce(a.bar, kbar, bs, dHd, a.spin_limit, a.unmet, [&](double t) {
          if constexpr (!BATCH) {
            if (!(t > 0.0)) s_done = 2;
            else s_alpha = (V)(rz / t);
          }
        })) {
      done = 3;
      break;
    }
    after_barrier(kbar - 1);
    // the pool counter of the previous iteration is dead (its claims preceded
    // the last barrier): clear it for the next one
    if (blockIdx.x == 0 && threadIdx.x == 0) a.bar->pool[(it + 1) & 1] = 0u;
    if (clock0) { const unsigned long long t = global_ns(); tph[2] += t - tlast; tlast = t; }
    V alpha = 0;
    if constexpr (!BATCH) {
      if (s_done) { done = s_done; break; }
      alpha = s_alpha;
    }
    // batches: alpha of scene sc (0 once finished; a breakdown finishes it)
    auto alpha_of = [&](int sc) -> V {
      if (sv.finished(sc, a.tol2)) return V(0);
      const double q = __ldcg(a.ring + (size_t)kb * a.nscene + sc);
      if (!(q > 0.0)) {
        if (blockIdx.x == 0) a.sflag[sc] = 2;
        return V(0);
      }
      return (V)(sv.rz(sc) / q);
    };
    // C: x += alpha d', r -= alpha q, z = M^-1 r, q = 0 ; r^T z
    acc = 0;
    if constexpr (!BATCH) {
      for (long long i = tid; i < a.nfree; i += 2 * nthr) {
        acc += update_free<T, V, true>(a, i, alpha, dn);
        if (i + nthr < a.nfree) acc += update_free<T, V, true>(a, i + nthr, alpha, dn);
      }
      apend = alpha;  // x += alpha d' in the next own-node pass (or after the loop)
      dpend = dn;
    } else {
      __syncthreads();  // everyone is done with the beta table
      for (int t = threadIdx.x; t < a.nscene; t += blockDim.x) tab[t] = alpha_of(t);
      __syncthreads();
      for (long long base = tid & ~31LL; base < a.nfree; base += nthr) {
        const long long i = base + lane;
        int key = -1;
        V v = 0;
        if (i < a.nfree) {
          key = a.node_scene[i];
          v = update_free<T, V, false>(a, i, tab[key], dn);
        }
        wacc_add(wa, shs, key, v, lane);
      }
      wacc_flush(wa, shs, lane);
    }
    for (long long bi = tid; bi < a.nb; bi += nthr) {
      const int i = a.nfree + (int)bi;
      const size_t o = 3 * ((size_t)a.nfree + 4 * (size_t)bi);
      V al = alpha;
      if constexpr (BATCH) al = tab[a.node_scene[a.nfree + 4 * bi]];
      for (int c = 0; c < 12; ++c) {
        if constexpr (BATCH) a.x[o + c] += al * dn[o + c];
        a.r[o + c] -= al * a.q[q_idx<V>(o + c)];
        a.q[q_idx<V>(o + c)] = 0;
      }
      const V v = precond_row<T, V>(i, a.nfree, a.Mi, a.r, a.z);
      if constexpr (BATCH) atomicAdd(&shs[a.node_scene[a.nfree + 4 * bi]], (double)v);
      else acc += v;
    }
    if constexpr (BATCH) flush_scene_sums(shs, a.ring, (int)(kbar & 7), a.nscene);
    bs = block_sum_v<V>(acc);
    if (clock0) { const unsigned long long t = global_ns(); tph[3] += t - tlast; tlast = t; }
    double rz_new = 0.0;
    const int kc = (int)(kbar & 7);
    if (!grid_reduce(a.bar, kbar, bs, rz_new, a.spin_limit, a.unmet, [&](double t) {
          if constexpr (!BATCH) {
            s_beta = (V)(t / rz);
            if (t <= a.tol2 * rz0) s_done = 1;
          }
        })) {
      done = 3;
      break;
    }
    after_barrier(kbar - 1);
    if (clock0) { const unsigned long long t = global_ns(); tph[4] += t - tlast; tlast = t; }
    ++it;
    if constexpr (!BATCH) {
      vb_next = s_beta;
      rz = rz_new;  // a register copy; only thread 0 of block 0 reports it
      done = s_done;
    } else {
      // iterations per scene: scenes that were still running this iteration
      if (blockIdx.x == 0)
        for (int t = threadIdx.x; t < a.nscene; t += blockDim.x)
          if (!sv.finished(t, a.tol2)) a.siters[t] += 1;
      cpp = cp;
      cp = kc;
      const scene_view<T, V> nv{&a, cp, cpp, kc};
      if (count_active(nv) == 0) done = 1;
    }
  }
  if constexpr (!BATCH) {
    // the last iteration's x update, on the nodes this thread owns (it wrote
    // their d' itself)
    if (apend != V(0))
      for (long long i = n0 + threadIdx.x; i < n1; i += blockDim.x)
        for (int c = 0; c < 3; ++c) a.x[3 * i + c] += apend * dpend[3 * i + c];
  }
  // a block that gave up may still have tile copies in flight: wait for them
  // before the block exits (bounded, but by a fixed limit far above a copy's
  // duration, independent of the barrier's wait limit)
  if (threadIdx.x == 0)
    for (int b = 0; b < 2; ++b)
      if ((inflight >> b) & 1u) mbar_wait_bounded(&mbar[b], (parity >> b) & 1u, kDrainPolls);
  __syncthreads();
  if (a.bt && threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    a.bt[blockIdx.x] = tbusy;
    a.bt[gridDim.x + blockIdx.x] = smid;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.sc->rz = rz;
    a.sc->rz0 = rz0;
    a.sc->done = done;
    a.sc->iters = it;
#pragma unroll
    for (int k = 0; k < 8; ++k) a.sc->t_ns[k] = k < 5 ? tph[k] : (k == 7 ? tph[5] : 0ull);
  }
  if (threadIdx.x == 0 && done == 3) dev_flag(a.status, DEV_TIMEOUT);
}

template <typename V>
__global__ void k_add_to(int n, double* __restrict__ p, const V* __restrict__ dx, double c) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] += c * (double)dx[i];
}
__global__ void k_sub_from(int n, const double* __restrict__ a, double* __restrict__ y) {  // y = a - y
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] - y[i];
}
// per-block max |x_i| into part[b] and an index holding it into part[nblk + b]
// (as a double; exact below 2^53)
__global__ void k_absmax(int n, const double* __restrict__ x, double* __restrict__ part) {
  double m = 0.0;
  long long at = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double a = fabs(x[i]);
    if (a > m) {
      m = a;
      at = i;
    }
  }
  __shared__ double sh[32];
  __shared__ long long shi[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double mo = __shfl_xor_sync(0xffffffffu, m, o);
    const long long ao = __shfl_xor_sync(0xffffffffu, at, o);
    if (mo > m || (mo == m && ao < at)) {
      m = mo;
      at = ao;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = m;
    shi[threadIdx.x >> 5] = at;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool in = threadIdx.x < (blockDim.x >> 5);
    double v = in ? sh[threadIdx.x] : 0.0;
    long long a = in ? shi[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double vo = __shfl_xor_sync(0xffffffffu, v, o);
      const long long ao = __shfl_xor_sync(0xffffffffu, a, o);
      if (vo > v || (vo == v && ao < a)) {
        v = vo;
        a = ao;
      }
    }
    if (threadIdx.x == 0) {
      part[blockIdx.x] = v;
      part[gridDim.x + blockIdx.x] = (double)a;
    }
  }
}
// per-block (a.b, b.b) partials into part[2 b], part[2 b + 1]
__global__ void k_dot2(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ part) {
  double ab = 0.0, bb = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double bi = b[i];
    ab += a[i] * bi;
    bb += bi * bi;
  }
  ab = block_sum(ab);
  bb = block_sum(bb);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ab;
    part[2 * blockIdx.x + 1] = bb;
  }
}
// r^T M^-1 r in FP64 (the refinement check of the FP32-mixed form)
template <typename T>
__global__ void k_rz64(int nfree, int nb, const T* __restrict__ Mi, const double* __restrict__ r, double* __restrict__ z,
                       double* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < nfree + nb) acc = precond_row<T, double>(i, nfree, Mi, r, z);
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// ---------------------------------------------------------------- host helpers
template <typename T, typename V>
yasps_status spmv_t(yasps_system* s, const V* x, V* y, const int* done) {
  const T* D = as<T>(s->diag);
  if (!done) {
    k_spmv_diag<T, V><<<blocks_for(s->nn, 256), 256, 0, s->stream>>>(s->nn, D, x, y);
    LAUNCH_CHECK(s, "k_spmv_diag");
  }
  if (s->Hs.nnzb > 0) {
    k_spmv_upper<T, V><<<blocks_for(s->Hs.nnzb, 256), 256, 0, s->stream>>>(
        s->Hs.nnzb, as<int>(s->Hs.row), as<int>(s->Hs.col), as<T>(s->Hs.vals), x, y, done);
    LAUNCH_CHECK(s, "k_spmv_upper(static)");
  }
  if (s->Hd.nnzb > 0) {
    k_spmv_upper<T, V><<<blocks_for(s->Hd.nnzb, 256), 256, 0, s->stream>>>(
        s->Hd.nnzb, as<int>(s->Hd.row), as<int>(s->Hd.col), as<T>(s->Hd.vals), x, y, done);
    LAUNCH_CHECK(s, "k_spmv_upper(dynamic)");
  }
  return YASPS_OK;
}

// grid of the persistent kernel: as many blocks as can be co-resident (a
// cooperative launch refuses a larger grid instead of deadlocking)
template <typename T, typename V, bool BATCH, typename CFG>
constexpr unsigned pcg_smem() {
  return stage_layout<T, CFG>::SMEM + (BATCH ? 16u * kMaxScenes : 0u);
}
template <typename T, typename V, bool BATCH, typename CFG>
yasps_status pcg_grid(yasps_system* s, int* G) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  CK(s, cudaGetDevice(&dev));
  CK(s, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(s, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) SYS_FAIL(s, YASPS_E_CUDA, "device does not support cooperative launches");
  const unsigned smem = pcg_smem<T, V, BATCH, CFG>();
  CK(s, cudaFuncSetAttribute(k_pcg_persistent<T, V, BATCH, CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
  CK(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<T, V, BATCH, CFG>, CFG::NTHR, smem));
  if (per_sm < 1) SYS_FAIL(s, YASPS_E_CUDA, "persistent PCG kernel cannot be resident");
  *G = sms * std::min(per_sm, CFG::MINB);
  return YASPS_OK;
}

// per-scene outputs of one batched launch
struct scene_out {
  std::vector<int> iters, flag;
};

// PCG in precision (T, V) on H dx = rhs (FP64 rhs); dx accumulated into p (FP64).
// Batches: stol2 (device, per scene) or null, per-scene iterations / flags out.
// D (nn nodes) and the free nodes' M^-1 packed symmetric for the PCG kernel
template <typename T>
__global__ void k_pack_sym(int nn, int nfree, const T* __restrict__ D, const T* __restrict__ Mi, T* __restrict__ Ds,
                           T* __restrict__ Ms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  auto pack = [](const T* A, T* S) {
    S[0] = A[0];
    S[1] = (T)0.5 * (A[1] + A[3]);
    S[2] = (T)0.5 * (A[2] + A[6]);
    S[3] = A[4];
    S[4] = (T)0.5 * (A[5] + A[7]);
    S[5] = A[8];
  };
  pack(D + 9 * (size_t)i, Ds + 6 * (size_t)i);
  if (i < nfree) pack(Mi + 9 * (size_t)i, Ms + 6 * (size_t)i);
}

template <typename T, typename V, bool BATCH, typename CFG>
yasps_status pcg_launch_cfg(yasps_system* s, const double* rhs, double* p, double tol, int maxit, const double* stol2,
                            int* iters, int* state, double* rel, scene_out* so, double rscale) {
  const int n3 = 3 * s->nn;
  for (int k = 0; k < 5; ++k) ENSURE(s, s->vec[k], sizeof(V) * (n3 + 4));
  ENSURE(s, s->vec[4], sizeof(V) * 4 * ((size_t)s->nn + 1));  // q: qlay<V>::S per node
  ENSURE(s, s->vec[8], sizeof(V) * (n3 + 4));
  int G = 0;
  RC((pcg_grid<T, V, BATCH, CFG>(s, &G)));
  const int ns = s->nscene;
  // scalars, barrier, and for batches: ring [8][ns], srz0, siters, sflag
  // pcg_dev (128 B), the barrier (cache-line aligned), then for batches the ring
  static_assert(sizeof(pcg_dev) <= 128, "pcg_dev exceeds its slot");
  constexpr size_t kHead = 128 + ((sizeof(pcg_bar) + 127) & ~(size_t)127);
  const size_t scal_bytes = kHead + (BATCH ? (size_t)ns * (8 * 8 + 8 + 4 + 4) + 64 : 0);
  ENSURE(s, s->scal, scal_bytes);
  char* base = static_cast<char*>(s->scal.p);
  pcg_dev* sc = reinterpret_cast<pcg_dev*>(base);
  pcg_bar* bar = reinterpret_cast<pcg_bar*>(base + 128);
  pcg_args<T, V> a;
  a.nn = s->nn;
  a.nfree = s->nfree;
  a.nb = s->nb;
  a.n_s = s->Hs.nnzb;
  a.n_d = s->Hd.nnzb;
  a.maxit = maxit;
  a.tol2 = tol * tol;
  a.row_s = as<int>(s->Hs.row);
  a.col_s = as<int>(s->Hs.col);
  a.val_s = as<T>(s->Hs.vals);
  a.row_d = as<int>(s->Hd.row);
  a.col_d = as<int>(s->Hd.col);
  a.val_d = as<T>(s->Hd.vals);
  a.D = as<T>(s->diag);
  a.Mi = as<T>(s->minv);
  ENSURE(s, s->dsym, sizeof(T) * 6 * (2 * (size_t)s->nn + 1));
  T* ds = as<T>(s->dsym);
  a.Ds = ds;
  a.Ms = ds + 6 * (size_t)s->nn;
  if (s->nn > 0) {
    k_pack_sym<T><<<blocks_for(s->nn, 256), 256, 0, s->stream>>>(s->nn, s->nfree, a.D, a.Mi, ds,
                                                                 ds + 6 * (size_t)s->nn);
    LAUNCH_CHECK(s, "k_pack_sym");
  }
  a.rhs = rhs;
  a.x = as<V>(s->vec[0]);
  a.r = as<V>(s->vec[1]);
  a.z = as<V>(s->vec[2]);
  a.q = as<V>(s->vec[4]);
  a.d0 = as<V>(s->vec[3]);
  a.d1 = as<V>(s->vec[8]);
  a.sc = sc;
  a.bar = bar;
  a.status = as<int>(s->status);
  a.spin_limit = s->wait_limit > 0 ? s->wait_limit : (1LL << 22);  // a few seconds of polling per wait
  a.rscale = rscale;
  a.bt = nullptr;
  if (s->prof_on) {
    ENSURE(s, s->pcg_bt, sizeof(unsigned long long) * (2 * (size_t)G + 1));
    a.bt = as<unsigned long long>(s->pcg_bt);
  }
  a.unmet = s->wait_unmet ? 1u : 0u;
  s->wait_unmet = false;
  a.nscene = ns;
  a.node_scene = BATCH ? as<int>(s->node_scene) : nullptr;
  a.ring = BATCH ? reinterpret_cast<double*>(base + kHead) : nullptr;
  a.srz0 = BATCH ? a.ring + 8 * (size_t)ns : nullptr;
  a.siters = BATCH ? reinterpret_cast<int*>(a.srz0 + ns) : nullptr;
  a.sflag = BATCH ? a.siters + ns : nullptr;
  a.stol2 = stol2;
  CK(s, cudaMemsetAsync(s->scal.p, 0, scal_bytes, s->stream));
  void* params[] = {&a};
  cudaEvent_t pk = prof_begin(s);
  CK(s, cudaLaunchCooperativeKernel((const void*)k_pcg_persistent<T, V, BATCH, CFG>, dim3(G), dim3(CFG::NTHR), params,
                                    pcg_smem<T, V, BATCH, CFG>(), s->stream));
  s->launches += 1;
  prof_end(s, YASPS_STAGE_PCG_KERNEL, pk, 0.0);
  pcg_dev h{};
  CK(s, cudaMemcpyAsync(&h, sc, sizeof(pcg_dev), cudaMemcpyDeviceToHost, s->stream));
  if (BATCH && so) {
    so->iters.assign(ns, 0);
    so->flag.assign(ns, 0);
    CK(s, cudaMemcpyAsync(so->iters.data(), a.siters, sizeof(int) * ns, cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaMemcpyAsync(so->flag.data(), a.sflag, sizeof(int) * ns, cudaMemcpyDeviceToHost, s->stream));
  }
  CK(s, cudaStreamSynchronize(s->stream));
  if (s->prof_on) {
    const double es = sizeof(T), vs = sizeof(V), nn = s->nn;
    const double nnzb = (double)s->Hs.nnzb + s->Hd.nnzb;
    // H d phase: blocks + column index + row pointer, D, z and d read, d' and q written
    // (D and M^-1 at 6 values per node: symmetric, read packed)
    const double spmv_bytes = nnzb * (9 * es + 4) + nn * 4 + nn * 6 * es + 3 * vs * nn * 4;
    // whole iteration: H d phase + update (x, d', r, q read; x, r, z, q written; M^-1)
    const double iter_bytes = spmv_bytes + 3 * vs * nn * 8 + nn * 6 * es;
    s->prof_acc[YASPS_STAGE_PCG_KERNEL].bytes += iter_bytes * h.iters;
    auto& sp = s->prof_acc[YASPS_STAGE_SPMV];
    sp.count += h.iters;
    sp.ms += (h.t_ns[0] + h.t_ns[1] + h.t_ns[2]) * 1e-6;
    for (int k = 0; k < 5; ++k) s->pcg_phase_ms[k] += h.t_ns[k] * 1e-6;
    s->pcg_phase_ms[7] += h.t_ns[7] * 1e-6;
    sp.bytes += spmv_bytes * h.iters;
    // load balance of the H d' phase: mean and max over the blocks of their busy time
    std::vector<unsigned long long> bt(2 * (size_t)G);
    CK(s, cudaMemcpyAsync(bt.data(), a.bt, sizeof(unsigned long long) * 2 * G, cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    double mean = 0.0, mx = 0.0;
    if ((int)s->pcg_busy_ns.size() != G) {
      s->pcg_busy_ns.assign(G, 0.0);
      s->pcg_busy_iters = 0;
    }
    s->pcg_busy_sm.resize(G);
    for (int b = 0; b < G; ++b) {
      mean += (double)bt[b];
      mx = std::max(mx, (double)bt[b]);
      s->pcg_busy_ns[b] += (double)bt[b];
      s->pcg_busy_sm[b] = (int)bt[G + b];
    }
    s->pcg_busy_iters += h.iters;
    s->pcg_phase_ms[5] += mean / G * 1e-6;
    s->pcg_phase_ms[6] += mx * 1e-6;
  }
  if (h.done == 3) SYS_FAIL(s, YASPS_E_TIMEOUT, "PCG grid barrier timed out");
  k_add_to<V><<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, p, a.x, 1.0 / rscale);
  LAUNCH_CHECK(s, "k_add_to");
  *iters = h.iters;
  *state = h.done;
  *rel = (h.rz0 > 0.0) ? std::sqrt(std::max(h.rz, 0.0) / h.rz0) : 0.0;
  return YASPS_OK;
}

// the launch configuration the system uses (s->pcg_variant)
template <typename T, typename V, bool BATCH>
yasps_status pcg_launch(yasps_system* s, const double* rhs, double* p, double tol, int maxit, const double* stol2,
                        int* iters, int* state, double* rel, scene_out* so, double rscale = 1.0) {
  switch (s->pcg_variant) {
    case 1:
      return pcg_launch_cfg<T, V, BATCH, typename pcg_variant<T, 1>::C>(s, rhs, p, tol, maxit, stol2, iters, state,
                                                                        rel, so, rscale);
    case 2:
      return pcg_launch_cfg<T, V, BATCH, typename pcg_variant<T, 2>::C>(s, rhs, p, tol, maxit, stol2, iters, state,
                                                                        rel, so, rscale);
    case 3:
      return pcg_launch_cfg<T, V, BATCH, typename pcg_variant<T, 3>::C>(s, rhs, p, tol, maxit, stol2, iters, state,
                                                                        rel, so, rscale);
    case 4:
      return pcg_launch_cfg<T, V, BATCH, typename pcg_variant<T, 4>::C>(s, rhs, p, tol, maxit, stol2, iters, state,
                                                                        rel, so, rscale);
    default:
      return pcg_launch_cfg<T, V, BATCH, typename pcg_variant<T, 0>::C>(s, rhs, p, tol, maxit, stol2, iters, state,
                                                                        rel, so, rscale);
  }
}

template <typename T, typename V>
yasps_status pcg_inner(yasps_system* s, const double* rhs, double* p, double tol, int maxit, int* iters, int* state,
                       double* rel, double rscale = 1.0) {
  return pcg_launch<T, V, false>(s, rhs, p, tol, maxit, nullptr, iters, state, rel, nullptr, rscale);
}

// r^T M^-1 r per scene in FP64 (the refinement check of a batch): warp-segmented
// by scene, run heads add into out[scene]
template <typename T>
__global__ void k_rz64_scene(int nfree, int nb, const T* __restrict__ Mi, const double* __restrict__ r,
                             double* __restrict__ z, const int* __restrict__ node_scene, double* __restrict__ out) {
  const long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL;
  const int lane = threadIdx.x & 31;
  const long long i = base + lane;
  const int nu = nfree + nb;
  double v = 0.0;
  int key = -1;
  if (i < nu) {
    v = precond_row<T, double>((int)i, nfree, Mi, r, z);
    key = node_scene[i < nfree ? i : nfree + 4 * (i - nfree)];
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int ko = __shfl_down_sync(0xffffffffu, key, off);
    const double vo = __shfl_down_sync(0xffffffffu, v, off);
    if (lane + off < 32 && ko == key) v += vo;
  }
  const int kp = __shfl_up_sync(0xffffffffu, key, 1);
  if (key >= 0 && (lane == 0 || kp != key)) atomicAdd(&out[key], v);
}

template <typename T>
yasps_status rz64(yasps_system* s, const double* r, double* out) {
  const int nu = s->nfree + s->nb;
  const int nblk = blocks_for(std::max(nu, 1), PT_);
  ENSURE(s, s->vec[5], sizeof(double) * (3 * (size_t)s->nn + 4));
  ENSURE(s, s->red, sizeof(double) * (nblk + 8));
  k_rz64<T><<<nblk, PT_, 0, s->stream>>>(s->nfree, s->nb, as<T>(s->minv), r, as<double>(s->vec[5]), as<double>(s->red));
  LAUNCH_CHECK(s, "k_rz64");
  std::vector<double> h(nblk);
  CK(s, cudaMemcpyAsync(h.data(), s->red.p, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  double acc = 0.0;
  for (double v : h) acc += v;
  *out = acc;
  return YASPS_OK;
}

}  // namespace

// ======================================================================== API
yasps_status pcg_solve_impl(yasps_system* s, const double* rhs, double* p, double tol, int maxit, int* iters,
                            double* rel_res, const double* x0);

yasps_status alloc_hessian(yasps_system* s) {
  const size_t es = (s->prm.precision == 1) ? sizeof(float) : sizeof(double);
  s->hess_precision = (s->prm.precision == 1) ? 1 : 0;
  ENSURE(s, s->diag, es * 9 * ((size_t)s->nn + 1));
  ENSURE(s, s->Hs.vals, es * 9 * ((size_t)s->Hs.nnzb + 1));
  ENSURE(s, s->Hd.vals, es * 9 * ((size_t)s->Hd.nnzb + 1));
  ENSURE(s, s->minv, es * (9 * (size_t)s->nfree + 144 * (size_t)s->nb + 1));
  ENSURE(s, s->grad, sizeof(double) * (3 * (size_t)s->nn + 1));
  return YASPS_OK;
}

yasps_status zero_system(yasps_system* s) {
  const size_t es = (s->hess_precision == 1) ? sizeof(float) : sizeof(double);
  CK(s, cudaMemsetAsync(s->grad.p, 0, sizeof(double) * 3 * (size_t)s->nn, s->stream));
  CK(s, cudaMemsetAsync(s->diag.p, 0, es * 9 * (size_t)s->nn, s->stream));
  if (s->Hs.nnzb) CK(s, cudaMemsetAsync(s->Hs.vals.p, 0, es * 9 * (size_t)s->Hs.nnzb, s->stream));
  if (s->Hd.nnzb) CK(s, cudaMemsetAsync(s->Hd.vals.p, 0, es * 9 * (size_t)s->Hd.nnzb, s->stream));
  return YASPS_OK;
}

template <typename T>
static yasps_status bjacobi_t(yasps_system* s) {
  int* st = as<int>(s->status);
  if (s->nfree > 0) {
    k_bj_free<T><<<blocks_for(s->nfree, 256), 256, 0, s->stream>>>(s->nfree, as<T>(s->diag), as<T>(s->minv), st);
    LAUNCH_CHECK(s, "k_bj_free");
  }
  if (s->nb > 0) {
    const bool dyn = s->Hd.nnzb > 0;
    k_bj_body<T><<<blocks_for(s->nb, 32), 32, 0, s->stream>>>(
        s->nb, s->nfree, as<T>(s->diag), as<int>(s->body_slot), as<T>(s->Hs.vals), dyn ? as<int>(s->Hd.row_ptr) : nullptr,
        dyn ? as<int>(s->Hd.col) : nullptr, dyn ? as<T>(s->Hd.vals) : nullptr, as<T>(s->minv), st);
    LAUNCH_CHECK(s, "k_bj_body");
  }
  return YASPS_OK;
}
yasps_status launch_bjacobi(yasps_system* s) {
  return s->hess_precision == 1 ? bjacobi_t<float>(s) : bjacobi_t<double>(s);
}

yasps_status spmv64(yasps_system* s, const double* x, double* y) {
  if (s->hess_precision == 1) return spmv_t<float, double>(s, x, y, nullptr);
  return spmv_t<double, double>(s, x, y, nullptr);
}

yasps_status pcg_solve(yasps_system* s, const double* rhs, double* p, double tol, int maxit, int* iters,
                       double* rel_res, const double* x0) {
  cudaEvent_t pa = prof_begin(s);
  yasps_status rc = pcg_solve_impl(s, rhs, p, tol, maxit, iters, rel_res, x0);
  prof_end(s, YASPS_STAGE_PCG, pa, 0.0);
  return rc;
}

// r^T M^-1 r per scene (FP64) into out[nscene]
template <typename T>
static yasps_status rz64_scene(yasps_system* s, const double* r, std::vector<double>& out) {
  const int nu = s->nfree + s->nb, ns = s->nscene;
  ENSURE(s, s->vec[5], sizeof(double) * (3 * (size_t)s->nn + 4));
  ENSURE(s, s->scene_buf, sizeof(double) * (2 * (size_t)ns + 4));
  double* acc = as<double>(s->scene_buf);
  CK(s, cudaMemsetAsync(acc, 0, sizeof(double) * ns, s->stream));
  k_rz64_scene<T><<<blocks_for(std::max(nu, 1), 256), 256, 0, s->stream>>>(s->nfree, s->nb, as<T>(s->minv), r,
                                                                          as<double>(s->vec[5]), as<int>(s->node_scene),
                                                                          acc);
  LAUNCH_CHECK(s, "k_rz64_scene");
  out.assign(ns, 0.0);
  CK(s, cudaMemcpyAsync(out.data(), acc, sizeof(double) * ns, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

// Batches: one PCG per scene, all in the same launches (per-scene alpha, beta
// and stopping test).  FP32-mixed: FP32 inner PCG, FP64 residual per scene,
// refinement sweeps until every scene meets the tolerance; a finished scene
// gets an inner tolerance of 1, so later sweeps leave it alone.
static yasps_status pcg_solve_batch(yasps_system* s, const double* rhs, double* p, double tol, int maxit, int* iters,
                                    double* rel_res) {
  const int n3 = 3 * s->nn, ns = s->nscene;
  scene_out so;
  int it = 0, state = 0;
  double rel = 0.0;
  s->scene_pcg.assign(ns, 0);
  auto take = [&](const scene_out& o) -> bool {  // true if some scene broke down
    bool broke = false;
    for (int k = 0; k < ns; ++k) {
      s->scene_pcg[k] += o.iters[k];
      broke |= o.flag[k] == 2;
    }
    return broke;
  };
  if (s->hess_precision != 1) {
    RC((pcg_launch<double, double, true>(s, rhs, p, tol, maxit, nullptr, &it, &state, &rel, &so)));
    if (iters) *iters = it;
    if (rel_res) *rel_res = state == 1 ? 0.0 : 1.0;
    if (take(so)) SYS_FAIL(s, YASPS_E_NAN, "PCG breakdown in a scene: d^T H d <= 0");
    if (state != 1) SYS_FAIL(s, YASPS_E_NOCONV, "PCG hit its iteration cap");
    return YASPS_OK;
  }
  ENSURE(s, s->vec[6], sizeof(double) * (n3 + 4));
  double* res = as<double>(s->vec[6]);
  std::vector<double> rz0, rz;
  RC(rz64_scene<float>(s, rhs, rz0));
  rz = rz0;
  std::vector<double> stol2(ns);
  int total = 0;
  bool all = false, broke = false;
  const int sweeps = std::max(1, s->prm.refine_sweeps);
  for (int sw = 0; sw < sweeps && !all; ++sw) {
    double live = 0.0;  // r^T M^-1 r of the scenes still solving
    for (int k = 0; k < ns; ++k) {
      const bool fin = !(rz[k] > tol * tol * rz0[k]);
      const double inner = fin ? 1.0 : std::max(tol * std::sqrt(rz0[k] / rz[k]), 5e-6);
      stol2[k] = inner * inner;
      if (!fin) live += rz[k];
    }
    // the FP32 solve works on the residual scaled to unit M^-1 norm over the
    // scenes still solving (kept away from FP32 underflow); scaled back in FP64
    const double rscale = live > 0.0 ? 1.0 / std::sqrt(live) : 1.0;
    ENSURE(s, s->scene_buf, sizeof(double) * (2 * (size_t)ns + 4));
    double* st_dev = as<double>(s->scene_buf) + ns;
    CK(s, cudaMemcpyAsync(st_dev, stol2.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s->stream));
    RC((pcg_launch<float, float, true>(s, sw == 0 ? rhs : res, p, tol, maxit - total, st_dev, &it, &state, &rel,
                                       &so, rscale)));
    total += it;
    broke |= take(so);
    RC(spmv64(s, p, res));
    k_sub_from<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, rhs, res);
    LAUNCH_CHECK(s, "k_sub_from");
    RC(rz64_scene<float>(s, res, rz));
    all = true;
    for (int k = 0; k < ns; ++k) all &= !(rz[k] > tol * tol * rz0[k]);
    if (total >= maxit || broke) break;
  }
  if (iters) *iters = total;
  double worst = 0.0;
  for (int k = 0; k < ns; ++k)
    if (rz0[k] > 0.0) worst = std::max(worst, std::sqrt(std::max(rz[k], 0.0) / rz0[k]));
  if (rel_res) *rel_res = worst;
  if (broke) SYS_FAIL(s, YASPS_E_NAN, "PCG breakdown in a scene: d^T H d <= 0");
  if (!all && total >= maxit) SYS_FAIL(s, YASPS_E_NOCONV, "PCG hit its iteration cap");
  return YASPS_OK;
}

yasps_status pcg_solve_impl(yasps_system* s, const double* rhs, double* p, double tol, int maxit, int* iters,
                            double* rel_res, const double* x0) {
  const int n3 = 3 * s->nn;
  if (maxit <= 0) maxit = 10 * n3;
  if (s->nscene > 1) x0 = nullptr;  // batches start cold
  if (x0) CK(s, cudaMemcpyAsync(p, x0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s->stream));
  else CK(s, cudaMemsetAsync(p, 0, sizeof(double) * n3, s->stream));
  if (s->nscene > 1) return pcg_solve_batch(s, rhs, p, tol, maxit, iters, rel_res);
  int it = 0, state = 0;
  double rel = 0.0;
  ENSURE(s, s->vec[6], sizeof(double) * (n3 + 4));
  double* res = as<double>(s->vec[6]);
  const bool mixed = s->hess_precision == 1;
  // the stopping test is relative to the right-hand side: r^T z <= tol^2 g^T M^-1 g
  double rz0 = 0.0, rz = 0.0;
  RC(mixed ? rz64<float>(s, rhs, &rz0) : rz64<double>(s, rhs, &rz0));
  // g^T M^-1 g: NaN from a non-finite right-hand side, negative from an
  // indefinite preconditioner block; exactly 0 means p = 0 solves it
  if (!(rz0 >= 0.0)) SYS_FAIL(s, YASPS_E_NAN, "PCG: non-finite right-hand side or indefinite preconditioner");
  if (!(rz0 > 0.0)) {
    CK(s, cudaMemsetAsync(p, 0, sizeof(double) * n3, s->stream));
    if (iters) *iters = 0;
    if (rel_res) *rel_res = 0.0;
    return YASPS_OK;
  }
  const double* r_cur = rhs;
  rz = rz0;
  if (x0) {  // warm start: solve for the correction of x0
    RC(spmv64(s, p, res));
    k_sub_from<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, rhs, res);
    LAUNCH_CHECK(s, "k_sub_from");
    RC(mixed ? rz64<float>(s, res, &rz) : rz64<double>(s, res, &rz));
    r_cur = res;
  }
  if (!mixed) {
    if (rz > tol * tol * rz0) {
      RC((pcg_inner<double, double>(s, r_cur, p, tol * std::sqrt(rz0 / rz), maxit, &it, &state, &rel)));
      rel *= std::sqrt(rz / rz0);
    } else {
      state = 1;
      rel = std::sqrt(rz / rz0);
    }
    if (iters) *iters = it;
    if (rel_res) *rel_res = rel;
    if (state == 2) SYS_FAIL(s, YASPS_E_NAN, "PCG breakdown: d^T H d <= 0");
    if (state != 1 && rel > tol) SYS_FAIL(s, YASPS_E_NOCONV, "PCG hit its iteration cap");
    return YASPS_OK;
  }
  // FP32-mixed: FP32 inner PCG, FP64 residual refinement
  int total = 0;
  const int sweeps = std::max(1, s->prm.refine_sweeps);
  for (int sw = 0; sw < sweeps && rz > tol * tol * rz0; ++sw) {
    const double inner_tol = std::max(tol * std::sqrt(rz0 / rz), 5e-6);
    // the FP32 solve sees the residual scaled to unit M^-1 norm (its vectors and
    // d^T H d stay far from FP32 underflow however small the residual gets);
    // the correction is scaled back in FP64
    RC((pcg_inner<float, float>(s, r_cur, p, inner_tol, maxit - total, &it, &state, &rel, 1.0 / std::sqrt(rz))));
    total += it;
    // FP64 residual res = rhs - H p
    RC(spmv64(s, p, res));
    k_sub_from<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, rhs, res);
    LAUNCH_CHECK(s, "k_sub_from");
    RC(rz64<float>(s, res, &rz));
    r_cur = res;
    if (total >= maxit || state == 2) break;
  }
  if (iters) *iters = total;
  const double r = std::sqrt(std::max(rz, 0.0) / rz0);
  if (rel_res) *rel_res = r;
  if (state == 2) SYS_FAIL(s, YASPS_E_NAN, "PCG breakdown: d^T H d <= 0");
  if (r > tol && total >= maxit) SYS_FAIL(s, YASPS_E_NOCONV, "PCG hit its iteration cap");
  return YASPS_OK;
}

// Autotuning of the PCG launch configuration on the system at hand: every
// variant runs `iters` iterations (tolerance 0) on the current assembly with
// the current gradient as right-hand side, timed with events after one
// warm-up launch; the fastest per iteration is kept.
template <typename T, typename V, bool BATCH>
static yasps_status autotune_t(yasps_system* s, int iters, int* variant, double* us) {
  const int n3 = 3 * s->nn;
  ENSURE(s, s->vec[6], sizeof(double) * (n3 + 4));
  double* pt = as<double>(s->vec[6]);
  const double* rhs = as<double>(s->grad);
  int best = 0;
  double best_us = 1e300;
  const bool prof = s->prof_on;
  s->prof_on = false;
  for (int v = 0; v < kPcgVariants; ++v) {
    s->pcg_variant = v;
    double t_us = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
      CK(s, cudaMemsetAsync(pt, 0, sizeof(double) * n3, s->stream));
      int it = 0, state = 0;
      double rel = 0.0;
      scene_out so;
      CK(s, cudaEventRecord(s->ev[6], s->stream));
      yasps_status rc = pcg_launch<T, V, BATCH>(s, rhs, pt, 0.0, iters, nullptr, &it, &state, &rel, &so);
      if (rc != YASPS_OK) {
        s->prof_on = prof;
        return rc;
      }
      CK(s, cudaEventRecord(s->ev[7], s->stream));
      CK(s, cudaEventSynchronize(s->ev[7]));
      float ms = 0.f;
      CK(s, cudaEventElapsedTime(&ms, s->ev[6], s->ev[7]));
      t_us = 1e3 * ms / std::max(it, 1);
    }
    if (us) us[v] = t_us;
    if (t_us < best_us) {
      best_us = t_us;
      best = v;
    }
  }
  s->prof_on = prof;
  s->pcg_variant = best;
  if (variant) *variant = best;
  return YASPS_OK;
}

yasps_status autotune_pcg(yasps_system* s, int iters, int* variant, double* us) {
  if (iters <= 0) iters = 30;
  const bool batch = s->nscene > 1;
  if (s->hess_precision == 1)
    return batch ? autotune_t<float, float, true>(s, iters, variant, us)
                 : autotune_t<float, float, false>(s, iters, variant, us);
  return batch ? autotune_t<double, double, true>(s, iters, variant, us)
               : autotune_t<double, double, false>(s, iters, variant, us);
}

yasps_status inf_norm(yasps_system* s, const double* x, int n, double* out_host, int* arg_host) {
  const int nblk = std::min(148 * 2, blocks_for(std::max(n, 1), 256));
  ENSURE(s, s->red, sizeof(double) * (2 * nblk + 8));
  k_absmax<<<nblk, 256, 0, s->stream>>>(n, x, as<double>(s->red));
  LAUNCH_CHECK(s, "k_absmax");
  std::vector<double> h(2 * nblk);
  CK(s, cudaMemcpyAsync(h.data(), s->red.p, sizeof(double) * 2 * nblk, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  double m = 0.0;
  int at = 0;
  for (int b = 0; b < nblk; ++b)
    if (h[b] > m) {
      m = h[b];
      at = (int)h[nblk + b];
    }
  *out_host = m;
  if (arg_host) *arg_host = at;
  return YASPS_OK;
}

yasps_status dot2(yasps_system* s, const double* a, const double* b, int n, double* ab_host, double* bb_host) {
  const int nblk = std::min(148 * 2, blocks_for(std::max(n, 1), 256));
  ENSURE(s, s->red, sizeof(double) * (2 * nblk + 8));
  k_dot2<<<nblk, 256, 0, s->stream>>>(n, a, b, as<double>(s->red));
  LAUNCH_CHECK(s, "k_dot2");
  std::vector<double> h(2 * nblk);
  CK(s, cudaMemcpyAsync(h.data(), s->red.p, sizeof(double) * 2 * nblk, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  double ab = 0.0, bb = 0.0;
  for (int k = 0; k < nblk; ++k) {
    ab += h[2 * k];
    bb += h[2 * k + 1];
  }
  *ab_host = ab;
  *bb_host = bb;
  return YASPS_OK;
}

yasps_status read_status(yasps_system* s, int* bits) {
  int h = 0;
  CK(s, cudaMemcpyAsync(&h, s->status.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  if (h) CK(s, cudaMemsetAsync(s->status.p, 0, sizeof(int), s->stream));
  *bits = h;
  return YASPS_OK;
}
