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
// PCG keeps its scalars (r^T z, alpha, beta, convergence flag) on the device.
// Dot products are two-level (per-block partials, then the last block to
// finish sums the partials in block order), so results do not depend on
// scheduling.  In the FP32-mixed form the inner PCG runs on FP32 vectors and
// FP32 blocks; an outer loop recomputes the residual g - H p in FP64 and
// solves for the correction (iterative refinement).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int PT_ = 256;  // threads per block for vector kernels
constexpr int kPcgChunk = 16;  // PCG iterations per CUDA graph launch

struct pcg_dev {
  double rz, rz_new, dq, alpha, beta, rz0, tol2;
  int done, iters, counter_dq, counter_rz, pad;
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
  // segmented suffix reduction of the U x contributions within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ro = __shfl_down_sync(0xffffffffu, r, o);
    const V b0 = shfl_down_v(a0, o), b1 = shfl_down_v(a1, o), b2 = shfl_down_v(a2, o);
    if (lane + o < 32 && ro == r) { a0 += b0; a1 += b1; a2 += b2; }
  }
  const int rp = __shfl_up_sync(0xffffffffu, r, 1);
  if (r >= 0 && (lane == 0 || rp != r)) {
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
  if (!(det > 0.0) || !isfinite(det)) {
    dev_flag(status, DEV_NAN);
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
    if (!(fabs(d) > 0.0)) { dev_flag(status, DEV_NAN); return; }
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

// ---------------------------------------------------------------- PCG kernels
// Last block to arrive sums the per-block partials in order.
__device__ __forceinline__ bool last_block(int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int t = atomicAdd(counter, 1);
    last = (t == (int)gridDim.x - 1);
  }
  __syncthreads();
  return last;
}
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
__device__ double sum_partials(const double* part, int n) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  return block_sum(v);
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

// init: r = rhs (- H p0 already folded into rhs by the caller), x = 0, z = M^-1 r, d = 0
template <typename T, typename V>
__global__ void k_pcg_init(int nfree, int nb, const double* __restrict__ rhs, const T* __restrict__ Mi, V* __restrict__ x,
                           V* __restrict__ r, V* __restrict__ z, V* __restrict__ d, double* __restrict__ part,
                           pcg_dev* sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nu = nfree + nb;
  V acc = 0;
  if (i < nu) {
    const int cnt = (i < nfree) ? 3 : 12;
    const size_t o = (i < nfree) ? 3 * (size_t)i : 3 * ((size_t)nfree + 4 * (size_t)(i - nfree));
    for (int c = 0; c < cnt; ++c) {
      r[o + c] = (V)rhs[o + c];
      x[o + c] = 0;
      d[o + c] = 0;
    }
  }
  __syncthreads();
  if (i < nu) acc = precond_row<T, V>(i, nfree, Mi, r, z);
  const double bs = (double)block_sum_v<V>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = bs;
  if (last_block(&sc->counter_rz)) {
    const double rz = sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
      sc->rz = rz;
      sc->rz0 = rz;
      sc->beta = 0.0;
      sc->iters = 0;
      sc->done = !(rz > 0.0) ? 1 : 0;
      sc->counter_rz = 0;
    }
  }
}

// d = z + beta d ; q = D d   (diagonal part of q = H d)
template <typename T, typename V>
__global__ void k_pcg_dir(int nn, const T* __restrict__ D, const V* __restrict__ z, V* __restrict__ d, V* __restrict__ q,
                          const pcg_dev* __restrict__ sc) {
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const V beta = (V)sc->beta;
  V dv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    dv[a] = z[3 * i + a] + beta * d[3 * i + a];
    d[3 * i + a] = dv[a];
  }
  const T* B = D + 9 * (size_t)i;
#pragma unroll
  for (int a = 0; a < 3; ++a) q[3 * i + a] = (V)B[3 * a] * dv[0] + (V)B[3 * a + 1] * dv[1] + (V)B[3 * a + 2] * dv[2];
}

// dq = d . q, alpha = rz / dq
template <typename V>
__global__ void k_pcg_alpha(int n3, const V* __restrict__ d, const V* __restrict__ q, double* __restrict__ part,
                            pcg_dev* sc) {
  if (sc->done) return;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x)
    acc += (double)d[i] * (double)q[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  if (last_block(&sc->counter_dq)) {
    const double dq = sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
      sc->dq = dq;
      sc->alpha = (dq > 0.0) ? sc->rz / dq : 0.0;
      if (!(dq > 0.0)) sc->done = 2;  // breakdown (H not positive definite on d)
      sc->counter_dq = 0;
    }
  }
}

// x += alpha d, r -= alpha q, z = M^-1 r, rz_new = r . z, beta, convergence
template <typename T, typename V>
__global__ void k_pcg_update(int nfree, int nb, const T* __restrict__ Mi, V* __restrict__ x, V* __restrict__ r,
                             V* __restrict__ z, const V* __restrict__ d, const V* __restrict__ q,
                             double* __restrict__ part, pcg_dev* sc) {
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nu = nfree + nb;
  const V alpha = (V)sc->alpha;
  V acc = 0;
  if (i < nu) {
    const int cnt = (i < nfree) ? 3 : 12;
    const size_t o = (i < nfree) ? 3 * (size_t)i : 3 * ((size_t)nfree + 4 * (size_t)(i - nfree));
    for (int c = 0; c < cnt; ++c) {
      x[o + c] += alpha * d[o + c];
      r[o + c] -= alpha * q[o + c];
    }
    acc = precond_row<T, V>(i, nfree, Mi, r, z);
  }
  const double bs = (double)block_sum_v<V>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = bs;
}

// ---------------------------------------------------------------- fused PCG iteration
// (1) d = z + beta d ; q = D d ; partial d^T D d
template <typename T, typename V>
__global__ void k_pcg_dir_dd(int nn, const T* __restrict__ D, const V* __restrict__ z, V* __restrict__ d,
                             V* __restrict__ q, const pcg_dev* __restrict__ sc, double* __restrict__ part) {
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  V accv = 0;
  if (i < nn) {
    const V beta = (V)sc->beta;
    V dv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dv[a] = z[3 * i + a] + beta * d[3 * i + a];
      d[3 * i + a] = dv[a];
    }
    const T* B = D + 9 * (size_t)i;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const V qa = (V)B[3 * a] * dv[0] + (V)B[3 * a + 1] * dv[1] + (V)B[3 * a + 2] * dv[2];
      q[3 * i + a] = qa;
      accv += dv[a] * qa;
    }
  }
  const double acc = (double)block_sum_v<V>(accv);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// (2) q += U d + U^T d over both upper parts (static blocks first, then
// dynamic), partial 2 d_r^T B d_c; the last block finishes d^T H d and alpha.
template <typename T, typename V>
__global__ void __launch_bounds__(256) k_spmv_both(int n_s, const int* __restrict__ row_s, const int* __restrict__ col_s,
                                                   const T* __restrict__ val_s, int n_d, const int* __restrict__ row_d,
                                                   const int* __restrict__ col_d, const T* __restrict__ val_d,
                                                   const V* __restrict__ x, V* __restrict__ y, pcg_dev* sc,
                                                   double* __restrict__ part, int n_dir_parts) {
  if (sc->done) return;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)n_s + n_d;
  const long long stride = (long long)gridDim.x * blockDim.x;
  V accv = 0;  // per-thread partial in the vector precision (FP64 ALU is scarce)
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
    const long long k = base + threadIdx.x;
    int r = -1;
    V a0 = 0, a1 = 0, a2 = 0;
    if (k < total) {
      const bool st = k < n_s;
      const long long kk = st ? k : k - n_s;
      r = st ? row_s[kk] : row_d[kk];
      const int c = st ? col_s[kk] : col_d[kk];
      const T* B = (st ? val_s : val_d) + 9 * (size_t)kk;
      T b[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) b[t] = B[t];
      const V xc0 = x[3 * c], xc1 = x[3 * c + 1], xc2 = x[3 * c + 2];
      const V xr0 = x[3 * r], xr1 = x[3 * r + 1], xr2 = x[3 * r + 2];
      a0 = (V)b[0] * xc0 + (V)b[1] * xc1 + (V)b[2] * xc2;
      a1 = (V)b[3] * xc0 + (V)b[4] * xc1 + (V)b[5] * xc2;
      a2 = (V)b[6] * xc0 + (V)b[7] * xc1 + (V)b[8] * xc2;
      accv += (V)2 * (xr0 * a0 + xr1 * a1 + xr2 * a2);
      atomicAdd(&y[3 * c], (V)b[0] * xr0 + (V)b[3] * xr1 + (V)b[6] * xr2);
      atomicAdd(&y[3 * c + 1], (V)b[1] * xr0 + (V)b[4] * xr1 + (V)b[7] * xr2);
      atomicAdd(&y[3 * c + 2], (V)b[2] * xr0 + (V)b[5] * xr1 + (V)b[8] * xr2);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ro = __shfl_down_sync(0xffffffffu, r, o);
      const V b0 = shfl_down_v(a0, o), b1 = shfl_down_v(a1, o), b2 = shfl_down_v(a2, o);
      if (lane + o < 32 && ro == r) { a0 += b0; a1 += b1; a2 += b2; }
    }
    const int rp = __shfl_up_sync(0xffffffffu, r, 1);
    if (r >= 0 && (lane == 0 || rp != r)) {
      atomicAdd(&y[3 * r], a0);
      atomicAdd(&y[3 * r + 1], a1);
      atomicAdd(&y[3 * r + 2], a2);
    }
  }
  const double acc = (double)block_sum_v<V>(accv);
  if (threadIdx.x == 0) part[n_dir_parts + blockIdx.x] = acc;
}

// one block: d^T H d from the partials in order, then alpha (a separate kernel:
// a grid-wide "last block" counter serialises thousands of same-address atomics)
__global__ void k_pcg_alpha_fin(const double* __restrict__ part, int nparts, pcg_dev* sc) {
  if (sc->done) return;
  const double dq = sum_partials(part, nparts);
  if (threadIdx.x == 0) {
    sc->dq = dq;
    sc->alpha = (dq > 0.0) ? sc->rz / dq : 0.0;
    if (!(dq > 0.0)) sc->done = 2;
  }
}
// one block: r^T z from the partials, beta, iteration count, convergence
__global__ void k_pcg_beta_fin(const double* __restrict__ part, int nparts, pcg_dev* sc) {
  if (sc->done) return;
  const double rz = sum_partials(part, nparts);
  if (threadIdx.x == 0) {
    sc->beta = rz / sc->rz;
    sc->rz = rz;
    sc->iters += 1;
    if (rz <= sc->tol2 * sc->rz0) sc->done = 1;
  }
}

template <typename V>
__global__ void k_add_to(int n, double* __restrict__ p, const V* __restrict__ dx) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] += (double)dx[i];
}
__global__ void k_sub_from(int n, const double* __restrict__ a, double* __restrict__ y) {  // y = a - y
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] - y[i];
}
__global__ void k_absmax(int n, const double* __restrict__ x, double* __restrict__ part) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  __shared__ double sh[32];
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    v = warp_max(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
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

// PCG in precision (T, V) on H dx = rhs (FP64 rhs); dx accumulated into p (FP64).
template <typename T, typename V>
yasps_status pcg_inner(yasps_system* s, const double* rhs, double* p, double tol, int maxit, int* iters, int* state,
                       double* rel) {
  const int n3 = 3 * s->nn;
  for (int k = 0; k < 5; ++k) ENSURE(s, s->vec[k], sizeof(V) * (n3 + 4));
  V *x = as<V>(s->vec[0]), *r = as<V>(s->vec[1]), *z = as<V>(s->vec[2]), *d = as<V>(s->vec[3]), *q = as<V>(s->vec[4]);
  const int nu = s->nfree + s->nb;
  const int nblk_u = blocks_for(std::max(nu, 1), PT_);
  const int nblk_dir = blocks_for(std::max(s->nn, 1), PT_);
  const long long nup = (long long)s->Hs.nnzb + s->Hd.nnzb;
  const int nblk_up = (int)std::max<long long>(1, (nup + PT_ - 1) / PT_);  // one block per thread
  ENSURE(s, s->scal, sizeof(pcg_dev) + 64);
  ENSURE(s, s->red, sizeof(double) * ((size_t)nblk_u + nblk_dir + nblk_up + 8));
  pcg_dev* sc = as<pcg_dev>(s->scal);
  double* part = as<double>(s->red);          // dir + SpMV partials
  double* part2 = part + nblk_dir + nblk_up;  // update partials
  pcg_dev h{};
  h.tol2 = tol * tol;
  const T* Mi = as<T>(s->minv);
  const T* D = as<T>(s->diag);
  // the iterations run on the library's own stream as CUDA graphs of
  // check_every iterations (3 kernels each), fenced to the caller's stream
  cudaStream_t cs = s->cstream;
  CK(s, cudaEventRecord(s->fence[0], s->stream));
  CK(s, cudaStreamWaitEvent(cs, s->fence[0], 0));
  CK(s, cudaMemcpyAsync(sc, &h, sizeof(pcg_dev), cudaMemcpyHostToDevice, cs));
  k_pcg_init<T, V><<<nblk_u, PT_, 0, cs>>>(s->nfree, s->nb, rhs, Mi, x, r, z, d, part, sc);
  LAUNCH_CHECK(s, "k_pcg_init");
  const int check_every = kPcgChunk;
  const double es = sizeof(T);
  const double spmv_bytes = (double)(s->Hs.nnzb + s->Hd.nnzb) * (9 * es + 4) + (double)s->nn * (9 * es + 4) +
                            4.0 * 3.0 * sizeof(V) * s->nn;
  const bool prof = s->prof_on;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  CK(s, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < check_every; ++k) {
    if (prof) cudaEventRecordWithFlags(s->spmv_ev[2 * k], cs, cudaEventRecordExternal);
    k_pcg_dir_dd<T, V><<<nblk_dir, PT_, 0, cs>>>(s->nn, D, z, d, q, sc, part);
    k_spmv_both<T, V><<<nblk_up, PT_, 0, cs>>>(s->Hs.nnzb, as<int>(s->Hs.row), as<int>(s->Hs.col), as<T>(s->Hs.vals),
                                               s->Hd.nnzb, as<int>(s->Hd.row), as<int>(s->Hd.col), as<T>(s->Hd.vals),
                                               d, q, sc, part, nblk_dir);
    if (prof) cudaEventRecordWithFlags(s->spmv_ev[2 * k + 1], cs, cudaEventRecordExternal);
    k_pcg_alpha_fin<<<1, 1024, 0, cs>>>(part, nblk_dir + nblk_up, sc);
    k_pcg_update<T, V><<<nblk_u, PT_, 0, cs>>>(s->nfree, s->nb, Mi, x, r, z, d, q, part2, sc);
    k_pcg_beta_fin<<<1, 1024, 0, cs>>>(part2, nblk_u, sc);
  }
  cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
  if (ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_check(s, ce, "PCG graph capture");
  }
  int it = 0;
  yasps_status rc = YASPS_OK;
  for (;;) {
    ce = cudaGraphLaunch(exec, cs);
    s->launches += 5LL * check_every;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, sc, sizeof(pcg_dev), cudaMemcpyDeviceToHost, cs);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
    if (ce != cudaSuccess) {
      rc = cuda_check(s, ce, "PCG graph launch");
      break;
    }
    if (prof) {  // only the products of iterations that really ran
      const int real = std::min(check_every, std::max(0, h.iters - it));
      for (int k = 0; k < real; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->spmv_ev[2 * k], s->spmv_ev[2 * k + 1]);
        auto& a = s->prof_acc[YASPS_STAGE_SPMV];
        a.count += 1;
        a.ms += ms;
        a.bytes += spmv_bytes;
      }
    }
    it += check_every;
    if (h.done || h.iters >= maxit || it >= maxit) break;
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  RC(rc);
  k_add_to<V><<<blocks_for(n3, 256), 256, 0, cs>>>(n3, p, x);
  LAUNCH_CHECK(s, "k_add_to");
  CK(s, cudaEventRecord(s->fence[1], cs));
  CK(s, cudaStreamWaitEvent(s->stream, s->fence[1], 0));
  *iters = h.iters;
  *state = h.done;
  *rel = (h.rz0 > 0.0) ? std::sqrt(std::max(h.rz, 0.0) / h.rz0) : 0.0;
  return YASPS_OK;
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
                            double* rel_res);

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
                       double* rel_res) {
  cudaEvent_t pa = prof_begin(s);
  yasps_status rc = pcg_solve_impl(s, rhs, p, tol, maxit, iters, rel_res);
  prof_end(s, YASPS_STAGE_PCG, pa, 0.0);
  return rc;
}

yasps_status pcg_solve_impl(yasps_system* s, const double* rhs, double* p, double tol, int maxit, int* iters,
                            double* rel_res) {
  const int n3 = 3 * s->nn;
  if (maxit <= 0) maxit = 10 * n3;
  CK(s, cudaMemsetAsync(p, 0, sizeof(double) * n3, s->stream));
  int it = 0, state = 0;
  double rel = 0.0;
  if (s->hess_precision != 1) {
    RC((pcg_inner<double, double>(s, rhs, p, tol, maxit, &it, &state, &rel)));
    if (iters) *iters = it;
    if (rel_res) *rel_res = rel;
    if (state == 2) SYS_FAIL(s, YASPS_E_NAN, "PCG breakdown: d^T H d <= 0");
    if (state != 1 && rel > tol) SYS_FAIL(s, YASPS_E_NOCONV, "PCG hit its iteration cap");
    return YASPS_OK;
  }
  // FP32-mixed: FP32 inner PCG, FP64 residual refinement
  ENSURE(s, s->vec[6], sizeof(double) * (n3 + 4));
  double* res = as<double>(s->vec[6]);
  double rz0 = 0.0, rz = 0.0;
  RC(rz64<float>(s, rhs, &rz0));
  if (!(rz0 > 0.0)) {
    if (iters) *iters = 0;
    if (rel_res) *rel_res = 0.0;
    return YASPS_OK;
  }
  rz = rz0;
  int total = 0;
  const int sweeps = std::max(1, s->prm.refine_sweeps);
  for (int sw = 0; sw < sweeps; ++sw) {
    const double inner_tol = std::max(tol * std::sqrt(rz0 / rz), 5e-6);
    if (sw == 0) {
      RC((pcg_inner<float, float>(s, rhs, p, inner_tol, maxit - total, &it, &state, &rel)));
    } else {
      RC((pcg_inner<float, float>(s, res, p, inner_tol, maxit - total, &it, &state, &rel)));
    }
    total += it;
    // FP64 residual res = rhs - H p
    RC(spmv64(s, p, res));
    k_sub_from<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, rhs, res);
    LAUNCH_CHECK(s, "k_sub_from");
    RC(rz64<float>(s, res, &rz));
    if (rz <= tol * tol * rz0 || total >= maxit || state == 2) break;
  }
  if (iters) *iters = total;
  const double r = std::sqrt(std::max(rz, 0.0) / rz0);
  if (rel_res) *rel_res = r;
  if (state == 2) SYS_FAIL(s, YASPS_E_NAN, "PCG breakdown: d^T H d <= 0");
  if (r > tol && total >= maxit) SYS_FAIL(s, YASPS_E_NOCONV, "PCG hit its iteration cap");
  return YASPS_OK;
}

yasps_status inf_norm(yasps_system* s, const double* x, int n, double* out_host) {
  const int nblk = std::min(148 * 2, blocks_for(std::max(n, 1), 256));
  ENSURE(s, s->red, sizeof(double) * (nblk + 8));
  k_absmax<<<nblk, 256, 0, s->stream>>>(n, x, as<double>(s->red));
  LAUNCH_CHECK(s, "k_absmax");
  std::vector<double> h(nblk);
  CK(s, cudaMemcpyAsync(h.data(), s->red.p, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  double m = 0.0;
  for (double v : h) m = std::max(m, v);
  *out_host = m;
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
