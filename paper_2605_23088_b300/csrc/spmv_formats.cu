// spmv_formats.cu -- the SpMV layout study (Sec. "Evaluation", the SpMV
// experiment; App. "SpMV"): y = A x for a symmetric 3x3-block matrix A =
// D + A_off held in one of four layouts, each with its own kernel, on caller
// arrays.  The library's PCG uses the first (upper blocks only, sorted by row,
// a per-block row index, rows reduced by a warp-segmented shuffle, transposes
// by atomics); the others are the alternatives the experiment compares it
// with: every off-diagonal block stored (no transposes, twice the blocks),
// and coordinate lists where every block adds its products with atomics.
#include <cuda_runtime.h>

#include "common.cuh"
#include "yasps.h"

namespace {

template <typename T, typename V>
__global__ void ks_diag(int nn, const T* __restrict__ D, const V* __restrict__ x, V* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const T* B = D + 9 * (size_t)i;
  const V x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
#pragma unroll
  for (int a = 0; a < 3; ++a) y[3 * i + a] = (V)B[3 * a] * x0 + (V)B[3 * a + 1] * x1 + (V)B[3 * a + 2] * x2;
}

template <typename V>
__device__ __forceinline__ V shfl_dn(V v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }

// one block per thread: B x_col into y_row (row-segmented warp reduction when
// SEG, one atomic per component and block otherwise) and, when SYM, B^T x_row
// into y_col by atomics
template <typename T, typename V, bool SEG, bool SYM>
__global__ void __launch_bounds__(256) ks_blocks(int nnzb, int nn, const int* __restrict__ row,
                                                 const int* __restrict__ col, const T* __restrict__ vals,
                                                 const V* __restrict__ x, V* __restrict__ y, int* __restrict__ bad) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int r = -1;
  V a0 = 0, a1 = 0, a2 = 0;
  if (k < nnzb) {
    r = row[k];
    const int c = col[k];
    if (r < 0 || r >= nn || c < 0 || c >= nn || (SYM && r >= c) || (!SYM && r == c)) {
      atomicOr(bad, 1);
      r = -1;
    } else {
      const T* B = vals + 9 * (size_t)k;
      T b[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) b[t] = B[t];
      const V xc0 = x[3 * c], xc1 = x[3 * c + 1], xc2 = x[3 * c + 2];
      a0 = (V)b[0] * xc0 + (V)b[1] * xc1 + (V)b[2] * xc2;
      a1 = (V)b[3] * xc0 + (V)b[4] * xc1 + (V)b[5] * xc2;
      a2 = (V)b[6] * xc0 + (V)b[7] * xc1 + (V)b[8] * xc2;
      if (SYM) {
        const V xr0 = x[3 * r], xr1 = x[3 * r + 1], xr2 = x[3 * r + 2];
        atomicAdd(&y[3 * c], (V)b[0] * xr0 + (V)b[3] * xr1 + (V)b[6] * xr2);
        atomicAdd(&y[3 * c + 1], (V)b[1] * xr0 + (V)b[4] * xr1 + (V)b[7] * xr2);
        atomicAdd(&y[3 * c + 2], (V)b[2] * xr0 + (V)b[5] * xr1 + (V)b[8] * xr2);
      }
    }
  }
  if (SEG) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ro = __shfl_down_sync(0xffffffffu, r, o);
      const V b0 = shfl_dn(a0, o), b1 = shfl_dn(a1, o), b2 = shfl_dn(a2, o);
      if (lane + o < 32 && ro == r) { a0 += b0; a1 += b1; a2 += b2; }
    }
    const int rp = __shfl_up_sync(0xffffffffu, r, 1);
    if (r >= 0 && (lane == 0 || rp != r)) {
      atomicAdd(&y[3 * r], a0);
      atomicAdd(&y[3 * r + 1], a1);
      atomicAdd(&y[3 * r + 2], a2);
    }
  } else if (r >= 0) {
    atomicAdd(&y[3 * r], a0);
    atomicAdd(&y[3 * r + 1], a1);
    atomicAdd(&y[3 * r + 2], a2);
  }
}

template <typename T>
yasps_status run(int format, int nn, int nnzb, const int* row, const int* col, const void* vals, const void* diag,
                 const void* x, void* y, cudaStream_t st, int* bad) {
  const T* D = static_cast<const T*>(diag);
  const T* Vv = static_cast<const T*>(vals);
  const T* X = static_cast<const T*>(x);
  T* Y = static_cast<T*>(y);
  if (nn > 0) ks_diag<T, T><<<blocks_for(nn, 256), 256, 0, st>>>(nn, D, X, Y);
  if (nnzb > 0) {
    const int g = blocks_for(nnzb, 256);
    switch (format) {
      case YASPS_SPMV_UPPER_BSR: ks_blocks<T, T, true, true><<<g, 256, 0, st>>>(nnzb, nn, row, col, Vv, X, Y, bad); break;
      case YASPS_SPMV_FULL_BSR: ks_blocks<T, T, true, false><<<g, 256, 0, st>>>(nnzb, nn, row, col, Vv, X, Y, bad); break;
      case YASPS_SPMV_FULL_BCOO: ks_blocks<T, T, false, false><<<g, 256, 0, st>>>(nnzb, nn, row, col, Vv, X, Y, bad); break;
      default: ks_blocks<T, T, false, true><<<g, 256, 0, st>>>(nnzb, nn, row, col, Vv, X, Y, bad); break;
    }
  }
  return cudaGetLastError() == cudaSuccess ? YASPS_OK : YASPS_E_CUDA;
}

}  // namespace

extern "C" yasps_status yasps_spmv_format(int format, int precision, int n_nodes, int nnzb, const int* row_dev,
                                          const int* col_dev, const void* vals_dev, const void* diag_dev,
                                          const void* x_dev, void* y_dev, int* flag_dev, void* cuda_stream) {
  if (format < 0 || format > 3 || (precision != 0 && precision != 1) || n_nodes < 0 || nnzb < 0 ||
      (n_nodes > 0 && (!diag_dev || !x_dev || !y_dev)) || (nnzb > 0 && (!row_dev || !col_dev || !vals_dev || !flag_dev)))
    return YASPS_E_INVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return precision == 0 ? run<double>(format, n_nodes, nnzb, row_dev, col_dev, vals_dev, diag_dev, x_dev, y_dev, st, flag_dev)
                        : run<float>(format, n_nodes, nnzb, row_dev, col_dev, vals_dev, diag_dev, x_dev, y_dev, st, flag_dev);
}
