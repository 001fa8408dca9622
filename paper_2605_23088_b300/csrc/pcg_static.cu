// pcg_static.cu -- block-Jacobi PCG on a caller-assembled block matrix that
// allocates no device memory.
//
// Who this is for: code that must not call cudaMalloc / cudaFree (or any
// allocating library routine) at solve time -- for example a solver step that
// runs inside another framework's fixed memory budget, a real-time loop that
// forbids allocation after start-up, or a host that hands us only its own
// buffers.  The caller passes the matrix, the right-hand side and the output;
// every temporary (the PCG vectors, the inverted diagonal blocks, reduction
// partials and scalars) lives in one file-scope __device__ array of fixed size,
// so the library never allocates on this path.
//
// Consequences of a shared fixed array:
//  * the array (about 11 MB) is held on every GPU that loads the library until
//    the process exits;
//  * problems larger than kMaxNodes nodes are rejected;
//  * every call uses the same array and leaves its contents behind; the call
//    clears what must start at zero itself, but two calls whose work overlaps
//    on the GPU (different streams, or different host threads on one device)
//    race on the array and give wrong results -- serialise them;
//  * the first call on a device looks up the array's device address (once per
//    device, with that device current); make that first call before any
//    stream capture;
//  * a call cannot itself be captured into a CUDA graph: it reads its
//    convergence scalars back to the host every 8 iterations;
//  * p_dev must not alias rhs_dev or any other input (the call zeroes p before
//    it has finished reading rhs).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "yasps.h"

namespace {

constexpr int kMaxNodes = 65536;
constexpr int kN3 = 3 * kMaxNodes;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = (kMaxNodes + kThreads - 1) / kThreads;  // node-parallel kernels
constexpr int kDotBlocks = 256;
// layout (doubles): r z d q | Minv (9 per node) | partials | scalars
constexpr size_t kOffR = 0, kOffZ = kN3, kOffD = 2 * (size_t)kN3, kOffQ = 3 * (size_t)kN3;
constexpr size_t kOffM = 4 * (size_t)kN3;
constexpr size_t kOffPart = kOffM + 9 * (size_t)kMaxNodes;
constexpr size_t kOffScal = kOffPart + 1024;
constexpr size_t kScratchDoubles = kOffScal + 16;

static __device__ __align__(256) double g_pcg_scratch[kScratchDoubles];

struct scal {  // lives at g_pcg_scratch + kOffScal
  double rz, rz0, alpha, beta, tol2;
  int done, iters;  // done: 0 running, 1 converged, 2 d^T H d <= 0, 3 iteration cap
  int max_iter;
};
// bits of the flag word (the last double of the array)
constexpr int kBadDiag = 1;   // a diagonal block that is not positive definite
constexpr int kBadIndex = 2;  // an upper block outside 0 <= row < col < n_nodes
static_assert(sizeof(scal) <= 16 * sizeof(double), "scalar block too large");

__device__ double blk_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// invert the 3x3 diagonal blocks; r = rhs, p = 0, d = 0, z = M^-1 r, partial r.z
__global__ void ks_init(int nn, const double* __restrict__ diag, const double* __restrict__ rhs, double* __restrict__ p,
                        double* S, double tol2, int max_iter, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double* r = S + kOffR;
  double* z = S + kOffZ;
  double* d = S + kOffD;
  double* M = S + kOffM;
  double acc = 0.0;
  if (i < nn) {
    const double* A = diag + 9 * (size_t)i;
    const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    double inv[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    // Sylvester's criterion: a symmetric 3x3 block is positive definite iff
    // its leading minors A00, A00 A11 - A01 A10 and det are all positive
    const double m2 = A[0] * A[4] - A[1] * A[3];
    if (A[0] > 0.0 && m2 > 0.0 && det > 0.0 && isfinite(det)) {
      inv[0] = c00 / det; inv[1] = (A[2] * A[7] - A[1] * A[8]) / det; inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
      inv[3] = c01 / det; inv[4] = (A[0] * A[8] - A[2] * A[6]) / det; inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
      inv[6] = c02 / det; inv[7] = (A[1] * A[6] - A[0] * A[7]) / det; inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    } else {
      atomicOr(bad, kBadDiag);
    }
    for (int t = 0; t < 9; ++t) M[9 * (size_t)i + t] = inv[t];
    for (int a = 0; a < 3; ++a) {
      r[3 * i + a] = rhs[3 * i + a];
      p[3 * i + a] = 0.0;
      d[3 * i + a] = 0.0;
    }
    for (int a = 0; a < 3; ++a) {
      const double za = inv[3 * a] * rhs[3 * i] + inv[3 * a + 1] * rhs[3 * i + 1] + inv[3 * a + 2] * rhs[3 * i + 2];
      z[3 * i + a] = za;
      acc += za * rhs[3 * i + a];
    }
  }
  acc = blk_sum(acc);
  if (threadIdx.x == 0) S[kOffPart + blockIdx.x] = acc;
  if (i == 0) {
    scal* sc = reinterpret_cast<scal*>(S + kOffScal);
    sc->tol2 = tol2;
    sc->beta = 0.0;
    sc->iters = 0;
    sc->done = 0;
    sc->max_iter = max_iter;
  }
}

// single block: total of the partials into rz (init) or, after an update, beta
__global__ void ks_finish_rz(int nparts, double* S, int first) {
  double v = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) v += S[kOffPart + k];
  v = blk_sum(v);
  if (threadIdx.x == 0) {
    scal* sc = reinterpret_cast<scal*>(S + kOffScal);
    if (first) {
      sc->rz = v;
      sc->rz0 = v;
      // r0 = 0 exactly: p = 0 is the solution; a negative or NaN r^T z means
      // an indefinite preconditioner block or a non-finite right-hand side
      if (v == 0.0) sc->done = 1;
      else if (!(v > 0.0)) sc->done = 2;
    } else if (!sc->done) {
      sc->beta = v / sc->rz;
      sc->rz = v;
      sc->iters += 1;
      if (v <= sc->tol2 * sc->rz0) sc->done = 1;
      else if (!(v == v)) sc->done = 2;
      else if (sc->iters >= sc->max_iter) sc->done = 3;
    }
  }
}

// d = z + beta d ; q = D d
__global__ void ks_dir(int nn, const double* __restrict__ diag, double* S) {
  const scal* sc = reinterpret_cast<const scal*>(S + kOffScal);
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double beta = sc->beta;
  double* z = S + kOffZ;
  double* d = S + kOffD;
  double* q = S + kOffQ;
  double dv[3];
  for (int a = 0; a < 3; ++a) {
    dv[a] = z[3 * i + a] + beta * d[3 * i + a];
    d[3 * i + a] = dv[a];
  }
  const double* B = diag + 9 * (size_t)i;
  for (int a = 0; a < 3; ++a) q[3 * i + a] = B[3 * a] * dv[0] + B[3 * a + 1] * dv[1] + B[3 * a + 2] * dv[2];
}

// q += U d + U^T d over upper blocks (row < col), one block per thread; a
// block outside 0 <= row < col < nn is skipped and flagged (the call then
// fails with YASPS_E_INVAL), so a bad index never addresses the array
__global__ void ks_upper(int nn, int nnzb, const int* __restrict__ row, const int* __restrict__ col,
                         const double* __restrict__ vals, double* S, int* bad) {
  const scal* sc = reinterpret_cast<const scal*>(S + kOffScal);
  if (sc->done) return;
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnzb) return;
  const double* d = S + kOffD;
  double* q = S + kOffQ;
  const int r = row[k], c = col[k];
  if (r < 0 || r >= c || c >= nn) {
    atomicOr(bad, kBadIndex);
    return;
  }
  const double* B = vals + 9 * (size_t)k;
  for (int a = 0; a < 3; ++a) {
    atomicAdd(&q[3 * r + a], B[3 * a] * d[3 * c] + B[3 * a + 1] * d[3 * c + 1] + B[3 * a + 2] * d[3 * c + 2]);
    atomicAdd(&q[3 * c + a], B[a] * d[3 * r] + B[3 + a] * d[3 * r + 1] + B[6 + a] * d[3 * r + 2]);
  }
}

__global__ void ks_dot_dq(int n3, double* S) {
  const scal* sc = reinterpret_cast<const scal*>(S + kOffScal);
  if (sc->done) return;
  const double* d = S + kOffD;
  const double* q = S + kOffQ;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) acc += d[i] * q[i];
  acc = blk_sum(acc);
  if (threadIdx.x == 0) S[kOffPart + blockIdx.x] = acc;
}
__global__ void ks_alpha(int nparts, double* S) {
  scal* sc = reinterpret_cast<scal*>(S + kOffScal);
  if (sc->done) return;
  double v = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) v += S[kOffPart + k];
  v = blk_sum(v);
  if (threadIdx.x == 0) {
    if (v > 0.0) sc->alpha = sc->rz / v;
    else sc->done = 2;  // d^T H d <= 0: the matrix is not positive definite
  }
}

// p += alpha d, r -= alpha q, z = M^-1 r, partial r.z
__global__ void ks_update(int nn, double* __restrict__ p, double* S) {
  const scal* sc = reinterpret_cast<const scal*>(S + kOffScal);
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < nn) {
    const double alpha = sc->alpha;
    double* r = S + kOffR;
    double* z = S + kOffZ;
    const double* d = S + kOffD;
    const double* q = S + kOffQ;
    const double* M = S + kOffM + 9 * (size_t)i;
    for (int a = 0; a < 3; ++a) {
      p[3 * i + a] += alpha * d[3 * i + a];
      r[3 * i + a] -= alpha * q[3 * i + a];
    }
    for (int a = 0; a < 3; ++a) {
      const double za = M[3 * a] * r[3 * i] + M[3 * a + 1] * r[3 * i + 1] + M[3 * a + 2] * r[3 * i + 2];
      z[3 * i + a] = za;
      acc += za * r[3 * i + a];
    }
  }
  acc = blk_sum(acc);
  if (threadIdx.x == 0) S[kOffPart + blockIdx.x] = acc;
}

// per-device address of g_pcg_scratch (a host-side name is not a device address)
std::mutex g_mu;
double* g_dev_ptr[64] = {};

void set_err(char* buf, int len, const char* msg) {
  if (buf && len > 0) snprintf(buf, (size_t)len, "%s", msg);
}

}  // namespace

extern "C" yasps_status yasps_pcg_solve_static(int n_nodes, int nnzb, const int* row_dev, const int* col_dev,
                                               const double* vals_dev, const double* diag_dev, const double* rhs_dev,
                                               double* p_dev, double rel_tol, int max_iter, void* cuda_stream,
                                               int* iters, double* rel_res, char* err, int err_len) {
  if (n_nodes < 0 || nnzb < 0 || (n_nodes > 0 && (!diag_dev || !rhs_dev || !p_dev)) ||
      (nnzb > 0 && (!row_dev || !col_dev || !vals_dev))) {
    set_err(err, err_len, "yasps_pcg_solve_static: bad arguments");
    return YASPS_E_INVAL;
  }
  if (n_nodes > 0 && (p_dev == rhs_dev || p_dev == diag_dev || (nnzb > 0 && p_dev == vals_dev))) {
    set_err(err, err_len, "yasps_pcg_solve_static: p_dev must not alias an input");
    return YASPS_E_INVAL;
  }
  if (n_nodes > kMaxNodes) {
    char m[160];
    snprintf(m, sizeof m, "yasps_pcg_solve_static: %d nodes exceed the fixed scratch capacity of %d nodes", n_nodes,
             kMaxNodes);
    set_err(err, err_len, m);
    return YASPS_E_CAPACITY;
  }
  if (iters) *iters = 0;
  if (rel_res) *rel_res = 0.0;
  if (n_nodes == 0) return YASPS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    set_err(err, err_len, "yasps_pcg_solve_static: no current CUDA device");
    return YASPS_E_CUDA;
  }
  double* S = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_pcg_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        set_err(err, err_len, "yasps_pcg_solve_static: cudaGetSymbolAddress of the scratch array failed");
        return YASPS_E_CUDA;
      }
      g_dev_ptr[dev] = static_cast<double*>(ptr);
    }
    S = g_dev_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int n3 = 3 * n_nodes;
  if (max_iter <= 0) max_iter = 10 * n3;
  const int nblk = (n_nodes + kThreads - 1) / kThreads;
  // a flag word for singular diagonal blocks: the last scalar slot
  int* bad = reinterpret_cast<int*>(S + kScratchDoubles - 1);
  if (cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    set_err(err, err_len, "yasps_pcg_solve_static: cudaMemsetAsync failed");
    return YASPS_E_CUDA;
  }
  ks_init<<<nblk, kThreads, 0, st>>>(n_nodes, diag_dev, rhs_dev, p_dev, S, rel_tol * rel_tol, max_iter, bad);
  ks_finish_rz<<<1, kThreads, 0, st>>>(nblk, S, 1);
  scal h{};
  int bad_h = 0;
  int launched = 0;
  for (;;) {
    for (int k = 0; k < 8; ++k) {
      ks_dir<<<nblk, kThreads, 0, st>>>(n_nodes, diag_dev, S);
      if (nnzb > 0)
        ks_upper<<<(nnzb + kThreads - 1) / kThreads, kThreads, 0, st>>>(n_nodes, nnzb, row_dev, col_dev, vals_dev, S,
                                                                        bad);
      ks_dot_dq<<<kDotBlocks, kThreads, 0, st>>>(n3, S);
      ks_alpha<<<1, kThreads, 0, st>>>(kDotBlocks, S);
      ks_update<<<nblk, kThreads, 0, st>>>(n_nodes, p_dev, S);
      ks_finish_rz<<<1, kThreads, 0, st>>>(nblk, S, 0);
    }
    launched += 8;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, S + kOffScal, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_err(err, err_len, cudaGetErrorString(e));
      return YASPS_E_CUDA;
    }
    if (h.done || (bad_h & kBadIndex) || launched >= max_iter) break;
  }
  if (iters) *iters = h.iters;
  const double rr = (h.rz0 > 0.0) ? std::sqrt(std::fmax(h.rz, 0.0) / h.rz0) : 0.0;
  if (rel_res) *rel_res = rr;
  if (bad_h & kBadIndex) {
    set_err(err, err_len, "yasps_pcg_solve_static: an upper block is outside 0 <= row < col < n_nodes");
    return YASPS_E_INVAL;
  }
  if ((bad_h & kBadDiag) || h.done == 2) {
    set_err(err, err_len,
            "yasps_pcg_solve_static: matrix not positive definite or non-finite input (indefinite diagonal block, "
            "r^T z <= 0 or NaN, or d^T H d <= 0)");
    return YASPS_E_NAN;
  }
  if (h.done != 1 && rr > rel_tol) {
    set_err(err, err_len, "yasps_pcg_solve_static: iteration cap reached");
    return YASPS_E_NOCONV;
  }
  return YASPS_OK;
}
