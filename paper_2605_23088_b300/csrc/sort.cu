// sort.cu -- device-wide exclusive scan, stable LSD radix sort of
// (64-bit key, int value) pairs, and the "gather block coordinates, sort
// lexicographically by (row, col), remove duplicates" construction of the
// compressed upper-triangular block layout (App. B, "Global Hessian
// Compression").
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

// exclusive scan of one value per thread across the block; *block_total gets the sum
__device__ int block_exclusive(int v, int* block_total) {
  __shared__ int warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const int before = (w > 0) ? warp_tot[w - 1] : 0;
  *block_total = warp_tot[nw - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void k_scan_reduce(const int* __restrict__ in, int n, int* __restrict__ bsum) {
  const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_I;
  int s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i)
    if (base + i < n) s += in[base + i];
  int tot;
  block_exclusive(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const int* in, int* out, int n, const int* __restrict__ boff, int* total) {
  const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_I;
  int v[SCAN_I];
  int s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  int tot;
  int run = block_exclusive(s, &tot) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
  for (int i = 0; i < SCAN_I; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *total = run;
}

// recursive scan; tmp holds the block sums of every level
yasps_status scan_rec(yasps_system* s, const int* in, int* out, int n, int* tmp, int* total_dev) {
  const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb <= 1) {
    k_scan_apply<<<1, SCAN_T, 0, s->stream>>>(in, out, n, nullptr, total_dev);
    LAUNCH_CHECK(s, "k_scan_apply");
    return YASPS_OK;
  }
  k_scan_reduce<<<nb, SCAN_T, 0, s->stream>>>(in, n, tmp);
  LAUNCH_CHECK(s, "k_scan_reduce");
  RC(scan_rec(s, tmp, tmp, nb, tmp + nb, nullptr));
  k_scan_apply<<<nb, SCAN_T, 0, s->stream>>>(in, out, n, tmp, total_dev);
  LAUNCH_CHECK(s, "k_scan_apply");
  return YASPS_OK;
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_T = 256, RS_ROUNDS = 16, RS_TILE = RS_T * RS_ROUNDS, RS_W = RS_T / 32;

__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int n, int shift, int* __restrict__ hist, int nblk) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const long long i = base + r * RS_T + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(int)((keys[i] >> shift) & 255u)], 1);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t* __restrict__ kin, const int* __restrict__ vin, uint64_t* __restrict__ kout,
                             int* __restrict__ vout, int n, int shift, const int* __restrict__ hist, int nblk) {
  __shared__ int off[256];
  __shared__ int wcnt[RS_W][257];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  off[tid] = hist[(long long)tid * nblk + blockIdx.x];
  const long long base = (long long)blockIdx.x * RS_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const long long i = base + r * RS_T + tid;
    const bool valid = i < n;
    uint64_t k = 0;
    int v = 0, d = 256;
    if (valid) {
      k = kin[i];
      v = vin[i];
      d = (int)((k >> shift) & 255u);
    }
#pragma unroll
    for (int q = 0; q < RS_W; ++q) wcnt[q][tid] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pos = off[d] + rank;
      for (int q = 0; q < w; ++q) pos += wcnt[q][d];
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
    int add = 0;
#pragma unroll
    for (int q = 0; q < RS_W; ++q) add += wcnt[q][tid];
    off[tid] += add;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- BSR from keys
__global__ void k_heads(const uint64_t* __restrict__ keys, int n, uint64_t sentinel, int* __restrict__ head) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  head[i] = (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
}
__global__ void k_bsr_fill(const uint64_t* __restrict__ keys, const int* __restrict__ vals, const int* __restrict__ pos,
                           int n, uint64_t sentinel, int nbits, int* __restrict__ col, int* __restrict__ row,
                           int* __restrict__ rowcnt, int* __restrict__ slot_of) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  if (k == sentinel) return;
  const bool head = (i == 0 || keys[i - 1] != k);
  const int u = pos[i] + (head ? 1 : 0) - 1;
  if (head) {
    const int r = (int)(k >> nbits), c = (int)(k & ((1ull << nbits) - 1ull));
    col[u] = c;
    row[u] = r;
    atomicAdd(&rowcnt[r], 1);
  }
  slot_of[vals[i]] = u;
}

}  // namespace

yasps_status scan_exclusive(yasps_system* s, const int* in, int* out, int n, int* total_host) {
  if (n <= 0) {
    if (total_host) *total_host = 0;
    return YASPS_OK;
  }
  // block sums of every level: n/2048 + n/2048^2 + ... < n/2000 + 8
  ENSURE(s, s->scan_tmp, sizeof(int) * ((size_t)n / 2000 + 64));
  int* tmp = as<int>(s->scan_tmp);
  int* total_dev = tmp + ((size_t)n / 2000 + 32);
  RC(scan_rec(s, in, out, n, tmp, total_dev));
  if (total_host) {
    CK(s, cudaMemcpyAsync(total_host, total_dev, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
  }
  return YASPS_OK;
}

// Small arrays (the dynamic contact keys: typically a few thousand): one
// block sorts (key, value) pairs in shared memory with a bitonic network,
// padded to a power of two with maximal entries.  Equal keys are ordered by
// value, so the result is a deterministic sort by key; one launch instead of
// a histogram, scan and scatter per 8-bit digit.
constexpr int kSmallSort = 16384;  // 12 bytes per entry: 192 KB of shared memory at most
__global__ void __launch_bounds__(1024) k_sort_small(uint64_t* __restrict__ keys, int* __restrict__ vals, int n, int m) {
  extern __shared__ __align__(16) unsigned char sort_smem[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(sort_smem);
  int* sv = reinterpret_cast<int*>(sk + m);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sk[i] = (i < n) ? keys[i] : ~0ull;
    sv[i] = (i < n) ? vals[i] : INT_MAX;
  }
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const uint64_t ka = sk[i], kb = sk[l];
          const int va = sv[i], vb = sv[l];
          const bool gt = (ka > kb) || (ka == kb && va > vb);
          if (gt == up) {
            sk[i] = kb; sk[l] = ka;
            sv[i] = vb; sv[l] = va;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    keys[i] = sk[i];
    vals[i] = sv[i];
  }
}

yasps_status radix_sort_pairs(yasps_system* s, uint64_t* keys, int* vals, uint64_t* keys_tmp, int* vals_tmp, int n,
                              int bits) {
  if (n <= 1) return YASPS_OK;
  if (n <= kSmallSort) {
    int m = 1;
    while (m < n) m <<= 1;  // padded size (a power of two)
    const size_t smem = (size_t)m * (sizeof(uint64_t) + sizeof(int));
    CK(s, cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)((size_t)kSmallSort * (sizeof(uint64_t) + sizeof(int)))));
    k_sort_small<<<1, 1024, smem, s->stream>>>(keys, vals, n, m);
    LAUNCH_CHECK(s, "k_sort_small");
    return YASPS_OK;
  }
  const int nblk = (n + RS_TILE - 1) / RS_TILE;
  gbuf& hist = s->ws[9];
  ENSURE(s, hist, sizeof(int) * 256 * (size_t)nblk);
  uint64_t *ka = keys, *kb = keys_tmp;
  int *va = vals, *vb = vals_tmp;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_rs_hist<<<nblk, RS_T, 0, s->stream>>>(ka, n, shift, as<int>(hist), nblk);
    LAUNCH_CHECK(s, "k_rs_hist");
    RC(scan_exclusive(s, as<int>(hist), as<int>(hist), 256 * nblk, nullptr));
    k_rs_scatter<<<nblk, RS_T, 0, s->stream>>>(ka, va, kb, vb, n, shift, as<int>(hist), nblk);
    LAUNCH_CHECK(s, "k_rs_scatter");
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    CK(s, cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s->stream));
    CK(s, cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, s->stream));
  }
  return YASPS_OK;
}

yasps_status bsr_from_keys(yasps_system* s, uint64_t* keys, int* vals, int n, bsr_struct& B, int* slot_of,
                           int n_contrib) {
  const int nbits = s->nbits;
  const uint64_t sent_id = (1ull << nbits) - 1ull;
  const uint64_t sentinel = (sent_id << nbits) | sent_id;
  if (n_contrib > 0) CK(s, cudaMemsetAsync(slot_of, 0xff, sizeof(int) * n_contrib, s->stream));
  ENSURE(s, B.row_ptr, sizeof(int) * (s->nn + 1));
  CK(s, cudaMemsetAsync(B.row_ptr.p, 0, sizeof(int) * (s->nn + 1), s->stream));
  if (n <= 0) {
    B.nnzb = 0;
    return YASPS_OK;
  }
  ENSURE(s, s->ws[6], sizeof(uint64_t) * n);
  ENSURE(s, s->ws[7], sizeof(int) * n);
  ENSURE(s, s->ws[8], sizeof(int) * n);
  RC(radix_sort_pairs(s, keys, vals, as<uint64_t>(s->ws[6]), as<int>(s->ws[7]), n, 2 * nbits));
  int* head = as<int>(s->ws[8]);
  k_heads<<<blocks_for(n, 256), 256, 0, s->stream>>>(keys, n, sentinel, head);
  LAUNCH_CHECK(s, "k_heads");
  int nnzb = 0;
  RC(scan_exclusive(s, head, head, n, &nnzb));
  B.nnzb = nnzb;
  ENSURE(s, B.col, sizeof(int) * (nnzb + 4));  // slack: bulk copies round up to 16 bytes
  ENSURE(s, B.row, sizeof(int) * (nnzb + 4));
  k_bsr_fill<<<blocks_for(n, 256), 256, 0, s->stream>>>(keys, vals, head, n, sentinel, nbits, as<int>(B.col),
                                                        as<int>(B.row), as<int>(B.row_ptr), slot_of);
  LAUNCH_CHECK(s, "k_bsr_fill");
  RC(scan_exclusive(s, as<int>(B.row_ptr), as<int>(B.row_ptr), s->nn + 1, nullptr));
  return YASPS_OK;
}
