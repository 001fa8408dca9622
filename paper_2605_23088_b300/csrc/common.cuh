// common.cuh -- device helpers shared by the library's kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "yasps.h"

#define YASPS_HD __host__ __device__ __forceinline__
#define YASPS_D __device__ __forceinline__

// Device-side error bits latched into the system's status word.
enum : int {
  DEV_OK = 0,
  DEV_CAPACITY = 1,  // a bounded list overflowed
  DEV_NAN = 2,       // non-finite value produced
  DEV_BADINDEX = 4,  // index out of range
  DEV_ITERCAP = 8,   // an iteration cap was reached (ACCD)
  DEV_TIMEOUT = 16,  // a bounded grid-barrier wait gave up
  DEV_INDEFINITE = 32,  // a block-Jacobi block is not positive definite (exact Hessians can be)
};

YASPS_D void dev_flag(int* status, int code) { atomicOr(status, code); }

inline int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 0x7fffffffLL) b = 0x7fffffffLL;
  return (int)b;
}

// ---------------------------------------------------------------- small vectors
template <typename T>
struct v3 {
  T x, y, z;
};
template <typename T>
YASPS_HD v3<T> operator+(v3<T> a, v3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
YASPS_HD v3<T> operator-(v3<T> a, v3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
YASPS_HD v3<T> operator*(T s, v3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T>
YASPS_HD T dot(v3<T> a, v3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
YASPS_HD v3<T> cross(v3<T> a, v3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

template <typename T>
YASPS_HD T comp3(v3<T> a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

YASPS_D v3<double> ld3(const double* p, int i) { return {p[3 * i], p[3 * i + 1], p[3 * i + 2]}; }
YASPS_D void st3(double* p, int i, v3<double> a) {
  p[3 * i] = a.x;
  p[3 * i + 1] = a.y;
  p[3 * i + 2] = a.z;
}

// Neumaier-compensated (value, compensation) pair for FP64 energy sums.
struct ksum {
  double s, c;
};
YASPS_HD void kadd(ksum& k, double v) {
  double t = k.s + v;
  if (fabs(k.s) >= fabs(v))
    k.c += (k.s - t) + v;
  else
    k.c += (v - t) + k.s;
  k.s = t;
}
YASPS_HD void kmerge(ksum& a, const ksum& b) {
  kadd(a, b.s);
  kadd(a, b.c);
}

// ---------------------------------------------------------------- warp helpers
YASPS_D double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
YASPS_D float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
YASPS_D double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// tree reduction of compensated sums down to lane 0 (fixed order: deterministic)
YASPS_D ksum warp_ksum(ksum k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ksum other{__shfl_down_sync(0xffffffffu, k.s, o), __shfl_down_sync(0xffffffffu, k.c, o)};
    kmerge(k, other);
  }
  return k;
}
// Block-wide compensated reduction; result valid in thread 0.  blockDim.x must
// be a multiple of 32 and at most 1024.
// Batches: warp-segmented FP64 sum over runs of equal keys (the runs must be
// contiguous across the lanes, as sorted keys are); the head lane of each run
// adds the run's sum into acc[key]; key < 0 adds nothing.  All 32 lanes of the
// warp must call.
YASPS_D void seg_add_global(double* acc, int key, double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int ko = __shfl_down_sync(0xffffffffu, key, off);
    const double vo = __shfl_down_sync(0xffffffffu, v, off);
    if (lane + off < 32 && ko == key) v += vo;
  }
  const int kp = __shfl_up_sync(0xffffffffu, key, 1);
  if (key >= 0 && (lane == 0 || kp != key)) atomicAdd(&acc[key], v);
}

YASPS_D ksum block_ksum(ksum k) {
  __shared__ double sh_s[32], sh_c[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  k = warp_ksum(k);
  if (lane == 0) { sh_s[w] = k.s; sh_c[w] = k.c; }
  __syncthreads();
  ksum r{0.0, 0.0};
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    if (lane < nw) r = ksum{sh_s[lane], sh_c[lane]};
    r = warp_ksum(r);
  }
  __syncthreads();
  return r;
}
