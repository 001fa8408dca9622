// eig.cuh -- PSD projection of small symmetric matrices on the device.
//
// Sec. "EVD and PSD Projection": Project(H) = V max(Lambda, 0) V^T, i.e. the
// negative eigenvalues of the local Hessian are set to zero.  Project(H) is
// unique even where eigenvectors are not, so any exact EVD gives the same
// matrix.  This is a cyclic Jacobi eigensolver specialised at compile time for
// the sizes the path needs (3k x 3k with k = 2, 3, 4 and the 6/9 F-spaces):
// every (p, q, k) loop is unrolled so that the matrix and the rotation
// accumulator stay in registers when they fit.
#pragma once
#include "common.cuh"

template <typename T>
struct eig_traits;
template <>
struct eig_traits<double> {
  static constexpr int max_sweeps = 12;
  static constexpr double rel_eps2 = 1e-30;  // stop when off(A)^2 <= eps^2 ||A||^2
};
template <>
struct eig_traits<float> {
  static constexpr int max_sweeps = 8;
  static constexpr float rel_eps2 = 1e-13f;
};

YASPS_D double jacobi_c(double t) { return 1.0 / sqrt(t * t + 1.0); }
YASPS_D float jacobi_c(float t) { return rsqrtf(t * t + 1.0f); }

// In place: A (N x N, row-major, symmetric) <- Project(A).
template <int N, typename T>
YASPS_D void project_psd(T* A) {
  T V[N * N];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) V[i * N + j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < eig_traits<T>::max_sweeps; ++sweep) {
    T off = 0, tot = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) {
      tot += A[p * N + p] * A[p * N + p];
#pragma unroll
      for (int q = p + 1; q < N; ++q) off += A[p * N + q] * A[p * N + q];
    }
    tot += T(2) * off;
    if (!(off > eig_traits<T>::rel_eps2 * tot)) break;
#pragma unroll
    for (int p = 0; p < N - 1; ++p) {
#pragma unroll
      for (int q = p + 1; q < N; ++q) {
        const T apq = A[p * N + q];
        if (apq != T(0)) {
          const T theta = (A[q * N + q] - A[p * N + p]) / (T(2) * apq);
          const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
          const T c = jacobi_c(t), s = t * c;
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const T akp = A[k * N + p], akq = A[k * N + q];
            A[k * N + p] = c * akp - s * akq;
            A[k * N + q] = s * akp + c * akq;
          }
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const T apk = A[p * N + k], aqk = A[q * N + k];
            A[p * N + k] = c * apk - s * aqk;
            A[q * N + k] = s * apk + c * aqk;
          }
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const T vkp = V[k * N + p], vkq = V[k * N + q];
            V[k * N + p] = c * vkp - s * vkq;
            V[k * N + q] = s * vkp + c * vkq;
          }
        }
      }
    }
  }
  T w[N];
#pragma unroll
  for (int k = 0; k < N; ++k) w[k] = A[k * N + k] > T(0) ? A[k * N + k] : T(0);
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      T s = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) s += V[i * N + k] * w[k] * V[j * N + k];
      A[i * N + j] = s;
      A[j * N + i] = s;
    }
}

// Eigen-decomposition of a small symmetric matrix: on return A's diagonal holds
// the eigenvalues and V's columns the eigenvectors (same cyclic Jacobi sweeps).
template <int N, typename T>
YASPS_D void eig_sym(T* A, T* V) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) V[i * N + j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < eig_traits<T>::max_sweeps; ++sweep) {
    T off = 0, tot = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) {
      tot += A[p * N + p] * A[p * N + p];
#pragma unroll
      for (int q = p + 1; q < N; ++q) off += A[p * N + q] * A[p * N + q];
    }
    tot += T(2) * off;
    if (!(off > eig_traits<T>::rel_eps2 * tot)) break;
#pragma unroll
    for (int p = 0; p < N - 1; ++p) {
#pragma unroll
      for (int q = p + 1; q < N; ++q) {
        const T apq = A[p * N + q];
        if (apq != T(0)) {
          const T theta = (A[q * N + q] - A[p * N + p]) / (T(2) * apq);
          const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
          const T c = jacobi_c(t), s = t * c;
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const T akp = A[k * N + p], akq = A[k * N + q];
            A[k * N + p] = c * akp - s * akq;
            A[k * N + q] = s * akp + c * akq;
          }
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const T apk = A[p * N + k], aqk = A[q * N + k];
            A[p * N + k] = c * apk - s * aqk;
            A[q * N + k] = s * apk + c * aqk;
          }
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const T vkp = V[k * N + p], vkq = V[k * N + q];
            V[k * N + p] = c * vkp - s * vkq;
            V[k * N + q] = s * vkp + c * vkq;
          }
        }
      }
    }
  }
}
