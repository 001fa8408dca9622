// bend.cu -- discrete-shell bending of cloth hinges (Grinspun et al. 2003):
//   Psi = kb (theta - theta_rest)^2 * 3 |e_rest|^2 / (A1_rest + A2_rest),
// theta the signed angle between the normals of the two triangles about the
// shared edge.  The gradient and Hessian of theta over the 12 hinge DOF are
// carried through the evaluation of theta by second-order forward-mode
// differentiation (value, gradient, packed upper-triangular Hessian), then
// Psi's Hessian 2 k w (grad theta grad theta^T + (theta - theta0) hess theta) is
// projected in the hinge's own 12-dim space.
#include "common.cuh"
#include "eig.cuh"
#include "internal.h"

namespace {

constexpr int NJ = 12, NH = NJ * (NJ + 1) / 2;

struct jet {
  double v;
  double g[NJ];
  double h[NH];  // packed upper triangle, row-major
};
__device__ __forceinline__ int hidx(int i, int j) { return i * NJ - i * (i - 1) / 2 + (j - i); }  // i <= j

__device__ jet jconst(double c) {
  jet r;
  r.v = c;
  for (int i = 0; i < NJ; ++i) r.g[i] = 0.0;
  for (int i = 0; i < NH; ++i) r.h[i] = 0.0;
  return r;
}
__device__ jet jvar(double c, int k) {
  jet r = jconst(c);
  r.g[k] = 1.0;
  return r;
}
__device__ jet operator+(const jet& a, const jet& b) {
  jet r;
  r.v = a.v + b.v;
  for (int i = 0; i < NJ; ++i) r.g[i] = a.g[i] + b.g[i];
  for (int i = 0; i < NH; ++i) r.h[i] = a.h[i] + b.h[i];
  return r;
}
__device__ jet operator-(const jet& a, const jet& b) {
  jet r;
  r.v = a.v - b.v;
  for (int i = 0; i < NJ; ++i) r.g[i] = a.g[i] - b.g[i];
  for (int i = 0; i < NH; ++i) r.h[i] = a.h[i] - b.h[i];
  return r;
}
__device__ jet operator*(const jet& a, const jet& b) {
  jet r;
  r.v = a.v * b.v;
  for (int i = 0; i < NJ; ++i) r.g[i] = a.v * b.g[i] + b.v * a.g[i];
  for (int i = 0; i < NJ; ++i)
    for (int j = i; j < NJ; ++j) {
      const int k = hidx(i, j);
      r.h[k] = a.v * b.h[k] + b.v * a.h[k] + a.g[i] * b.g[j] + a.g[j] * b.g[i];
    }
  return r;
}
// r = f(a) given f, f', f''
__device__ jet junary(const jet& a, double f, double df, double d2f) {
  jet r;
  r.v = f;
  for (int i = 0; i < NJ; ++i) r.g[i] = df * a.g[i];
  for (int i = 0; i < NJ; ++i)
    for (int j = i; j < NJ; ++j) {
      const int k = hidx(i, j);
      r.h[k] = df * a.h[k] + d2f * a.g[i] * a.g[j];
    }
  return r;
}
__device__ jet jsqrt(const jet& a) {
  const double s = sqrt(a.v);
  return junary(a, s, 0.5 / s, -0.25 / (s * a.v));
}
__device__ jet jinv(const jet& a) { return junary(a, 1.0 / a.v, -1.0 / (a.v * a.v), 2.0 / (a.v * a.v * a.v)); }
// theta = atan2(y, x)
__device__ jet jatan2(const jet& y, const jet& x) {
  const double r2 = x.v * x.v + y.v * y.v, r4 = r2 * r2;
  const double ty = x.v / r2, tx = -y.v / r2;
  const double tyy = -2.0 * x.v * y.v / r4, txx = 2.0 * x.v * y.v / r4, txy = (y.v * y.v - x.v * x.v) / r4;
  jet r;
  r.v = atan2(y.v, x.v);
  for (int i = 0; i < NJ; ++i) r.g[i] = ty * y.g[i] + tx * x.g[i];
  for (int i = 0; i < NJ; ++i)
    for (int j = i; j < NJ; ++j) {
      const int k = hidx(i, j);
      r.h[k] = ty * y.h[k] + tx * x.h[k] + tyy * y.g[i] * y.g[j] + txx * x.g[i] * x.g[j] +
               txy * (x.g[i] * y.g[j] + y.g[i] * x.g[j]);
    }
  return r;
}
struct jv3 {
  jet c[3];
};
__device__ jv3 jsub3(const jv3& a, const jv3& b) {
  jv3 r;
  for (int k = 0; k < 3; ++k) r.c[k] = a.c[k] - b.c[k];
  return r;
}
__device__ jet jdot3(const jv3& a, const jv3& b) { return a.c[0] * b.c[0] + a.c[1] * b.c[1] + a.c[2] * b.c[2]; }
__device__ jv3 jcross3(const jv3& a, const jv3& b) {
  jv3 r;
  r.c[0] = a.c[1] * b.c[2] - a.c[2] * b.c[1];
  r.c[1] = a.c[2] * b.c[0] - a.c[0] * b.c[2];
  r.c[2] = a.c[0] * b.c[1] - a.c[1] * b.c[0];
  return r;
}

template <typename T>
__global__ void __launch_bounds__(64) k_bend(int nh, const int* __restrict__ hv, const int* __restrict__ hn,
                                            const double* __restrict__ hrest, const int* __restrict__ hslot,
                                            const double* __restrict__ P, double h2, int project, double* __restrict__ g,
                                            T* __restrict__ diag, T* __restrict__ vals) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nh) return;
  jv3 X[4];
  for (int a = 0; a < 4; ++a) {
    const int v = hv[4 * e + a];
    for (int c = 0; c < 3; ++c) X[a].c[c] = jvar(P[3 * v + c], 3 * a + c);
  }
  const jv3 ed = jsub3(X[1], X[0]);
  const jv3 n1 = jcross3(ed, jsub3(X[2], X[0]));
  const jv3 n2 = jcross3(jsub3(X[0], X[1]), jsub3(X[3], X[1]));
  const jet le = jsqrt(jdot3(ed, ed));
  const jet sn = jdot3(jcross3(n1, n2), ed) * jinv(le);
  const jet th = jatan2(sn, jdot3(n1, n2));
  const double dth = th.v - hrest[2 * e];
  const double kw = hrest[2 * e + 1] * h2;
  int nodes[4];
  for (int a = 0; a < 4; ++a) nodes[a] = hn[4 * e + a];
  for (int a = 0; a < 4; ++a) {
    if (nodes[a] < 0) continue;
    for (int c = 0; c < 3; ++c) atomicAdd(&g[3 * nodes[a] + c], 2.0 * kw * dth * th.g[3 * a + c]);
  }
  T H[144];
  for (int i = 0; i < NJ; ++i)
    for (int j = i; j < NJ; ++j) {
      const T v = (T)(2.0 * kw * (th.g[i] * th.g[j] + dth * th.h[hidx(i, j)]));
      H[i * NJ + j] = v;
      H[j * NJ + i] = v;
    }
  if (project) project_psd<12, T>(H);
  for (int a = 0; a < 4; ++a)
    for (int b = a; b < 4; ++b) {
      if (nodes[a] < 0 || nodes[b] < 0) continue;
      T* d;
      bool tr = false;
      if (a == b) d = diag + 9 * (size_t)nodes[a];
      else {
        const int q = (a == 0) ? b - 1 : (a == 1 ? b + 1 : 5);
        d = vals + 9 * (size_t)hslot[6 * e + q];
        tr = nodes[a] > nodes[b];
      }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          atomicAdd(d + 3 * i + j, tr ? H[(3 * b + i) * NJ + 3 * a + j] : H[(3 * a + i) * NJ + 3 * b + j]);
    }
}

template <typename T>
yasps_status bend_t(yasps_system* s, int project) {
  k_bend<T><<<blocks_for(s->nh, 64), 64, 0, s->stream>>>(s->nh, as<int>(s->hinge_v), as<int>(s->hinge_n),
                                                        as<double>(s->hinge_rest), as<int>(s->hinge_slot),
                                                        as<double>(s->P), s->prm.dt * s->prm.dt, project,
                                                        as<double>(s->grad), as<T>(s->diag), as<T>(s->Hs.vals));
  LAUNCH_CHECK(s, "k_bend");
  return YASPS_OK;
}

}  // namespace

yasps_status launch_bend(yasps_system* s, int project) {
  if (s->nh == 0) return YASPS_OK;
  return s->hess_precision == 1 ? bend_t<float>(s, project) : bend_t<double>(s, project);
}
