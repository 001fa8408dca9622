// bend.cu -- discrete-shell bending of cloth hinges (Grinspun et al. 2003):
//   Psi = kb (theta - theta_rest)^2 * 3 |e_rest|^2 / (A1_rest + A2_rest),
// theta the signed angle between the normals of triangles (x0, x1, xa) and
// (x1, x0, xb) about the shared edge.
//
// With e = x1 - x0, u = xa - x0, w = xb - x0 the normals are n1 = e x u and
// n2 = w x e, and
//   theta = atan2(S, C),  S = (n1 x n2).e / |e| = -|e| [e, u, w],
//                         C = n1 . n2 = (e.w)(e.u) - |e|^2 (u.w),
// so its gradient and Hessian in the 9 variables (e, u, w) follow from those of
// the scalar products (closed forms below).  The map from the 12 hinge DOF to
// (e, u, w) is linear, so the 12 x 12 Hessian is J^T H9 J with no curvature
// term; Psi's Hessian 2 k w (grad theta grad theta^T + (theta - theta0) hess
// theta) is projected in the hinge's own 12-dim space.
#include "common.cuh"
#include "eig.cuh"
#include "internal.h"

namespace {

__device__ __forceinline__ int lc3(int i, int j, int k) {  // Levi-Civita symbol
  return (i == j || j == k || i == k) ? 0 : (((j - i + 3) % 3 == 1) ? 1 : -1);
}

// theta and its gradient (12) / Hessian (12 x 12, row-major) w.r.t. (x0, x1, xa, xb)
__device__ void hinge_theta_derivs(const double* x, double* th, double* g12, double* H12) {
  double e[3], u[3], w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    e[k] = x[3 + k] - x[k];
    u[k] = x[6 + k] - x[k];
    w[k] = x[9 + k] - x[k];
  }
  const double Q = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
  const double L = sqrt(Q);
  const double uxw[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  const double wxe[3] = {w[1] * e[2] - w[2] * e[1], w[2] * e[0] - w[0] * e[2], w[0] * e[1] - w[1] * e[0]};
  const double exu[3] = {e[1] * u[2] - e[2] * u[1], e[2] * u[0] - e[0] * u[2], e[0] * u[1] - e[1] * u[0]};
  const double tau = e[0] * uxw[0] + e[1] * uxw[1] + e[2] * uxw[2];
  const double A = e[0] * w[0] + e[1] * w[1] + e[2] * w[2];
  const double B = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
  const double R = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
  const double S = -L * tau, C = A * B - Q * R;
  // gradients over z = (e, u, w)
  double gL[9] = {0}, gt[9], gA[9] = {0}, gB[9] = {0}, gQ[9] = {0}, gR[9] = {0};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gL[k] = e[k] / L;
    gt[k] = uxw[k]; gt[3 + k] = wxe[k]; gt[6 + k] = exu[k];
    gA[k] = w[k]; gA[6 + k] = e[k];
    gB[k] = u[k]; gB[3 + k] = e[k];
    gQ[k] = 2.0 * e[k];
    gR[3 + k] = w[k]; gR[6 + k] = u[k];
  }
  double gS[9], gC[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    gS[i] = -(tau * gL[i] + L * gt[i]);
    gC[i] = B * gA[i] + A * gB[i] - R * gQ[i] - Q * gR[i];
  }
  const double D = S * S + C * C;
  *th = atan2(S, C);
  double g9[9], v9[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    g9[i] = (C * gS[i] - S * gC[i]) / D;
    v9[i] = 2.0 * S * gS[i] + 2.0 * C * gC[i];
  }
  // Hessians of S and C over z, entry by entry
  double H9[81];
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int br = r / 3, i = r % 3, bq = q / 3, j = q % 3;
      // d2 L (e,e), d2 tau, d2 A, d2 B, d2 Q, d2 R
      const double HLrq = (br == 0 && bq == 0) ? ((i == j ? 1.0 : 0.0) - e[i] * e[j] / Q) / L : 0.0;
      double Htrq = 0.0;
      if (br != bq) {
        // tau = eps_abc e_a u_b w_c
        const double* third = (br != 0 && bq != 0) ? e : ((br != 1 && bq != 1) ? u : w);
        const int tb = 3 - br - bq;  // block of the third vector
        int idx[3];
        idx[br] = i; idx[bq] = j;
        double s = 0.0;
        for (int k = 0; k < 3; ++k) {
          idx[tb] = k;
          s += lc3(idx[0], idx[1], idx[2]) * third[k];
        }
        Htrq = s;
      }
      const double d = (i == j) ? 1.0 : 0.0;
      const double HArq = ((br == 0 && bq == 2) || (br == 2 && bq == 0)) ? d : 0.0;
      const double HBrq = ((br == 0 && bq == 1) || (br == 1 && bq == 0)) ? d : 0.0;
      const double HQrq = (br == 0 && bq == 0) ? 2.0 * d : 0.0;
      const double HRrq = ((br == 1 && bq == 2) || (br == 2 && bq == 1)) ? d : 0.0;
      const double HS = -(tau * HLrq + gL[r] * gt[q] + gt[r] * gL[q] + L * Htrq);
      const double HC = gA[r] * gB[q] + gB[r] * gA[q] + B * HArq + A * HBrq - gR[r] * gQ[q] - gQ[r] * gR[q] -
                        R * HQrq - Q * HRrq;
      H9[9 * r + q] = (C * HS - S * HC + gC[r] * gS[q] - gS[r] * gC[q]) / D - (C * gS[r] - S * gC[r]) * v9[q] / (D * D);
    }
  // symmetrise and map z -> x: e = x1 - x0, u = xa - x0, w = xb - x0
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int q = r + 1; q < 9; ++q) {
      const double m = 0.5 * (H9[9 * r + q] + H9[9 * q + r]);
      H9[9 * r + q] = m;
      H9[9 * q + r] = m;
    }
  const double cf[3][4] = {{-1, 1, 0, 0}, {-1, 0, 1, 0}, {-1, 0, 0, 1}};
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int i = 0; i < 3; ++i) g12[3 * v + i] = cf[0][v] * g9[i] + cf[1][v] * g9[3 + i] + cf[2][v] * g9[6 + i];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          double s = 0.0;
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) s += cf[r][v] * cf[q][t] * H9[9 * (3 * r + i) + 3 * q + j];
          H12[12 * (3 * v + i) + 3 * t + j] = s;
        }
}

template <typename T>
__global__ void __launch_bounds__(128) k_bend(int nh, const int* __restrict__ hv, const int* __restrict__ hn,
                                             const double* __restrict__ hrest, const int* __restrict__ hslot,
                                             const double* __restrict__ P, double h2, int project,
                                             double* __restrict__ g, T* __restrict__ diag, T* __restrict__ vals) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nh) return;
  double x[12];
  int nodes[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int v = hv[4 * e + a];
    nodes[a] = hn[4 * e + a];
    x[3 * a] = P[3 * v]; x[3 * a + 1] = P[3 * v + 1]; x[3 * a + 2] = P[3 * v + 2];
  }
  double th, gt[12], Ht[144];
  hinge_theta_derivs(x, &th, gt, Ht);
  const double dth = th - hrest[2 * e];
  const double kw = hrest[2 * e + 1] * h2;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (nodes[a] < 0) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(&g[3 * nodes[a] + c], 2.0 * kw * dth * gt[3 * a + c]);
  }
  T H[144];
#pragma unroll
  for (int i = 0; i < 12; ++i)
#pragma unroll
    for (int j = 0; j < 12; ++j) H[12 * i + j] = (T)(2.0 * kw * (gt[i] * gt[j] + dth * Ht[12 * i + j]));
  if (project) project_psd<12, T>(H);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) {
      if (nodes[a] < 0 || nodes[b] < 0) continue;
      T* d;
      bool tr = false;
      if (a == b) {
        d = diag + 9 * (size_t)nodes[a];
      } else {
        const int q = (a == 0) ? b - 1 : (a == 1 ? b + 1 : 5);
        d = vals + 9 * (size_t)hslot[6 * e + q];
        tr = nodes[a] > nodes[b];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          atomicAdd(d + 3 * i + j, tr ? H[12 * (3 * b + i) + 3 * a + j] : H[12 * (3 * a + i) + 3 * b + j]);
    }
}

template <typename T>
yasps_status bend_t(yasps_system* s, int project) {
  k_bend<T><<<blocks_for(s->nh, 128), 128, 0, s->stream>>>(s->nh, as<int>(s->hinge_v), as<int>(s->hinge_n),
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
