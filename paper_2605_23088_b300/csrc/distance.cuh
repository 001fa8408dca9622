// distance.cuh -- contact distances for point-triangle, edge-edge and
// point-plane pairs (Sec. "UNION": collision pairs as dynamic primitives).
//
// Classification and the squared distance s that decides membership in the
// active set (s < dhat^2) are evaluated in FP64 with explicitly rounded
// operations (__dmul_rn / __dadd_rn / __dsub_rn are never fused into FMAs), in
// a fixed operation order:  dot(a,b) = (a.x*b.x + a.y*b.y) + a.z*b.z,
// cross(a,b) = (a.y*b.z - a.z*b.y, a.z*b.x - a.x*b.z, a.x*b.y - a.y*b.x).
// The closest-feature regions of a triangle follow the Voronoi-region tests of
// Ericson, "Real-Time Collision Detection" (2005), Sec. 5.1.5; the closed
// interval (<= 0) goes to the lower-dimensional feature.
//
// Derivatives of s are hand-derived for the four distance types (PP, PE,
// point-plane of a triangle, line-line of two edges) and consumed by the
// barrier kernels.
#pragma once
#include "common.cuh"

namespace dist {

using d3 = v3<double>;

YASPS_D double mul(double a, double b) { return __dmul_rn(a, b); }
YASPS_D double add(double a, double b) { return __dadd_rn(a, b); }
YASPS_D double sub(double a, double b) { return __dsub_rn(a, b); }
YASPS_D double dv(double a, double b) { return __ddiv_rn(a, b); }
YASPS_D d3 vsub(d3 a, d3 b) { return {sub(a.x, b.x), sub(a.y, b.y), sub(a.z, b.z)}; }
YASPS_D double vdot(d3 a, d3 b) { return add(add(mul(a.x, b.x), mul(a.y, b.y)), mul(a.z, b.z)); }
YASPS_D d3 vcross(d3 a, d3 b) {
  return {sub(mul(a.y, b.z), mul(a.z, b.y)), sub(mul(a.z, b.x), mul(a.x, b.z)), sub(mul(a.x, b.y), mul(a.y, b.x))};
}

enum { PP = 0, PE = 1, PT = 2, EE = 3 };

YASPS_D double s_pp(d3 p, d3 a) {
  d3 e = vsub(p, a);
  return vdot(e, e);
}
YASPS_D double s_pe(d3 p, d3 a, d3 b) {
  d3 e = vsub(b, a), w = vsub(p, a);
  d3 c = vcross(w, e);
  return dv(vdot(c, c), vdot(e, e));
}
YASPS_D double s_ptplane(d3 p, d3 a, d3 b, d3 c) {
  d3 n = vcross(vsub(b, a), vsub(c, a));
  double t = vdot(vsub(p, a), n);
  return dv(mul(t, t), vdot(n, n));
}
YASPS_D double s_eeline(d3 a0, d3 a1, d3 b0, d3 b1) {
  d3 cr = vcross(vsub(a1, a0), vsub(b1, b0));
  double t = vdot(vsub(a0, b0), cr);
  return dv(mul(t, t), vdot(cr, cr));
}

// Local vertex ids of a PT pair: 0 = point, 1..3 = triangle (a, b, c).
// subtype 0/1/2: nearest vertex a/b/c; 3: edge ab; 4: edge bc; 5: edge ca; 6: face.
YASPS_D int pt_classify(d3 p, d3 a, d3 b, d3 c, double* s) {
  d3 ab = vsub(b, a), ac = vsub(c, a), ap = vsub(p, a);
  double d1 = vdot(ab, ap), d2 = vdot(ac, ap);
  if (d1 <= 0.0 && d2 <= 0.0) { *s = s_pp(p, a); return 0; }
  d3 bp = vsub(p, b);
  double d3_ = vdot(ab, bp), d4 = vdot(ac, bp);
  if (d3_ >= 0.0 && d4 <= d3_) { *s = s_pp(p, b); return 1; }
  double vc = sub(mul(d1, d4), mul(d3_, d2));
  if (vc <= 0.0 && d1 >= 0.0 && d3_ <= 0.0) { *s = s_pe(p, a, b); return 3; }
  d3 cp = vsub(p, c);
  double d5 = vdot(ab, cp), d6 = vdot(ac, cp);
  if (d6 >= 0.0 && d5 <= d6) { *s = s_pp(p, c); return 2; }
  double vb = sub(mul(d5, d2), mul(d1, d6));
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) { *s = s_pe(p, c, a); return 5; }
  double va = sub(mul(d3_, d6), mul(d5, d4));
  if (va <= 0.0 && sub(d4, d3_) >= 0.0 && sub(d5, d6) >= 0.0) { *s = s_pe(p, b, c); return 4; }
  *s = s_ptplane(p, a, b, c);
  return 6;
}

// point vs segment (u, v): 0 nearest u, 1 nearest v, 2 interior
YASPS_D int pe_classify(d3 p, d3 u, d3 v, double* s) {
  d3 e = vsub(v, u), w = vsub(p, u);
  double t = vdot(w, e);
  if (t <= 0.0) { *s = vdot(w, w); return 0; }
  double ee = vdot(e, e);
  if (t >= ee) { *s = s_pp(p, v); return 1; }
  *s = s_pe(p, u, v);
  return 2;
}

constexpr double kEEParallelEps = 1e-10;

// Local vertex ids of an EE pair: 0,1 = edge a; 2,3 = edge b.  subtype 0 =
// line-line interior; 1 + 3k + r for endpoint case k (a0|b, a1|b, b0|a, b1|a)
// and point-segment result r.  Near-parallel edges (|da x db|^2 <= eps |da|^2
// |db|^2) always use the endpoint cases.
YASPS_D int ee_classify(d3 a0, d3 a1, d3 b0, d3 b1, double* s) {
  d3 da = vsub(a1, a0), db = vsub(b1, b0), w = vsub(a0, b0);
  d3 cr = vcross(da, db);
  double A = vdot(da, da), B = vdot(da, db), C = vdot(db, db), D = vdot(da, w), E = vdot(db, w);
  double den = vdot(cr, cr);
  if (den > mul(mul(kEEParallelEps, A), C)) {
    double sn = sub(mul(B, E), mul(C, D)), tn = sub(mul(A, E), mul(B, D));
    if (sn > 0.0 && sn < den && tn > 0.0 && tn < den) {
      *s = s_eeline(a0, a1, b0, b1);
      return 0;
    }
  }
  double best = 0.0;
  int bk = -1, br = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const d3 P = (k == 0) ? a0 : (k == 1) ? a1 : (k == 2) ? b0 : b1;
    const d3 U = (k < 2) ? b0 : a0;
    const d3 V = (k < 2) ? b1 : a1;
    double sk;
    int r = pe_classify(P, U, V, &sk);
    if (bk < 0 || sk < best) { best = sk; bk = k; br = r; }
  }
  *s = best;
  return 1 + 3 * bk + br;
}

// Distance type and the local vertices it involves, in the order the
// derivative routines expect: PP (p, a), PE (p, a, b), PT (p, a, b, c),
// EE (a0, a1, b0, b1).
struct dclass {
  int dtype, n;
  int loc[4];
};
YASPS_D dclass pt_dclass(int st) {
  switch (st) {
    case 0: return {PP, 2, {0, 1, 0, 0}};
    case 1: return {PP, 2, {0, 2, 0, 0}};
    case 2: return {PP, 2, {0, 3, 0, 0}};
    case 3: return {PE, 3, {0, 1, 2, 0}};
    case 4: return {PE, 3, {0, 2, 3, 0}};
    case 5: return {PE, 3, {0, 3, 1, 0}};
    default: return {PT, 4, {0, 1, 2, 3}};
  }
}
YASPS_D dclass ee_dclass(int st) {
  if (st == 0) return {EE, 4, {0, 1, 2, 3}};
  const int k = (st - 1) / 3, r = (st - 1) % 3;
  const int pv = k, uu = (k < 2) ? 2 : 0, vv = (k < 2) ? 3 : 1;
  if (r == 0) return {PP, 2, {pv, uu, 0, 0}};
  if (r == 1) return {PP, 2, {pv, vv, 0, 0}};
  return {PE, 3, {pv, uu, vv, 0}};
}

// ---------------------------------------------------------------- derivatives
// Gradient g (3n) and Hessian H (3n x 3n, row-major) of s for the classified
// local vertices y[0..n-1].  Ordinary FP64 arithmetic: compared with a
// tolerance, not bit-exactly.

// PP: s = |p - a|^2
YASPS_D void ds_pp(const d3* y, double* g, double* H) {
  d3 w = y[0] - y[1];
  const double wv[3] = {w.x, w.y, w.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) { g[i] = 2.0 * wv[i]; g[3 + i] = -2.0 * wv[i]; }
#pragma unroll
  for (int i = 0; i < 36; ++i) H[i] = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    H[i * 6 + i] = 2.0; H[(3 + i) * 6 + 3 + i] = 2.0;
    H[i * 6 + 3 + i] = -2.0; H[(3 + i) * 6 + i] = -2.0;
  }
}

// PE: s = |w|^2 - (w.e)^2/|e|^2, w = p - a, e = b - a
YASPS_D void ds_pe(const d3* y, double* g, double* H) {
  d3 wv = y[0] - y[1], ev = y[2] - y[1];
  const double w[3] = {wv.x, wv.y, wv.z}, e[3] = {ev.x, ev.y, ev.z};
  const double u = dot(wv, ev), L = dot(ev, ev);
  double gw[3], ge[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gw[i] = 2.0 * w[i] - 2.0 * u * e[i] / L;
    ge[i] = -2.0 * u * w[i] / L + 2.0 * u * u * e[i] / (L * L);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) { g[i] = gw[i]; g[6 + i] = ge[i]; g[3 + i] = -gw[i] - ge[i]; }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double d = (i == j) ? 1.0 : 0.0;
      const double ww = 2.0 * d - 2.0 * e[i] * e[j] / L;
      const double we = -2.0 * e[i] * w[j] / L - 2.0 * u * d / L + 4.0 * u * e[i] * e[j] / (L * L);
      const double ew = -2.0 * e[j] * w[i] / L - 2.0 * u * d / L + 4.0 * u * e[j] * e[i] / (L * L);
      const double ee = -2.0 * w[i] * w[j] / L + 4.0 * u * (w[i] * e[j] + e[i] * w[j]) / (L * L) +
                        2.0 * u * u * d / (L * L) - 8.0 * u * u * e[i] * e[j] / (L * L * L);
      // map (w, e) -> (p, a, b): w = p - a, e = b - a
      H[(0 + i) * 9 + 0 + j] = ww;
      H[(0 + i) * 9 + 6 + j] = we;
      H[(6 + i) * 9 + 0 + j] = ew;
      H[(6 + i) * 9 + 6 + j] = ee;
      H[(0 + i) * 9 + 3 + j] = -ww - we;
      H[(3 + i) * 9 + 0 + j] = -ww - ew;
      H[(6 + i) * 9 + 3 + j] = -ew - ee;
      H[(3 + i) * 9 + 6 + j] = -we - ee;
      H[(3 + i) * 9 + 3 + j] = ww + we + ew + ee;
    }
}

// s = (w.n)^2 / (n.n), n = e1 x e2, in the variables (w, e1, e2): gradient
// (9) and Hessian (9x9).  Shared by the point-plane (PT) and line-line (EE) types.
YASPS_D void ds_wn(d3 wv, d3 e1v, d3 e2v, double* g9, double* H9) {
  const d3 nv = cross(e1v, e2v);
  const double w[3] = {wv.x, wv.y, wv.z}, n[3] = {nv.x, nv.y, nv.z}, e1[3] = {e1v.x, e1v.y, e1v.z},
               e2[3] = {e2v.x, e2v.y, e2v.z};
  const double t = dot(wv, nv), N = dot(nv, nv);
  double gw[3], gn[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gw[i] = 2.0 * t * n[i] / N;
    gn[i] = 2.0 * t * w[i] / N - 2.0 * t * t * n[i] / (N * N);
  }
  double Hwn[9], Hnn[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double d = (i == j) ? 1.0 : 0.0;
      H9[9 * i + j] = 2.0 * n[i] * n[j] / N;
      Hwn[3 * i + j] = 2.0 * (n[i] * w[j] + t * d) / N - 4.0 * t * n[i] * n[j] / (N * N);
      Hnn[3 * i + j] = 2.0 * w[i] * w[j] / N - 4.0 * t * (w[i] * n[j] + n[i] * w[j]) / (N * N) -
                       2.0 * t * t * d / (N * N) + 8.0 * t * t * n[i] * n[j] / (N * N * N);
    }
  // dn/de1 = -[e2]x, dn/de2 = [e1]x  (row k, column a); Jn = [J1 J2] is 3 x 6
  const double Jn[18] = {0, e2[2], -e2[1], 0, -e1[2], e1[1],
                         -e2[2], 0, e2[0], e1[2], 0, -e1[0],
                         e2[1], -e2[0], 0, -e1[1], e1[0], 0};
#pragma unroll
  for (int i = 0; i < 3; ++i) g9[i] = gw[i];
#pragma unroll
  for (int c = 0; c < 6; ++c) g9[3 + c] = gn[0] * Jn[c] + gn[1] * Jn[6 + c] + gn[2] * Jn[12 + c];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double s = Hwn[3 * i] * Jn[c] + Hwn[3 * i + 1] * Jn[6 + c] + Hwn[3 * i + 2] * Jn[12 + c];
      H9[9 * i + 3 + c] = s;
      H9[9 * (3 + c) + i] = s;
    }
  double T[18];  // Hnn Jn (3 x 6)
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 6; ++c) T[6 * k + c] = Hnn[3 * k] * Jn[c] + Hnn[3 * k + 1] * Jn[6 + c] + Hnn[3 * k + 2] * Jn[12 + c];
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) H9[9 * (3 + r) + 3 + c] = Jn[r] * T[c] + Jn[6 + r] * T[6 + c] + Jn[12 + r] * T[12 + c];
  // curvature of n: d2 n_k / de1_i de2_j = eps_kij -> block (e1, e2) = sum_k gn_k eps_kij
  const double M[9] = {0, gn[2], -gn[1], -gn[2], 0, gn[0], gn[1], -gn[0], 0};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      H9[9 * (3 + i) + 6 + j] += M[3 * i + j];
      H9[9 * (6 + j) + 3 + i] += M[3 * i + j];
    }
}

// Map (w, e1, e2) derivatives to the 4 vertices: variable group r is
// sum_v coef[r][v] y_v.
YASPS_D void map_wn_to_verts(const double (&coef)[3][4], const double* g9, const double* H9, double* g, double* H) {
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      g[3 * v + i] = coef[0][v] * g9[i] + coef[1][v] * g9[3 + i] + coef[2][v] * g9[6 + i];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          double s = 0;
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) s += coef[r][v] * coef[q][u] * H9[9 * (3 * r + i) + 3 * q + j];
          H[12 * (3 * v + i) + 3 * u + j] = s;
        }
}

// ---- warp-cooperative form of ds_wn + map_wn_to_verts (the same formulas):
// the scalars are formed by every lane, the 18 entries of Hwn and Hnn, the 81
// of H9 and the 144 of H by different lanes.  One lane doing all of it issues
// a few thousand FP64 instructions; a warp instruction with a single active
// lane costs about as much FP64 pipe time as a full one, so spreading the
// entries over the lanes cuts the pipe time about 16 times.
struct wn_scratch {
  double Hwn[9], Hnn[9], gw[3], gn[3], g9[9], H9[81];
};
YASPS_D double comp(const d3& v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }
// entry c (0..5) of row k of Jn = [dn/de1 dn/de2] (3 x 6), as in ds_wn
YASPS_D double jn(const d3& e1, const d3& e2, int k, int c) {
  const d3& e = (c < 3) ? e2 : e1;
  const double sg = (c < 3) ? -1.0 : 1.0;  // dn/de1 = -[e2]x, dn/de2 = [e1]x
  const int a = c % 3;
  if (k == a) return 0.0;
  // [v]x (row k, column a) = -eps_kab v_b
  const int b = 3 - k - a;
  const double eps = ((k + 1) % 3 == a) ? 1.0 : -1.0;
  return sg * (-eps) * comp(e, b);
}
// all 32 lanes call; g (12) and H (144) are written to shared memory
YASPS_D void ds_wn_warp(d3 wv, d3 e1v, d3 e2v, const double (&coef)[3][4], wn_scratch& S, double* g, double* H,
                        int lane) {
  const d3 nv = cross(e1v, e2v);
  const double t = dot(wv, nv), N = dot(nv, nv);
  if (lane < 9) {
    const int i = lane / 3, j = lane % 3;
    const double d = (i == j) ? 1.0 : 0.0;
    S.Hwn[lane] = 2.0 * (comp(nv, i) * comp(wv, j) + t * d) / N - 4.0 * t * comp(nv, i) * comp(nv, j) / (N * N);
  } else if (lane < 18) {
    const int i = (lane - 9) / 3, j = (lane - 9) % 3;
    const double d = (i == j) ? 1.0 : 0.0;
    const double wi = comp(wv, i), wj = comp(wv, j), ni = comp(nv, i), nj = comp(nv, j);
    S.Hnn[lane - 9] = 2.0 * wi * wj / N - 4.0 * t * (wi * nj + ni * wj) / (N * N) - 2.0 * t * t * d / (N * N) +
                      8.0 * t * t * ni * nj / (N * N * N);
  } else if (lane < 21) {
    const int i = lane - 18;
    S.gw[i] = 2.0 * t * comp(nv, i) / N;
  } else if (lane < 24) {
    const int i = lane - 21;
    S.gn[i] = 2.0 * t * comp(wv, i) / N - 2.0 * t * t * comp(nv, i) / (N * N);
  }
  __syncwarp();
  if (lane < 9) S.g9[lane] = lane < 3 ? S.gw[lane]
                                      : S.gn[0] * jn(e1v, e2v, 0, lane - 3) + S.gn[1] * jn(e1v, e2v, 1, lane - 3) +
                                            S.gn[2] * jn(e1v, e2v, 2, lane - 3);
  for (int e = lane; e < 81; e += 32) {
    const int r = e / 9, c = e % 9;
    double h;
    if (r < 3 && c < 3) {
      h = 2.0 * comp(nv, r) * comp(nv, c) / N;
    } else if (r < 3 || c < 3) {
      const int i = r < 3 ? r : c, cc = (r < 3 ? c : r) - 3;
      h = S.Hwn[3 * i] * jn(e1v, e2v, 0, cc) + S.Hwn[3 * i + 1] * jn(e1v, e2v, 1, cc) +
          S.Hwn[3 * i + 2] * jn(e1v, e2v, 2, cc);
    } else {
      const int rr = r - 3, cc = c - 3;
      double T3[3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        T3[k] = S.Hnn[3 * k] * jn(e1v, e2v, 0, cc) + S.Hnn[3 * k + 1] * jn(e1v, e2v, 1, cc) +
                S.Hnn[3 * k + 2] * jn(e1v, e2v, 2, cc);
      h = jn(e1v, e2v, 0, rr) * T3[0] + jn(e1v, e2v, 1, rr) * T3[1] + jn(e1v, e2v, 2, rr) * T3[2];
      // curvature of n: block (e1, e2) and its transpose, M = sum_k gn_k eps_kij
      // (row e1_i, column e2_j or its transpose; eps_kij = +1 when j = i + 1 mod 3)
      const int i = rr < 3 ? rr : cc, j = rr < 3 ? cc - 3 : rr - 3;
      if ((rr < 3) != (cc < 3) && i != j) h += S.gn[3 - i - j] * (((i + 1) % 3 == j) ? 1.0 : -1.0);
    }
    S.H9[e] = h;
  }
  __syncwarp();
  if (lane < 12) {
    const int v = lane / 3, i = lane % 3;
    g[lane] = coef[0][v] * S.g9[i] + coef[1][v] * S.g9[3 + i] + coef[2][v] * S.g9[6 + i];
  }
  for (int e = lane; e < 144; e += 32) {
    const int row = e / 12, col = e % 12;
    const int v = row / 3, i = row % 3, u = col / 3, j = col % 3;
    double acc = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) acc += coef[r][v] * coef[q][u] * S.H9[9 * (3 * r + i) + 3 * q + j];
    H[e] = acc;
  }
  __syncwarp();
}

// PT (point-plane): w = p - a, e1 = b - a, e2 = c - a
YASPS_D void ds_pt(const d3* y, double* g, double* H) {
  double g9[9], H9[81];
  ds_wn(y[0] - y[1], y[2] - y[1], y[3] - y[1], g9, H9);
  const double coef[3][4] = {{1, -1, 0, 0}, {0, -1, 1, 0}, {0, -1, 0, 1}};
  map_wn_to_verts(coef, g9, H9, g, H);
}
// EE (line-line): w = a0 - b0, e1 = a1 - a0, e2 = b1 - b0
YASPS_D void ds_ee(const d3* y, double* g, double* H) {
  double g9[9], H9[81];
  ds_wn(y[0] - y[2], y[1] - y[0], y[3] - y[2], g9, H9);
  const double coef[3][4] = {{1, 0, -1, 0}, {-1, 1, 0, 0}, {0, 0, -1, 1}};
  map_wn_to_verts(coef, g9, H9, g, H);
}

}  // namespace dist
