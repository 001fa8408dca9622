/*
 * oracle.c -- plain FP64 CPU oracle of the IPC Newton hot path (YASPS,
 * arxiv 2605.23088).  TEST INFRASTRUCTURE ONLY: it is called by the test
 * suite, by the smoke check and by the benchmark's CPU-baseline leg, never by
 * the library.  It shares no code with the CUDA path.
 *
 * Design rules of this file:
 *  - every energy is written once as a plain formula over "jets"
 *    (value, gradient, Hessian carried through each operation, i.e. exact
 *    second-order forward-mode differentiation), so no derivative is derived
 *    by hand here;
 *  - PSD projection is a textbook cyclic Jacobi eigendecomposition followed by
 *    clamping negative eigenvalues to zero (Sec. "EVD and PSD Projection");
 *  - the projection is done in the space the paper prescribes: F-space for the
 *    Neo-Hookean tet (Sec. "Eigendecomposition: Manual Optimization"),
 *    F(3x2)-space for the membrane, the element's own space for bending and
 *    the affine orthogonality term, position space for contact barriers whose
 *    parameterisations are linear (Sec. "Projecting in reduced coordinates");
 *  - assembly collects upper-triangular 3x3 block contributions, sorts them by
 *    (row, col) and merges duplicates (App. B "Global Hessian Compression");
 *  - the linear solve is block-Jacobi PCG on H p = g, p not negated
 *    (Sec. "Solution Extraction", Sec. 8 "Solver", App. D "Preconditioner").
 *
 * Built with -ffp-contract=off so that the contact-distance arithmetic is
 * evaluated exactly in the written order (no fused multiply-adds).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EXPORT __attribute__((visibility("default")))

/* ======================================================================== */
/* jets: f, df/dz (n), d2f/dz2 (n x n) for n <= 12 independent variables      */
/* ======================================================================== */
#define JMAX 12
typedef struct { double v; double g[JMAX]; double h[JMAX * JMAX]; } jet;
static _Thread_local int JN = 0;

static jet jc(double c) { jet r; memset(&r, 0, sizeof r); r.v = c; return r; }
static jet jvar(double c, int i) { jet r = jc(c); r.g[i] = 1.0; return r; }
static jet jadd(jet a, jet b) {
  jet r; r.v = a.v + b.v;
  for (int i = 0; i < JN; ++i) r.g[i] = a.g[i] + b.g[i];
  for (int i = 0; i < JN * JN; ++i) r.h[i] = a.h[i] + b.h[i];
  return r;
}
static jet jsub(jet a, jet b) {
  jet r; r.v = a.v - b.v;
  for (int i = 0; i < JN; ++i) r.g[i] = a.g[i] - b.g[i];
  for (int i = 0; i < JN * JN; ++i) r.h[i] = a.h[i] - b.h[i];
  return r;
}
static jet jscale(jet a, double c) {
  jet r; r.v = a.v * c;
  for (int i = 0; i < JN; ++i) r.g[i] = a.g[i] * c;
  for (int i = 0; i < JN * JN; ++i) r.h[i] = a.h[i] * c;
  return r;
}
static jet jaddc(jet a, double c) { a.v += c; return a; }
static jet jmul(jet a, jet b) {
  jet r; r.v = a.v * b.v;
  for (int i = 0; i < JN; ++i) r.g[i] = a.v * b.g[i] + b.v * a.g[i];
  for (int i = 0; i < JN; ++i)
    for (int j = 0; j < JN; ++j)
      r.h[i * JN + j] = a.v * b.h[i * JN + j] + b.v * a.h[i * JN + j] + a.g[i] * b.g[j] + b.g[i] * a.g[j];
  return r;
}
/* unary chain rule: r = f(a), given f(a.v), f'(a.v), f''(a.v) */
static jet junary(jet a, double f, double df, double d2f) {
  jet r; r.v = f;
  for (int i = 0; i < JN; ++i) r.g[i] = df * a.g[i];
  for (int i = 0; i < JN; ++i)
    for (int j = 0; j < JN; ++j) r.h[i * JN + j] = df * a.h[i * JN + j] + d2f * a.g[i] * a.g[j];
  return r;
}
static jet jlog(jet a) { return junary(a, log(a.v), 1.0 / a.v, -1.0 / (a.v * a.v)); }
static jet jsqrt(jet a) { double s = sqrt(a.v); return junary(a, s, 0.5 / s, -0.25 / (s * a.v)); }
static jet jinv(jet a) { return junary(a, 1.0 / a.v, -1.0 / (a.v * a.v), 2.0 / (a.v * a.v * a.v)); }
static jet jdiv(jet a, jet b) { return jmul(a, jinv(b)); }
static jet jsq(jet a) { return jmul(a, a); }
/* theta = atan2(y, x) as a function of two jets */
static jet jatan2(jet y, jet x) {
  double r2 = x.v * x.v + y.v * y.v;
  double ty = x.v / r2, tx = -y.v / r2;
  double r4 = r2 * r2;
  double tyy = -2.0 * x.v * y.v / r4, txx = 2.0 * x.v * y.v / r4, txy = (y.v * y.v - x.v * x.v) / r4;
  jet r; r.v = atan2(y.v, x.v);
  for (int i = 0; i < JN; ++i) r.g[i] = ty * y.g[i] + tx * x.g[i];
  for (int i = 0; i < JN; ++i)
    for (int j = 0; j < JN; ++j)
      r.h[i * JN + j] = ty * y.h[i * JN + j] + tx * x.h[i * JN + j] + tyy * y.g[i] * y.g[j] + txx * x.g[i] * x.g[j] +
                        txy * (x.g[i] * y.g[j] + y.g[i] * x.g[j]);
  return r;
}
typedef struct { jet c[3]; } jvec;
static jvec jv_sub(jvec a, jvec b) { jvec r; for (int k = 0; k < 3; ++k) r.c[k] = jsub(a.c[k], b.c[k]); return r; }
static jet jv_dot(jvec a, jvec b) { return jadd(jadd(jmul(a.c[0], b.c[0]), jmul(a.c[1], b.c[1])), jmul(a.c[2], b.c[2])); }
static jvec jv_cross(jvec a, jvec b) {
  jvec r;
  r.c[0] = jsub(jmul(a.c[1], b.c[2]), jmul(a.c[2], b.c[1]));
  r.c[1] = jsub(jmul(a.c[2], b.c[0]), jmul(a.c[0], b.c[2]));
  r.c[2] = jsub(jmul(a.c[0], b.c[1]), jmul(a.c[1], b.c[0]));
  return r;
}
static jvec jv_vars(const double* x, int first) { jvec r; for (int k = 0; k < 3; ++k) r.c[k] = jvar(x[k], first + k); return r; }

/* ======================================================================== */
/* dense symmetric eigen-decomposition (cyclic Jacobi) and PSD projection    */
/* ======================================================================== */
/* A (n x n, row-major, symmetric) -> w (eigenvalues), V (columns = vectors). */
OR_EXPORT int or_eig_sym(int n, const double* Ain, double* w, double* V) {
  double A[48 * 48];
  if (n > 48) return -1;
  memcpy(A, Ain, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  int sweep;
  for (sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        tot += A[p * n + q] * A[p * n + q];
        if (p != q) off += A[p * n + q] * A[p * n + q];
      }
    if (off == 0.0 || off <= 1e-34 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) { /* columns p, q */
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* rows p, q */
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
  return sweep;
}

/* out = V max(w, 0) V^T  (setting negative eigenvalues to zero) */
OR_EXPORT void or_project_psd(int n, const double* A, double* out) {
  double w[48], V[48 * 48];
  or_eig_sym(n, A, w, V);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        if (w[k] > 0.0) s += V[i * n + k] * w[k] * V[j * n + k];
      out[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i) /* exact symmetry */
    for (int j = i + 1; j < n; ++j) {
      double m = 0.5 * (out[i * n + j] + out[j * n + i]);
      out[i * n + j] = out[j * n + i] = m;
    }
}

/* ======================================================================== */
/* material constants                                                        */
/* ======================================================================== */
OR_EXPORT void or_lame(double E, double nu, double* mu, double* lam) {
  *mu = E / (2.0 * (1.0 + nu));
  *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}
/* plane-stress Lame constants for the membrane */
OR_EXPORT void or_lame_ps(double E, double nu, double* mu, double* lam) {
  *mu = E / (2.0 * (1.0 + nu));
  *lam = E * nu / (1.0 - nu * nu);
}

static void inv3(const double* M, double* Mi, double* det) {
  double a = M[0], b = M[1], c = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], i = M[8];
  double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
  double D = a * A + b * B + c * C;
  *det = D;
  Mi[0] = A / D; Mi[1] = -(b * i - c * h) / D; Mi[2] = (b * f - c * e) / D;
  Mi[3] = B / D; Mi[4] = (a * i - c * g) / D; Mi[5] = -(a * f - c * d) / D;
  Mi[6] = C / D; Mi[7] = -(a * h - b * g) / D; Mi[8] = (a * e - b * d) / D;
}

/* rest shape of a tet: Dm = [X1-X0, X2-X0, X3-X0] (columns), Dm^-1, volume */
OR_EXPORT int or_tet_rest(const double* X, double* Dminv, double* vol) {
  double Dm[9], det;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) Dm[i * 3 + k] = X[(k + 1) * 3 + i] - X[i];
  inv3(Dm, Dminv, &det);
  *vol = det / 6.0;
  return det > 0 ? 0 : -1;
}

/* ======================================================================== */
/* Stable Neo-Hookean (Eq. snh):                                             */
/*   Psi(F) = mu/2 (I_C - 3) - mu/2 log(I_C + 1) + lam/2 (J - alpha)^2,      */
/*   I_C = ||F||_F^2, J = det F, alpha = 1 + 3 mu / (4 lam)                  */
/* with F = Ds Dm^-1.  Hessian projected in F-space (9x9), then J_F^T P J_F  */
/* ======================================================================== */
static jet snh_psi_jet(const double* F, double mu, double lam) {
  JN = 9;
  jet f[9];
  for (int i = 0; i < 9; ++i) f[i] = jvar(F[i], i);
  jet Ic = jc(0.0);
  for (int i = 0; i < 9; ++i) Ic = jadd(Ic, jsq(f[i]));
  /* det of row-major F */
  jet J = jsub(jadd(jmul(f[0], jsub(jmul(f[4], f[8]), jmul(f[5], f[7]))),
                    jmul(f[2], jsub(jmul(f[3], f[7]), jmul(f[4], f[6])))),
               jmul(f[1], jsub(jmul(f[3], f[8]), jmul(f[5], f[6]))));
  double alpha = 1.0 + 3.0 * mu / (4.0 * lam);
  jet t1 = jscale(jaddc(Ic, -3.0), 0.5 * mu);
  jet t2 = jscale(jlog(jaddc(Ic, 1.0)), -0.5 * mu);
  jet t3 = jscale(jsq(jaddc(J, -alpha)), 0.5 * lam);
  return jadd(jadd(t1, t2), t3);
}

/* density-level F-space quantities (no volume factor) */
OR_EXPORT void or_snh_Fspace(const double* F, double mu, double lam, double* psi, double* P, double* dPdF) {
  jet r = snh_psi_jet(F, mu, lam);
  *psi = r.v;
  if (P) for (int i = 0; i < 9; ++i) P[i] = r.g[i];
  if (dPdF) for (int i = 0; i < 81; ++i) dPdF[i] = r.h[i];
}

/* dF/dx for F = Ds Dm^-1, F row-major (index 3i+j), x = 4 vertices x 3 */
static void tet_dFdx(const double* Dminv, double* Jf /*9 x 12*/) {
  memset(Jf, 0, sizeof(double) * 108);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s0 = 0.0;
      for (int a = 1; a < 4; ++a) {
        double w = Dminv[(a - 1) * 3 + j];
        Jf[(3 * i + j) * 12 + 3 * a + i] = w;
        s0 += w;
      }
      Jf[(3 * i + j) * 12 + 0 + i] = -s0;
    }
}

/* Jt P J for J (m x n), P (m x m): out (n x n) */
static void JtPJ(int m, int n, const double* J, const double* P, double* out) {
  double T[48 * 48];
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int b = 0; b < m; ++b) s += P[a * m + b] * J[b * n + c];
      T[a * n + c] = s;
    }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int a = 0; a < m; ++a) s += J[a * n + r] * T[a * n + c];
      out[r * n + c] = s;
    }
}

/* Per-tet energy V*Psi, gradient (12) and Hessian (12x12, F-space projected
 * when project != 0, exact otherwise). x, X: 4 vertices x 3 (current, rest). */
OR_EXPORT int or_snh_local(const double* x, const double* X, double mu, double lam, int project,
                           double* E, double* g, double* H) {
  double Dminv[9], vol;
  if (or_tet_rest(X, Dminv, &vol)) return -1;
  double F[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += (x[(k + 1) * 3 + i] - x[i]) * Dminv[k * 3 + j];
      F[3 * i + j] = s;
    }
  jet r = snh_psi_jet(F, mu, lam);
  double Jf[108];
  tet_dFdx(Dminv, Jf);
  if (E) *E = vol * r.v;
  if (g)
    for (int c = 0; c < 12; ++c) {
      double s = 0.0;
      for (int a = 0; a < 9; ++a) s += Jf[a * 12 + c] * r.g[a];
      g[c] = vol * s;
    }
  if (H) {
    double Pf[81];
    if (project) or_project_psd(9, r.h, Pf); else memcpy(Pf, r.h, sizeof Pf);
    JtPJ(9, 12, Jf, Pf, H);
    for (int i = 0; i < 144; ++i) H[i] *= vol;
  }
  return 0;
}

/* ======================================================================== */
/* StVK membrane (textbook; the paper's cloth uses Baraff-Witkin):            */
/*   F (3x2) = [x1-x0, x2-x0] Dm^-1,  E = (F^T F - I)/2,                       */
/*   Psi = A t (mu ||E||^2 + lam/2 tr(E)^2), plane-stress Lame constants.     */
/* Hessian projected in F-space (6x6).                                        */
/* ======================================================================== */
OR_EXPORT int or_tri_rest(const double* X, double* Dminv /*2x2*/, double* area) {
  double e1[3], e2[3];
  for (int k = 0; k < 3; ++k) { e1[k] = X[3 + k] - X[k]; e2[k] = X[6 + k] - X[k]; }
  double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  double u[3] = {e1[0] / l1, e1[1] / l1, e1[2] / l1};
  double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  double v[3] = {(n[1] * u[2] - n[2] * u[1]) / ln, (n[2] * u[0] - n[0] * u[2]) / ln, (n[0] * u[1] - n[1] * u[0]) / ln};
  /* 2D rest edge vectors in the orthonormal frame (u, v) */
  double Dm[4] = {l1, e2[0] * u[0] + e2[1] * u[1] + e2[2] * u[2], 0.0, e2[0] * v[0] + e2[1] * v[1] + e2[2] * v[2]};
  double det = Dm[0] * Dm[3] - Dm[1] * Dm[2];
  Dminv[0] = Dm[3] / det; Dminv[1] = -Dm[1] / det; Dminv[2] = -Dm[2] / det; Dminv[3] = Dm[0] / det;
  *area = 0.5 * ln;
  return det > 0 ? 0 : -1;
}

static jet stvk_psi_jet(const double* F /*3x2 row-major*/, double mu, double lam) {
  JN = 6;
  jet f[6];
  for (int i = 0; i < 6; ++i) f[i] = jvar(F[i], i);
  /* C = F^T F (2x2) */
  jet C00 = jadd(jadd(jmul(f[0], f[0]), jmul(f[2], f[2])), jmul(f[4], f[4]));
  jet C01 = jadd(jadd(jmul(f[0], f[1]), jmul(f[2], f[3])), jmul(f[4], f[5]));
  jet C11 = jadd(jadd(jmul(f[1], f[1]), jmul(f[3], f[3])), jmul(f[5], f[5]));
  jet E00 = jscale(jaddc(C00, -1.0), 0.5), E11 = jscale(jaddc(C11, -1.0), 0.5), E01 = jscale(C01, 0.5);
  jet nrm = jadd(jadd(jsq(E00), jsq(E11)), jscale(jsq(E01), 2.0));
  jet tr = jadd(E00, E11);
  return jadd(jscale(nrm, mu), jscale(jsq(tr), 0.5 * lam));
}

/* Baraff-Witkin stretch and shear (Baraff and Witkin 1998) as a function of
 * the 3x2 deformation gradient F = [f_u f_v] over the rest (u, v) frame:
 *   Psi = kst/2 ((|f_u| - 1)^2 + (|f_v| - 1)^2) + ksh/2 (f_u . f_v)^2,
 * the cloth of the paper's benchmarks (Sec. "Cloths on Bunny on Cloth");
 * projected in its 6x6 F-space (Sec. "Eigendecomposition: Manual
 * Optimization"). */
static jet bw_psi_jet(const double* F /*3x2 row-major*/, double kst, double ksh) {
  JN = 6;
  jet f[6];
  for (int i = 0; i < 6; ++i) f[i] = jvar(F[i], i);
  jet lu = jsqrt(jadd(jadd(jsq(f[0]), jsq(f[2])), jsq(f[4])));
  jet lv = jsqrt(jadd(jadd(jsq(f[1]), jsq(f[3])), jsq(f[5])));
  jet c = jadd(jadd(jmul(f[0], f[1]), jmul(f[2], f[3])), jmul(f[4], f[5]));
  jet st = jadd(jsq(jaddc(lu, -1.0)), jsq(jaddc(lv, -1.0)));
  return jadd(jscale(st, 0.5 * kst), jscale(jsq(c), 0.5 * ksh));
}

/* membrane element (model 0 StVK with Lame constants a = mu, b = lam;
 * model 1 Baraff-Witkin with a = kst, b = ksh): energy area * thick * Psi(F),
 * F = [x1 - x0, x2 - x0] Dm^-1, Hessian J_F^T Project(d2Psi/dF2) J_F */
static int membrane_local(int model, const double* x, const double* X, double a, double b, double thick,
                          int project, double* E, double* g, double* H) {
  double Dminv[4], area;
  if (or_tri_rest(X, Dminv, &area)) return -1;
  double F[6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 2; ++j)
      F[2 * i + j] = (x[3 + i] - x[i]) * Dminv[0 * 2 + j] + (x[6 + i] - x[i]) * Dminv[1 * 2 + j];
  jet r = model == 1 ? bw_psi_jet(F, a, b) : stvk_psi_jet(F, a, b);
  double Jf[6 * 9];
  memset(Jf, 0, sizeof Jf);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 2; ++j) {
      double w1 = Dminv[0 * 2 + j], w2 = Dminv[1 * 2 + j];
      Jf[(2 * i + j) * 9 + 3 + i] = w1;
      Jf[(2 * i + j) * 9 + 6 + i] = w2;
      Jf[(2 * i + j) * 9 + 0 + i] = -(w1 + w2);
    }
  double k = area * thick;
  if (E) *E = k * r.v;
  if (g)
    for (int c = 0; c < 9; ++c) {
      double s = 0.0;
      for (int q = 0; q < 6; ++q) s += Jf[q * 9 + c] * r.g[q];
      g[c] = k * s;
    }
  if (H) {
    double Pf[36];
    if (project) or_project_psd(6, r.h, Pf); else memcpy(Pf, r.h, sizeof Pf);
    JtPJ(6, 9, Jf, Pf, H);
    for (int i = 0; i < 81; ++i) H[i] *= k;
  }
  return 0;
}
OR_EXPORT int or_stvk_local(const double* x, const double* X, double mu, double lam, double thick, int project,
                            double* E, double* g, double* H) {
  return membrane_local(0, x, X, mu, lam, thick, project, E, g, H);
}
OR_EXPORT int or_bw_local(const double* x, const double* X, double kst, double ksh, double thick, int project,
                          double* E, double* g, double* H) {
  return membrane_local(1, x, X, kst, ksh, thick, project, E, g, H);
}

/* ======================================================================== */
/* Discrete-shell bending (Grinspun et al. 2003):                             */
/*   Psi = kb (theta - theta_rest)^2 * 3 |e_rest|^2 / (A1_rest + A2_rest)     */
/* hinge (e0, e1, a, b): triangles (e0, e1, a) and (e1, e0, b); theta is the  */
/* signed angle between their normals about the shared edge.                 */
/* ======================================================================== */
static jet hinge_theta_jet(const double* x) {
  JN = 12;
  jvec x0 = jv_vars(x, 0), x1 = jv_vars(x + 3, 3), xa = jv_vars(x + 6, 6), xb = jv_vars(x + 9, 9);
  jvec e = jv_sub(x1, x0);
  jvec n1 = jv_cross(e, jv_sub(xa, x0));
  jvec n2 = jv_cross(jv_sub(x0, x1), jv_sub(xb, x1));
  jet le = jsqrt(jv_dot(e, e));
  jvec c = jv_cross(n1, n2);
  jet sn = jdiv(jv_dot(c, e), le);
  jet cs = jv_dot(n1, n2);
  return jatan2(sn, cs);
}
static double hinge_theta_plain(const double* x) {
  jet t = hinge_theta_jet(x);
  return t.v;
}
OR_EXPORT void or_hinge_rest(const double* X, double* theta0, double* weight) {
  *theta0 = hinge_theta_plain(X);
  double e[3], a1[3], a2[3];
  for (int k = 0; k < 3; ++k) { e[k] = X[3 + k] - X[k]; a1[k] = X[6 + k] - X[k]; a2[k] = X[9 + k] - X[3 + k]; }
  double c1[3] = {e[1] * a1[2] - e[2] * a1[1], e[2] * a1[0] - e[0] * a1[2], e[0] * a1[1] - e[1] * a1[0]};
  double c2[3] = {e[1] * a2[2] - e[2] * a2[1], e[2] * a2[0] - e[0] * a2[2], e[0] * a2[1] - e[1] * a2[0]};
  double A1 = 0.5 * sqrt(c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]);
  double A2 = 0.5 * sqrt(c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2]);
  double le2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
  *weight = 3.0 * le2 / (A1 + A2);
}
OR_EXPORT int or_bend_local(const double* x, const double* X, double kb, int project, double* E, double* g, double* H) {
  double th0, wgt;
  or_hinge_rest(X, &th0, &wgt);
  jet th = hinge_theta_jet(x);
  jet psi = jscale(jsq(jaddc(th, -th0)), kb * wgt);
  if (E) *E = psi.v;
  if (g) for (int i = 0; i < 12; ++i) g[i] = psi.g[i];
  if (H) { if (project) or_project_psd(12, psi.h, H); else memcpy(H, psi.h, sizeof(double) * 144); }
  return 0;
}

/* ======================================================================== */
/* Affine-body orthogonality: kv * 1/2 ||A^T A - I||_F^2, A = [c1 c2 c3]       */
/* (columns are the three A-nodes of the body).  Projected in its 9x9 space. */
/* ======================================================================== */
OR_EXPORT int or_abd_ortho_local(const double* A /*c1,c2,c3*/, double kv, int project, double* E, double* g, double* H) {
  JN = 9;
  jvec c[3];
  for (int k = 0; k < 3; ++k) c[k] = jv_vars(A + 3 * k, 3 * k);
  jet s = jc(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      jet d = jv_dot(c[i], c[j]);
      if (i == j) d = jaddc(d, -1.0);
      s = jadd(s, jsq(d));
    }
  s = jscale(s, 0.5 * kv);
  if (E) *E = s.v;
  if (g) for (int i = 0; i < 9; ++i) g[i] = s.g[i];
  if (H) { if (project) or_project_psd(9, s.h, H); else memcpy(H, s.h, sizeof(double) * 81); }
  return 0;
}

/* ======================================================================== */
/* contact distances with closest-feature classification                     */
/* (operation order fixed; no contraction)                                   */
/* ======================================================================== */
static inline void vsub(const double* a, const double* b, double* r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static inline double vdot(const double* a, const double* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }
static inline void vcross(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

enum { D_PP = 0, D_PE = 1, D_PT = 2, D_EE = 3 };
typedef struct { int dtype; int nloc; int loc[4]; } dclass;

static double d_pp(const double* p, const double* a) { double e[3]; vsub(p, a, e); return vdot(e, e); }
static double d_pe(const double* p, const double* a, const double* b) {
  double e[3], w[3], c[3];
  vsub(b, a, e); vsub(p, a, w); vcross(w, e, c);
  return vdot(c, c) / vdot(e, e);
}
static double d_ptplane(const double* p, const double* a, const double* b, const double* c) {
  double ab[3], ac[3], n[3], w[3];
  vsub(b, a, ab); vsub(c, a, ac); vcross(ab, ac, n); vsub(p, a, w);
  double t = vdot(w, n);
  return t * t / vdot(n, n);
}
static double d_eeline(const double* a0, const double* a1, const double* b0, const double* b1) {
  double da[3], db[3], w[3], cr[3];
  vsub(a1, a0, da); vsub(b1, b0, db); vsub(a0, b0, w); vcross(da, db, cr);
  double t = vdot(w, cr);
  return t * t / vdot(cr, cr);
}

/* point-triangle: local vertices 0 = p, 1..3 = triangle.  Returns subtype
 * 0/1/2: nearest triangle vertex a/b/c; 3: edge ab; 4: edge bc; 5: edge ca; 6: interior */
OR_EXPORT int or_pt_classify(const double* p, const double* a, const double* b, const double* c, double* s_out) {
  double ab[3], ac[3], ap[3], bp[3], cp[3];
  vsub(b, a, ab); vsub(c, a, ac); vsub(p, a, ap);
  double d1 = vdot(ab, ap), d2 = vdot(ac, ap);
  int st;
  if (d1 <= 0.0 && d2 <= 0.0) { st = 0; goto done; }
  vsub(p, b, bp);
  double d3 = vdot(ab, bp), d4 = vdot(ac, bp);
  if (d3 >= 0.0 && d4 <= d3) { st = 1; goto done; }
  double vc = d1 * d4 - d3 * d2;
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) { st = 3; goto done; }
  vsub(p, c, cp);
  double d5 = vdot(ab, cp), d6 = vdot(ac, cp);
  if (d6 >= 0.0 && d5 <= d6) { st = 2; goto done; }
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) { st = 5; goto done; }
  double va = d3 * d6 - d5 * d4;
  if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) { st = 4; goto done; }
  st = 6;
done:
  if (s_out) {
    switch (st) {
      case 0: *s_out = d_pp(p, a); break;
      case 1: *s_out = d_pp(p, b); break;
      case 2: *s_out = d_pp(p, c); break;
      case 3: *s_out = d_pe(p, a, b); break;
      case 4: *s_out = d_pe(p, b, c); break;
      case 5: *s_out = d_pe(p, c, a); break;
      default: *s_out = d_ptplane(p, a, b, c); break;
    }
  }
  return st;
}
static dclass pt_dclass(int st) {
  static const dclass T[7] = {
      {D_PP, 2, {0, 1, 0, 0}}, {D_PP, 2, {0, 2, 0, 0}}, {D_PP, 2, {0, 3, 0, 0}},
      {D_PE, 3, {0, 1, 2, 0}}, {D_PE, 3, {0, 2, 3, 0}}, {D_PE, 3, {0, 3, 1, 0}},
      {D_PT, 4, {0, 1, 2, 3}}};
  return T[st];
}

/* point-segment with closed-interval rule: returns 0 = nearest u, 1 = nearest v, 2 = interior */
static int pe_classify(const double* p, const double* u, const double* v, double* s) {
  double e[3], w[3];
  vsub(v, u, e); vsub(p, u, w);
  double t = vdot(w, e);
  if (t <= 0.0) { *s = vdot(w, w); return 0; }
  double ee = vdot(e, e);
  if (t >= ee) { *s = d_pp(p, v); return 1; }
  *s = d_pe(p, u, v);
  return 2;
}

#define EE_PARALLEL_EPS 1e-10
/* edge-edge: local vertices 0,1 = edge a; 2,3 = edge b.  Subtype 0 = interior
 * (line-line); 1 + 3*k + r for endpoint case k (a0 vs b, a1 vs b, b0 vs a,
 * b1 vs a) and result r (0 nearest first seg vertex, 1 second, 2 interior). */
OR_EXPORT int or_ee_classify(const double* a0, const double* a1, const double* b0, const double* b1, double* s_out) {
  double da[3], db[3], w[3], cr[3];
  vsub(a1, a0, da); vsub(b1, b0, db); vsub(a0, b0, w); vcross(da, db, cr);
  double A = vdot(da, da), B = vdot(da, db), C = vdot(db, db), D = vdot(da, w), Ee = vdot(db, w);
  double den = vdot(cr, cr);
  if (den > EE_PARALLEL_EPS * A * C) {
    double sn = B * Ee - C * D, tn = A * Ee - B * D;
    if (sn > 0.0 && sn < den && tn > 0.0 && tn < den) {
      if (s_out) *s_out = d_eeline(a0, a1, b0, b1);
      return 0;
    }
  }
  const double* P[4] = {a0, a1, b0, b1};
  const double* U[4] = {b0, b0, a0, a0};
  const double* V[4] = {b1, b1, a1, a1};
  double best = 0.0;
  int bk = -1, br = 0;
  for (int k = 0; k < 4; ++k) {
    double s;
    int r = pe_classify(P[k], U[k], V[k], &s);
    if (bk < 0 || s < best) { best = s; bk = k; br = r; }
  }
  if (s_out) *s_out = best;
  return 1 + 3 * bk + br;
}
static dclass ee_dclass(int st) {
  dclass d;
  if (st == 0) { d.dtype = D_EE; d.nloc = 4; d.loc[0] = 0; d.loc[1] = 1; d.loc[2] = 2; d.loc[3] = 3; return d; }
  int k = (st - 1) / 3, r = (st - 1) % 3;
  static const int pv[4] = {0, 1, 2, 3}, uu[4] = {2, 2, 0, 0}, vv[4] = {3, 3, 1, 1};
  d.loc[0] = pv[k];
  if (r == 0) { d.dtype = D_PP; d.nloc = 2; d.loc[1] = uu[k]; }
  else if (r == 1) { d.dtype = D_PP; d.nloc = 2; d.loc[1] = vv[k]; }
  else { d.dtype = D_PE; d.nloc = 3; d.loc[1] = uu[k]; d.loc[2] = vv[k]; }
  d.loc[3] = 0;
  return d;
}

/* squared distance of the classified feature pair as a jet over 3*nloc vars */
static jet dist_jet(const dclass* dc, const double* xloc /*4 x 3 local vertices*/) {
  JN = 3 * dc->nloc;
  jvec v[4];
  for (int i = 0; i < dc->nloc; ++i) v[i] = jv_vars(xloc + 3 * dc->loc[i], 3 * i);
  switch (dc->dtype) {
    case D_PP: { jvec e = jv_sub(v[0], v[1]); return jv_dot(e, e); }
    case D_PE: {
      jvec e = jv_sub(v[2], v[1]), w = jv_sub(v[0], v[1]);
      jvec c = jv_cross(w, e);
      return jdiv(jv_dot(c, c), jv_dot(e, e));
    }
    case D_PT: {
      jvec n = jv_cross(jv_sub(v[2], v[1]), jv_sub(v[3], v[1]));
      jet t = jv_dot(jv_sub(v[0], v[1]), n);
      return jdiv(jsq(t), jv_dot(n, n));
    }
    default: {
      jvec cr = jv_cross(jv_sub(v[1], v[0]), jv_sub(v[3], v[2]));
      jet t = jv_dot(jv_sub(v[0], v[2]), cr);
      return jdiv(jsq(t), jv_dot(cr, cr));
    }
  }
}

/* ======================================================================== */
/* barrier (E7): form 0 = -(s - sh)^2 ln(s/sh)  (IPC, squared distances)     */
/*               form 1 = (s - sh)^2 ln^2(s/sh) (the paper's PP listing)     */
/* ======================================================================== */
static jet barrier_jet(jet s, double sh, int form) {
  if (s.v >= sh) return jc(0.0);
  jet d = jaddc(s, -sh);
  jet l = jlog(jscale(s, 1.0 / sh));
  if (form == 1) return jmul(jsq(d), jsq(l));
  return jscale(jmul(jsq(d), l), -1.0);
}
OR_EXPORT void or_barrier_scalar(double s, double sh, int form, double* b, double* db, double* d2b) {
  int save = JN;
  JN = 1;
  jet r = barrier_jet(jvar(s, 0), sh, form);
  *b = r.v; *db = r.g[0]; *d2b = r.h[0];
  JN = save;
}

/* Contact pair in position space: kind 0 = PT (4 verts), 1 = EE (4 verts),
 * 2 = PG (1 vert + plane).  Returns kappa*b, gradient (3*nv) and projected
 * (or exact) Hessian in position space for all nv local vertices.        */
OR_EXPORT int or_pair_local(int kind, const double* xloc, const double* plane, double kappa, double sh, int form,
                            int project, double* E, double* g, double* H, int* subtype) {
  int nv = (kind == 2) ? 1 : 4;
  int n = 3 * nv;
  jet bj;
  dclass dc;
  if (kind == 2) {
    JN = 3;
    jvec p = jv_vars(xloc, 0);
    jet d = jaddc(jadd(jadd(jscale(p.c[0], plane[0]), jscale(p.c[1], plane[1])), jscale(p.c[2], plane[2])), -plane[3]);
    bj = barrier_jet(jsq(d), sh, form);
    dc.dtype = -1; dc.nloc = 1; dc.loc[0] = 0;
    if (subtype) *subtype = 0;
  } else {
    int st = (kind == 0) ? or_pt_classify(xloc, xloc + 3, xloc + 6, xloc + 9, NULL)
                         : or_ee_classify(xloc, xloc + 3, xloc + 6, xloc + 9, NULL);
    if (subtype) *subtype = st;
    dc = (kind == 0) ? pt_dclass(st) : ee_dclass(st);
    jet s = dist_jet(&dc, xloc);
    bj = barrier_jet(s, sh, form);
  }
  /* scatter from the classified local variables to all nv vertices */
  int m = 3 * dc.nloc;
  double Hl[144], Hp[144];
  for (int i = 0; i < m * m; ++i) Hl[i] = kappa * bj.h[i];
  if (project) or_project_psd(m, Hl, Hp); else memcpy(Hp, Hl, sizeof(double) * m * m);
  if (E) *E = kappa * bj.v;
  if (g) {
    memset(g, 0, sizeof(double) * n);
    for (int i = 0; i < dc.nloc; ++i)
      for (int k = 0; k < 3; ++k) g[3 * dc.loc[i] + k] += kappa * bj.g[3 * i + k];
  }
  if (H) {
    memset(H, 0, sizeof(double) * n * n);
    for (int i = 0; i < dc.nloc; ++i)
      for (int j = 0; j < dc.nloc; ++j)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            H[(3 * dc.loc[i] + a) * n + 3 * dc.loc[j] + b] += Hp[(3 * i + a) * m + 3 * j + b];
  }
  return 0;
}

/* ======================================================================== */
/* additive CCD (Li, Kaufman, Jiang 2021, "Codimensional IPC", ACCD):        */
/* conservative advancement along x + t dx, t in [0, tmax], keeping a gap of */
/* at least gap_s times the starting distance.                              */
/* ======================================================================== */
static double pair_dist2(int kind, const double* x) {
  double s;
  if (kind == 0) or_pt_classify(x, x + 3, x + 6, x + 9, &s);
  else or_ee_classify(x, x + 3, x + 6, x + 9, &s);
  return s;
}
OR_EXPORT double or_accd(int kind, const double* x0, const double* dx0, double gap_s, double tmax, int max_iter, int* iters) {
  double x[12], dx[12], mean[3] = {0, 0, 0};
  memcpy(x, x0, sizeof x);
  memcpy(dx, dx0, sizeof dx);
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) mean[k] += 0.25 * dx[3 * i + k];
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 3; ++k) dx[3 * i + k] -= mean[k];
  double nrm[4];
  for (int i = 0; i < 4; ++i) nrm[i] = sqrt(vdot(dx + 3 * i, dx + 3 * i));
  double lp;
  if (kind == 0) lp = nrm[0] + fmax(nrm[1], fmax(nrm[2], nrm[3]));
  else lp = fmax(nrm[0], nrm[1]) + fmax(nrm[2], nrm[3]);
  if (iters) *iters = 0;
  if (lp == 0.0) return tmax;
  double d = sqrt(pair_dist2(kind, x));
  double gap = gap_s * d;
  double t = 0.0, tl = (1.0 - gap_s) * d / lp;
  for (int it = 0; it < max_iter; ++it) {
    for (int i = 0; i < 12; ++i) x[i] += tl * dx[i];
    d = sqrt(pair_dist2(kind, x));
    if (iters) *iters = it + 1;
    if (t > 0.0 && d < gap) return t;
    t += tl;
    if (t > tmax) return tmax;
    tl = (1.0 - gap_s) * d / lp;
  }
  return t; /* iteration cap: t is still a safe (conservative) bound */
}
/* point-plane: exact linear trajectory */
OR_EXPORT double or_pg_ccd(const double* p, const double* dp, const double* plane, double gap_s, double tmax) {
  double d0 = (plane[0] * p[0] + plane[1] * p[1]) + plane[2] * p[2] - plane[3];
  double v = (plane[0] * dp[0] + plane[1] * dp[1]) + plane[2] * dp[2];
  if (v >= 0.0) return tmax;
  double t = (1.0 - gap_s) * d0 / (-v);
  return t < tmax ? t : tmax;
}

/* ======================================================================== */
/* system                                                                     */
/* ======================================================================== */
typedef struct {
  int nv, nt, nc, nh, nb, nst, nse, nsv, np, nfix;
  double* rest; int* vbody; int* tets; double *tE, *tnu, *trho;
  int* tris; double *cE, *cnu, *cth, *crho;
  int* hinges; double* hkb;
  double *bmass, *bvol, *bkappa;
  int *stris, *sedges, *sverts;
  double* planes;
  int* fixed; double* fixvel;
  /* params */
  double dt, dhat, kappa, grav[3], newton_tol, pcg_tol, gap_s;
  int pcg_max, newton_max, ls_max, form, ccd_max_iter;
  /* derived */
  int nn, nfree;
  int* vnode;     /* free: node; body: first node of its body; fixed: -1 */
  int* vfixed;    /* 1 if fixed */
  double* vr;     /* body-relative rest position r (3 per vertex) */
  double* vmass;
  double* xfix;   /* current positions of fixed vertices (3 per vertex, others unused) */
  double* nodemass; /* free nodes: m; bodies: 4x4 scalar mass matrix (16 per body) */
  double *tmu, *tlam, *cmu, *clam;
  int cmodel;  /* membrane model: 0 StVK (cmu, clam), 1 Baraff-Witkin (cE stretch, cshear) */
  double* cshear;
  int ne;        /* cage-embedded vertices (vert_body -2) */
  int* emb_of;   /* [nv] embedding row or -1 */
  int* emb_cage; /* [ne][8] cage vertex ids */
  double* emb_w; /* [ne][8] trilinear weights */
  /* adaptive barrier stiffness (off unless set): bounds, distance threshold, state */
  int kadapt, kinit;
  double kmin, kmax, kdmin, dmin_prev;
} osys;

static void* dupa(const void* p, size_t bytes) {
  if (bytes == 0) return calloc(1, 8);
  void* r = malloc(bytes);
  memcpy(r, p, bytes);
  return r;
}

OR_EXPORT void* or_create(int nv, const double* rest, const int* vbody,
                          int nfix, const int* fixed, const double* fixvel,
                          int nt, const int* tets, const double* tE, const double* tnu, const double* trho,
                          int nc, const int* tris, const double* cE, const double* cnu, const double* cth, const double* crho,
                          int nh, const int* hinges, const double* hkb,
                          int nb, const double* bmass, const double* bvol, const double* bkappa,
                          int nst, const int* stris, int nse, const int* sedges, int nsv, const int* sverts,
                          int np, const double* planes,
                          const double* fparams /* dt, dhat, kappa, gx, gy, gz, newton_tol, pcg_tol, gap_s */,
                          const int* iparams /* pcg_max, newton_max, ls_max, barrier_form, ccd_max_iter */) {
  osys* S = calloc(1, sizeof(osys));
  S->nv = nv; S->nt = nt; S->nc = nc; S->nh = nh; S->nb = nb; S->nst = nst; S->nse = nse; S->nsv = nsv; S->np = np; S->nfix = nfix;
  S->rest = dupa(rest, sizeof(double) * 3 * nv);
  S->vbody = dupa(vbody, sizeof(int) * nv);
  S->fixed = dupa(fixed, sizeof(int) * nfix);
  S->fixvel = dupa(fixvel, sizeof(double) * 3 * nfix);
  S->tets = dupa(tets, sizeof(int) * 4 * nt);
  S->tE = dupa(tE, sizeof(double) * nt); S->tnu = dupa(tnu, sizeof(double) * nt); S->trho = dupa(trho, sizeof(double) * nt);
  S->tris = dupa(tris, sizeof(int) * 3 * nc);
  S->cE = dupa(cE, sizeof(double) * nc); S->cnu = dupa(cnu, sizeof(double) * nc);
  S->cth = dupa(cth, sizeof(double) * nc); S->crho = dupa(crho, sizeof(double) * nc);
  S->hinges = dupa(hinges, sizeof(int) * 4 * nh); S->hkb = dupa(hkb, sizeof(double) * nh);
  S->bmass = dupa(bmass, sizeof(double) * nb); S->bvol = dupa(bvol, sizeof(double) * nb); S->bkappa = dupa(bkappa, sizeof(double) * nb);
  S->stris = dupa(stris, sizeof(int) * 3 * nst); S->sedges = dupa(sedges, sizeof(int) * 2 * nse); S->sverts = dupa(sverts, sizeof(int) * nsv);
  S->planes = dupa(planes, sizeof(double) * 4 * np);
  S->dt = fparams[0]; S->dhat = fparams[1]; S->kappa = fparams[2];
  S->grav[0] = fparams[3]; S->grav[1] = fparams[4]; S->grav[2] = fparams[5];
  S->newton_tol = fparams[6]; S->pcg_tol = fparams[7]; S->gap_s = fparams[8];
  S->pcg_max = iparams[0]; S->newton_max = iparams[1]; S->ls_max = iparams[2]; S->form = iparams[3]; S->ccd_max_iter = iparams[4];

  /* DOF layout (App. A "Gradient Size Computation"): free vertices first
   * (3 DOF each), then 4 nodes (t, A col 1..3) per affine body.  Fixed
   * vertices carry no DOF. */
  S->vfixed = calloc(nv, sizeof(int));
  for (int i = 0; i < nfix; ++i) S->vfixed[fixed[i]] = 1;
  S->vnode = malloc(sizeof(int) * nv);
  int nf = 0;
  for (int v = 0; v < nv; ++v) {
    if (S->vfixed[v]) S->vnode[v] = -1;
    else if (vbody[v] == -1) S->vnode[v] = nf++;
    else if (vbody[v] <= -2) S->vnode[v] = -2; /* cage-embedded: or_set_embedding gives its map */
  }
  S->nfree = nf;
  S->nn = nf + 4 * nb;
  for (int v = 0; v < nv; ++v)
    if (!S->vfixed[v] && vbody[v] >= 0) S->vnode[v] = nf + 4 * vbody[v];
  /* lumped vertex masses: rho V / 4 per tet vertex, rho A t / 3 per cloth
   * vertex, body mass spread uniformly over the body's vertices */
  S->vmass = calloc(nv, sizeof(double));
  S->tmu = malloc(sizeof(double) * (nt + 1)); S->tlam = malloc(sizeof(double) * (nt + 1));
  for (int e = 0; e < nt; ++e) {
    double X[12], Dminv[9], vol;
    for (int a = 0; a < 4; ++a) memcpy(X + 3 * a, rest + 3 * tets[4 * e + a], sizeof(double) * 3);
    or_tet_rest(X, Dminv, &vol);
    for (int a = 0; a < 4; ++a) S->vmass[tets[4 * e + a]] += trho[e] * vol / 4.0;
    or_lame(tE[e], tnu[e], &S->tmu[e], &S->tlam[e]);
  }
  S->cmu = malloc(sizeof(double) * (nc + 1)); S->clam = malloc(sizeof(double) * (nc + 1));
  for (int e = 0; e < nc; ++e) {
    double X[9], Dminv[4], area;
    for (int a = 0; a < 3; ++a) memcpy(X + 3 * a, rest + 3 * tris[3 * e + a], sizeof(double) * 3);
    or_tri_rest(X, Dminv, &area);
    for (int a = 0; a < 3; ++a) S->vmass[tris[3 * e + a]] += crho[e] * area * cth[e] / 3.0;
    or_lame_ps(cE[e], cnu[e], &S->cmu[e], &S->clam[e]);
  }
  int* bcount = calloc(nb + 1, sizeof(int));
  double* bcen = calloc(3 * (nb + 1), sizeof(double));
  for (int v = 0; v < nv; ++v)
    if (vbody[v] >= 0) {
      bcount[vbody[v]]++;
      for (int k = 0; k < 3; ++k) bcen[3 * vbody[v] + k] += rest[3 * v + k];
    }
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 3; ++k) bcen[3 * b + k] /= bcount[b];
  S->vr = calloc((size_t)3 * nv + 3, sizeof(double));
  for (int v = 0; v < nv; ++v)
    if (vbody[v] >= 0) {
      S->vmass[v] = bmass[vbody[v]] / bcount[vbody[v]];
      for (int k = 0; k < 3; ++k) S->vr[3 * v + k] = rest[3 * v + k] - bcen[3 * vbody[v] + k];
    }
  /* node mass: free m I3; body M_ab = sum_v m_v w_a w_b, w = (1, r1, r2, r3) */
  S->nodemass = calloc(nf + 16 * nb + 1, sizeof(double));
  for (int v = 0; v < nv; ++v) {
    if (S->vfixed[v] || vbody[v] <= -2) continue; /* embedded vertices carry no mass */
    if (vbody[v] < 0) S->nodemass[S->vnode[v]] = S->vmass[v];
    else {
      double w[4] = {1.0, S->vr[3 * v], S->vr[3 * v + 1], S->vr[3 * v + 2]};
      double* M = S->nodemass + nf + 16 * vbody[v];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) M[4 * a + b] += S->vmass[v] * w[a] * w[b];
    }
  }
  S->xfix = calloc((size_t)3 * nv + 3, sizeof(double));
  for (int v = 0; v < nv; ++v)
    if (S->vfixed[v]) memcpy(S->xfix + 3 * v, rest + 3 * v, sizeof(double) * 3);
  free(bcount);
  free(bcen);
  return S;
}

OR_EXPORT void or_destroy(void* p) {
  osys* S = p;
  if (!S) return;
  void* ptrs[] = {S->rest, S->vbody, S->tets, S->tE, S->tnu, S->trho, S->tris, S->cE, S->cnu, S->cth, S->crho, S->hinges,
                  S->hkb, S->bmass, S->bvol, S->bkappa, S->stris, S->sedges, S->sverts, S->planes, S->fixed, S->fixvel,
                  S->vnode, S->vfixed, S->vr, S->vmass, S->xfix, S->nodemass, S->tmu, S->tlam, S->cmu, S->clam,
                  S->cshear, S->emb_of, S->emb_cage, S->emb_w};
  for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) free(ptrs[i]);
  free(S);
}

OR_EXPORT int or_num_nodes(void* p) { return ((osys*)p)->nn; }
OR_EXPORT int or_num_free(void* p) { return ((osys*)p)->nfree; }
/* cage embedding (Sec. "Caged Bunny"): vertex verts[e] (vert_body -2) sits
 * at sum_k w[e][k] x(cage[e][k]) over its cage cell's 8 free vertices */
OR_EXPORT void or_set_embedding(void* p, int ne, const int* verts, const int* cage, const double* w) {
  osys* S = p;
  S->ne = ne;
  free(S->emb_of); free(S->emb_cage); free(S->emb_w);
  S->emb_of = malloc(sizeof(int) * (S->nv + 1));
  for (int v = 0; v < S->nv; ++v) S->emb_of[v] = -1;
  for (int e = 0; e < ne; ++e) S->emb_of[verts[e]] = e;
  S->emb_cage = dupa(cage, sizeof(int) * 8 * (ne > 0 ? ne : 1));
  S->emb_w = dupa(w, sizeof(double) * 8 * (ne > 0 ? ne : 1));
}
/* membrane model of the cloth triangles: 0 StVK (default), 1 Baraff-Witkin
 * with the stretch stiffness in tri_E and shear[e] the shear stiffness */
OR_EXPORT void or_set_cloth_model(void* p, int model, const double* shear) {
  osys* S = p;
  S->cmodel = model;
  free(S->cshear);
  S->cshear = NULL;
  if (model == 1) S->cshear = dupa(shear, sizeof(double) * (S->nc > 0 ? S->nc : 1));
}
OR_EXPORT void or_vertex_info(void* p, int* vnode, double* vr, double* vmass) {
  osys* S = p;
  memcpy(vnode, S->vnode, sizeof(int) * S->nv);
  memcpy(vr, S->vr, sizeof(double) * 3 * S->nv);
  memcpy(vmass, S->vmass, sizeof(double) * S->nv);
}

/* vertex -> (up to 8) node ids and weights; position p = sum w_k x[node_k]
 * (Sec. "UNION": free -> itself; affine -> (t, A1, A2, A3) with weights
 * (1, r1, r2, r3); cage-embedded -> the 8 nodes of its cage cell with its
 * trilinear weights, Sec. "Caged Bunny") */
static int vmap(const osys* S, int v, int* nodes, double* w) {
  if (S->vfixed[v]) return 0;
  if (S->vbody[v] <= -2) {
    const int e = S->emb_of[v];
    for (int k = 0; k < 8; ++k) { nodes[k] = S->vnode[S->emb_cage[8 * e + k]]; w[k] = S->emb_w[8 * e + k]; }
    return 8;
  }
  if (S->vbody[v] < 0) { nodes[0] = S->vnode[v]; w[0] = 1.0; return 1; }
  int b0 = S->vnode[v];
  for (int k = 0; k < 4; ++k) nodes[k] = b0 + k;
  w[0] = 1.0; w[1] = S->vr[3 * v]; w[2] = S->vr[3 * v + 1]; w[3] = S->vr[3 * v + 2];
  return 4;
}
static void vpos(const osys* S, const double* x, int v, double* p) {
  if (S->vfixed[v]) { memcpy(p, S->xfix + 3 * v, sizeof(double) * 3); return; }
  int nodes[8]; double w[8];
  int m = vmap(S, v, nodes, w);
  p[0] = p[1] = p[2] = 0.0;
  for (int k = 0; k < m; ++k)
    for (int c = 0; c < 3; ++c) p[c] += w[k] * x[3 * nodes[k] + c];
}
OR_EXPORT void or_vertex_positions(void* p, const double* x, double* P) {
  osys* S = p;
  for (int v = 0; v < S->nv; ++v) vpos(S, x, v, P + 3 * v);
}
OR_EXPORT void or_initial_state(void* p, const double* vel0, double* x, double* v) {
  osys* S = p;
  memset(x, 0, sizeof(double) * 3 * S->nn);
  memset(v, 0, sizeof(double) * 3 * S->nn);
  for (int i = 0; i < S->nv; ++i)
    if (!S->vfixed[i] && S->vbody[i] == -1)
      for (int c = 0; c < 3; ++c) { x[3 * S->vnode[i] + c] = S->rest[3 * i + c]; v[3 * S->vnode[i] + c] = vel0[3 * i + c]; }
  for (int b = 0; b < S->nb; ++b) {
    int b0 = S->nfree + 4 * b;
    /* t = body centre: any body vertex minus its r */
    for (int i = 0; i < S->nv; ++i)
      if (S->vbody[i] == b) {
        for (int c = 0; c < 3; ++c) x[3 * b0 + c] = S->rest[3 * i + c] - S->vr[3 * i + c];
        break;
      }
    for (int k = 0; k < 3; ++k) x[3 * (b0 + 1 + k) + k] = 1.0; /* A = I */
  }
}
OR_EXPORT void or_set_fixed_positions(void* p, const double* xfix_all /* 3*nv, only fixed rows read */) {
  osys* S = p;
  for (int i = 0; i < S->nfix; ++i) memcpy(S->xfix + 3 * S->fixed[i], xfix_all + 3 * S->fixed[i], sizeof(double) * 3);
}
OR_EXPORT void or_get_fixed_positions(void* p, double* xfix_all) {
  osys* S = p;
  memcpy(xfix_all, S->xfix, sizeof(double) * 3 * S->nv);
}

/* ------------------------------------------------------------------------ */
/* contact pairs (D6, E8): PT, EE, PG with s < dhat^2                        */
/* ------------------------------------------------------------------------ */
typedef struct { int a, b, st; } opair;
typedef struct { opair* p; int n, cap; } plist;
static void pl_push(plist* L, int a, int b, int st) {
  if (L->n == L->cap) { L->cap = L->cap ? 2 * L->cap : 1024; L->p = realloc(L->p, sizeof(opair) * L->cap); }
  L->p[L->n].a = a; L->p[L->n].b = b; L->p[L->n].st = st; L->n++;
}
static int cmp_pair(const void* x, const void* y) {
  const opair *A = x, *B = y;
  if (A->a != B->a) return A->a < B->a ? -1 : 1;
  if (A->b != B->b) return A->b < B->b ? -1 : 1;
  return 0;
}
/* exclusions: shared vertex, same affine body, all vertices fixed */
static int pt_excluded(const osys* S, int v, const int* t) {
  if (v == t[0] || v == t[1] || v == t[2]) return 1;
  int bv = S->vbody[v];
  if (bv >= 0 && bv == S->vbody[t[0]]) return 1;
  if (S->vfixed[v] && S->vfixed[t[0]] && S->vfixed[t[1]] && S->vfixed[t[2]]) return 1;
  return 0;
}
static int ee_excluded(const osys* S, const int* e, const int* f) {
  if (e[0] == f[0] || e[0] == f[1] || e[1] == f[0] || e[1] == f[1]) return 1;
  int be = S->vbody[e[0]];
  if (be >= 0 && be == S->vbody[f[0]]) return 1;
  if (S->vfixed[e[0]] && S->vfixed[e[1]] && S->vfixed[f[0]] && S->vfixed[f[1]]) return 1;
  return 0;
}

/* Candidate pairs between two sets of axis-aligned boxes (A queried against
 * a uniform grid built on B).  A conservative filter only: the pair set is
 * decided afterwards by the exact distance test.  same != 0 keeps only j > i. */
typedef struct { int* a; int* b; long n, cap; } cand;
static void cand_push(cand* C, int i, int j) {
  if (C->n == C->cap) { C->cap = C->cap ? 2 * C->cap : 4096; C->a = realloc(C->a, sizeof(int) * C->cap); C->b = realloc(C->b, sizeof(int) * C->cap); }
  C->a[C->n] = i; C->b[C->n] = j; C->n++;
}
static int aabb_overlap(const double* alo, const double* ahi, const double* blo, const double* bhi) {
  for (int c = 0; c < 3; ++c)
    if (ahi[c] < blo[c] || bhi[c] < alo[c]) return 0;
  return 1;
}
static void box_pairs(int nA, const double* Alo, const double* Ahi, int nB, const double* Blo, const double* Bhi,
                      int same, int brute, cand* C) {
  C->n = 0;
  if (nA == 0 || nB == 0) return;
  if (brute) {
    for (int i = 0; i < nA; ++i)
      for (int j = same ? i + 1 : 0; j < nB; ++j)
        if (aabb_overlap(Alo + 3 * i, Ahi + 3 * i, Blo + 3 * j, Bhi + 3 * j)) cand_push(C, i, j);
    return;
  }
  double gl[3] = {1e300, 1e300, 1e300}, gh[3] = {-1e300, -1e300, -1e300}, ext = 0.0;
  for (int j = 0; j < nB; ++j)
    for (int c = 0; c < 3; ++c) {
      if (Blo[3 * j + c] < gl[c]) gl[c] = Blo[3 * j + c];
      if (Bhi[3 * j + c] > gh[c]) gh[c] = Bhi[3 * j + c];
      if (Bhi[3 * j + c] - Blo[3 * j + c] > ext) ext = Bhi[3 * j + c] - Blo[3 * j + c];
    }
  double span = 0.0;
  for (int c = 0; c < 3; ++c) if (gh[c] - gl[c] > span) span = gh[c] - gl[c];
  double cell = ext > 0.0 ? ext : 1.0;
  if (span / cell > 256.0) cell = span / 256.0;
  int dim[3];
  for (int c = 0; c < 3; ++c) dim[c] = (int)((gh[c] - gl[c]) / cell) + 1;
  long ncell = (long)dim[0] * dim[1] * dim[2];
  int* start = calloc(ncell + 2, sizeof(int));
  int c0[3], c1[3];
#define CELLS(lo, hi)                                                    \
  for (int c = 0; c < 3; ++c) {                                         \
    int a_ = (int)floor(((lo)[c] - gl[c]) / cell), b_ = (int)floor(((hi)[c] - gl[c]) / cell); \
    c0[c] = a_ < 0 ? 0 : (a_ > dim[c] - 1 ? dim[c] - 1 : a_);           \
    c1[c] = b_ < 0 ? 0 : (b_ > dim[c] - 1 ? dim[c] - 1 : b_);           \
  }
  for (int j = 0; j < nB; ++j) {
    CELLS(Blo + 3 * j, Bhi + 3 * j);
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) start[((long)z * dim[1] + y) * dim[0] + x + 1]++;
  }
  for (long i = 0; i < ncell; ++i) start[i + 1] += start[i];
  int* items = malloc(sizeof(int) * (start[ncell] + 1));
  int* fill = calloc(ncell + 1, sizeof(int));
  for (int j = 0; j < nB; ++j) {
    CELLS(Blo + 3 * j, Bhi + 3 * j);
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) {
          long id = ((long)z * dim[1] + y) * dim[0] + x;
          items[start[id] + fill[id]++] = j;
        }
  }
  int* seen = malloc(sizeof(int) * nB);
  for (int j = 0; j < nB; ++j) seen[j] = -1;
  for (int i = 0; i < nA; ++i) {
    CELLS(Alo + 3 * i, Ahi + 3 * i);
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) {
          long id = ((long)z * dim[1] + y) * dim[0] + x;
          for (int q = start[id]; q < start[id + 1]; ++q) {
            int j = items[q];
            if (seen[j] == i) continue;
            seen[j] = i;
            if (same && j <= i) continue;
            if (aabb_overlap(Alo + 3 * i, Ahi + 3 * i, Blo + 3 * j, Bhi + 3 * j)) cand_push(C, i, j);
          }
        }
  }
#undef CELLS
  free(start); free(items); free(fill); free(seen);
}
static void aabb_of(const double* P, const int* ids, int k, double* lo, double* hi) {
  for (int c = 0; c < 3; ++c) { lo[c] = P[3 * ids[0] + c]; hi[c] = lo[c]; }
  for (int i = 1; i < k; ++i)
    for (int c = 0; c < 3; ++c) { double v = P[3 * ids[i] + c]; if (v < lo[c]) lo[c] = v; if (v > hi[c]) hi[c] = v; }
}
/* boxes of k-vertex primitives over positions P0 (and P1 if given: swept), grown by infl */
static void prim_boxes(const double* P0, const double* P1, const int* prims, int n, int k, double infl, double* lo, double* hi) {
  for (int e = 0; e < n; ++e) {
    aabb_of(P0, prims + k * e, k, lo + 3 * e, hi + 3 * e);
    if (P1) {
      double l1[3], h1[3];
      aabb_of(P1, prims + k * e, k, l1, h1);
      for (int c = 0; c < 3; ++c) { lo[3 * e + c] = fmin(lo[3 * e + c], l1[c]); hi[3 * e + c] = fmax(hi[3 * e + c], h1[c]); }
    }
    for (int c = 0; c < 3; ++c) { lo[3 * e + c] -= infl; hi[3 * e + c] += infl; }
  }
}

/* Detect all pairs at vertex positions P.  brute != 0 -> O(n^2) enumeration. */
static void detect(const osys* S, const double* P, int brute, plist* PT, plist* EE, plist* PG) {
  double sh = S->dhat * S->dhat;
  PT->n = EE->n = PG->n = 0;
  for (int i = 0; i < S->nsv; ++i) {
    int v = S->sverts[i];
    if (S->vfixed[v]) continue;
    for (int k = 0; k < S->np; ++k) {
      const double* pl = S->planes + 4 * k;
      double d = vdot(pl, P + 3 * v) - pl[3];
      if (d > 0.0 && d * d < sh) pl_push(PG, v, k, 0);
    }
  }
  if (S->nst == 0) return;
  int nmax = S->nsv > S->nst ? S->nsv : S->nst;
  if (S->nse > nmax) nmax = S->nse;
  double *alo = malloc(sizeof(double) * 3 * nmax), *ahi = malloc(sizeof(double) * 3 * nmax);
  double *blo = malloc(sizeof(double) * 3 * nmax), *bhi = malloc(sizeof(double) * 3 * nmax);
  cand C = {0};
  prim_boxes(P, NULL, S->sverts, S->nsv, 1, S->dhat, alo, ahi);
  prim_boxes(P, NULL, S->stris, S->nst, 3, 0.0, blo, bhi);
  box_pairs(S->nsv, alo, ahi, S->nst, blo, bhi, 0, brute, &C);
  for (long q = 0; q < C.n; ++q) {
    int v = S->sverts[C.a[q]], t = C.b[q];
    const int* tv = S->stris + 3 * t;
    if (pt_excluded(S, v, tv)) continue;
    double s;
    int st = or_pt_classify(P + 3 * v, P + 3 * tv[0], P + 3 * tv[1], P + 3 * tv[2], &s);
    if (s < sh) pl_push(PT, v, t, st);
  }
  prim_boxes(P, NULL, S->sedges, S->nse, 2, S->dhat, alo, ahi);
  prim_boxes(P, NULL, S->sedges, S->nse, 2, 0.0, blo, bhi);
  box_pairs(S->nse, alo, ahi, S->nse, blo, bhi, 1, brute, &C);
  for (long q = 0; q < C.n; ++q) {
    int i = C.a[q], j = C.b[q];
    const int *e = S->sedges + 2 * i, *f = S->sedges + 2 * j;
    if (ee_excluded(S, e, f)) continue;
    double s;
    int st = or_ee_classify(P + 3 * e[0], P + 3 * e[1], P + 3 * f[0], P + 3 * f[1], &s);
    if (s < sh) pl_push(EE, i, j, st);
  }
  free(C.a); free(C.b); free(alo); free(ahi); free(blo); free(bhi);
  qsort(PT->p, PT->n, sizeof(opair), cmp_pair);
  qsort(EE->p, EE->n, sizeof(opair), cmp_pair);
  qsort(PG->p, PG->n, sizeof(opair), cmp_pair);
}

/* Exported detection; outputs (a, b, subtype) triples sorted by (a, b).
 * Returns 0, or -1 when a capacity is exceeded (counts are still written). */
OR_EXPORT int or_detect_pairs(void* p, const double* x, int brute, int cap, int* pt, int* npt, int* ee, int* nee, int* pg, int* npg) {
  osys* S = p;
  double* P = malloc(sizeof(double) * 3 * S->nv);
  or_vertex_positions(S, x, P);
  plist A = {0}, B = {0}, C = {0};
  detect(S, P, brute, &A, &B, &C);
  *npt = A.n; *nee = B.n; *npg = C.n;
  int rc = 0;
  if (A.n > cap || B.n > cap || C.n > cap) rc = -1;
  else {
    for (int i = 0; i < A.n; ++i) { pt[3 * i] = A.p[i].a; pt[3 * i + 1] = A.p[i].b; pt[3 * i + 2] = A.p[i].st; }
    for (int i = 0; i < B.n; ++i) { ee[3 * i] = B.p[i].a; ee[3 * i + 1] = B.p[i].b; ee[3 * i + 2] = B.p[i].st; }
    for (int i = 0; i < C.n; ++i) { pg[3 * i] = C.p[i].a; pg[3 * i + 1] = C.p[i].b; pg[3 * i + 2] = 0; }
  }
  free(A.p); free(B.p); free(C.p); free(P);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* energies                                                                  */
/* ------------------------------------------------------------------------ */
/* x_tilde = x_t + h v_t + h^2 M^-1 f_gravity: gravity moves free nodes and
 * the body translation node; with body-centred r the A-nodes get no force. */
OR_EXPORT void or_xtilde(void* p, const double* xt, const double* vt, double* xtil) {
  osys* S = p;
  double h = S->dt;
  for (int i = 0; i < S->nn; ++i)
    for (int c = 0; c < 3; ++c) xtil[3 * i + c] = xt[3 * i + c] + h * vt[3 * i + c];
  for (int i = 0; i < S->nfree; ++i)
    for (int c = 0; c < 3; ++c) xtil[3 * i + c] += h * h * S->grav[c];
  for (int b = 0; b < S->nb; ++b)
    for (int c = 0; c < 3; ++c) xtil[3 * (S->nfree + 4 * b) + c] += h * h * S->grav[c];
}

/* Neumaier compensated accumulator */
typedef struct { double s, c; } ksum;
static void kadd(ksum* k, double v) {
  double t = k->s + v;
  if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v; else k->c += (v - t) + k->s;
  k->s = t;
}
static double kval(const ksum* k) { return k->s + k->c; }

static void gather_pos(const osys* S, const double* P, const int* ids, int k, double* out) {
  for (int i = 0; i < k; ++i) memcpy(out + 3 * i, P + 3 * ids[i], sizeof(double) * 3);
}

/* term energies: out[0] inertia, [1] tets, [2] membrane, [3] bending, [4] ABD
 * orthogonality, [5] barrier; elastic terms already multiplied by h^2.      */
static void energy_terms(const osys* S, const double* x, const double* xtil, const double* P, const plist* PT,
                         const plist* EE, const plist* PG, double* out) {
  double h2 = S->dt * S->dt;
  ksum k[6];
  memset(k, 0, sizeof k);
  for (int i = 0; i < S->nfree; ++i) {
    double d[3];
    vsub(x + 3 * i, xtil + 3 * i, d);
    kadd(&k[0], 0.5 * S->nodemass[i] * vdot(d, d));
  }
  for (int b = 0; b < S->nb; ++b) {
    const double* M = S->nodemass + S->nfree + 16 * b;
    int b0 = S->nfree + 4 * b;
    double e = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) {
        double da[3], dc[3];
        vsub(x + 3 * (b0 + a), xtil + 3 * (b0 + a), da);
        vsub(x + 3 * (b0 + c), xtil + 3 * (b0 + c), dc);
        e += M[4 * a + c] * vdot(da, dc);
      }
    kadd(&k[0], 0.5 * e);
  }
  double* et = malloc(sizeof(double) * (S->nt + S->nc + S->nh + 1));
#pragma omp parallel for schedule(static)
  for (int e = 0; e < S->nt; ++e) {
    double xl[12], Xl[12];
    gather_pos(S, P, S->tets + 4 * e, 4, xl);
    gather_pos(S, S->rest, S->tets + 4 * e, 4, Xl);
    or_snh_local(xl, Xl, S->tmu[e], S->tlam[e], 0, &et[e], NULL, NULL);
  }
  for (int e = 0; e < S->nt; ++e) kadd(&k[1], h2 * et[e]);
  for (int e = 0; e < S->nc; ++e) {
    double xl[9], Xl[9], E;
    gather_pos(S, P, S->tris + 3 * e, 3, xl);
    gather_pos(S, S->rest, S->tris + 3 * e, 3, Xl);
    if (S->cmodel == 1) or_bw_local(xl, Xl, S->cE[e], S->cshear[e], S->cth[e], 0, &E, NULL, NULL);
    else or_stvk_local(xl, Xl, S->cmu[e], S->clam[e], S->cth[e], 0, &E, NULL, NULL);
    kadd(&k[2], h2 * E);
  }
  for (int e = 0; e < S->nh; ++e) {
    double xl[12], Xl[12], E;
    gather_pos(S, P, S->hinges + 4 * e, 4, xl);
    gather_pos(S, S->rest, S->hinges + 4 * e, 4, Xl);
    or_bend_local(xl, Xl, S->hkb[e], 0, &E, NULL, NULL);
    kadd(&k[3], h2 * E);
  }
  for (int b = 0; b < S->nb; ++b) {
    double E;
    or_abd_ortho_local(x + 3 * (S->nfree + 4 * b + 1), S->bkappa[b] * S->bvol[b], 0, &E, NULL, NULL);
    kadd(&k[4], h2 * E);
  }
  double sh = S->dhat * S->dhat;
  for (int i = 0; i < PT->n; ++i) {
    int ids[4] = {PT->p[i].a, S->stris[3 * PT->p[i].b], S->stris[3 * PT->p[i].b + 1], S->stris[3 * PT->p[i].b + 2]};
    double xl[12], E;
    gather_pos(S, P, ids, 4, xl);
    or_pair_local(0, xl, NULL, S->kappa, sh, S->form, 0, &E, NULL, NULL, NULL);
    kadd(&k[5], E);
  }
  for (int i = 0; i < EE->n; ++i) {
    const int *e = S->sedges + 2 * EE->p[i].a, *f = S->sedges + 2 * EE->p[i].b;
    int ids[4] = {e[0], e[1], f[0], f[1]};
    double xl[12], E;
    gather_pos(S, P, ids, 4, xl);
    or_pair_local(1, xl, NULL, S->kappa, sh, S->form, 0, &E, NULL, NULL, NULL);
    kadd(&k[5], E);
  }
  for (int i = 0; i < PG->n; ++i) {
    double E;
    or_pair_local(2, P + 3 * PG->p[i].a, S->planes + 4 * PG->p[i].b, S->kappa, sh, S->form, 0, &E, NULL, NULL, NULL);
    kadd(&k[5], E);
  }
  for (int i = 0; i < 6; ++i) out[i] = kval(&k[i]);
  free(et);
}

OR_EXPORT double or_energy(void* p, const double* x, const double* xtil, int brute, double* terms) {
  osys* S = p;
  double* P = malloc(sizeof(double) * 3 * S->nv);
  or_vertex_positions(S, x, P);
  plist A = {0}, B = {0}, C = {0};
  detect(S, P, brute, &A, &B, &C);
  double t[6];
  energy_terms(S, x, xtil, P, &A, &B, &C, t);
  ksum k = {0, 0};
  for (int i = 0; i < 6; ++i) kadd(&k, t[i]);
  if (terms) memcpy(terms, t, sizeof t);
  free(A.p); free(B.p); free(C.p); free(P);
  return kval(&k);
}

/* ------------------------------------------------------------------------ */
/* assembly (App. A index rules, App. B compression)                          */
/* ------------------------------------------------------------------------ */
typedef struct { int r, c; double v[9]; } contrib;
typedef struct { contrib* a; long n, cap; } clist;
static void cl_push(clist* L, int r, int c, const double* blk /*3x3, row-major, block (r,c)*/) {
  if (L->n == L->cap) { L->cap = L->cap ? 2 * L->cap : 4096; L->a = realloc(L->a, sizeof(contrib) * L->cap); }
  contrib* q = &L->a[L->n++];
  if (r <= c) { q->r = r; q->c = c; memcpy(q->v, blk, sizeof(double) * 9); }
  else { q->r = c; q->c = r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) q->v[3 * i + j] = blk[3 * j + i]; }
}
static int cmp_contrib(const void* x, const void* y) {
  const contrib *A = x, *B = y;
  if (A->r != B->r) return A->r < B->r ? -1 : 1;
  if (A->c != B->c) return A->c < B->c ? -1 : 1;
  return 0;
}

/* Scatter a local position-space gradient / Hessian over k vertices into node
 * space through each vertex's UNION Jacobian (free: I3; body: [I3, r1 I3,
 * r2 I3, r3 I3]); node blocks that several local vertices share are merged
 * before they are emitted (Sec. "Hessian Code Generation", local compression). */
static void scatter_local(const osys* S, const int* verts, int k, const double* gl, const double* Hl, double* g, clist* L) {
  int un[32], nu = 0;
  double W[4][32];
  memset(W, 0, sizeof W);
  for (int i = 0; i < k; ++i) {
    int nodes[8]; double w[8];
    int m = vmap(S, verts[i], nodes, w);
    for (int q = 0; q < m; ++q) {
      int u;
      for (u = 0; u < nu; ++u) if (un[u] == nodes[q]) break;
      if (u == nu) un[nu++] = nodes[q];
      W[i][u] += w[q];
    }
  }
  int n = 3 * k;
  for (int u = 0; u < nu; ++u)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += W[i][u] * gl[3 * i + c];
      g[3 * un[u] + c] += s;
    }
  if (!L) return;
  for (int u = 0; u < nu; ++u)
    for (int w2 = 0; w2 < nu; ++w2) {
      if (un[u] > un[w2]) continue;
      double blk[9] = {0};
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
          double f = W[i][u] * W[j][w2];
          if (f == 0.0) continue;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) blk[3 * a + b] += f * Hl[(3 * i + a) * n + 3 * j + b];
        }
      cl_push(L, un[u], un[w2], blk);
    }
}

typedef struct {
  int nn, nnzb;
  int* rowptr; int* col; double* vals; double* diag;
} obsr;
static void bsr_free(obsr* B) { free(B->rowptr); free(B->col); free(B->vals); free(B->diag); memset(B, 0, sizeof *B); }
static void bsr_from(const osys* S, clist* L, obsr* B) {
  qsort(L->a, L->n, sizeof(contrib), cmp_contrib);
  B->nn = S->nn;
  B->diag = calloc(9 * S->nn + 1, sizeof(double));
  B->rowptr = calloc(S->nn + 1, sizeof(int));
  long nu = 0;
  for (long i = 0; i < L->n; ++i)
    if (L->a[i].r != L->a[i].c && (i == 0 || L->a[i].r != L->a[i - 1].r || L->a[i].c != L->a[i - 1].c)) nu++;
  B->nnzb = (int)nu;
  B->col = malloc(sizeof(int) * (nu + 1));
  B->vals = calloc(9 * nu + 1, sizeof(double));
  long q = -1;
  int lr = -1, lc = -1;
  for (long i = 0; i < L->n; ++i) {
    contrib* c = &L->a[i];
    if (c->r == c->c) {
      for (int t = 0; t < 9; ++t) B->diag[9 * c->r + t] += c->v[t];
      continue;
    }
    if (c->r != lr || c->c != lc) {
      ++q;
      B->col[q] = c->c;
      B->rowptr[c->r + 1]++;
      lr = c->r; lc = c->c;
    }
    for (int t = 0; t < 9; ++t) B->vals[9 * q + t] += c->v[t];
  }
  for (int r = 0; r < S->nn; ++r) B->rowptr[r + 1] += B->rowptr[r];
}

typedef struct {
  obsr Hs, Hd;       /* static (elastic, inertia, ABD) and dynamic (barrier) parts */
  double* g;
  plist PT, EE, PG;
  double E;
} oasm;
static oasm* G_ASM = NULL; /* last assembly, for export */

/* Assemble g and the projected H at x (Sec. "Solution Extraction": H dx = g). */
OR_EXPORT int or_assemble(void* p, const double* x, const double* xtil, int brute, int project) {
  osys* S = p;
  if (G_ASM) { bsr_free(&G_ASM->Hs); bsr_free(&G_ASM->Hd); free(G_ASM->g); free(G_ASM->PT.p); free(G_ASM->EE.p); free(G_ASM->PG.p); free(G_ASM); }
  oasm* A = calloc(1, sizeof(oasm));
  G_ASM = A;
  double h2 = S->dt * S->dt;
  double* P = malloc(sizeof(double) * 3 * S->nv);
  or_vertex_positions(S, x, P);
  A->g = calloc(3 * S->nn + 1, sizeof(double));
  clist Ls = {0}, Ld = {0};
  /* inertia: g = M (x - xtilde), H = M */
  for (int i = 0; i < S->nfree; ++i) {
    double m = S->nodemass[i];
    for (int c = 0; c < 3; ++c) A->g[3 * i + c] += m * (x[3 * i + c] - xtil[3 * i + c]);
    double blk[9] = {m, 0, 0, 0, m, 0, 0, 0, m};
    cl_push(&Ls, i, i, blk);
  }
  for (int b = 0; b < S->nb; ++b) {
    const double* M = S->nodemass + S->nfree + 16 * b;
    int b0 = S->nfree + 4 * b;
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) {
        for (int k = 0; k < 3; ++k) A->g[3 * (b0 + a) + k] += M[4 * a + c] * (x[3 * (b0 + c) + k] - xtil[3 * (b0 + c) + k]);
        if (a <= c) { double m = M[4 * a + c]; double blk[9] = {m, 0, 0, 0, m, 0, 0, 0, m}; cl_push(&Ls, b0 + a, b0 + c, blk); }
      }
    /* orthogonality on the three A-nodes */
    double gl[9], Hl[81];
    or_abd_ortho_local(x + 3 * (b0 + 1), S->bkappa[b] * S->bvol[b], project, NULL, gl, Hl);
    for (int i = 0; i < 3; ++i)
      for (int c = 0; c < 3; ++c) A->g[3 * (b0 + 1 + i) + c] += h2 * gl[3 * i + c];
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) {
        double blk[9];
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) blk[3 * a + c] = h2 * Hl[(3 * i + a) * 9 + 3 * j + c];
        cl_push(&Ls, b0 + 1 + i, b0 + 1 + j, blk);
      }
  }
  /* elastic elements */
  for (int e = 0; e < S->nt; ++e) {
    double xl[12], Xl[12], gl[12], Hl[144];
    gather_pos(S, P, S->tets + 4 * e, 4, xl);
    gather_pos(S, S->rest, S->tets + 4 * e, 4, Xl);
    or_snh_local(xl, Xl, S->tmu[e], S->tlam[e], project, NULL, gl, Hl);
    for (int i = 0; i < 12; ++i) gl[i] *= h2;
    for (int i = 0; i < 144; ++i) Hl[i] *= h2;
    scatter_local(S, S->tets + 4 * e, 4, gl, Hl, A->g, &Ls);
  }
  for (int e = 0; e < S->nc; ++e) {
    double xl[9], Xl[9], gl[9], Hl[81];
    gather_pos(S, P, S->tris + 3 * e, 3, xl);
    gather_pos(S, S->rest, S->tris + 3 * e, 3, Xl);
    if (S->cmodel == 1) or_bw_local(xl, Xl, S->cE[e], S->cshear[e], S->cth[e], project, NULL, gl, Hl);
    else or_stvk_local(xl, Xl, S->cmu[e], S->clam[e], S->cth[e], project, NULL, gl, Hl);
    for (int i = 0; i < 9; ++i) gl[i] *= h2;
    for (int i = 0; i < 81; ++i) Hl[i] *= h2;
    scatter_local(S, S->tris + 3 * e, 3, gl, Hl, A->g, &Ls);
  }
  for (int e = 0; e < S->nh; ++e) {
    double xl[12], Xl[12], gl[12], Hl[144];
    gather_pos(S, P, S->hinges + 4 * e, 4, xl);
    gather_pos(S, S->rest, S->hinges + 4 * e, 4, Xl);
    or_bend_local(xl, Xl, S->hkb[e], project, NULL, gl, Hl);
    for (int i = 0; i < 12; ++i) gl[i] *= h2;
    for (int i = 0; i < 144; ++i) Hl[i] *= h2;
    scatter_local(S, S->hinges + 4 * e, 4, gl, Hl, A->g, &Ls);
  }
  /* contact barrier (dynamic part) */
  detect(S, P, brute, &A->PT, &A->EE, &A->PG);
  double sh = S->dhat * S->dhat;
  for (int i = 0; i < A->PT.n; ++i) {
    int ids[4] = {A->PT.p[i].a, S->stris[3 * A->PT.p[i].b], S->stris[3 * A->PT.p[i].b + 1], S->stris[3 * A->PT.p[i].b + 2]};
    double xl[12], gl[12], Hl[144];
    gather_pos(S, P, ids, 4, xl);
    or_pair_local(0, xl, NULL, S->kappa, sh, S->form, project, NULL, gl, Hl, NULL);
    scatter_local(S, ids, 4, gl, Hl, A->g, &Ld);
  }
  for (int i = 0; i < A->EE.n; ++i) {
    const int *e = S->sedges + 2 * A->EE.p[i].a, *f = S->sedges + 2 * A->EE.p[i].b;
    int ids[4] = {e[0], e[1], f[0], f[1]};
    double xl[12], gl[12], Hl[144];
    gather_pos(S, P, ids, 4, xl);
    or_pair_local(1, xl, NULL, S->kappa, sh, S->form, project, NULL, gl, Hl, NULL);
    scatter_local(S, ids, 4, gl, Hl, A->g, &Ld);
  }
  for (int i = 0; i < A->PG.n; ++i) {
    int ids[1] = {A->PG.p[i].a};
    double gl[3], Hl[9];
    or_pair_local(2, P + 3 * ids[0], S->planes + 4 * A->PG.p[i].b, S->kappa, sh, S->form, project, NULL, gl, Hl, NULL);
    scatter_local(S, ids, 1, gl, Hl, A->g, &Ld);
  }
  bsr_from(S, &Ls, &A->Hs);
  bsr_from(S, &Ld, &A->Hd);
  free(Ls.a); free(Ld.a); free(P);
  return 0;
}

/* which: 0 static, 1 dynamic.  Pass NULL arrays to query nnzb only. */
OR_EXPORT int or_export_bsr(int which, int* nnzb, int* rowptr, int* col, double* vals, double* diag) {
  if (!G_ASM) return -1;
  obsr* B = which ? &G_ASM->Hd : &G_ASM->Hs;
  *nnzb = B->nnzb;
  if (rowptr) memcpy(rowptr, B->rowptr, sizeof(int) * (B->nn + 1));
  if (col) memcpy(col, B->col, sizeof(int) * B->nnzb);
  if (vals) memcpy(vals, B->vals, sizeof(double) * 9 * B->nnzb);
  if (diag) memcpy(diag, B->diag, sizeof(double) * 9 * B->nn);
  return 0;
}
OR_EXPORT int or_export_grad(void* p, double* g) {
  osys* S = p;
  if (!G_ASM) return -1;
  memcpy(g, G_ASM->g, sizeof(double) * 3 * S->nn);
  return 0;
}

/* y = (Hs + Hd) x with symmetric upper storage */
static void bsr_apply_add(const obsr* B, const double* x, double* y) {
  for (int r = 0; r < B->nn; ++r) {
    const double* D = B->diag + 9 * r;
    for (int a = 0; a < 3; ++a) y[3 * r + a] += D[3 * a] * x[3 * r] + D[3 * a + 1] * x[3 * r + 1] + D[3 * a + 2] * x[3 * r + 2];
    for (int q = B->rowptr[r]; q < B->rowptr[r + 1]; ++q) {
      int c = B->col[q];
      const double* V = B->vals + 9 * q;
      for (int a = 0; a < 3; ++a) {
        y[3 * r + a] += V[3 * a] * x[3 * c] + V[3 * a + 1] * x[3 * c + 1] + V[3 * a + 2] * x[3 * c + 2];
        y[3 * c + a] += V[a] * x[3 * r] + V[3 + a] * x[3 * r + 1] + V[6 + a] * x[3 * r + 2];
      }
    }
  }
}
OR_EXPORT int or_spmv(void* p, const double* x, double* y) {
  osys* S = p;
  if (!G_ASM) return -1;
  memset(y, 0, sizeof(double) * 3 * S->nn);
  bsr_apply_add(&G_ASM->Hs, x, y);
  bsr_apply_add(&G_ASM->Hd, x, y);
  return 0;
}

/* block-Jacobi inverse: 3x3 per free node, 12x12 per affine body (its four
 * nodes together), gathered from both parts of H (App. D).              */
static void dense_inv(int n, const double* A, double* Ai) {
  double M[12 * 24];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i * 2 * n + j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (fabs(M[r * 2 * n + c]) > fabs(M[piv * 2 * n + c])) piv = r;
    if (piv != c) for (int j = 0; j < 2 * n; ++j) { double t = M[c * 2 * n + j]; M[c * 2 * n + j] = M[piv * 2 * n + j]; M[piv * 2 * n + j] = t; }
    double d = M[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        double f = M[r * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[c * 2 * n + j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ai[i * n + j] = M[i * 2 * n + n + j];
}
static double* precond_build(const osys* S) {
  double* Minv = calloc(9 * S->nfree + 144 * S->nb + 1, sizeof(double));
  for (int i = 0; i < S->nfree; ++i) {
    double D[9];
    for (int t = 0; t < 9; ++t) D[t] = G_ASM->Hs.diag[9 * i + t] + G_ASM->Hd.diag[9 * i + t];
    dense_inv(3, D, Minv + 9 * i);
  }
  for (int b = 0; b < S->nb; ++b) {
    int b0 = S->nfree + 4 * b;
    double A[144] = {0};
    const obsr* parts[2] = {&G_ASM->Hs, &G_ASM->Hd};
    for (int pp = 0; pp < 2; ++pp) {
      const obsr* B = parts[pp];
      for (int a = 0; a < 4; ++a) {
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) A[(3 * a + i) * 12 + 3 * a + j] += B->diag[9 * (b0 + a) + 3 * i + j];
        for (int q = B->rowptr[b0 + a]; q < B->rowptr[b0 + a + 1]; ++q) {
          int c = B->col[q] - b0;
          if (c < 0 || c > 3) continue;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              A[(3 * a + i) * 12 + 3 * c + j] += B->vals[9 * q + 3 * i + j];
              A[(3 * c + j) * 12 + 3 * a + i] += B->vals[9 * q + 3 * i + j];
            }
        }
      }
    }
    dense_inv(12, A, Minv + 9 * S->nfree + 144 * b);
  }
  return Minv;
}
static void precond_apply(const osys* S, const double* Minv, const double* r, double* z) {
  for (int i = 0; i < S->nfree; ++i)
    for (int a = 0; a < 3; ++a) {
      const double* M = Minv + 9 * i + 3 * a;
      z[3 * i + a] = M[0] * r[3 * i] + M[1] * r[3 * i + 1] + M[2] * r[3 * i + 2];
    }
  for (int b = 0; b < S->nb; ++b) {
    const double* M = Minv + 9 * S->nfree + 144 * b;
    int o = 3 * (S->nfree + 4 * b);
    for (int i = 0; i < 12; ++i) {
      double s = 0.0;
      for (int j = 0; j < 12; ++j) s += M[12 * i + j] * r[o + j];
      z[o + i] = s;
    }
  }
}
static double dotn(int n, const double* a, const double* b) {
  ksum k = {0, 0};
  for (int i = 0; i < n; ++i) kadd(&k, a[i] * b[i]);
  return kval(&k);
}

/* PCG on H p = rhs (H from the last assembly).  Stop when r^T z <= tol^2 r0^T z0. */
OR_EXPORT int or_pcg(void* p, const double* rhs, double* x, double tol, int maxit, int* iters) {
  osys* S = p;
  if (!G_ASM) return -1;
  int n = 3 * S->nn;
  double* Minv = precond_build(S);
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n),
         *q = malloc(sizeof(double) * n);
  memset(x, 0, sizeof(double) * n);
  memcpy(r, rhs, sizeof(double) * n);
  precond_apply(S, Minv, r, z);
  memcpy(d, z, sizeof(double) * n);
  double rz = dotn(n, r, z), rz0 = rz;
  int it = 0;
  if (rz0 > 0.0) {
    for (it = 0; it < maxit; ++it) {
      if (rz <= tol * tol * rz0) break;
      or_spmv(S, d, q);
      double alpha = rz / dotn(n, d, q);
      for (int i = 0; i < n; ++i) { x[i] += alpha * d[i]; r[i] -= alpha * q[i]; }
      precond_apply(S, Minv, r, z);
      double rzn = dotn(n, r, z);
      double beta = rzn / rz;
      rz = rzn;
      for (int i = 0; i < n; ++i) d[i] = z[i] + beta * d[i];
    }
  }
  if (iters) *iters = it;
  free(Minv); free(r); free(z); free(d); free(q);
  return (rz0 > 0.0 && rz > tol * tol * rz0) ? -5 : 0;
}

/* ------------------------------------------------------------------------ */
/* CCD step bound along x - alpha p, alpha in [0, 1]                        */
/* ------------------------------------------------------------------------ */
OR_EXPORT double or_ccd_bound(void* p, const double* x, const double* dir, int brute) {
  osys* S = p;
  int nv = S->nv;
  double *P0 = malloc(sizeof(double) * 3 * nv), *P1 = malloc(sizeof(double) * 3 * nv), *D = malloc(sizeof(double) * 3 * nv);
  double* x1 = malloc(sizeof(double) * 3 * S->nn);
  for (int i = 0; i < 3 * S->nn; ++i) x1[i] = x[i] - dir[i];
  or_vertex_positions(S, x, P0);
  or_vertex_positions(S, x1, P1);
  for (int i = 0; i < 3 * nv; ++i) D[i] = P1[i] - P0[i];
  double t = 1.0;
  /* point-ground: exact */
  for (int i = 0; i < S->nsv; ++i) {
    int v = S->sverts[i];
    if (S->vfixed[v]) continue;
    for (int k = 0; k < S->np; ++k) {
      double tk = or_pg_ccd(P0 + 3 * v, D + 3 * v, S->planes + 4 * k, S->gap_s, 1.0);
      if (tk < t) t = tk;
    }
  }
  /* PT and EE candidates: swept boxes over the full step, grown by dhat on
   * the query side, taken in the frame that moves with the mean vertex
   * displacement u (end positions P1 - u).  A translation common to every
   * vertex changes no distance at any time of the step, so these boxes hold
   * every pair that comes within dhat, as boxes swept in place do; the
   * candidate set, and with it the bound, no longer depends on how fast the
   * scene moves as a whole. */
  double u[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < nv; ++i)
    for (int c = 0; c < 3; ++c) u[c] += D[3 * i + c];
  for (int c = 0; c < 3; ++c) u[c] /= (nv > 0 ? nv : 1);
  double* P1s = malloc(sizeof(double) * 3 * nv);
  for (int i = 0; i < nv; ++i)
    for (int c = 0; c < 3; ++c) P1s[3 * i + c] = P1[3 * i + c] - u[c];
  int nmax = S->nsv > S->nst ? S->nsv : S->nst;
  if (S->nse > nmax) nmax = S->nse;
  double *alo = malloc(sizeof(double) * 3 * (nmax + 1)), *ahi = malloc(sizeof(double) * 3 * (nmax + 1));
  double *blo = malloc(sizeof(double) * 3 * (nmax + 1)), *bhi = malloc(sizeof(double) * 3 * (nmax + 1));
  cand C = {0};
  prim_boxes(P0, P1s, S->sverts, S->nsv, 1, S->dhat, alo, ahi);
  prim_boxes(P0, P1s, S->stris, S->nst, 3, 0.0, blo, bhi);
  box_pairs(S->nsv, alo, ahi, S->nst, blo, bhi, 0, brute, &C);
  for (long q = 0; q < C.n; ++q) {
    int v = S->sverts[C.a[q]];
    const int* tv = S->stris + 3 * C.b[q];
    if (pt_excluded(S, v, tv)) continue;
    int ids[4] = {v, tv[0], tv[1], tv[2]};
    double xl[12], dl[12];
    gather_pos(S, P0, ids, 4, xl);
    gather_pos(S, D, ids, 4, dl);
    double tk = or_accd(0, xl, dl, S->gap_s, 1.0, S->ccd_max_iter, NULL);
    if (tk < t) t = tk;
  }
  prim_boxes(P0, P1s, S->sedges, S->nse, 2, S->dhat, alo, ahi);
  prim_boxes(P0, P1s, S->sedges, S->nse, 2, 0.0, blo, bhi);
  box_pairs(S->nse, alo, ahi, S->nse, blo, bhi, 1, brute, &C);
  for (long q = 0; q < C.n; ++q) {
    const int *e = S->sedges + 2 * C.a[q], *f = S->sedges + 2 * C.b[q];
    if (ee_excluded(S, e, f)) continue;
    int ids[4] = {e[0], e[1], f[0], f[1]};
    double xl[12], dl[12];
    gather_pos(S, P0, ids, 4, xl);
    gather_pos(S, D, ids, 4, dl);
    double tk = or_accd(1, xl, dl, S->gap_s, 1.0, S->ccd_max_iter, NULL);
    if (tk < t) t = tk;
  }
  free(C.a); free(C.b); free(alo); free(ahi); free(blo); free(bhi);
  free(P0); free(P1); free(P1s); free(D); free(x1);
  return t;
}

/* ------------------------------------------------------------------------ */
/* adaptive barrier stiffness (reading c5).  kappa is chosen at the start   */
/* of a step and frozen for it.  The first step that starts with contact    */
/* pairs takes the kappa that best balances the barrier gradient g_B        */
/* (kappa = 1) against the gradient of the rest of the potential g_E,       */
/* argmin_k |g_E + k g_B| = -g_E.g_B / g_B.g_B, clamped to [kmin, kmax]     */
/* (kmin until then).  Later steps double it, up to kmax, when the smallest */
/* pair distance at the step's start is below kdmin and smaller than at the */
/* previous step's start.  Off by default: kappa stays the parameter.       */
/*                                                                          */
/* kmin <= 0 derives the lower bound from the scene: the stiffness at which */
/* the barrier alone holds the weight of an average vertex (total mass /    */
/* vertex count) at half the activation distance.  In this potential the   */
/* weight enters as m h^2 |g| (inertia term with x_tilde = x + h v + h^2 g) */
/* and the barrier as kappa |db/dd|, d the distance, so                     */
/*   kmin = m h^2 |g| / |db/dd (dhat / 2)|,  db/dd = 2 d b'(d^2).           */
/* |g| = 0 takes standard gravity.  kmax <= 0 takes 1e4 kmin.               */
/* ------------------------------------------------------------------------ */
static double kappa_lower_bound(const osys* S) {
  double m = 0.0;
  for (int v = 0; v < S->nv; ++v) m += S->vmass[v];
  m /= (S->nv > 0 ? S->nv : 1);
  double gn = sqrt(S->grav[0] * S->grav[0] + S->grav[1] * S->grav[1] + S->grav[2] * S->grav[2]);
  if (!(gn > 0.0)) gn = 9.80665;
  const double d = 0.5 * S->dhat;
  double b, db, d2b;
  or_barrier_scalar(d * d, S->dhat * S->dhat, S->form, &b, &db, &d2b);
  return m * S->dt * S->dt * gn / fabs(2.0 * d * db);
}
OR_EXPORT void or_set_kappa_adaptive(void* p, int on, double kmin, double kmax, double kdmin) {
  osys* S = p;
  S->kadapt = on;
  S->kinit = 0;
  S->kmin = kmin > 0.0 ? kmin : kappa_lower_bound(S);
  S->kmax = kmax > 0.0 ? kmax : 1e4 * S->kmin;
  S->kdmin = kdmin;
  S->dmin_prev = INFINITY;
}
OR_EXPORT void or_get_kappa_bounds(void* p, double* kmin, double* kmax) {
  const osys* S = p;
  *kmin = S->kmin;
  *kmax = S->kmax;
}
OR_EXPORT double or_get_kappa(void* p) { return ((const osys*)p)->kappa; }

/* smallest distance over the pairs within dhat at positions P (INFINITY if none) */
static double min_pair_distance(const osys* S, const double* P, int brute) {
  plist PT = {0}, EE = {0}, PG = {0};
  detect(S, P, brute, &PT, &EE, &PG);
  double m2 = INFINITY;
  for (int q = 0; q < PT.n; ++q) {
    const int v = PT.p[q].a;
    const int* tv = S->stris + 3 * PT.p[q].b;
    double s2;
    or_pt_classify(P + 3 * v, P + 3 * tv[0], P + 3 * tv[1], P + 3 * tv[2], &s2);
    if (s2 < m2) m2 = s2;
  }
  for (int q = 0; q < EE.n; ++q) {
    const int *e = S->sedges + 2 * EE.p[q].a, *f = S->sedges + 2 * EE.p[q].b;
    double s2;
    or_ee_classify(P + 3 * e[0], P + 3 * e[1], P + 3 * f[0], P + 3 * f[1], &s2);
    if (s2 < m2) m2 = s2;
  }
  for (int q = 0; q < PG.n; ++q) {
    const double* pl = S->planes + 4 * PG.p[q].b;
    const double d = vdot(pl, P + 3 * PG.p[q].a) - pl[3];
    if (d * d < m2) m2 = d * d;
  }
  free(PT.p); free(EE.p); free(PG.p);
  return sqrt(m2);
}

static void kappa_update(osys* S, const double* x, const double* xtil, int brute) {
  const int n = 3 * S->nn;
  double* P = malloc(sizeof(double) * 3 * S->nv);
  or_vertex_positions(S, x, P);
  const double dmin = min_pair_distance(S, P, brute);
  if (!S->kinit) {
    if (isfinite(dmin)) {
      double *gE = malloc(sizeof(double) * n), num = 0.0, den = 0.0;
      S->kappa = 0.0;
      or_assemble(S, x, xtil, brute, 0);
      memcpy(gE, G_ASM->g, sizeof(double) * n);
      S->kappa = 1.0;
      or_assemble(S, x, xtil, brute, 0);
      for (int i = 0; i < n; ++i) {
        const double gB = G_ASM->g[i] - gE[i];
        num += gE[i] * gB;
        den += gB * gB;
      }
      double k = (den > 0.0) ? -num / den : S->kmin;
      if (!(k >= S->kmin)) k = S->kmin;
      if (k > S->kmax) k = S->kmax;
      S->kappa = k;
      S->kinit = 1;
      free(gE);
    } else {
      S->kappa = S->kmin;
    }
  } else if (dmin < S->kdmin && dmin < S->dmin_prev) {
    S->kappa = fmin(2.0 * S->kappa, S->kmax);
  }
  S->dmin_prev = dmin;
  free(P);
}

/* ------------------------------------------------------------------------ */
/* one implicit time step: Newton on the incremental potential              */
/* ------------------------------------------------------------------------ */
/* stats: [0] newton iters, [1] pcg iters total, [2] last alpha, [3] final ||p||inf,
 *        [4] n_pt, [5] n_ee, [6] n_pg, [7] line-search failures,
 *        [8] the step's barrier stiffness kappa                            */
OR_EXPORT int or_step(void* p, double* x, double* v, int brute, double* stats) {
  osys* S = p;
  int n = 3 * S->nn;
  double h = S->dt;
  /* prescribed vertices move with their velocity */
  for (int i = 0; i < S->nfix; ++i)
    for (int c = 0; c < 3; ++c) S->xfix[3 * S->fixed[i] + c] += h * S->fixvel[3 * i + c];
  double *xt = malloc(sizeof(double) * n), *xtil = malloc(sizeof(double) * n), *g = malloc(sizeof(double) * n),
         *dir = malloc(sizeof(double) * n), *xtrial = malloc(sizeof(double) * n);
  memcpy(xt, x, sizeof(double) * n);
  or_xtilde(S, x, v, xtil);
  if (S->kadapt) kappa_update(S, x, xtil, brute);
  int rc = 0, it, pcg_total = 0, ls_fail = 0;
  double alpha = 0.0, pinf = 0.0;
  for (it = 0; it < S->newton_max; ++it) {
    or_assemble(S, x, xtil, brute, 1);
    memcpy(g, G_ASM->g, sizeof(double) * n);
    int pit = 0;
    or_pcg(S, g, dir, S->pcg_tol, S->pcg_max, &pit);
    pcg_total += pit;
    pinf = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(dir[i]) > pinf) pinf = fabs(dir[i]);
    if (pinf <= S->newton_tol) break;
    alpha = or_ccd_bound(S, x, dir, brute);
    double E0 = or_energy(S, x, xtil, brute, NULL);
    int ls;
    for (ls = 0; ls < S->ls_max; ++ls) {
      for (int i = 0; i < n; ++i) xtrial[i] = x[i] - alpha * dir[i];
      double E1 = or_energy(S, xtrial, xtil, brute, NULL);
      /* a decrease, up to the rounding of the energy sums (reading c15):
       * differences below 1e-12 |E0| are not resolved by FP64 element energies */
      if (E1 <= E0 + 1e-12 * fabs(E0)) break;
      alpha *= 0.5;
    }
    if (ls == S->ls_max) { ls_fail++; rc = -6; break; }
    memcpy(x, xtrial, sizeof(double) * n);
  }
  if (it == S->newton_max && rc == 0) rc = -5;
  for (int i = 0; i < n; ++i) v[i] = (x[i] - xt[i]) / h;
  if (stats) {
    stats[0] = it; stats[1] = pcg_total; stats[2] = alpha; stats[3] = pinf;
    stats[4] = G_ASM ? G_ASM->PT.n : 0; stats[5] = G_ASM ? G_ASM->EE.n : 0; stats[6] = G_ASM ? G_ASM->PG.n : 0;
    stats[7] = ls_fail;
    stats[8] = S->kappa;
  }
  free(xt); free(xtil); free(g); free(dir); free(xtrial);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* adjoint of one implicit step (form 2 of the hot path; the paper lists     */
/* differentiable simulation as future work, Sec. "Conclusion and Future     */
/* Work", so this follows the implicit-function theorem on the step's        */
/* optimality condition grad E(x_{t+1}; x_t, v_t, E) = 0)                    */
/* ------------------------------------------------------------------------ */
/* per-tet Young's moduli (Poisson ratios kept): mu, lam follow (reading c2) */
OR_EXPORT void or_set_tet_young(void* p, const double* E) {
  osys* S = p;
  for (int e = 0; e < S->nt; ++e) {
    S->tE[e] = E[e];
    or_lame(E[e], S->tnu[e], &S->tmu[e], &S->tlam[e]);
  }
}

/* y = M x with the lumped node masses (free: m I3; body: 4x4 (x) I3) */
static void mass_apply(const osys* S, const double* x, double* y) {
  for (int i = 0; i < S->nfree; ++i)
    for (int c = 0; c < 3; ++c) y[3 * i + c] = S->nodemass[i] * x[3 * i + c];
  for (int b = 0; b < S->nb; ++b) {
    const double* M = S->nodemass + S->nfree + 16 * b;
    int b0 = S->nfree + 4 * b;
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int k = 0; k < 4; ++k) s += M[4 * a + k] * x[3 * (b0 + k) + c];
        y[3 * (b0 + a) + c] = s;
      }
  }
}

/* One reverse step.  With v_{t+1} = (x_{t+1} - x_t)/h and the optimality
 * condition, given xbar = dL/dx_{t+1} and vbar = dL/dv_{t+1} (total
 * derivatives of everything downstream):
 *   H lambda = xbar + vbar / h          (H: the EXACT Hessian at x_{t+1})
 *   dL/dx_t  = M lambda - vbar / h      (x_tilde = x_t + h v_t + h^2 g)
 *   dL/dv_t  = h M lambda
 *   dL/dE_e -= h^2 lambda^T d(grad V Psi_e)/dE_e = h^2 lambda_e^T grad(V Psi_e) / E_e
 * because Psi_SNH is linear in E at a fixed Poisson ratio (mu, lam are both
 * proportional to E and alpha = 1 + 3 mu / (4 lam) does not change).  Ebar
 * is accumulated (not overwritten).  Returns the PCG status. */
OR_EXPORT int or_adjoint_step(void* p, const double* xt, const double* vt, const double* xnext, const double* xbar,
                              const double* vbar, double tol, int maxit, double* xbar_prev, double* vbar_prev,
                              double* Ebar, int* iters) {
  osys* S = p;
  int n = 3 * S->nn;
  double h = S->dt, h2 = h * h;
  double *xtil = malloc(sizeof(double) * (n + 1)), *rhs = malloc(sizeof(double) * (n + 1)),
         *lam = malloc(sizeof(double) * (n + 1)), *Ml = malloc(sizeof(double) * (n + 1));
  or_xtilde(S, xt, vt, xtil);
  or_assemble(S, xnext, xtil, 0, 0);
  for (int i = 0; i < n; ++i) rhs[i] = xbar[i] + vbar[i] / h;
  int rc = or_pcg(S, rhs, lam, tol, maxit, iters);
  mass_apply(S, lam, Ml);
  for (int i = 0; i < n; ++i) {
    xbar_prev[i] = Ml[i] - vbar[i] / h;
    vbar_prev[i] = h * Ml[i];
  }
  double* P = malloc(sizeof(double) * 3 * (S->nv + 1));
  or_vertex_positions(S, xnext, P);
  for (int e = 0; e < S->nt; ++e) {
    double xl[12], Xl[12], gl[12], Hl[144];
    gather_pos(S, P, S->tets + 4 * e, 4, xl);
    gather_pos(S, S->rest, S->tets + 4 * e, 4, Xl);
    or_snh_local(xl, Xl, S->tmu[e], S->tlam[e], 0, NULL, gl, Hl);
    double acc = 0.0;
    for (int a = 0; a < 4; ++a) {
      int nodes[8];
      double w[8];
      int m = vmap(S, S->tets[4 * e + a], nodes, w);
      for (int c = 0; c < 3; ++c) {
        double lv = 0.0;
        for (int k = 0; k < m; ++k) lv += w[k] * lam[3 * nodes[k] + c];
        acc += lv * gl[3 * a + c];
      }
    }
    Ebar[e] -= h2 * acc / S->tE[e];
  }
  free(P); free(xtil); free(rhs); free(lam); free(Ml);
  return rc;
}

OR_EXPORT int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
