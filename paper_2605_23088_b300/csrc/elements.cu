// elements.cu -- static (fixed-connectivity) terms of the incremental potential:
// inertia, stable Neo-Hookean tets (Eq. snh, projected in F-space as in Sec.
// "Eigendecomposition: Manual Optimization"), StVK membrane triangles, discrete-
// shell hinges, and the affine-body orthogonality term 1/2 ||A^T A - I||_F^2.
// Each element kernel evaluates its local gradient (FP64) and PSD-projected
// Hessian (precision T), maps local vertices to global nodes through the JOIN
// of its connectivity, and scatters with atomic additions into the static BSR
// (App. B "Assembly") whose slots were fixed when the system was built.
#include <algorithm>

#include "common.cuh"
#include "eig.cuh"
#include "internal.h"

namespace {

// local pair q of a 4-vertex element: (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
__host__ __device__ __forceinline__ int pairA(int q) { return q < 3 ? 0 : (q < 5 ? 1 : 2); }
__host__ __device__ __forceinline__ int pairB(int q) { return q < 3 ? q + 1 : (q < 5 ? q - 1 : 3); }

__device__ __forceinline__ int pair_index4(int a, int b) {  // a < b, 4 local vertices
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}
__device__ __forceinline__ int pair_index3(int a, int b) { return a == 0 ? b - 1 : 2; }

// ---------------------------------------------------------------- rest shape
__device__ void inv3(const double* M, double* Mi, double* det) {
  const double a = M[0], b = M[1], c = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], i = M[8];
  const double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
  const double D = a * A + b * B + c * C;
  *det = D;
  Mi[0] = A / D; Mi[1] = -(b * i - c * h) / D; Mi[2] = (b * f - c * e) / D;
  Mi[3] = B / D; Mi[4] = (a * i - c * g) / D; Mi[5] = -(a * f - c * d) / D;
  Mi[6] = C / D; Mi[7] = -(a * h - b * g) / D; Mi[8] = (a * e - b * d) / D;
}

__global__ void k_rest_tet(int nt, const int* __restrict__ tv, const double* __restrict__ rest,
                           const double* __restrict__ E, const double* __restrict__ nu, const double* __restrict__ rho,
                           double* __restrict__ out, double* __restrict__ vmass, int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  int v[4];
  for (int a = 0; a < 4; ++a) v[a] = tv[4 * e + a];
  double Dm[9];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) Dm[3 * i + k] = rest[3 * v[k + 1] + i] - rest[3 * v[0] + i];
  double Mi[9], det;
  inv3(Dm, Mi, &det);
  if (!(det > 0.0)) dev_flag(status, DEV_BADINDEX);
  const double vol = det / 6.0;
  const double mu = E[e] / (2.0 * (1.0 + nu[e]));
  const double lam = E[e] * nu[e] / ((1.0 + nu[e]) * (1.0 - 2.0 * nu[e]));
  double* o = out + 12 * (size_t)e;
  for (int k = 0; k < 9; ++k) o[k] = Mi[k];
  o[9] = vol; o[10] = mu; o[11] = lam;
  for (int a = 0; a < 4; ++a) atomicAdd(&vmass[v[a]], rho[e] * vol / 4.0);
}

__global__ void k_rest_tri(int nc, const int* __restrict__ tv, const double* __restrict__ rest,
                           const double* __restrict__ E, const double* __restrict__ nu, const double* __restrict__ th,
                           const double* __restrict__ rho, int model, double* __restrict__ out,
                           double* __restrict__ vmass, int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc) return;
  const int v0 = tv[3 * e], v1 = tv[3 * e + 1], v2 = tv[3 * e + 2];
  const v3<double> X0 = ld3(rest, v0), e1 = ld3(rest, v1) - X0, e2 = ld3(rest, v2) - X0;
  const double l1 = sqrt(dot(e1, e1));
  const v3<double> u = (1.0 / l1) * e1;
  const v3<double> n = cross(e1, e2);
  const double ln = sqrt(dot(n, n));
  const v3<double> w = (1.0 / ln) * cross(n, u);
  // rest edge vectors in the orthonormal in-plane frame (u, w)
  const double D00 = l1, D01 = dot(e2, u), D10 = 0.0, D11 = dot(e2, w);
  const double det = D00 * D11 - D01 * D10;
  if (!(det > 0.0)) dev_flag(status, DEV_BADINDEX);
  double* o = out + 8 * (size_t)e;
  o[0] = D11 / det; o[1] = -D01 / det; o[2] = -D10 / det; o[3] = D00 / det;
  const double area = 0.5 * ln;
  o[4] = area * th[e];
  if (model == 1) {  // Baraff-Witkin: stretch and shear stiffness (nu holds the shear stiffness)
    o[5] = E[e];
    o[6] = nu[e];
    o[7] = 1.0;
  } else {
    o[5] = E[e] / (2.0 * (1.0 + nu[e]));          // mu
    o[6] = E[e] * nu[e] / (1.0 - nu[e] * nu[e]);  // plane-stress lambda
    o[7] = 0.0;
  }
  const double m = rho[e] * area * th[e] / 3.0;
  atomicAdd(&vmass[v0], m); atomicAdd(&vmass[v1], m); atomicAdd(&vmass[v2], m);
}

// signed dihedral angle of hinge (e0, e1, a, b): angle between the normals of
// triangles (e0, e1, a) and (e1, e0, b) about the shared edge
__device__ double hinge_theta(v3<double> x0, v3<double> x1, v3<double> xa, v3<double> xb) {
  const v3<double> e = x1 - x0;
  const v3<double> n1 = cross(e, xa - x0), n2 = cross(x0 - x1, xb - x1);
  const double le = sqrt(dot(e, e));
  return atan2(dot(cross(n1, n2), e) / le, dot(n1, n2));
}

__global__ void k_rest_hinge(int nh, const int* __restrict__ hv, const double* __restrict__ rest,
                             const double* __restrict__ kb, double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nh) return;
  const v3<double> x0 = ld3(rest, hv[4 * e]), x1 = ld3(rest, hv[4 * e + 1]), xa = ld3(rest, hv[4 * e + 2]),
                   xb = ld3(rest, hv[4 * e + 3]);
  const v3<double> ed = x1 - x0;
  const v3<double> c1 = cross(ed, xa - x0), c2 = cross(ed, xb - x1);
  const double A1 = 0.5 * sqrt(dot(c1, c1)), A2 = 0.5 * sqrt(dot(c2, c2));
  out[2 * e] = hinge_theta(x0, x1, xa, xb);
  out[2 * e + 1] = kb[e] * 3.0 * dot(ed, ed) / (A1 + A2);
}

__global__ void k_nodes_of(int n, int k, const int* __restrict__ ev, const int* __restrict__ vnode,
                           const int* __restrict__ vbody, int* __restrict__ en, int* status) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * k) return;
  const int v = ev[i];
  if (vbody[v] != -1) dev_flag(status, DEV_BADINDEX);  // elastic elements act on free / fixed vertices
  en[i] = vnode[v];
}

__global__ void k_free_nodemass(int nv, const int* __restrict__ vnode, const int* __restrict__ vbody,
                                const double* __restrict__ vmass, double* __restrict__ nodemass) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  if (vbody[v] == -1 && vnode[v] >= 0) nodemass[vnode[v]] = vmass[v];
}

// ---------------------------------------------------------------- static sparsity keys
__device__ __forceinline__ uint64_t pack_key(int a, int b, int nbits) {
  const uint64_t sent = (1ull << nbits) - 1ull;
  if (a < 0 || b < 0 || a == b) return (sent << nbits) | sent;
  const uint64_t r = (uint64_t)min(a, b), c = (uint64_t)max(a, b);
  return (r << nbits) | c;
}
// elements with k local nodes (k = 3: 3 pairs, k = 4: 6 pairs) -> keys [n * npairs]
__global__ void k_elem_keys(int n, int k, const int* __restrict__ en, int nbits, int id_base, uint64_t* __restrict__ keys,
                            int* __restrict__ vals) {
  const int np = (k == 4) ? 6 : 3;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * np) return;
  const int e = (int)(i / np), q = (int)(i % np);
  int a, b;
  if (k == 4) { a = pairA(q); b = pairB(q); }
  else { a = (q == 2) ? 1 : 0; b = (q == 0) ? 1 : 2; }
  keys[i] = pack_key(en[k * e + a], en[k * e + b], nbits);
  vals[i] = id_base + (int)i;
}
__global__ void k_body_keys(int nb, int nfree, int nbits, int id_base, uint64_t* __restrict__ keys, int* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * 6) return;
  const int b = i / 6, q = i % 6;
  const int b0 = nfree + 4 * b;
  keys[i] = pack_key(b0 + pairA(q), b0 + pairB(q), nbits);
  vals[i] = id_base + i;
}

// ---------------------------------------------------------------- positions
// p = t + r1 A_1 + r2 A_2 + r3 A_3 for body vertices (the UNION branch of the
// affine parameterisation), x[node] for free vertices, the prescribed position
// for fixed vertices.  Explicitly rounded, in a fixed order, so that positions
// agree bit-for-bit with a plain evaluation of the same sum.
__global__ void k_positions(int nv, const int* __restrict__ vnode, const int* __restrict__ vbody,
                            const double* __restrict__ vr, const int* __restrict__ enode,
                            const double* __restrict__ ew, const double* __restrict__ xfix,
                            const double* __restrict__ x, double* __restrict__ P) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int n = vnode[v];
  if (n < 0) {
    for (int c = 0; c < 3; ++c) P[3 * v + c] = xfix[3 * v + c];
  } else if (vbody[v] <= -2) {  // cage-embedded: sum_k w_k x(cage node k), in order
    const int e = -2 - vbody[v];
    for (int c = 0; c < 3; ++c) {
      double p = 0.0;
      for (int k = 0; k < 8; ++k) p = __dadd_rn(p, __dmul_rn(ew[8 * e + k], x[3 * enode[8 * e + k] + c]));
      P[3 * v + c] = p;
    }
  } else if (vbody[v] < 0) {
    for (int c = 0; c < 3; ++c) P[3 * v + c] = x[3 * n + c];
  } else {
    const double r1 = vr[3 * v], r2 = vr[3 * v + 1], r3 = vr[3 * v + 2];
    for (int c = 0; c < 3; ++c) {
      double p = __dadd_rn(0.0, __dmul_rn(1.0, x[3 * n + c]));
      p = __dadd_rn(p, __dmul_rn(r1, x[3 * (n + 1) + c]));
      p = __dadd_rn(p, __dmul_rn(r2, x[3 * (n + 2) + c]));
      p = __dadd_rn(p, __dmul_rn(r3, x[3 * (n + 3) + c]));
      P[3 * v + c] = p;
    }
  }
}

// x_tilde = x_t + h v_t + h^2 M^-1 f_gravity (free nodes and body translation nodes)
__global__ void k_xtilde(int nn, int nfree, double h, double gx, double gy, double gz, const double* __restrict__ xt,
                         const double* __restrict__ vt, double* __restrict__ xtil) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const bool grav = (i < nfree) || (((i - nfree) & 3) == 0);
  const double g[3] = {gx, gy, gz};
  for (int c = 0; c < 3; ++c) {
    double v = xt[3 * i + c] + h * vt[3 * i + c];
    if (grav) v += h * h * g[c];
    xtil[3 * i + c] = v;
  }
}

// ---------------------------------------------------------------- inertia
template <typename T>
__global__ void k_inertia_free(int nfree, const double* __restrict__ m, const double* __restrict__ x,
                               const double* __restrict__ xtil, double* __restrict__ g, T* __restrict__ diag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nfree) return;
  const double mi = m[i];
  for (int c = 0; c < 3; ++c) g[3 * i + c] += mi * (x[3 * i + c] - xtil[3 * i + c]);
  diag[9 * i + 0] += (T)mi;
  diag[9 * i + 4] += (T)mi;
  diag[9 * i + 8] += (T)mi;
}

template <typename T>
__global__ void k_inertia_body(int nb, int nfree, const double* __restrict__ Mb, const int* __restrict__ slot,
                               const double* __restrict__ x, const double* __restrict__ xtil, double* __restrict__ g,
                               T* __restrict__ diag, T* __restrict__ vals) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double* M = Mb + 16 * b;
  const int b0 = nfree + 4 * b;
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int q = 0; q < 4; ++q) s += M[4 * a + q] * (x[3 * (b0 + q) + c] - xtil[3 * (b0 + q) + c]);
      atomicAdd(&g[3 * (b0 + a) + c], s);
    }
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) atomicAdd(&diag[9 * (b0 + a) + 4 * c], (T)M[5 * a]);
  for (int q = 0; q < 6; ++q) {
    const double m = M[4 * pairA(q) + pairB(q)];
    T* d = vals + 9 * (size_t)slot[6 * b + q];
    for (int c = 0; c < 3; ++c) atomicAdd(&d[4 * c], (T)m);
  }
}

// ---------------------------------------------------------------- shared scatter
// d[0..8] += B[0..8] for one 3x3 block.  FP32: vector atomics (16- and 8-byte
// reductions) where the block's address allows; a block starts at 36 bytes
// times its index, so at one of four offsets mod 16 and in 3 or 4 operations
// instead of 9.  FP64: scalar atomics.
__device__ __forceinline__ void add_block9(double* d, const double* B) {
#pragma unroll
  for (int t = 0; t < 9; ++t) atomicAdd(d + t, B[t]);
}
__device__ __forceinline__ void add_block9(float* d, const float* B) {
  const int off = (int)((reinterpret_cast<uintptr_t>(d) >> 2) & 3);  // floats past a 16-byte boundary
  if (off == 0) {  // 4 + 4 + 1
    atomicAdd(reinterpret_cast<float4*>(d), make_float4(B[0], B[1], B[2], B[3]));
    atomicAdd(reinterpret_cast<float4*>(d + 4), make_float4(B[4], B[5], B[6], B[7]));
    atomicAdd(d + 8, B[8]);
  } else if (off == 1) {  // 1 + 2 + 4 + 2
    atomicAdd(d, B[0]);
    atomicAdd(reinterpret_cast<float2*>(d + 1), make_float2(B[1], B[2]));
    atomicAdd(reinterpret_cast<float4*>(d + 3), make_float4(B[3], B[4], B[5], B[6]));
    atomicAdd(reinterpret_cast<float2*>(d + 7), make_float2(B[7], B[8]));
  } else if (off == 2) {  // 2 + 4 + 2 + 1
    atomicAdd(reinterpret_cast<float2*>(d), make_float2(B[0], B[1]));
    atomicAdd(reinterpret_cast<float4*>(d + 2), make_float4(B[2], B[3], B[4], B[5]));
    atomicAdd(reinterpret_cast<float2*>(d + 6), make_float2(B[6], B[7]));
    atomicAdd(d + 8, B[8]);
  } else {  // 1 + 4 + 4
    atomicAdd(d, B[0]);
    atomicAdd(reinterpret_cast<float4*>(d + 1), make_float4(B[1], B[2], B[3], B[4]));
    atomicAdd(reinterpret_cast<float4*>(d + 5), make_float4(B[5], B[6], B[7], B[8]));
  }
}

// Add the k x k grid of 3x3 blocks  Bab = scale * sum_{j,l} w[a][j] w[b][l] Hf[(i,j),(m,l)]
// (Hf in an F-space of dimension 3*nc, nc = 3 for tets, 2 for membranes)
// for every local pair a <= b into diag / vals.
template <typename T, int K, int NC>
__device__ __forceinline__ void scatter_fspace(const T* Hf, const double (*w)[NC], double scale, const int* nodes,
                                               const int* slots, T* diag, T* vals) {
  constexpr int NF = 3 * NC;
  // the weights and the scale in T once: in the FP32-mixed form every
  // double-to-float conversion is an instruction on the (scarce) FP64 pipe
  T wt[K][NC];
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int j = 0; j < NC; ++j) wt[a][j] = (T)w[a][j];
  const T sct = (T)scale;
  // Y[a][i][(m,l)] = sum_j w[a][j] Hf[(i,j),(m,l)]
#pragma unroll
  for (int a = 0; a < K; ++a) {
    T Y[3][NF];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int q = 0; q < NF; ++q) {
        T s = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) s += wt[a][j] * Hf[(NC * i + j) * NF + q];
        Y[i][q] = s;
      }
#pragma unroll
    for (int b = a; b < K; ++b) {
      if (nodes[a] < 0 || nodes[b] < 0) continue;
      T B[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          T s = 0;
#pragma unroll
          for (int l = 0; l < NC; ++l) s += Y[i][NC * m + l] * wt[b][l];
          B[3 * i + m] = sct * s;
        }
      if (a == b) {
        add_block9(diag + 9 * (size_t)nodes[a], B);
      } else {
        const int sl = slots[(K == 4) ? pair_index4(a, b) : pair_index3(a, b)];
        if (nodes[a] > nodes[b]) {  // the stored block is the transpose
          T Bt[9];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int m = 0; m < 3; ++m) Bt[3 * i + m] = B[3 * m + i];
          add_block9(vals + 9 * (size_t)sl, Bt);
        } else {
          add_block9(vals + 9 * (size_t)sl, B);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- stable Neo-Hookean
struct snh_state {
  double F[9], Ic, J, alpha, mu, lam, vol;
};

__device__ __forceinline__ int lc(int i, int j, int k) {  // Levi-Civita for i,j,k in {0,1,2}
  return (i == j || j == k || i == k) ? 0 : (((j - i + 3) % 3 == 1) ? 1 : -1);
}

// PSD projection of the F-space Hessian c1 I + c2 f f^T + lam g g^T + c4 d2J/dF2
// in closed form.  With the signed SVD F = U diag(s) V^T (U, V rotations) the
// nine eigenvectors are U E V^T for: the three "scaling" directions E = diag(w)
// (w an eigenvector of the 3x3 matrix A_ii = c1 + c2 s_i^2 + lam g_i^2,
// A_ij = c2 s_i s_j + lam g_i g_j + c4 s_k, g_i = s_j s_k), and for each pair
// (i, j) a "twist" E = (e_i e_j^T - e_j e_i^T)/sqrt2 with eigenvalue c1 + c4 s_k
// and a "flip" E = (e_i e_j^T + e_j e_i^T)/sqrt2 with eigenvalue c1 - c4 s_k
// (d2J/dF2 is 0 / -s_k / +s_k on those subspaces).  Negative eigenvalues are
// dropped.  The result equals the EVD projection of the assembled 9x9 matrix.
template <typename T>
__device__ __forceinline__ void snh_project_fspace(const T* F, T c1, T c2, T lam, T c4, T* P) {
  // F^T F and its eigen-decomposition (descending), V a rotation
  T C[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  T V[9];
  eig_sym<3, T>(C, V);
  T w[3] = {C[0], C[4], C[8]};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2 - a; ++b)
      if (w[b] < w[b + 1]) {
        const T tw = w[b]; w[b] = w[b + 1]; w[b + 1] = tw;
#pragma unroll
        for (int r = 0; r < 3; ++r) { const T tv = V[3 * r + b]; V[3 * r + b] = V[3 * r + b + 1]; V[3 * r + b + 1] = tv; }
      }
  const T detV = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) + V[2] * (V[3] * V[7] - V[4] * V[6]);
  if (detV < T(0)) { V[2] = -V[2]; V[5] = -V[5]; V[8] = -V[8]; }
  T v[3][3], u[3][3], s[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) v[c][r] = V[3 * r + c];
  s[0] = sqrt(w[0] > T(0) ? w[0] : T(0));
  s[1] = sqrt(w[1] > T(0) ? w[1] : T(0));
  T Fv[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) Fv[c][r] = F[3 * r] * v[c][0] + F[3 * r + 1] * v[c][1] + F[3 * r + 2] * v[c][2];
  {
    T n0 = sqrt(Fv[0][0] * Fv[0][0] + Fv[0][1] * Fv[0][1] + Fv[0][2] * Fv[0][2]);
    if (!(n0 > T(0))) { u[0][0] = 1; u[0][1] = 0; u[0][2] = 0; }
    else { u[0][0] = Fv[0][0] / n0; u[0][1] = Fv[0][1] / n0; u[0][2] = Fv[0][2] / n0; }
    T d = u[0][0] * Fv[1][0] + u[0][1] * Fv[1][1] + u[0][2] * Fv[1][2];
    T x1 = Fv[1][0] - d * u[0][0], y1 = Fv[1][1] - d * u[0][1], z1 = Fv[1][2] - d * u[0][2];
    T n1 = sqrt(x1 * x1 + y1 * y1 + z1 * z1);
    if (!(n1 > T(1e-30))) {  // any unit vector orthogonal to u0
      const T ax = fabs(u[0][0]) < T(0.9) ? T(1) : T(0), ay = ax > T(0) ? T(0) : T(1);
      x1 = ay * u[0][2]; y1 = -ax * u[0][2]; z1 = ax * u[0][1] - ay * u[0][0];
      n1 = sqrt(x1 * x1 + y1 * y1 + z1 * z1);
    }
    u[1][0] = x1 / n1; u[1][1] = y1 / n1; u[1][2] = z1 / n1;
    u[2][0] = u[0][1] * u[1][2] - u[0][2] * u[1][1];
    u[2][1] = u[0][2] * u[1][0] - u[0][0] * u[1][2];
    u[2][2] = u[0][0] * u[1][1] - u[0][1] * u[1][0];
  }
  s[2] = u[2][0] * Fv[2][0] + u[2][1] * Fv[2][1] + u[2][2] * Fv[2][2];  // signed
  const T g[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
  T A[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      A[3 * i + j] = (i == j) ? c1 + c2 * s[i] * s[i] + lam * g[i] * g[i]
                              : c2 * s[i] * s[j] + lam * g[i] * g[j] + c4 * s[3 - i - j];
  T W[9];
  eig_sym<3, T>(A, W);
#pragma unroll
  for (int k = 0; k < 81; ++k) P[k] = T(0);
  // rank-one update with q = vec(sum_t a_t u_{i_t} v_{j_t}^T)
  auto add_mode = [&](T lamb, const T* coef /*9: E in the SVD frame*/) {
    if (!(lamb > T(0))) return;
    T q[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T acc = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            if (coef[3 * a + b] != T(0)) acc += coef[3 * a + b] * u[a][r] * v[b][c];
        q[3 * r + c] = acc;
      }
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
      for (int c = r; c < 9; ++c) P[9 * r + c] += lamb * q[r] * q[c];
  };
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    T coef[9] = {W[m], 0, 0, 0, W[3 + m], 0, 0, 0, W[6 + m]};
    add_mode(A[4 * m], coef);
  }
  const T h = T(0.70710678118654752440);
#pragma unroll
  for (int pr = 0; pr < 3; ++pr) {
    const int i = (pr == 2) ? 1 : 0, j = (pr == 0) ? 1 : 2, k = 3 - i - j;
    T ct[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, cf[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    ct[3 * i + j] = h; ct[3 * j + i] = -h;
    cf[3 * i + j] = h; cf[3 * j + i] = h;
    add_mode(c1 + c4 * s[k], ct);
    add_mode(c1 - c4 * s[k], cf);
  }
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int c = 0; c < r; ++c) P[9 * r + c] = P[9 * c + r];
}

template <typename T>
__global__ void __launch_bounds__(128) k_snh(int nt, const int* __restrict__ tv, const int* __restrict__ tn,
                                             const double* __restrict__ trest, const int* __restrict__ tslot,
                                             const double* __restrict__ P, double h2, int project,
                                             double* __restrict__ g, T* __restrict__ diag, T* __restrict__ vals) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  const int4 v = reinterpret_cast<const int4*>(tv)[e];
  const int4 n4 = reinterpret_cast<const int4*>(tn)[e];
  const int nodes[4] = {n4.x, n4.y, n4.z, n4.w};
  const double* R = trest + 12 * (size_t)e;
  double Dmi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Dmi[k] = R[k];
  const double vol = R[9], mu = R[10], lam = R[11];
  const v3<double> x0 = ld3(P, v.x);
  const v3<double> d1 = ld3(P, v.y) - x0, d2 = ld3(P, v.z) - x0, d3_ = ld3(P, v.w) - x0;
  const double Ds[9] = {d1.x, d2.x, d3_.x, d1.y, d2.y, d3_.y, d1.z, d2.z, d3_.z};
  double F[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F[3 * i + j] = Ds[3 * i] * Dmi[j] + Ds[3 * i + 1] * Dmi[3 + j] + Ds[3 * i + 2] * Dmi[6 + j];
  double Ic = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) Ic += F[k] * F[k];
  // cofactor matrix C = dJ/dF
  double C[9];
  C[0] = F[4] * F[8] - F[5] * F[7]; C[1] = F[5] * F[6] - F[3] * F[8]; C[2] = F[3] * F[7] - F[4] * F[6];
  C[3] = F[2] * F[7] - F[1] * F[8]; C[4] = F[0] * F[8] - F[2] * F[6]; C[5] = F[1] * F[6] - F[0] * F[7];
  C[6] = F[1] * F[5] - F[2] * F[4]; C[7] = F[2] * F[3] - F[0] * F[5]; C[8] = F[0] * F[4] - F[1] * F[3];
  const double J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
  const double alpha = 1.0 + 0.75 * mu / lam;
  const double c1 = mu * (1.0 - 1.0 / (Ic + 1.0));
  const double c4 = lam * (J - alpha);
  // first Piola-Kirchhoff stress dPsi/dF and the gradient w.r.t. the 4 vertices
  double Pk[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Pk[k] = c1 * F[k] + c4 * C[k];
  double w[4][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    w[1][j] = Dmi[j]; w[2][j] = Dmi[3 + j]; w[3][j] = Dmi[6 + j];
    w[0][j] = -(Dmi[j] + Dmi[3 + j] + Dmi[6 + j]);
  }
  const double sc = vol * h2;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (nodes[a] < 0) continue;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double gi = sc * (Pk[3 * i] * w[a][0] + Pk[3 * i + 1] * w[a][1] + Pk[3 * i + 2] * w[a][2]);
      atomicAdd(&g[3 * nodes[a] + i], gi);
    }
  }
  // d2Psi/dF2 = c1 I + c2 f f^T + lam c c^T + c4 d2J/dF2  (f = vec F, c = vec cof F)
  const T c2 = (T)(2.0 * mu / ((Ic + 1.0) * (Ic + 1.0)));
  T Hf[81];
  T Ft[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Ft[k] = (T)F[k];
  if (project) {
    snh_project_fspace<T>(Ft, (T)c1, c2, (T)lam, (T)c4, Hf);
  } else {
    T Ct[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Ct[k] = (T)C[k];
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const int i = r / 3, j = r % 3, k = q / 3, l = q % 3;
        T hj = 0;
        if (i != k && j != l) {
          const int m = 3 - i - k, nn = 3 - j - l;
          hj = (T)(lc(i, k, m) * lc(j, l, nn)) * Ft[3 * m + nn];
        }
        Hf[9 * r + q] = ((r == q) ? (T)c1 : T(0)) + c2 * Ft[r] * Ft[q] + (T)lam * Ct[r] * Ct[q] + (T)c4 * hj;
      }
  }
  const int* sl = tslot + 6 * (size_t)e;
  int slots[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) slots[q] = sl[q];
  scatter_fspace<T, 4, 3>(Hf, w, sc, nodes, slots, diag, vals);
}

// ---------------------------------------------------------------- adjoint (form 2)
// Parameter derivative of the tet term for the implicit-step adjoint.  At a
// fixed Poisson ratio mu and lam are both proportional to E and alpha = 1 +
// 3 mu / (4 lam) does not change, so Psi_SNH (Eq. snh) is linear in E and
// d(h^2 grad V Psi_e)/dE_e = h^2 grad(V Psi_e) / E_e.  Each tet adds
// -lambda_e . that to Ebar_e (lambda_e: the adjoint at its 4 nodes, 0 on fixed
// vertices); the gradient is formed exactly as in k_snh.
__global__ void __launch_bounds__(128) k_snh_young_adj(int nt, const int* __restrict__ tv, const int* __restrict__ tn,
                                                       const double* __restrict__ trest, const double* __restrict__ tE,
                                                       const double* __restrict__ P, const double* __restrict__ lamv,
                                                       double h2, double* __restrict__ Ebar) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  const int4 v = reinterpret_cast<const int4*>(tv)[e];
  const int4 n4 = reinterpret_cast<const int4*>(tn)[e];
  const int nodes[4] = {n4.x, n4.y, n4.z, n4.w};
  const double* R = trest + 12 * (size_t)e;
  double Dmi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Dmi[k] = R[k];
  const double vol = R[9], mu = R[10], lam = R[11];
  const v3<double> x0 = ld3(P, v.x);
  const v3<double> d1 = ld3(P, v.y) - x0, d2 = ld3(P, v.z) - x0, d3_ = ld3(P, v.w) - x0;
  const double Ds[9] = {d1.x, d2.x, d3_.x, d1.y, d2.y, d3_.y, d1.z, d2.z, d3_.z};
  double F[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F[3 * i + j] = Ds[3 * i] * Dmi[j] + Ds[3 * i + 1] * Dmi[3 + j] + Ds[3 * i + 2] * Dmi[6 + j];
  double Ic = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) Ic += F[k] * F[k];
  double C[9];
  C[0] = F[4] * F[8] - F[5] * F[7]; C[1] = F[5] * F[6] - F[3] * F[8]; C[2] = F[3] * F[7] - F[4] * F[6];
  C[3] = F[2] * F[7] - F[1] * F[8]; C[4] = F[0] * F[8] - F[2] * F[6]; C[5] = F[1] * F[6] - F[0] * F[7];
  C[6] = F[1] * F[5] - F[2] * F[4]; C[7] = F[2] * F[3] - F[0] * F[5]; C[8] = F[0] * F[4] - F[1] * F[3];
  const double J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
  const double alpha = 1.0 + 0.75 * mu / lam;
  const double c1 = mu * (1.0 - 1.0 / (Ic + 1.0));
  const double c4 = lam * (J - alpha);
  double Pk[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Pk[k] = c1 * F[k] + c4 * C[k];
  double w[4][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    w[1][j] = Dmi[j]; w[2][j] = Dmi[3 + j]; w[3][j] = Dmi[6 + j];
    w[0][j] = -(Dmi[j] + Dmi[3 + j] + Dmi[6 + j]);
  }
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (nodes[a] < 0) continue;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      acc += lamv[3 * nodes[a] + i] * vol * (Pk[3 * i] * w[a][0] + Pk[3 * i + 1] * w[a][1] + Pk[3 * i + 2] * w[a][2]);
  }
  Ebar[e] -= h2 * acc / tE[e];
}

// per-tet Young's moduli at fixed Poisson ratios: mu, lam as in k_rest_tet
__global__ void k_set_young(int nt, const double* __restrict__ E, const double* __restrict__ nu,
                            double* __restrict__ tE, double* __restrict__ trest, int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  const double Ee = E[e];
  if (!(Ee > 0.0) || !isfinite(Ee)) dev_flag(status, DEV_NAN);
  tE[e] = Ee;
  trest[12 * (size_t)e + 10] = Ee / (2.0 * (1.0 + nu[e]));
  trest[12 * (size_t)e + 11] = Ee * nu[e] / ((1.0 + nu[e]) * (1.0 - 2.0 * nu[e]));
}

// ---------------------------------------------------------------- StVK membrane
template <typename T>
__global__ void __launch_bounds__(128) k_membrane(int nc, const int* __restrict__ cv, const int* __restrict__ cn,
                                                  const double* __restrict__ crest, const int* __restrict__ cslot,
                                                  const double* __restrict__ P, double h2, int project,
                                                  double* __restrict__ g, T* __restrict__ diag, T* __restrict__ vals) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc) return;
  const int nodes[3] = {cn[3 * e], cn[3 * e + 1], cn[3 * e + 2]};
  const double* R = crest + 8 * (size_t)e;
  const double Dm[4] = {R[0], R[1], R[2], R[3]};
  const double at = R[4], mu = R[5], lam = R[6];
  const v3<double> x0 = ld3(P, cv[3 * e]);
  const v3<double> a1 = ld3(P, cv[3 * e + 1]) - x0, a2 = ld3(P, cv[3 * e + 2]) - x0;
  const double A1[3] = {a1.x, a1.y, a1.z}, A2[3] = {a2.x, a2.y, a2.z};
  double F[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) F[2 * i + j] = A1[i] * Dm[j] + A2[i] * Dm[2 + j];
  // first Piola-Kirchhoff stress P = dPsi/dF (3x2) and d2Psi/dF2 (6x6, index 2 i + j)
  double Pk[6];
  T Hf[36];
  if (R[7] == 0.0) {
    // StVK: E = (F^T F - I) / 2, S = 2 mu E + lam tr(E) I, P = F S;
    // d2Psi/dF2 [(i,j),(k,l)] = d_ik S_lj + mu (F_il F_kj + (F F^T)_ik d_jl) + lam F_ij F_kl
    const double E00 = 0.5 * (F[0] * F[0] + F[2] * F[2] + F[4] * F[4] - 1.0);
    const double E11 = 0.5 * (F[1] * F[1] + F[3] * F[3] + F[5] * F[5] - 1.0);
    const double E01 = 0.5 * (F[0] * F[1] + F[2] * F[3] + F[4] * F[5]);
    const double tr = E00 + E11;
    const double S[4] = {2 * mu * E00 + lam * tr, 2 * mu * E01, 2 * mu * E01, 2 * mu * E11 + lam * tr};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) Pk[2 * i + j] = F[2 * i] * S[j] + F[2 * i + 1] * S[2 + j];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int i = r / 2, j = r % 2, k = q / 2, l = q % 2;
        const double FFt = F[2 * i] * F[2 * k] + F[2 * i + 1] * F[2 * k + 1];
        double v = (i == k ? S[2 * l + j] : 0.0) + mu * (F[2 * i + l] * F[2 * k + j] + (j == l ? FFt : 0.0)) +
                   lam * F[2 * i + j] * F[2 * k + l];
        Hf[6 * r + q] = (T)v;
      }
  } else {
    // Baraff-Witkin: Psi = kst/2 ((|fu| - 1)^2 + (|fv| - 1)^2) + ksh/2 (fu.fv)^2 (mu, lam hold kst, ksh)
    const double kst = mu, ksh = lam;
    const double fu[3] = {F[0], F[2], F[4]}, fv[3] = {F[1], F[3], F[5]};
    const double nu_ = fmax(sqrt(fu[0] * fu[0] + fu[1] * fu[1] + fu[2] * fu[2]), 1e-12);
    const double nv_ = fmax(sqrt(fv[0] * fv[0] + fv[1] * fv[1] + fv[2] * fv[2]), 1e-12);
    const double c = fu[0] * fv[0] + fu[1] * fv[1] + fu[2] * fv[2];
    const double su = kst * (1.0 - 1.0 / nu_), sv = kst * (1.0 - 1.0 / nv_);
    const double tu = kst / (nu_ * nu_ * nu_), tv = kst / (nv_ * nv_ * nv_);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Pk[2 * i] = su * fu[i] + ksh * c * fv[i];
      Pk[2 * i + 1] = sv * fv[i] + ksh * c * fu[i];
    }
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int i = r / 2, j = r % 2, k = q / 2, l = q % 2;
        const double d = (i == k) ? 1.0 : 0.0;
        double v;
        if (j == 0 && l == 0) v = su * d + tu * fu[i] * fu[k] + ksh * fv[i] * fv[k];
        else if (j == 1 && l == 1) v = sv * d + tv * fv[i] * fv[k] + ksh * fu[i] * fu[k];
        else if (j == 0) v = ksh * (fv[i] * fu[k] + c * d);
        else v = ksh * (fu[i] * fv[k] + c * d);
        Hf[6 * r + q] = (T)v;
      }
  }
  double w[3][2];
#pragma unroll
  for (int j = 0; j < 2; ++j) { w[1][j] = Dm[j]; w[2][j] = Dm[2 + j]; w[0][j] = -(Dm[j] + Dm[2 + j]); }
  const double sc = at * h2;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (nodes[a] < 0) continue;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double sg = 0.0;
#pragma unroll
      for (int j = 0; j < 2; ++j) sg += Pk[2 * i + j] * w[a][j];
      atomicAdd(&g[3 * nodes[a] + i], sc * sg);
    }
  }
  if (project) project_psd<6, T>(Hf);
  int slots[3] = {cslot[3 * e], cslot[3 * e + 1], cslot[3 * e + 2]};
  scatter_fspace<T, 3, 2>(Hf, w, sc, nodes, slots, diag, vals);
}

// ---------------------------------------------------------------- affine orthogonality
template <typename T>
__global__ void k_abd(int nb, int nfree, const double* __restrict__ kv, const int* __restrict__ bslot,
                      const double* __restrict__ x, double h2, int project, double* __restrict__ g,
                      T* __restrict__ diag, T* __restrict__ vals) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int a0 = nfree + 4 * b + 1;  // the three A-column nodes
  v3<double> c[3];
  for (int k = 0; k < 3; ++k) c[k] = ld3(x, a0 + k);
  double G[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[i][j] = dot(c[i], c[j]) - (i == j ? 1.0 : 0.0);
  const double k2 = 2.0 * kv[b] * h2;
  for (int k = 0; k < 3; ++k) {
    v3<double> s = {0, 0, 0};
    for (int j = 0; j < 3; ++j) s = s + G[k][j] * c[j];
    atomicAdd(&g[3 * (a0 + k)], k2 * s.x);
    atomicAdd(&g[3 * (a0 + k) + 1], k2 * s.y);
    atomicAdd(&g[3 * (a0 + k) + 2], k2 * s.z);
  }
  // H_kl = 2 kv [d_kl sum_j c_j c_j^T + c_l c_k^T + G_kl I]
  T H[81];
  double cc[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int q = 0; q < 3; ++q) s += comp3(c[q], i) * comp3(c[q], j);
      cc[i][j] = s;
    }
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double v = comp3(c[l], i) * comp3(c[k], j) + (i == j ? G[k][l] : 0.0) + (k == l ? cc[i][j] : 0.0);
          H[9 * (3 * k + i) + 3 * l + j] = (T)(k2 * v);
        }
  if (project) project_psd<9, T>(H);
  for (int k = 0; k < 3; ++k)
    for (int l = k; l < 3; ++l) {
      if (k == l) {
        T* d = diag + 9 * (size_t)(a0 + k);
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) atomicAdd(d + 3 * i + j, H[9 * (3 * k + i) + 3 * k + j]);
      } else {
        const int q = (k == 0) ? (l == 1 ? 3 : 4) : 5;  // node pairs (1,2) (1,3) (2,3)
        T* d = vals + 9 * (size_t)bslot[6 * b + q];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) atomicAdd(d + 3 * i + j, H[9 * (3 * k + i) + 3 * l + j]);
      }
    }
}

// ---------------------------------------------------------------- energies (FP64, compensated)
constexpr int EN_T = 256, EN_MAXB = 148 * 4;

// Every energy kernel walks its items in warp-uniform strides.  With sacc set
// (batches) each item's energy goes to its scene's accumulator (warp-segmented
// by scene; items are sorted by scene); otherwise into the compensated block
// partials.
struct scene_acc {
  const int* vscene;      // [nv] vertex -> scene
  const int* node_scene;  // [nn] node -> scene
  double* acc;            // [nscene] or null
};
__device__ __forceinline__ void add_energy(const scene_acc& sa, ksum& k, int key, double v) {
  if (sa.acc) seg_add_global(sa.acc, key, v);
  else kadd(k, v);
}

__global__ void k_energy_inertia(int nfree, int nb, const double* __restrict__ m, const double* __restrict__ x,
                                 const double* __restrict__ xtil, ksum* __restrict__ part, scene_acc sa) {
  ksum k{0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long first = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL;
  for (long long base = first; base < nfree; base += stride) {
    const long long i = base + lane;
    double e = 0.0;
    int key = -1;
    if (i < nfree) {
      double s = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double d = x[3 * i + c] - xtil[3 * i + c];
        s += d * d;
      }
      e = 0.5 * m[i] * s;
      key = sa.acc ? sa.node_scene[i] : 0;
    }
    add_energy(sa, k, key, e);
  }
  for (long long base = first; base < nb; base += stride) {
    const long long b = base + lane;
    double e = 0.0;
    int key = -1;
    if (b < nb) {
      const double* M = m + nfree + 16 * b;
      const long long b0 = nfree + 4 * b;
      for (int a = 0; a < 4; ++a)
        for (int q = 0; q < 4; ++q)
          for (int c = 0; c < 3; ++c)
            e += M[4 * a + q] * (x[3 * (b0 + a) + c] - xtil[3 * (b0 + a) + c]) *
                 (x[3 * (b0 + q) + c] - xtil[3 * (b0 + q) + c]);
      e *= 0.5;
      key = sa.acc ? sa.node_scene[b0] : 0;
    }
    add_energy(sa, k, key, e);
  }
  k = block_ksum(k);
  if (threadIdx.x == 0) part[blockIdx.x] = k;
}

__global__ void k_energy_snh(int nt, const int* __restrict__ tv, const double* __restrict__ trest,
                             const double* __restrict__ P, double h2, ksum* __restrict__ part, scene_acc sa) {
  ksum k{0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < nt; base += stride) {
    const long long e = base + lane;
    double val = 0.0;
    int key = -1;
    if (e < nt) {
      const int4 v = reinterpret_cast<const int4*>(tv)[e];
      const double* R = trest + 12 * (size_t)e;
      const v3<double> x0 = ld3(P, v.x);
      const v3<double> d1 = ld3(P, v.y) - x0, d2 = ld3(P, v.z) - x0, d3_ = ld3(P, v.w) - x0;
      const double Ds[9] = {d1.x, d2.x, d3_.x, d1.y, d2.y, d3_.y, d1.z, d2.z, d3_.z};
      double F[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[3 * i + j] = Ds[3 * i] * R[j] + Ds[3 * i + 1] * R[3 + j] + Ds[3 * i + 2] * R[6 + j];
      double Ic = 0.0;
      for (int q = 0; q < 9; ++q) Ic += F[q] * F[q];
      const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                       F[2] * (F[3] * F[7] - F[4] * F[6]);
      const double mu = R[10], lam = R[11];
      const double alpha = 1.0 + 0.75 * mu / lam;
      const double psi = 0.5 * mu * (Ic - 3.0) - 0.5 * mu * log(Ic + 1.0) + 0.5 * lam * (J - alpha) * (J - alpha);
      val = h2 * R[9] * psi;
      key = sa.acc ? sa.vscene[v.x] : 0;
    }
    add_energy(sa, k, key, val);
  }
  k = block_ksum(k);
  if (threadIdx.x == 0) part[blockIdx.x] = k;
}

__global__ void k_energy_membrane(int nc, const int* __restrict__ cv, const double* __restrict__ crest,
                                  const double* __restrict__ P, double h2, ksum* __restrict__ part, scene_acc sa) {
  ksum k{0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < nc; base += stride) {
    const long long e = base + lane;
    double val = 0.0;
    int key = -1;
    if (e < nc) {
      const double* R = crest + 8 * (size_t)e;
      const v3<double> x0 = ld3(P, cv[3 * e]);
      const v3<double> a1 = ld3(P, cv[3 * e + 1]) - x0, a2 = ld3(P, cv[3 * e + 2]) - x0;
      const v3<double> f0 = R[0] * a1 + R[2] * a2, f1 = R[1] * a1 + R[3] * a2;  // columns of F
      double psi;
      if (R[7] == 0.0) {  // StVK
        const double E00 = 0.5 * (dot(f0, f0) - 1.0), E11 = 0.5 * (dot(f1, f1) - 1.0), E01 = 0.5 * dot(f0, f1);
        const double tr = E00 + E11;
        psi = R[5] * (E00 * E00 + E11 * E11 + 2.0 * E01 * E01) + 0.5 * R[6] * tr * tr;
      } else {  // Baraff-Witkin stretch and shear
        const double su = sqrt(dot(f0, f0)) - 1.0, sv = sqrt(dot(f1, f1)) - 1.0, c = dot(f0, f1);
        psi = 0.5 * R[5] * (su * su + sv * sv) + 0.5 * R[6] * c * c;
      }
      val = h2 * R[4] * psi;
      key = sa.acc ? sa.vscene[cv[3 * e]] : 0;
    }
    add_energy(sa, k, key, val);
  }
  k = block_ksum(k);
  if (threadIdx.x == 0) part[blockIdx.x] = k;
}

__global__ void k_energy_bend(int nh, const int* __restrict__ hv, const double* __restrict__ hrest,
                              const double* __restrict__ P, double h2, ksum* __restrict__ part, scene_acc sa) {
  ksum k{0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < nh; base += stride) {
    const long long e = base + lane;
    double val = 0.0;
    int key = -1;
    if (e < nh) {
      const double th =
          hinge_theta(ld3(P, hv[4 * e]), ld3(P, hv[4 * e + 1]), ld3(P, hv[4 * e + 2]), ld3(P, hv[4 * e + 3]));
      const double d = th - hrest[2 * e];
      val = h2 * hrest[2 * e + 1] * d * d;
      key = sa.acc ? sa.vscene[hv[4 * e]] : 0;
    }
    add_energy(sa, k, key, val);
  }
  k = block_ksum(k);
  if (threadIdx.x == 0) part[blockIdx.x] = k;
}

__global__ void k_energy_abd(int nb, int nfree, const double* __restrict__ kv, const double* __restrict__ x, double h2,
                             ksum* __restrict__ part, scene_acc sa) {
  ksum k{0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < nb; base += stride) {
    const long long b = base + lane;
    double val = 0.0;
    int key = -1;
    if (b < nb) {
      const long long a0 = nfree + 4 * b + 1;
      double s = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const double d = dot(ld3(x, (int)(a0 + i)), ld3(x, (int)(a0 + j))) - (i == j ? 1.0 : 0.0);
          s += d * d;
        }
      val = h2 * 0.5 * kv[b] * s;
      key = sa.acc ? sa.node_scene[a0 - 1] : 0;
    }
    add_energy(sa, k, key, val);
  }
  k = block_ksum(k);
  if (threadIdx.x == 0) part[blockIdx.x] = k;
}

// sum each term's partials in order (one block per term)
__global__ void k_reduce_parts(const ksum* __restrict__ part, int nparts, int stride, double* __restrict__ out) {
  ksum k{0.0, 0.0};
  const ksum* p = part + (size_t)blockIdx.x * stride;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) kmerge(k, p[i]);
  k = block_ksum(k);
  if (threadIdx.x == 0) out[blockIdx.x] = k.s + k.c;
}

template <typename T>
yasps_status eval_static_t(yasps_system* s, const double* x, const double* xtil, int mask, int project) {
  const double h2 = s->prm.dt * s->prm.dt;
  T* diag = as<T>(s->diag);
  T* vals = as<T>(s->Hs.vals);
  double* g = as<double>(s->grad);
  const double* P = as<double>(s->P);
  if ((mask & YASPS_TERM_INERTIA) && s->nfree > 0) {
    k_inertia_free<T><<<blocks_for(s->nfree, 256), 256, 0, s->stream>>>(s->nfree, as<double>(s->nodemass), x, xtil, g, diag);
    LAUNCH_CHECK(s, "k_inertia_free");
  }
  if ((mask & YASPS_TERM_INERTIA) && s->nb > 0) {
    k_inertia_body<T><<<blocks_for(s->nb, 64), 64, 0, s->stream>>>(s->nb, s->nfree, as<double>(s->nodemass) + s->nfree,
                                                                  as<int>(s->body_slot), x, xtil, g, diag, vals);
    LAUNCH_CHECK(s, "k_inertia_body");
  }
  if ((mask & YASPS_TERM_TET) && s->nt > 0) {
    // algorithmic bytes: per-tet inputs once, positions once, unique outputs once
    const double bytes = (double)s->nt * (16 + 16 + 96 + 24) + 24.0 * s->nv + 24.0 * s->nn +
                         (double)sizeof(T) * 9.0 * ((double)s->Hs.nnzb + s->nn);
    cudaEvent_t pa = prof_begin(s);
    k_snh<T><<<blocks_for(s->nt, 128), 128, 0, s->stream>>>(s->nt, as<int>(s->tet_v), as<int>(s->tet_n),
                                                           as<double>(s->tet_rest), as<int>(s->tet_slot), P, h2,
                                                           project, g, diag, vals);
    LAUNCH_CHECK(s, "k_snh");
    prof_end(s, YASPS_STAGE_TET, pa, bytes);
  }
  if ((mask & YASPS_TERM_MEMBRANE) && s->nc > 0) {
    k_membrane<T><<<blocks_for(s->nc, 128), 128, 0, s->stream>>>(s->nc, as<int>(s->tri_v), as<int>(s->tri_n),
                                                                as<double>(s->tri_rest), as<int>(s->tri_slot), P, h2,
                                                                project, g, diag, vals);
    LAUNCH_CHECK(s, "k_membrane");
  }
  if ((mask & YASPS_TERM_BEND) && s->nh > 0) {
    RC(launch_bend(s, project));
  }
  if ((mask & YASPS_TERM_ABD) && s->nb > 0) {
    k_abd<T><<<blocks_for(s->nb, 64), 64, 0, s->stream>>>(s->nb, s->nfree, as<double>(s->body_kv), as<int>(s->body_slot),
                                                          x, h2, project, g, diag, vals);
    LAUNCH_CHECK(s, "k_abd");
  }
  return YASPS_OK;
}

}  // namespace

// ======================================================================== API
yasps_status setup_rest(yasps_system* s, const double* tE, const double* tnu, const double* trho, const double* cE,
                        const double* cnu, const double* cth, const double* crho, const double* hkb) {
  int* st = as<int>(s->status);
  if (s->nt > 0) {
    k_rest_tet<<<blocks_for(s->nt, 128), 128, 0, s->stream>>>(s->nt, as<int>(s->tet_v), as<double>(s->rest), tE, tnu,
                                                             trho, as<double>(s->tet_rest), as<double>(s->vmass), st);
    LAUNCH_CHECK(s, "k_rest_tet");
    k_nodes_of<<<blocks_for(4LL * s->nt, 256), 256, 0, s->stream>>>(s->nt, 4, as<int>(s->tet_v), as<int>(s->vnode),
                                                                   as<int>(s->vbody), as<int>(s->tet_n), st);
    LAUNCH_CHECK(s, "k_nodes_of");
  }
  if (s->nc > 0) {
    k_rest_tri<<<blocks_for(s->nc, 128), 128, 0, s->stream>>>(s->nc, as<int>(s->tri_v), as<double>(s->rest), cE, cnu,
                                                             cth, crho, s->cloth_model, as<double>(s->tri_rest),
                                                             as<double>(s->vmass), st);
    LAUNCH_CHECK(s, "k_rest_tri");
    k_nodes_of<<<blocks_for(3LL * s->nc, 256), 256, 0, s->stream>>>(s->nc, 3, as<int>(s->tri_v), as<int>(s->vnode),
                                                                   as<int>(s->vbody), as<int>(s->tri_n), st);
    LAUNCH_CHECK(s, "k_nodes_of");
  }
  if (s->nh > 0) {
    k_rest_hinge<<<blocks_for(s->nh, 128), 128, 0, s->stream>>>(s->nh, as<int>(s->hinge_v), as<double>(s->rest), hkb,
                                                               as<double>(s->hinge_rest));
    LAUNCH_CHECK(s, "k_rest_hinge");
    k_nodes_of<<<blocks_for(4LL * s->nh, 256), 256, 0, s->stream>>>(s->nh, 4, as<int>(s->hinge_v), as<int>(s->vnode),
                                                                   as<int>(s->vbody), as<int>(s->hinge_n), st);
    LAUNCH_CHECK(s, "k_nodes_of");
  }
  if (s->nv > 0) {
    k_free_nodemass<<<blocks_for(s->nv, 256), 256, 0, s->stream>>>(s->nv, as<int>(s->vnode), as<int>(s->vbody),
                                                                  as<double>(s->vmass), as<double>(s->nodemass));
    LAUNCH_CHECK(s, "k_free_nodemass");
  }
  return YASPS_OK;
}

yasps_status launch_snh_young_adj(yasps_system* s, const double* P, const double* lam, double h2, double* Ebar) {
  if (s->nt == 0) return YASPS_OK;
  k_snh_young_adj<<<blocks_for(s->nt, 128), 128, 0, s->stream>>>(s->nt, as<int>(s->tet_v), as<int>(s->tet_n),
                                                                 as<double>(s->tet_rest), as<double>(s->tet_E), P, lam,
                                                                 h2, Ebar);
  LAUNCH_CHECK(s, "k_snh_young_adj");
  return YASPS_OK;
}

yasps_status launch_set_young(yasps_system* s, const double* E) {
  if (s->nt == 0) return YASPS_OK;
  k_set_young<<<blocks_for(s->nt, 256), 256, 0, s->stream>>>(s->nt, E, as<double>(s->tet_nu), as<double>(s->tet_E),
                                                             as<double>(s->tet_rest), as<int>(s->status));
  LAUNCH_CHECK(s, "k_set_young");
  return YASPS_OK;
}

yasps_status static_sparsity(yasps_system* s) {
  const long long n_tet = 6LL * s->nt, n_tri = 3LL * s->nc, n_h = 6LL * s->nh, n_b = 6LL * s->nb;
  const long long n = n_tet + n_tri + n_h + n_b;
  if (n > 0x7fffffffLL) SYS_FAIL(s, YASPS_E_INVAL, "scene too large for 32-bit contribution ids");
  ENSURE(s, s->ws[0], sizeof(uint64_t) * (n + 1));
  ENSURE(s, s->ws[1], sizeof(int) * (n + 1));
  ENSURE(s, s->ws[2], sizeof(int) * (n + 1));
  uint64_t* keys = as<uint64_t>(s->ws[0]);
  int* vals = as<int>(s->ws[1]);
  int* slot_of = as<int>(s->ws[2]);
  long long off = 0;
  if (s->nt) {
    k_elem_keys<<<blocks_for(n_tet, 256), 256, 0, s->stream>>>(s->nt, 4, as<int>(s->tet_n), s->nbits, (int)off, keys + off, vals + off);
    LAUNCH_CHECK(s, "k_elem_keys");
  }
  off += n_tet;
  if (s->nc) {
    k_elem_keys<<<blocks_for(n_tri, 256), 256, 0, s->stream>>>(s->nc, 3, as<int>(s->tri_n), s->nbits, (int)off, keys + off, vals + off);
    LAUNCH_CHECK(s, "k_elem_keys");
  }
  off += n_tri;
  if (s->nh) {
    k_elem_keys<<<blocks_for(n_h, 256), 256, 0, s->stream>>>(s->nh, 4, as<int>(s->hinge_n), s->nbits, (int)off, keys + off, vals + off);
    LAUNCH_CHECK(s, "k_elem_keys");
  }
  off += n_h;
  if (s->nb) {
    k_body_keys<<<blocks_for(n_b, 256), 256, 0, s->stream>>>(s->nb, s->nfree, s->nbits, (int)off, keys + off, vals + off);
    LAUNCH_CHECK(s, "k_body_keys");
  }
  RC(bsr_from_keys(s, keys, vals, (int)n, s->Hs, slot_of, (int)n));
  off = 0;
  if (s->nt) CK(s, cudaMemcpyAsync(s->tet_slot.p, slot_of + off, sizeof(int) * n_tet, cudaMemcpyDeviceToDevice, s->stream));
  off += n_tet;
  if (s->nc) CK(s, cudaMemcpyAsync(s->tri_slot.p, slot_of + off, sizeof(int) * n_tri, cudaMemcpyDeviceToDevice, s->stream));
  off += n_tri;
  if (s->nh) CK(s, cudaMemcpyAsync(s->hinge_slot.p, slot_of + off, sizeof(int) * n_h, cudaMemcpyDeviceToDevice, s->stream));
  off += n_h;
  if (s->nb) CK(s, cudaMemcpyAsync(s->body_slot.p, slot_of + off, sizeof(int) * n_b, cudaMemcpyDeviceToDevice, s->stream));
  return YASPS_OK;
}

yasps_status launch_positions(yasps_system* s, const double* x, double* P) {
  if (s->nv == 0) return YASPS_OK;
  k_positions<<<blocks_for(s->nv, 256), 256, 0, s->stream>>>(s->nv, as<int>(s->vnode), as<int>(s->vbody),
                                                             as<double>(s->vr), as<int>(s->emb_node),
                                                             as<double>(s->emb_w), as<double>(s->xfix), x, P);
  LAUNCH_CHECK(s, "k_positions");
  return YASPS_OK;
}

yasps_status launch_xtilde(yasps_system* s, const double* xt, const double* vt, double* xtil) {
  if (s->nn == 0) return YASPS_OK;
  k_xtilde<<<blocks_for(s->nn, 256), 256, 0, s->stream>>>(s->nn, s->nfree, s->prm.dt, s->prm.gravity[0],
                                                         s->prm.gravity[1], s->prm.gravity[2], xt, vt, xtil);
  LAUNCH_CHECK(s, "k_xtilde");
  return YASPS_OK;
}

yasps_status launch_eval_static(yasps_system* s, const double* x, const double* xtil, int mask, int project) {
  if (s->hess_precision == 1) return eval_static_t<float>(s, x, xtil, mask, project);
  return eval_static_t<double>(s, x, xtil, mask, project);
}

yasps_status energy_static(yasps_system* s, const double* x, const double* xtil, double* out5, double* sacc) {
  const scene_acc sa{sacc ? as<int>(s->vscene) : nullptr, sacc ? as<int>(s->node_scene) : nullptr, sacc};
  const double h2 = s->prm.dt * s->prm.dt;
  const int stride = EN_MAXB;
  ENSURE(s, s->red, sizeof(ksum) * 5 * stride + 64);
  ksum* part = as<ksum>(s->red);
  CK(s, cudaMemsetAsync(part, 0, sizeof(ksum) * 5 * stride, s->stream));
  const double* P = as<double>(s->P);
  auto nblk = [](long long n) { return (int)std::min<long long>(EN_MAXB, std::max<long long>(1, (n + EN_T - 1) / EN_T)); };
  k_energy_inertia<<<nblk(std::max(s->nfree, s->nb)), EN_T, 0, s->stream>>>(s->nfree, s->nb, as<double>(s->nodemass), x,
                                                                            xtil, part, sa);
  LAUNCH_CHECK(s, "k_energy_inertia");
  if (s->nt) {
    k_energy_snh<<<nblk(s->nt), EN_T, 0, s->stream>>>(s->nt, as<int>(s->tet_v), as<double>(s->tet_rest), P, h2,
                                                      part + stride, sa);
    LAUNCH_CHECK(s, "k_energy_snh");
  }
  if (s->nc) {
    k_energy_membrane<<<nblk(s->nc), EN_T, 0, s->stream>>>(s->nc, as<int>(s->tri_v), as<double>(s->tri_rest), P, h2,
                                                          part + 2 * stride, sa);
    LAUNCH_CHECK(s, "k_energy_membrane");
  }
  if (s->nh) {
    k_energy_bend<<<nblk(s->nh), EN_T, 0, s->stream>>>(s->nh, as<int>(s->hinge_v), as<double>(s->hinge_rest), P, h2,
                                                      part + 3 * stride, sa);
    LAUNCH_CHECK(s, "k_energy_bend");
  }
  if (s->nb) {
    k_energy_abd<<<nblk(s->nb), EN_T, 0, s->stream>>>(s->nb, s->nfree, as<double>(s->body_kv), x, h2, part + 4 * stride,
                                                      sa);
    LAUNCH_CHECK(s, "k_energy_abd");
  }
  if (sacc) return YASPS_OK;  // batches: the per-scene sums are the result
  double* out_dev = reinterpret_cast<double*>(part + 5 * stride);
  k_reduce_parts<<<5, 256, 0, s->stream>>>(part, stride, stride, out_dev);
  LAUNCH_CHECK(s, "k_reduce_parts");
  CK(s, cudaMemcpyAsync(out5, out_dev, sizeof(double) * 5, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}
