// contact.cu -- the dynamic (collision) part of the IPC Newton step.
//
//  * broadphase: a uniform grid over the boxes of one primitive set (counting
//    sort into cells), queried by the boxes of the other; each overlapping box
//    pair is reported once, in the cell holding the minimum corner of the
//    boxes' intersection;
//  * narrow phase: exact FP64 squared distances with closest-feature
//    classification (distance.cuh); a pair is active when s < dhat^2.  Pair
//    lists are canonical: sorted by (a, b) (Sec. "UNION": collision pairs are a
//    dynamic primitive whose connectivity is rebuilt at run time);
//  * the dynamic BSR layout of H_dynamic (Sec. "Index Computation"): the upper
//    block keys of every pair's node set, sorted and made unique (App. B);
//  * barrier evaluation: b(s), its position-space gradient and Hessian,
//    projected in position space (the reduced-coordinate projection of Sec.
//    "EVD and PSD Projection", valid because free and affine parameterisations
//    are linear), then mapped to nodes through the UNION Jacobian of each
//    vertex (I3 for a free vertex, [I3, r1 I3, r2 I3, r3 I3] for an affine one,
//    Sec. "Differentiation of Unioned Attributes") with duplicate nodes merged
//    (Sec. "Hessian Code Generation", local compression);
//  * the CCD step bound: additive CCD (Li, Kaufman and Jiang 2021, ACCD) on
//    swept-box candidates, exact for point-plane pairs.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "distance.cuh"
#include "eig.cuh"
#include "internal.h"

using dist::d3;

namespace {

// ---------------------------------------------------------------- boxes and grid
// The grid works on FP32 copies of the boxes rounded outward (a conservative
// superset); pairs that pass the FP32 test are confirmed on the exact FP64
// boxes, so candidate sets are those of the FP64 boxes while the per-item work
// stays off the (scarce) FP64 pipe.
struct gridp {
  float lo[3];
  float inv;
  int dim[3];
};

__device__ __forceinline__ int cell_coord(float v, float lo, float inv, int dim) {
  const float f = floorf((v - lo) * inv);
  return (f < 0.0f) ? 0 : (f > (float)(dim - 1) ? dim - 1 : (int)f);
}

struct boxes {  // n boxes, 3 per corner, FP64 exact + FP32 outward-rounded copies
  const double *lo, *hi;
  const float *lof, *hif;
};
struct boxw {
  double *lo, *hi;
  float *lof, *hif;
  // batches: every scene's boxes are moved to its own cell of a lattice with
  // this spacing, so the grid does not stack the (overlapping) scenes; pairs
  // across scenes are excluded anyway, so this only saves work
  const int* vscene;
  double spacing;
  // swept boxes: per-scene sums of the vertex displacements (x, y, z, count
  // in rows of nsc) or null.  The end positions are moved back by their
  // scene's mean displacement: a common translation of every vertex changes
  // no distance at any time of the step, so boxes swept in that moving frame
  // are as conservative as boxes swept in place, and much smaller when a
  // scene moves as a whole (a falling pile)
  const double* shift;
  int nsc;
  operator boxes() const { return boxes{lo, hi, lof, hif}; }
};
__device__ __forceinline__ void scene_offset(int sc, double spacing, double* off) {
  off[0] = (double)(sc & 7) * spacing;
  off[1] = (double)((sc >> 3) & 7) * spacing;
  off[2] = (double)(sc >> 6) * spacing;
}

// box of k-vertex primitive e at positions P0 (and P1 when swept), before
// growth: l, h; off: its scene's lattice offset
__device__ __forceinline__ void prim_hull(int e, int k, const int* __restrict__ idx, const double* __restrict__ P0,
                                          const double* __restrict__ P1, const boxw& out, double* l, double* h,
                                          double* off) {
  const int v0 = idx[k * e];
  for (int c = 0; c < 3; ++c) l[c] = h[c] = P0[3 * v0 + c];
  for (int a = 1; a < k; ++a) {
    const int v = idx[k * e + a];
    for (int c = 0; c < 3; ++c) { l[c] = fmin(l[c], P0[3 * v + c]); h[c] = fmax(h[c], P0[3 * v + c]); }
  }
  if (P1) {
    double u[3] = {0.0, 0.0, 0.0};
    if (out.shift) {
      const int sc = out.vscene ? out.vscene[v0] : 0;
      const double cnt = out.shift[3 * out.nsc + sc];
      if (cnt > 0.0)
        for (int c = 0; c < 3; ++c) u[c] = out.shift[c * out.nsc + sc] / cnt;
    }
    double l1[3], h1[3];
    for (int c = 0; c < 3; ++c) l1[c] = h1[c] = P1[3 * v0 + c] - u[c];
    for (int a = 1; a < k; ++a) {
      const int v = idx[k * e + a];
      for (int c = 0; c < 3; ++c) {
        const double q = P1[3 * v + c] - u[c];
        l1[c] = fmin(l1[c], q);
        h1[c] = fmax(h1[c], q);
      }
    }
    for (int c = 0; c < 3; ++c) {
      // the rounding of P1 - u: a few ulps of the operands
      const double r = out.shift ? 4.0 * DBL_EPSILON * (fmax(fabs(l1[c]), fabs(h1[c])) + fabs(u[c])) : 0.0;
      l[c] = fmin(l[c], l1[c] - r);
      h[c] = fmax(h[c], h1[c] + r);
    }
  }
  for (int c = 0; c < 3; ++c) off[c] = 0.0;
  if (out.vscene) scene_offset(out.vscene[v0], out.spacing, off);
}
// the box grown by infl: FP64 and outward-rounded FP32
__device__ __forceinline__ void put_box(const boxw& out, int e, const double* l, const double* h, const double* off,
                                        double infl) {
  for (int c = 0; c < 3; ++c) {
    const double lc = l[c] - infl + off[c], hc = h[c] + infl + off[c];
    out.lo[3 * e + c] = lc;
    out.hi[3 * e + c] = hc;
    out.lof[3 * e + c] = __double2float_rd(lc);
    out.hif[3 * e + c] = __double2float_ru(hc);
  }
}
// boxes of k-vertex primitives at positions P0 (and P1 when swept), grown by infl
__global__ void k_boxes(int n, int k, const int* __restrict__ idx, const double* __restrict__ P0,
                        const double* __restrict__ P1, double infl, boxw out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double l[3], h[3], off[3];
  prim_hull(e, k, idx, P0, P1, out, l, h, off);
  put_box(out, e, l, h, off, infl);
}
// a set queried against itself (edges): its query boxes (grown by infl) and
// its grid boxes (not grown) from one hull
__global__ void k_boxes_self(int n, int k, const int* __restrict__ idx, const double* __restrict__ P0,
                             const double* __restrict__ P1, double infl, boxw query, boxw grid) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double l[3], h[3], off[3];
  prim_hull(e, k, idx, P0, P1, query, l, h, off);
  put_box(query, e, l, h, off, infl);
  put_box(grid, e, l, h, off, 0.0);
}

// per-scene sums of the vertex displacements D and vertex counts into
// acc[4][ns] (rows x, y, z, count).  One scene: per-block sums, one atomic per
// block and row; batches (vertices sorted by scene): one atomic per run of a
// scene within a warp
__global__ void k_disp_sum(int nv, const double* __restrict__ D, const int* __restrict__ vscene, int ns,
                           double* __restrict__ acc) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  if (!vscene) {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
      for (int c = 0; c < 3; ++c) t[c] += D[3 * i + c];
      t[3] += 1.0;
    }
    __shared__ double sh[4][32];
    for (int c = 0; c < 4; ++c) {
      double v = t[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sh[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
      atomicAdd(acc + threadIdx.x, v);
    }
    return;
  }
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < nv; base += stride) {
    const long long i = base + lane;
    const bool in = i < nv;
    const int key = in ? vscene[i] : -1;
    for (int c = 0; c < 3; ++c) seg_add_global(acc + (size_t)c * ns, key, in ? D[3 * i + c] : 0.0);
    seg_add_global(acc + 3 * (size_t)ns, key, in ? 1.0 : 0.0);
  }
}

// min of lo, max of hi, max extent over n boxes -> out[7] (per-block partials first)
__global__ void k_box_reduce(int n, const double* __restrict__ lo, const double* __restrict__ hi, double* __restrict__ part) {
  // min lo (3), max hi (3), max extent, sum of per-box largest extents
  double r[8] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300, 0.0, 0.0};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double ext = 0.0;
    for (int c = 0; c < 3; ++c) {
      r[c] = fmin(r[c], lo[3 * e + c]);
      r[3 + c] = fmax(r[3 + c], hi[3 * e + c]);
      ext = fmax(ext, hi[3 * e + c] - lo[3 * e + c]);
    }
    r[6] = fmax(r[6], ext);
    r[7] += ext;
  }
  __shared__ double sh[8][32];
  for (int q = 0; q < 8; ++q) {
    double v = r[q];
    for (int o = 16; o > 0; o >>= 1) {
      double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = (q < 3) ? fmin(v, w) : (q < 7 ? fmax(v, w) : v + w);
    }
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int q = threadIdx.x;
    double v = sh[q][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      v = (q < 3) ? fmin(v, sh[q][w]) : (q < 7 ? fmax(v, sh[q][w]) : v + sh[q][w]);
    part[8 * blockIdx.x + q] = v;
  }
}

__device__ __forceinline__ void cell_range(const gridp& G, const float* lo, const float* hi, int* c0, int* c1) {
  for (int c = 0; c < 3; ++c) {
    c0[c] = cell_coord(lo[c], G.lo[c], G.inv, G.dim[c]);
    c1[c] = cell_coord(hi[c], G.lo[c], G.inv, G.dim[c]);
  }
}

__global__ void k_grid_count(int n, const float* __restrict__ lo, const float* __restrict__ hi, gridp G,
                             int* __restrict__ cnt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  int c0[3], c1[3];
  cell_range(G, lo + 3 * e, hi + 3 * e, c0, c1);
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) atomicAdd(&cnt[((long long)z * G.dim[1] + y) * G.dim[0] + x], 1);
}
// Each cell's entries are stored as packed records (FP32 box + primitive id,
// 32 bytes), so a query walks a cell as one contiguous stream instead of
// gathering every box by primitive id.
__global__ void k_grid_fill(int n, const float* __restrict__ lo, const float* __restrict__ hi, gridp G,
                            const int* __restrict__ start, int* __restrict__ fill, float4* __restrict__ pk) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  int c0[3], c1[3];
  const float* l = lo + 3 * e;
  const float* h = hi + 3 * e;
  cell_range(G, l, h, c0, c1);
  const float4 r0 = make_float4(l[0], l[1], l[2], __int_as_float(e));
  const float4 r1 = make_float4(h[0], h[1], h[2], 0.0f);
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        const long long id = ((long long)z * G.dim[1] + y) * G.dim[0] + x;
        const int q = start[id] + atomicAdd(&fill[id], 1);
        pk[2 * (size_t)q] = r0;
        pk[2 * (size_t)q + 1] = r1;
      }
}

struct grid_dev {
  gridp G;
  const int* start;
  const float4* pk;  // [entries][2]: (lo, id), (hi, 0)
  boxes B;
};

// Visit every B box overlapping A box i once (min-corner rule on the FP32
// boxes, then the exact FP64 overlap test).  upper: only B ids above i (a set
// queried against itself, each unordered pair once), skipped on the record's
// id before its box is read.
template <class F>
__device__ __forceinline__ void grid_visit(const grid_dev& g, const boxes& A, int i, F&& f, bool upper = false,
                                           int sub = 0, int gsz = 1) {
  // the query box in registers (f writes through pointers the compiler cannot
  // tell apart from it)
  float alf[3], ahf[3];
  double alo[3], ahi[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    alf[c] = A.lof[3 * i + c];
    ahf[c] = A.hif[3 * i + c];
    alo[c] = A.lo[3 * i + c];
    ahi[c] = A.hi[3 * i + c];
  }
  int c0[3], c1[3];
  cell_range(g.G, alf, ahf, c0, c1);
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        const long long id = ((long long)z * g.G.dim[1] + y) * g.G.dim[0] + x;
        const int qe = g.start[id + 1];
        // records sub, sub + gsz, ... of the cell (a group of gsz lanes shares a query)
        int q = g.start[id] + sub;
        // one record ahead: the next record's 32 bytes load while this one is tested
        float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
        if (q < qe) {
          n0 = g.pk[2 * (size_t)q];
          n1 = g.pk[2 * (size_t)q + 1];
        }
        for (; q < qe; q += gsz) {
          const float4 r0 = n0, r1 = n1;
          if (q + gsz < qe) {
            n0 = g.pk[2 * (size_t)(q + gsz)];
            n1 = g.pk[2 * (size_t)(q + gsz) + 1];
          }
          const int j = __float_as_int(r0.w);
          if (upper && j <= i) continue;
          const float blf[3] = {r0.x, r0.y, r0.z};
          const float bhf[3] = {r1.x, r1.y, r1.z};
          if (ahf[0] < blf[0] || bhf[0] < alf[0] || ahf[1] < blf[1] || bhf[1] < alf[1] || ahf[2] < blf[2] ||
              bhf[2] < alf[2])
            continue;
          // report only in the cell of the FP32 intersection's minimum corner
          const int mx = cell_coord(fmaxf(alf[0], blf[0]), g.G.lo[0], g.G.inv, g.G.dim[0]);
          const int my = cell_coord(fmaxf(alf[1], blf[1]), g.G.lo[1], g.G.inv, g.G.dim[1]);
          const int mz = cell_coord(fmaxf(alf[2], blf[2]), g.G.lo[2], g.G.inv, g.G.dim[2]);
          if (mx != x || my != y || mz != z) continue;
          const double* bl = g.B.lo + 3 * j;
          const double* bh = g.B.hi + 3 * j;
          if (ahi[0] < bl[0] || bh[0] < alo[0] || ahi[1] < bl[1] || bh[1] < alo[1] || ahi[2] < bl[2] || bh[2] < alo[2])
            continue;
          f(j);
        }
      }
}

// ---------------------------------------------------------------- exclusions
struct topo {
  const int *vnode, *vbody, *stri, *sedge, *svert;
  int* status;
  const int* vscene;  // scene of each vertex in a batch, else null: pairs never cross scenes
  const int* enode;   // [ne][8] cage nodes of embedded vertices
  const double* ew;   // [ne][8] their weights
};
__device__ __forceinline__ bool pt_excluded(const topo& T, int v, int t0, int t1, int t2) {
  if (v == t0 || v == t1 || v == t2) return true;
  if (T.vscene && T.vscene[v] != T.vscene[t0]) return true;
  const int bv = T.vbody[v];
  if (bv >= 0 && bv == T.vbody[t0]) return true;
  if (T.vnode[v] < 0 && T.vnode[t0] < 0 && T.vnode[t1] < 0 && T.vnode[t2] < 0) return true;
  return false;
}
__device__ __forceinline__ bool ee_excluded(const topo& T, int e0, int e1, int f0, int f1) {
  if (e0 == f0 || e0 == f1 || e1 == f0 || e1 == f1) return true;
  if (T.vscene && T.vscene[e0] != T.vscene[f0]) return true;
  const int be = T.vbody[e0];
  if (be >= 0 && be == T.vbody[f0]) return true;
  if (T.vnode[e0] < 0 && T.vnode[e1] < 0 && T.vnode[f0] < 0 && T.vnode[f1] < 0) return true;
  return false;
}

// A lower bound of the squared distance between the primitives of a pair
// (point vs triangle: kind 0, y0 | y1 y2 y3; segment vs segment: kind 1,
// y0 y1 | y2 y3): the squared distance between their axis-aligned boxes.  A
// few FP64 operations instead of the exact classification, which is skipped
// whenever the bound already exceeds what matters (dhat^2, or the CCD step);
// the comparisons keep a 1e-9 relative margin, so every skipped pair is one the
// exact test would also have rejected.
__device__ __forceinline__ double pair_lb2(int kind, d3 y0, d3 y1, d3 y2, d3 y3) {
  const double alo[3] = {kind == 0 ? y0.x : fmin(y0.x, y1.x), kind == 0 ? y0.y : fmin(y0.y, y1.y),
                         kind == 0 ? y0.z : fmin(y0.z, y1.z)};
  const double ahi[3] = {kind == 0 ? y0.x : fmax(y0.x, y1.x), kind == 0 ? y0.y : fmax(y0.y, y1.y),
                         kind == 0 ? y0.z : fmax(y0.z, y1.z)};
  double blo[3] = {fmin(y2.x, y3.x), fmin(y2.y, y3.y), fmin(y2.z, y3.z)};
  double bhi[3] = {fmax(y2.x, y3.x), fmax(y2.y, y3.y), fmax(y2.z, y3.z)};
  if (kind == 0) {
    blo[0] = fmin(blo[0], y1.x); blo[1] = fmin(blo[1], y1.y); blo[2] = fmin(blo[2], y1.z);
    bhi[0] = fmax(bhi[0], y1.x); bhi[1] = fmax(bhi[1], y1.y); bhi[2] = fmax(bhi[2], y1.z);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double g = fmax(fmax(alo[c] - bhi[c], blo[c] - ahi[c]), 0.0);
    s += g * g;
  }
  return s;
}
__device__ __forceinline__ bool surely_apart(double lb2, double sh) { return lb2 > sh * (1.0 + 1e-9); }

// A second conservative test for pairs the box bound keeps: the distance
// between two convex sets is at least their gap along any axis u, and the
// projections of a point, a segment or a triangle are extreme at its
// vertices.  Two axes: the common normal (triangle normal; e1 x e2 for two
// segments) and the direction between the primitives' centres.  The gap is
// formed relative to y0 in FP64 and compared with the same 1e-9 relative
// margin; an axis of zero length is skipped.  Most candidate pairs lie a few
// millimetres apart, beyond dhat, and stop here instead of in the exact
// classification.
__device__ __forceinline__ double sat_lb2(int kind, d3 y0, d3 y1, d3 y2, d3 y3) {
  const d3 a1 = y1 - y0, b0 = y2 - y0, b1 = y3 - y0;  // y0 at the origin
  d3 ax[2];
  if (kind == 0) {  // point y0, triangle y1 y2 y3
    ax[0] = cross(b0 - a1, b1 - a1);
    ax[1] = a1 + b0 + b1;  // three times the centroid
  } else {  // segments y0 y1 and y2 y3
    ax[0] = cross(a1, b1 - b0);
    ax[1] = (b0 + b1) - a1;  // twice the centre difference
  }
  double best = 0.0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const d3 u = ax[k];
    const double n2 = dot(u, u);
    if (!(n2 > 0.0)) continue;
    const double pa0 = 0.0, pa1 = dot(u, a1), pb0 = dot(u, b0), pb1 = dot(u, b1);
    double lo_a, hi_a, lo_b, hi_b;
    if (kind == 0) {  // the point alone on one side, the triangle's three vertices on the other
      lo_a = hi_a = pa0;
      lo_b = fmin(pa1, fmin(pb0, pb1));
      hi_b = fmax(pa1, fmax(pb0, pb1));
    } else {
      lo_a = fmin(pa0, pa1);
      hi_a = fmax(pa0, pa1);
      lo_b = fmin(pb0, pb1);
      hi_b = fmax(pb0, pb1);
    }
    const double gap = fmax(lo_b - hi_a, lo_a - hi_b);
    if (gap > 0.0) best = fmax(best, gap * gap / n2);
  }
  return best;  // a squared lower bound of the distance (0: no axis separates)
}
__device__ __forceinline__ bool sat_apart(int kind, d3 y0, d3 y1, d3 y2, d3 y3, double sh) {
  return surely_apart(sat_lb2(kind, y0, y1, y2, y3), sh);
}

// ---- single-precision prefilters of the candidate kernels
// The tests above run on the FP64 pipe, which bounds the candidate kernels on
// this part.  The candidate kernels therefore first run the same two bounds
// in FP32 on single-precision copies of the vertex arrays (one rounding per
// component), each reduced by a bound on every rounding involved, so that the
// FP32 value never exceeds the exact bound.  A pair the FP32 test rejects is
// one the FP64 test rejects too; only the others take the FP64 path.
constexpr float kU32 = 5.9604645e-8f;  // 2^-24, the FP32 unit roundoff

__device__ __forceinline__ float3 ldf3(const float4* p, int i) {
  const float4 v = p[i];
  return make_float3(v.x, v.y, v.z);
}
__device__ __forceinline__ float3 f3sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float f3dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 f3cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float f3amax(float3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }
__device__ __forceinline__ float f3l1(float3 a) { return fabsf(a.x) + fabsf(a.y) + fabsf(a.z); }

// FP32 copy of a 3-per-vertex FP64 array, 16 bytes per vertex
__global__ void k_f32_copy(int n, const double* __restrict__ a, float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float4((float)a[3 * i], (float)a[3 * i + 1], (float)a[3 * i + 2], 0.0f);
}

// A lower bound of the squared distance of a pair (kind and vertex order as
// in pair_lb2) from the FP32 copies y of its vertices, valid for the exact
// FP64 positions: the larger of the box bound and the separating-axis bound.
// Every copied component is within u |y| of the exact one (u = 2^-24); the
// box gaps lose that twice and one rounding of the subtraction; a projection
// onto an axis a (any axis gives a valid bound, so a's own rounding does not
// matter) is off by at most |a|_1 (2u X + u A) for the differences plus
// 3u |a|_1 A for the dot product, where X bounds the coordinates and A the
// differences; both bounds are taken twice over.  The result never exceeds
// the exact bound.
__device__ __forceinline__ float lb2_f32(int kind, float3 y0, float3 y1, float3 y2, float3 y3) {
  const float u = kU32;
  const float X = fmaxf(fmaxf(f3amax(y0), f3amax(y1)), fmaxf(f3amax(y2), f3amax(y3)));
  const float dl = 2.0f * u * X;
  float alo[3], ahi[3], blo[3], bhi[3];
  const float a0[3] = {y0.x, y0.y, y0.z}, a1v[3] = {y1.x, y1.y, y1.z}, b0v[3] = {y2.x, y2.y, y2.z},
              b1v[3] = {y3.x, y3.y, y3.z};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (kind == 0) {
      alo[c] = ahi[c] = a0[c];
      blo[c] = fminf(a1v[c], fminf(b0v[c], b1v[c]));
      bhi[c] = fmaxf(a1v[c], fmaxf(b0v[c], b1v[c]));
    } else {
      alo[c] = fminf(a0[c], a1v[c]);
      ahi[c] = fmaxf(a0[c], a1v[c]);
      blo[c] = fminf(b0v[c], b1v[c]);
      bhi[c] = fmaxf(b0v[c], b1v[c]);
    }
  }
  float sb = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float g = fmaxf(alo[c] - bhi[c], blo[c] - ahi[c]);
    g = g * (1.0f - 2.0f * u) - 2.0f * dl;
    if (g > 0.0f) sb += g * g;
  }
  float best = sb * (1.0f - 8.0f * u);
  const float3 a1 = f3sub(y1, y0), b0 = f3sub(y2, y0), b1 = f3sub(y3, y0);
  const float A = fmaxf(f3amax(a1), fmaxf(f3amax(b0), f3amax(b1)));
  float3 ax[2];
  if (kind == 0) {
    ax[0] = f3cross(f3sub(b0, a1), f3sub(b1, a1));
    ax[1] = make_float3(a1.x + b0.x + b1.x, a1.y + b0.y + b1.y, a1.z + b0.z + b1.z);
  } else {
    ax[0] = f3cross(a1, f3sub(b1, b0));
    ax[1] = make_float3(b0.x + b1.x - a1.x, b0.y + b1.y - a1.y, b0.z + b1.z - a1.z);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float3 w = ax[k];
    const float n2 = f3dot(w, w);
    if (!(n2 > 1e-30f)) continue;  // keeps the products out of the subnormal range
    const float pa1 = f3dot(w, a1), pb0 = f3dot(w, b0), pb1 = f3dot(w, b1);
    float lo_a, hi_a, lo_b, hi_b;
    if (kind == 0) {
      lo_a = hi_a = 0.0f;
      lo_b = fminf(pa1, fminf(pb0, pb1));
      hi_b = fmaxf(pa1, fmaxf(pb0, pb1));
    } else {
      lo_a = fminf(0.0f, pa1);
      hi_a = fmaxf(0.0f, pa1);
      lo_b = fminf(pb0, pb1);
      hi_b = fmaxf(pb0, pb1);
    }
    const float E = f3l1(w) * (4.0f * u * X + 8.0f * u * A);
    const float g = fmaxf(lo_b - hi_a, lo_a - hi_b) * (1.0f - 2.0f * u) - 2.0f * E;
    if (g > 0.0f) best = fmaxf(best, (g * g) / (n2 * (1.0f + 8.0f * u)) * (1.0f - 4.0f * u));
  }
  return best;
}
__device__ __forceinline__ float lb2_f32(int kind, const float4* pf, const int* ids) {
  return lb2_f32(kind, ldf3(pf, ids[0]), ldf3(pf, ids[1]), ldf3(pf, ids[2]), ldf3(pf, ids[3]));
}
// An upper bound of max_k |dx_k - m| (m the mean of the exact dx_k) from the
// FP32 copies d_k: the copies, the mean and the differences add at most
// 7 u Dm per component (Dm bounds the components), taken twice over.
__device__ __forceinline__ float motion_hi_f32(const float3* d) {
  const float u = kU32;
  float Dm = 0.0f;
  float3 m = make_float3(0.0f, 0.0f, 0.0f);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    Dm = fmaxf(Dm, f3amax(d[i]));
    m.x += 0.25f * d[i].x; m.y += 0.25f * d[i].y; m.z += 0.25f * d[i].z;
  }
  float mx2 = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float3 c = f3sub(d[i], m);
    mx2 = fmaxf(mx2, f3dot(c, c));
  }
  return sqrtf(mx2) * (1.0f + 8.0f * u) + 1.7320508f * 16.0f * u * Dm;
}

// ---------------------------------------------------------------- barrier scalar
struct bder {
  double b, db, d2b;
};
__host__ __device__ __forceinline__ bder barrier_fn(double s, double sh, int form) {
  if (!(s < sh)) return {0.0, 0.0, 0.0};
  const double d = s - sh, L = log(s / sh);
  if (form == 1)
    return {d * d * L * L, 2.0 * d * L * L + 2.0 * d * d * L / s,
            2.0 * L * L + 8.0 * d * L / s + 2.0 * d * d / (s * s) - 2.0 * d * d * L / (s * s)};
  return {-d * d * L, -2.0 * d * L - d * d / s, -2.0 * L - 4.0 * d / s + d * d / (s * s)};
}

// ---------------------------------------------------------------- detection
// mode 0: count, mode 1: write + sort segment, mode 2: accumulate kappa * b(s)
__global__ void k_pt_query(int total, int nsv, topo T, const double* __restrict__ P, const float4* __restrict__ Pf,
                           grid_dev g, boxes A, double sh, int mode, int* __restrict__ cnt,
                           const int* __restrict__ off, int* __restrict__ out, double kappa, int form,
                           ksum* __restrict__ part) {
  const float shf = (float)sh * (1.0f + 1e-6f);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  ksum acc{0.0, 0.0};
  if (i < nsv) {
    const int v = T.svert[i];
    const d3 p = ld3(P, v);
    int c = 0;
    const int base = (mode == 1) ? off[i] : 0;
    const int lim = (mode == 1) ? ((i + 1 < nsv) ? off[i + 1] : total) : 0;
    grid_visit(g, A, i, [&](int t) {
      const int t0 = T.stri[3 * t], t1 = T.stri[3 * t + 1], t2 = T.stri[3 * t + 2];
      if (pt_excluded(T, v, t0, t1, t2)) return;
      const int ids[4] = {v, t0, t1, t2};
      if (Pf && lb2_f32(0, Pf, ids) > shf) return;  // FP32 prefilter
      const d3 q0 = ld3(P, t0), q1 = ld3(P, t1), q2 = ld3(P, t2);
      if (surely_apart(pair_lb2(0, p, q0, q1, q2), sh) || sat_apart(0, p, q0, q1, q2, sh)) return;
      double s;
      const int st = dist::pt_classify(p, q0, q1, q2, &s);
      if (!(s < sh)) return;
      if (mode == 1) {
        if (base + c >= lim) { dev_flag(T.status, DEV_CAPACITY); return; }
        int* o = out + 3 * (size_t)(base + c);
        o[0] = v; o[1] = t; o[2] = st;
      } else if (mode == 2) {
        kadd(acc, kappa * barrier_fn(s, sh, form).b);
      }
      ++c;
    });
    if (mode == 0) cnt[i] = c;
    if (mode == 1) {  // insertion sort of this vertex's partners by triangle id
      c = min(c, lim - base);
      int* o = out + 3 * (size_t)base;
      for (int a = 1; a < c; ++a) {
        const int kb = o[3 * a + 1], ks = o[3 * a + 2];
        int q = a - 1;
        while (q >= 0 && o[3 * q + 1] > kb) {
          o[3 * (q + 1) + 1] = o[3 * q + 1];
          o[3 * (q + 1) + 2] = o[3 * q + 2];
          --q;
        }
        o[3 * (q + 1) + 1] = kb;
        o[3 * (q + 1) + 2] = ks;
      }
    }
  }
  if (mode == 2) {
    acc = block_ksum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
  }
}

__global__ void k_ee_query(int total, int nse, topo T, const double* __restrict__ P, const float4* __restrict__ Pf,
                           grid_dev g, boxes A, double sh, int mode, int* __restrict__ cnt,
                           const int* __restrict__ off, int* __restrict__ out, double kappa, int form,
                           ksum* __restrict__ part) {
  const float shf = (float)sh * (1.0f + 1e-6f);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  ksum acc{0.0, 0.0};
  if (i < nse) {
    const int e0 = T.sedge[2 * i], e1 = T.sedge[2 * i + 1];
    const d3 a0 = ld3(P, e0), a1 = ld3(P, e1);
    int c = 0;
    const int base = (mode == 1) ? off[i] : 0;
    const int lim = (mode == 1) ? ((i + 1 < nse) ? off[i + 1] : total) : 0;
    grid_visit(g, A, i, [&](int j) {
      if (j <= i) return;
      const int f0 = T.sedge[2 * j], f1 = T.sedge[2 * j + 1];
      if (ee_excluded(T, e0, e1, f0, f1)) return;
      const int ids[4] = {e0, e1, f0, f1};
      if (Pf && lb2_f32(1, Pf, ids) > shf) return;  // FP32 prefilter
      const d3 b0 = ld3(P, f0), b1 = ld3(P, f1);
      if (surely_apart(pair_lb2(1, a0, a1, b0, b1), sh) || sat_apart(1, a0, a1, b0, b1, sh)) return;
      double s;
      const int st = dist::ee_classify(a0, a1, b0, b1, &s);
      if (!(s < sh)) return;
      if (mode == 1) {
        if (base + c >= lim) { dev_flag(T.status, DEV_CAPACITY); return; }
        int* o = out + 3 * (size_t)(base + c);
        o[0] = i; o[1] = j; o[2] = st;
      } else if (mode == 2) {
        kadd(acc, kappa * barrier_fn(s, sh, form).b);
      }
      ++c;
    }, true);
    if (mode == 0) cnt[i] = c;
    if (mode == 1) {
      c = min(c, lim - base);
      int* o = out + 3 * (size_t)base;
      for (int a = 1; a < c; ++a) {
        const int kb = o[3 * a + 1], ks = o[3 * a + 2];
        int q = a - 1;
        while (q >= 0 && o[3 * q + 1] > kb) {
          o[3 * (q + 1) + 1] = o[3 * q + 1];
          o[3 * (q + 1) + 2] = o[3 * q + 2];
          --q;
        }
        o[3 * (q + 1) + 1] = kb;
        o[3 * (q + 1) + 2] = ks;
      }
    }
  }
  if (mode == 2) {
    acc = block_ksum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
  }
}

// point-plane pairs: d = n.p - c, active when d > 0 and d^2 < dhat^2
__global__ void k_pg_query(int total, int nsv, int npl, topo T, const double* __restrict__ P, const double* __restrict__ planes,
                           double sh, int mode, int* __restrict__ cnt, const int* __restrict__ off,
                           int* __restrict__ out, double kappa, int form, ksum* __restrict__ part,
                           double* __restrict__ sacc = nullptr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  ksum acc{0.0, 0.0};
  int key = -1;
  if (i < nsv && sacc) key = T.vscene[T.svert[i]];
  if (i < nsv) {
    const int v = T.svert[i];
    int c = 0;
    if (T.vnode[v] >= 0) {
      const d3 p = ld3(P, v);
      for (int k = 0; k < npl; ++k) {
        const double* pl = planes + 4 * k;
        const double d = dist::sub(dist::vdot(d3{pl[0], pl[1], pl[2]}, p), pl[3]);
        const double s = dist::mul(d, d);
        if (!(d > 0.0 && s < sh)) continue;
        if (mode == 1) {
          const int lim = (i + 1 < nsv) ? off[i + 1] : total;
          if (off[i] + c >= lim) { dev_flag(T.status, DEV_CAPACITY); break; }
          int* o = out + 3 * (size_t)(off[i] + c);
          o[0] = v; o[1] = k; o[2] = 0;
        } else if (mode == 2) {
          kadd(acc, kappa * barrier_fn(s, sh, form).b);
        }
        ++c;
      }
    }
    if (mode == 0) cnt[i] = c;
  }
  if (mode == 2) {
    if (sacc) {  // batches: per scene (surface vertices are sorted, so are their scenes)
      seg_add_global(sacc, key, acc.s + acc.c);
    } else {
      acc = block_ksum(acc);
      if (threadIdx.x == 0) part[blockIdx.x] = acc;
    }
  }
}

// ---------------------------------------------------------------- pair node sets
// Nodes and weights of a vertex through its UNION branch (App. A index rules):
// The UNION map of a vertex: the nodes its position depends on and the
// weights (its Jacobian is w_k I3 per node).  Free -> 1 node (w = 1); affine
// -> 4 nodes (t, A1, A2, A3; w = 1, r1, r2, r3); cage-embedded -> the 8 nodes
// of its cage cell (trilinear weights); fixed -> none.
constexpr int kMaxVertNodes = 8;
constexpr int kMaxPairNodes = 4 * kMaxVertNodes;  // before merging
struct vmapd {
  int n;
  int node[kMaxVertNodes];
  double w[kMaxVertNodes];
};
__device__ __forceinline__ vmapd vertex_map(int v, const topo& T, const double* vr) {
  vmapd m;
  const int n = T.vnode[v];
  if (n < 0) { m.n = 0; return m; }
  const int b = T.vbody[v];
  if (b == -1) { m.n = 1; m.node[0] = n; m.w[0] = 1.0; return m; }
  if (b <= -2) {
    const int e = -2 - b;
    m.n = 8;
    for (int k = 0; k < 8; ++k) { m.node[k] = T.enode[8 * e + k]; m.w[k] = T.ew[8 * e + k]; }
    return m;
  }
  m.n = 4;
  for (int k = 0; k < 4; ++k) m.node[k] = n + k;
  m.w[0] = 1.0; m.w[1] = vr[3 * v]; m.w[2] = vr[3 * v + 1]; m.w[3] = vr[3 * v + 2];
  return m;
}

// sorted unique node list of up to 4 vertices (<= 32 before merging)
struct nodeset {
  int m;
  int node[kMaxPairNodes];
};
__device__ __forceinline__ nodeset pair_nodes(const int* ids, int k, const topo& T, const double* vr) {
  nodeset S;
  S.m = 0;
  for (int a = 0; a < k; ++a) {
    const vmapd vm = vertex_map(ids[a], T, vr);
    for (int q = 0; q < vm.n; ++q) {
      const int nd = vm.node[q];
      int pos = 0;
      bool dup = false;
      for (; pos < S.m; ++pos) {
        if (S.node[pos] == nd) { dup = true; break; }
        if (S.node[pos] > nd) break;
      }
      if (dup) continue;
      for (int r = S.m; r > pos; --r) S.node[r] = S.node[r - 1];
      S.node[pos] = nd;
      ++S.m;
    }
  }
  return S;
}
// index of key (u < w) in the lexicographic enumeration of pairs of m items
__device__ __forceinline__ int pair_rank(int u, int w, int m) { return u * (2 * m - u - 1) / 2 + (w - u - 1); }

__device__ __forceinline__ void pair_vertices(int kind, int pidx, const int* pairs, const topo& T, int* ids, int* k) {
  const int* pr = pairs + 3 * (size_t)pidx;
  if (kind == 0) {
    ids[0] = pr[0];
    ids[1] = T.stri[3 * pr[1]]; ids[2] = T.stri[3 * pr[1] + 1]; ids[3] = T.stri[3 * pr[1] + 2];
    *k = 4;
  } else if (kind == 1) {
    ids[0] = T.sedge[2 * pr[0]]; ids[1] = T.sedge[2 * pr[0] + 1];
    ids[2] = T.sedge[2 * pr[1]]; ids[3] = T.sedge[2 * pr[1] + 1];
    *k = 4;
  } else {
    ids[0] = pr[0];
    *k = 1;
  }
}

// number of upper off-diagonal keys per pair; pairs are PT, then EE, then PG
__global__ void k_pair_nkeys(int npt, int nee, int npg, const int* __restrict__ pt, const int* __restrict__ ee,
                             const int* __restrict__ pg, topo T, const double* __restrict__ vr, int* __restrict__ nk) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npt + nee + npg) return;
  const int kind = p < npt ? 0 : (p < npt + nee ? 1 : 2);
  const int li = p - (kind == 0 ? 0 : (kind == 1 ? npt : npt + nee));
  int ids[4], k;
  pair_vertices(kind, li, kind == 0 ? pt : (kind == 1 ? ee : pg), T, ids, &k);
  const nodeset S = pair_nodes(ids, k, T, vr);
  nk[p] = S.m * (S.m - 1) / 2;
}
__global__ void k_pair_keys(int npt, int nee, int npg, const int* __restrict__ pt, const int* __restrict__ ee,
                            const int* __restrict__ pg, topo T, const double* __restrict__ vr,
                            const int* __restrict__ koff, int nbits, uint64_t* __restrict__ keys, int* __restrict__ vals) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npt + nee + npg) return;
  const int kind = p < npt ? 0 : (p < npt + nee ? 1 : 2);
  const int li = p - (kind == 0 ? 0 : (kind == 1 ? npt : npt + nee));
  int ids[4], k;
  pair_vertices(kind, li, kind == 0 ? pt : (kind == 1 ? ee : pg), T, ids, &k);
  const nodeset S = pair_nodes(ids, k, T, vr);
  int o = koff[p];
  for (int u = 0; u < S.m; ++u)
    for (int w = u + 1; w < S.m; ++w) {
      keys[o] = ((uint64_t)S.node[u] << nbits) | (uint64_t)S.node[w];
      vals[o] = o;
      ++o;
    }
}

// ---------------------------------------------------------------- barrier evaluation
template <int N, typename T>
__device__ __forceinline__ void project_n(T* H) {
  project_psd<N, T>(H);
}

// PT / EE barrier pairs (kind 0 = PT, 1 = EE) in two passes.
//
// k_barrier_prep, one thread per pair: the exact FP64 classification (closest
// feature), the squared distance and the barrier derivatives b'(s), b''(s).
// FP64 is scarce on this part and a warp instruction costs about the same
// FP64 pipe time with one active lane as with 32, so this scalar work runs 32
// pairs per warp instruction instead of on one lane of a warp per pair.
//
// k_barrier_pair, one warp per pair: every distance type is written in
// reduced variables z = C y (PP: w = p - a; PE: w = p - a, e = b - a; PT and
// EE: (w, e1, e2) as in the distance functions), C = coef (x) I3 with k = 1,
// 2, 3 rows of small integers over the n = k + 1 classified vertices.  The
// position-space Hessian is C^T H_z C with H_z = kappa (b'' g_z g_z^T + b'
// d2s/dz2) (R x R, R = 3k).  With C C^T = L L^T (L = chol(coef coef^T) (x) I3)
// the rows of Q = L^-1 C are orthonormal, C = L Q, and
//   Project(C^T H_z C) = Q^T Project(L^T H_z L) Q
// exactly: a Jacobi solve on R = 3, 6, 9 instead of 6, 9, 12, and no
// position-space Hessian is formed before the projection.  The gradient stays
// FP64 (g_y = C^T g_z); in the FP32-mixed form the R x R Hessians, the
// projection and the product are FP32.  The result is then mapped through the
// UNION weights of the pair's vertices, duplicate nodes merged, and scattered.
template <typename T>
struct bar_ws {
  double gz[9];    // ds/dz
  T gzf[9];        // the same in T
  T Hz[81];        // kappa (b'' gz gz^T + b' d2s/dz2), then K = L^T Hz L, then Project(K)
  T V[81];         // Jacobi rotations
  T Hy[144];       // Q^T Project(K) Q (n3 x n3)
  T cs[5], sn[5];
  double W[4][kMaxPairNodes];
  int node[kMaxPairNodes];
  int m;
};

// reduced-coordinate constants per distance type (PP, PE, PT, EE): coef (k x
// n), L = chol(coef coef^T) (k x k, lower) and Q = L^-1 coef (k x n)
struct bar_tables {
  double coef[4][3][4];
  double L[4][3][3];
  double Q[4][3][4];
  float Lf[4][3][3];
  float Qf[4][3][4];
  int k[4];
};
__device__ __forceinline__ double tab_L(const bar_tables& t, double, int d, int r, int a) { return t.L[d][r][a]; }
__device__ __forceinline__ float tab_L(const bar_tables& t, float, int d, int r, int a) { return t.Lf[d][r][a]; }
__device__ __forceinline__ double tab_Q(const bar_tables& t, double, int d, int r, int v) { return t.Q[d][r][v]; }
__device__ __forceinline__ float tab_Q(const bar_tables& t, float, int d, int r, int v) { return t.Qf[d][r][v]; }

// Project(A) = V max(Lambda, 0) V^T for the N x N symmetric A in shared
// memory (row-major), by one warp: cyclic Jacobi with N/2 disjoint rotations
// per step in the round-robin order (N - 1 steps per sweep), the same rotation
// formula and stopping rule as project_psd; then the product, upper triangle
// first, mirrored.  N is a compile-time size (6, 9, 12: PP, PE, PT/EE), so the
// index arithmetic of the sweeps is constant divisions.
template <typename T, int N>
__device__ void warp_project(T* A, T* V, T* cs, T* sn, int lane) {
  constexpr int NP = N + (N & 1);  // even count for the round-robin (index N is a dummy when N is odd)
  constexpr int M = NP / 2;
  for (int e = lane; e < N * N; e += 32) V[e] = (e / N == e % N) ? T(1) : T(0);
  __syncwarp();
  // the pair (a, b), a < b, of rotation i in step st
  auto rot = [](int st, int i, int& pp, int& qq) {
    const int a = (i == 0) ? 0 : 1 + (st + i) % (NP - 1);
    const int b = (i == 0) ? 1 + st : 1 + (st - i + NP - 1) % (NP - 1);
    pp = min(a, b);
    qq = max(a, b);
  };
  for (int sweep = 0; sweep < eig_traits<T>::max_sweeps; ++sweep) {
    T off = 0, tot = 0;
    for (int e = lane; e < N * N; e += 32) {
      const int r = e / N, c = e % N;
      const T a = A[e];
      if (r == c) tot += a * a;
      else if (r < c) off += a * a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    tot += T(2) * off;
    if (!(off > eig_traits<T>::rel_eps2 * tot)) break;
    for (int st = 0; st < NP - 1; ++st) {
      if (lane < M) {
        int pp, qq;
        rot(st, lane, pp, qq);
        T c = 1, sg = 0;
        if (qq < N) {
          const T apq = A[pp * N + qq];
          if (apq != T(0)) {
            const T theta = (A[qq * N + qq] - A[pp * N + pp]) / (T(2) * apq);
            const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
            c = jacobi_c(t);
            sg = t * c;
          }
        }
        cs[lane] = c;
        sn[lane] = sg;
      }
      __syncwarp();
      // columns of A and V: A <- A J, V <- V J
      for (int e = lane; e < M * N; e += 32) {
        const int i = e / N, k = e % N;
        int pp, qq;
        rot(st, i, pp, qq);
        const T c = cs[i], sg = sn[i];
        if (qq >= N || sg == T(0)) continue;
        const T akp = A[k * N + pp], akq = A[k * N + qq];
        A[k * N + pp] = c * akp - sg * akq;
        A[k * N + qq] = sg * akp + c * akq;
        const T vkp = V[k * N + pp], vkq = V[k * N + qq];
        V[k * N + pp] = c * vkp - sg * vkq;
        V[k * N + qq] = sg * vkp + c * vkq;
      }
      __syncwarp();
      // rows of A: A <- J^T A
      for (int e = lane; e < M * N; e += 32) {
        const int i = e / N, k = e % N;
        int pp, qq;
        rot(st, i, pp, qq);
        const T c = cs[i], sg = sn[i];
        if (qq >= N || sg == T(0)) continue;
        const T apk = A[pp * N + k], aqk = A[qq * N + k];
        A[pp * N + k] = c * apk - sg * aqk;
        A[qq * N + k] = sg * apk + c * aqk;
      }
      __syncwarp();
    }
  }
  T lam[N];
#pragma unroll
  for (int k = 0; k < N; ++k) lam[k] = (A[k * N + k] > T(0)) ? A[k * N + k] : T(0);
  __syncwarp();
  constexpr int NO = (N * N + 31) / 32;  // entries a lane visits (upper ones kept)
  T outv[NO];
  int oute[NO];
  int no = 0;
  for (int e = lane; e < N * N; e += 32) {
    const int r = e / N, c = e % N;
    if (r > c) continue;
    T acc = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) acc += V[r * N + k] * lam[k] * V[c * N + k];
    outv[no] = acc;
    oute[no] = e;
    ++no;
  }
  __syncwarp();
  for (int q = 0; q < no; ++q) {
    const int e = oute[q], r = e / N, c = e % N;
    A[r * N + c] = outv[q];
    A[c * N + r] = outv[q];
  }
  __syncwarp();
}

// one thread per PT / EE pair: info[p] = active | dtype << 1 | loc0 << 3 | loc1
// << 5 | loc2 << 7 | loc3 << 9 (loc: the classified vertices among the pair's
// four), bd[p] = (b'(s), b''(s)).  Pairs are PT then EE (kind by index).
__global__ void k_barrier_prep(int npt, int nee, const int* __restrict__ pt, const int* __restrict__ ee, topo Tp,
                               const double* __restrict__ P, double sh, int form, int* __restrict__ info,
                               double2* __restrict__ bd) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npt + nee) return;
  const int kind = p < npt ? 0 : 1;
  int ids[4], k;
  pair_vertices(kind, kind == 0 ? p : p - npt, kind == 0 ? pt : ee, Tp, ids, &k);
  d3 y[4];
  for (int a = 0; a < 4; ++a) y[a] = ld3(P, ids[a]);
  double sd;
  dist::dclass dc;
  if (kind == 0) dc = dist::pt_dclass(dist::pt_classify(y[0], y[1], y[2], y[3], &sd));
  else dc = dist::ee_dclass(dist::ee_classify(y[0], y[1], y[2], y[3], &sd));
  const bool active = (sd < sh) && (sd > 0.0);
  int code = active ? 1 : 0;
  code |= dc.dtype << 1;
  for (int q = 0; q < 4; ++q) code |= (q < dc.n ? dc.loc[q] : 0) << (3 + 2 * q);
  info[p] = code;
  if (active) {
    const bder b = barrier_fn(sd, sh, form);
    bd[p] = make_double2(b.db, b.d2b);
  }
}

// ds/dz and d2s/dz2 (times kappa b', plus kappa b'' gz gz^T) of one pair in its
// reduced variables z, by the lanes of one warp; gz (FP64) and Hz (T) in
// shared memory.  z: PP w (3); PE (w, e) (6); PT / EE (w, e1, e2) (9).
template <typename T>
__device__ void bar_reduced(int dtype, const d3* yl, double kappa, double db, double d2b, bar_ws<T>& w, int lane) {
  using dist::comp;
  if (dtype == dist::PP) {
    const d3 wv = yl[0] - yl[1];
    if (lane < 3) {
      w.gz[lane] = 2.0 * comp(wv, lane);
      w.gzf[lane] = (T)w.gz[lane];
    }
    __syncwarp();
    if (lane < 9) {
      const int i = lane / 3, j = lane % 3;
      w.Hz[lane] = (T)kappa * ((T)d2b * w.gzf[i] * w.gzf[j] + (T)db * ((i == j) ? T(2) : T(0)));
    }
  } else if (dtype == dist::PE) {
    // s = |w|^2 - (w.e)^2 / |e|^2
    const d3 wv = yl[0] - yl[1], ev = yl[2] - yl[1];
    const double u = dot(wv, ev), L = dot(ev, ev), iLd = 1.0 / L;
    if (lane < 3) w.gz[lane] = 2.0 * comp(wv, lane) - 2.0 * u * comp(ev, lane) * iLd;
    else if (lane < 6) {
      const int i = lane - 3;
      w.gz[lane] = -2.0 * u * comp(wv, i) * iLd + 2.0 * u * u * comp(ev, i) * iLd * iLd;
    }
    if (lane < 6) w.gzf[lane] = (T)w.gz[lane];
    __syncwarp();
    // blocks (w,w), (w,e), (e,w), (e,e) of the 6 x 6 Hessian, in T
    const T uf = (T)u, iL = (T)iLd;
    for (int e = lane; e < 36; e += 32) {
      const int r = e / 6, c = e % 6, i = r % 3, j = c % 3;
      const T wi = (T)comp(wv, i), wj = (T)comp(wv, j), ei = (T)comp(ev, i), ej = (T)comp(ev, j);
      const T d = (i == j) ? T(1) : T(0);
      T h;
      if (r < 3 && c < 3) h = T(2) * d - T(2) * ei * ej * iL;
      else if (r < 3) h = -T(2) * ei * wj * iL - T(2) * uf * d * iL + T(4) * uf * ei * ej * iL * iL;
      else if (c < 3) h = -T(2) * ej * wi * iL - T(2) * uf * d * iL + T(4) * uf * ej * ei * iL * iL;
      else
        h = -T(2) * wi * wj * iL + T(4) * uf * (wi * ej + ei * wj) * iL * iL + T(2) * uf * uf * d * iL * iL -
            T(8) * uf * uf * ei * ej * iL * iL * iL;
      w.Hz[e] = (T)kappa * ((T)d2b * w.gzf[r] * w.gzf[c] + (T)db * h);
    }
  } else {
    // s = (w.n)^2 / (n.n), n = e1 x e2
    d3 wv, e1v, e2v;
    if (dtype == dist::PT) {
      wv = yl[0] - yl[1]; e1v = yl[2] - yl[1]; e2v = yl[3] - yl[1];
    } else {
      wv = yl[0] - yl[2]; e1v = yl[1] - yl[0]; e2v = yl[3] - yl[2];
    }
    const d3 nv = cross(e1v, e2v);
    const double t = dot(wv, nv), N = dot(nv, nv), iNd = 1.0 / N;
    // gradient (FP64): lanes 0-2 dw, 3-8 de1, de2 through dn/de = [-[e2]x, [e1]x]
    if (lane < 9) {
      double g;
      if (lane < 3) g = 2.0 * t * comp(nv, lane) * iNd;
      else {
        const int c = lane - 3;
        g = 0.0;
        for (int q = 0; q < 3; ++q)
          g += (2.0 * t * comp(wv, q) * iNd - 2.0 * t * t * comp(nv, q) * iNd * iNd) * dist::jn(e1v, e2v, q, c);
      }
      w.gz[lane] = g;
      w.gzf[lane] = (T)g;
    }
    __syncwarp();
    // Hessian entries in T from T copies of the FP64 vectors and scalars
    const T tf = (T)t, iN = (T)iNd;
    const T wf[3] = {(T)wv.x, (T)wv.y, (T)wv.z}, nf[3] = {(T)nv.x, (T)nv.y, (T)nv.z};
    const T e1f[3] = {(T)e1v.x, (T)e1v.y, (T)e1v.z}, e2f[3] = {(T)e2v.x, (T)e2v.y, (T)e2v.z};
    // entry (q, c) of Jn = dn/d(e1, e2) (3 x 6)
    auto jnf = [&](int q, int c) -> T {
      const T* e = (c < 3) ? e2f : e1f;
      const T sg = (c < 3) ? T(-1) : T(1);
      const int a = c % 3;
      if (q == a) return T(0);
      const int b = 3 - q - a;
      const T eps = ((q + 1) % 3 == a) ? T(1) : T(-1);
      return sg * (-eps) * e[b];
    };
    auto hwn = [&](int i, int j) -> T {
      return T(2) * (nf[i] * wf[j] + (i == j ? tf : T(0))) * iN - T(4) * tf * nf[i] * nf[j] * iN * iN;
    };
    auto hnn = [&](int i, int j) -> T {
      return T(2) * wf[i] * wf[j] * iN - T(4) * tf * (wf[i] * nf[j] + nf[i] * wf[j]) * iN * iN -
             (i == j ? T(2) * tf * tf * iN * iN : T(0)) + T(8) * tf * tf * nf[i] * nf[j] * iN * iN * iN;
    };
    for (int e = lane; e < 81; e += 32) {
      const int r = e / 9, c = e % 9;
      T h;
      if (r < 3 && c < 3) {
        h = T(2) * nf[r] * nf[c] * iN;
      } else if (r < 3 || c < 3) {
        const int i = r < 3 ? r : c, cc = (r < 3 ? c : r) - 3;
        h = hwn(i, 0) * jnf(0, cc) + hwn(i, 1) * jnf(1, cc) + hwn(i, 2) * jnf(2, cc);
      } else {
        const int rr = r - 3, cc = c - 3;
        T t3[3];
        for (int q = 0; q < 3; ++q) t3[q] = hnn(q, 0) * jnf(0, cc) + hnn(q, 1) * jnf(1, cc) + hnn(q, 2) * jnf(2, cc);
        h = jnf(0, rr) * t3[0] + jnf(1, rr) * t3[1] + jnf(2, rr) * t3[2];
        // curvature of n: the (e1, e2) block and its transpose, sum_k gn_k eps_kij
        const int i = rr < 3 ? rr : cc, j = rr < 3 ? cc - 3 : rr - 3;
        if ((rr < 3) != (cc < 3) && i != j) {
          const int kk = 3 - i - j;
          const T gn = T(2) * tf * wf[kk] * iN - T(2) * tf * tf * nf[kk] * iN * iN;
          h += gn * (((i + 1) % 3 == j) ? T(1) : T(-1));
        }
      }
      w.Hz[e] = (T)kappa * ((T)d2b * w.gzf[r] * w.gzf[c] + (T)db * h);
    }
  }
  __syncwarp();
}

// STAGE 0: the whole pair in one pass (the warp projects K itself when
// `project`); STAGE 1: up to K = L^T Hz L, which goes to kbuf[p] (R x R) with
// g_z to gzbuf[p]; STAGE 2: K (projected by k_project_pairs) and g_z back from
// there, then the position-space blocks, the gradient and the scatter.
template <typename T, int STAGE>
__global__ void __launch_bounds__(128) k_barrier_pair(int npairs, int npt, const int* __restrict__ pt,
                                                       const int* __restrict__ ee, topo Tp,
                                                       const double* __restrict__ vr, const double* __restrict__ P,
                                                       const int* __restrict__ info, const double2* __restrict__ bd,
                                                       double kappa, int project, bar_tables tb,
                                                       const int* __restrict__ koff, const int* __restrict__ dslot,
                                                       double* __restrict__ g, T* __restrict__ diag,
                                                       T* __restrict__ vals, int* status, T* __restrict__ kbuf,
                                                       double* __restrict__ gzbuf) {
  __shared__ bar_ws<T> wsp[4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int p = blockIdx.x * 4 + wid;
  if (p >= npairs) return;  // warp-uniform
  const int code = info[p];
  if (!(code & 1)) return;  // warp-uniform: not within dhat
  bar_ws<T>& w = wsp[wid];
  const int dtype = (code >> 1) & 3;
  const int kind = p < npt ? 0 : 1;
  int ids[4], kv;
  pair_vertices(kind, kind == 0 ? p : p - npt, kind == 0 ? pt : ee, Tp, ids, &kv);
  const int nloc = (dtype == dist::PP) ? 2 : (dtype == dist::PE ? 3 : 4);
  int loc[4];
  d3 yl[4];
  for (int q = 0; q < 4; ++q) {
    loc[q] = (code >> (3 + 2 * q)) & 3;
    if (STAGE != 2) yl[q] = ld3(P, ids[loc[q]]);
  }
  const double2 b2 = bd[p];
  const int k = tb.k[dtype], R = 3 * k, n3 = 3 * nloc;
  if (STAGE != 2) {
    bar_reduced<T>(dtype, yl, kappa, b2.x, b2.y, w, lane);
    // K = L^T Hz L (R x R), into V as scratch, then back into Hz
    for (int e = lane; e < R * R; e += 32) {
      const int ra = e / R, ca = e % R, a = ra / 3, i = ra % 3, b = ca / 3, j = ca % 3;
      T acc = 0;
      for (int r = a; r < k; ++r)
        for (int q = b; q < k; ++q) acc += tab_L(tb, T(), dtype, r, a) * tab_L(tb, T(), dtype, q, b) * w.Hz[R * (3 * r + i) + 3 * q + j];
      w.V[e] = acc;
    }
    __syncwarp();
    if constexpr (STAGE == 1) {
      for (int e = lane; e < R * R; e += 32) kbuf[81 * (size_t)p + e] = w.V[e];
      if (lane < R) gzbuf[9 * (size_t)p + lane] = w.gz[lane];
      return;
    } else {
      for (int e = lane; e < R * R; e += 32) w.Hz[e] = w.V[e];
      __syncwarp();
      if (project) {
        if (R == 9) warp_project<T, 9>(w.Hz, w.V, w.cs, w.sn, lane);
        else if (R == 6) warp_project<T, 6>(w.Hz, w.V, w.cs, w.sn, lane);
        else warp_project<T, 3>(w.Hz, w.V, w.cs, w.sn, lane);
      }
    }
  } else {
    for (int e = lane; e < R * R; e += 32) w.Hz[e] = kbuf[81 * (size_t)p + e];
    if (lane < R) w.gz[lane] = gzbuf[9 * (size_t)p + lane];
  }
  // merged node set and the UNION weights of the classified vertices (integer
  // work and loads; lane 0)
  if (lane == 0) {
    const nodeset S = pair_nodes(ids, kv, Tp, vr);
    w.m = S.m;
    for (int u = 0; u < S.m; ++u) w.node[u] = S.node[u];
    for (int q = 0; q < nloc; ++q) {
      for (int u = 0; u < S.m; ++u) w.W[q][u] = 0.0;
      const vmapd vm = vertex_map(ids[loc[q]], Tp, vr);
      for (int a = 0; a < vm.n; ++a) {
        int u = 0;
        while (S.node[u] != vm.node[a]) ++u;
        w.W[q][u] += vm.w[a];
      }
    }
  }
  __syncwarp();
  // position space: Hy = Q^T K Q (n3 x n3)
  for (int e = lane; e < n3 * n3; e += 32) {
    const int row = e / n3, col = e % n3, v = row / 3, i = row % 3, u = col / 3, j = col % 3;
    T acc = 0;
    for (int r = 0; r < k; ++r)
      for (int q = 0; q < k; ++q) acc += tab_Q(tb, T(), dtype, r, v) * tab_Q(tb, T(), dtype, q, u) * w.Hz[R * (3 * r + i) + 3 * q + j];
    w.Hy[e] = acc;
  }
  __syncwarp();
  // gradient rows of the merged nodes (FP64): g_y = C^T g_z, times kappa b'
  const int M = w.m;
  if (lane < M) {
    double gu[3] = {0, 0, 0};
    bool any = false;
    for (int q = 0; q < nloc; ++q)
      if (w.W[q][lane] != 0.0) {
        any = true;
        for (int i = 0; i < 3; ++i) {
          double gq = 0.0;
          for (int r = 0; r < k; ++r) gq += tb.coef[dtype][r][q] * w.gz[3 * r + i];
          gu[i] += w.W[q][lane] * kappa * b2.x * gq;
        }
      }
    if (any)
      for (int i = 0; i < 3; ++i) atomicAdd(&g[3 * w.node[lane] + i], gu[i]);
  }
  // Hessian blocks (u <= w) of the merged nodes, one per lane at a time
  const int kbase = koff[p];
  const int nb = M * (M + 1) / 2;
  for (int e = lane; e < nb; e += 32) {
    int u = 0, rem = e;
    while (rem >= M - u) { rem -= M - u; ++u; }
    const int v2 = u + rem;
    T B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool any = false;
    for (int q = 0; q < nloc; ++q) {
      if (w.W[q][u] == 0.0) continue;
      for (int r = 0; r < nloc; ++r) {
        const double f = w.W[q][u] * w.W[r][v2];
        if (f == 0.0) continue;
        any = true;
        const T ff = (T)f;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) B[3 * i + j] += ff * w.Hy[(3 * q + i) * n3 + 3 * r + j];
      }
    }
    if (!any) continue;
    T* d;
    if (u == v2) d = diag + 9 * (size_t)w.node[u];
    else {
      const int sl = dslot[kbase + pair_rank(u, v2, M)];
      if (sl < 0) { dev_flag(status, DEV_BADINDEX); continue; }
      d = vals + 9 * (size_t)sl;
    }
    for (int t = 0; t < 9; ++t) atomicAdd(d + t, B[t]);
  }
}

// The projection of the stored K of every active PT / EE pair, one pair per
// thread (cyclic Jacobi in registers, project_psd): a warp projects 32 pairs
// at once, where the warp-parallel sweeps of k_barrier_pair<., 0> project one
// with a long chain of dependent shared-memory steps.  Pairs of one warp with
// different sizes (R = 3, 6, 9) take the branches in turn.
template <typename T, int R>
__device__ __forceinline__ void project_slot(T* __restrict__ kb) {
  T A[R * R];
#pragma unroll
  for (int e = 0; e < R * R; ++e) A[e] = kb[e];
  project_psd<R, T>(A);
#pragma unroll
  for (int e = 0; e < R * R; ++e) kb[e] = A[e];
}
template <typename T>
__global__ void __launch_bounds__(128) k_project_pairs(int npairs, const int* __restrict__ info, bar_tables tb,
                                                        T* __restrict__ kbuf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int code = info[p];
  if (!(code & 1)) return;
  const int R = 3 * tb.k[(code >> 1) & 3];
  T* kb = kbuf + 81 * (size_t)p;
  if (R == 9) project_slot<T, 9>(kb);
  else if (R == 6) project_slot<T, 6>(kb);
  else project_slot<T, 3>(kb);
}

// smallest squared distance over the PT, EE and PG pair lists (the adaptive
// barrier stiffness and the Newton records).  Squared distances are
// non-negative, so their bit patterns order like their values.
__global__ void k_pairs_min_s(int npt, int nee, int npg, const int* __restrict__ pt, const int* __restrict__ ee,
                              const int* __restrict__ pg, topo T, const double* __restrict__ P,
                              const double* __restrict__ planes, unsigned long long* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double sd = __builtin_huge_val();
  if (p < npt + nee) {
    const int kind = p < npt ? 0 : 1;
    int ids[4], k;
    pair_vertices(kind, kind == 0 ? p : p - npt, kind == 0 ? pt : ee, T, ids, &k);
    d3 y[4];
    for (int a = 0; a < 4; ++a) y[a] = ld3(P, ids[a]);
    if (kind == 0) dist::pt_classify(y[0], y[1], y[2], y[3], &sd);
    else dist::ee_classify(y[0], y[1], y[2], y[3], &sd);
  } else if (p < npt + nee + npg) {
    const int q = p - npt - nee;
    const double* pl = planes + 4 * pg[3 * q + 1];
    const double d = dist::sub(dist::vdot(d3{pl[0], pl[1], pl[2]}, ld3(P, pg[3 * q])), pl[3]);
    sd = dist::mul(d, d);
  }
  unsigned long long b = (unsigned long long)__double_as_longlong(sd);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long bo = __shfl_xor_sync(0xffffffffu, b, o);
    b = bo < b ? bo : b;
  }
  if ((threadIdx.x & 31) == 0 && p - (int)(threadIdx.x & 31) < npt + nee + npg) atomicMin(out, b);
}

// point-plane pairs: s = d^2, grad s = 2 d n, hess s = 2 n n^T; the position-
// space Hessian kappa (4 d^2 b'' + 2 b') n n^T is rank one: its projection
// keeps it when the eigenvalue kappa (4 d^2 b'' + 2 b') |n|^2 is positive.
template <typename T>
__global__ void k_barrier_pg(int npg, int pair_base, const int* __restrict__ pg, topo Tp, const double* __restrict__ vr,
                             const double* __restrict__ P, const double* __restrict__ planes, double sh, double kappa,
                             int form, int project, const int* __restrict__ koff, const int* __restrict__ dslot,
                             double* __restrict__ g, T* __restrict__ diag, T* __restrict__ vals, int* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npg) return;
  const int v = pg[3 * p], k = pg[3 * p + 1];
  const double* pl = planes + 4 * k;
  const d3 x = ld3(P, v);
  const double d = dist::sub(dist::vdot(d3{pl[0], pl[1], pl[2]}, x), pl[3]);
  const double s = dist::mul(d, d);
  if (!(s < sh) || !(d > 0.0)) return;
  const bder bd = barrier_fn(s, sh, form);
  const double nv[3] = {pl[0], pl[1], pl[2]};
  const double lam = kappa * (4.0 * d * d * bd.d2b + 2.0 * bd.db);
  const double hc = (project && lam < 0.0) ? 0.0 : lam;
  vmapd vm = vertex_map(v, Tp, vr);
  // the pair's dynamic keys follow the sorted node order (a cage's nodes need not be sorted)
  for (int a = 1; a < vm.n; ++a)
    for (int b = a; b > 0 && vm.node[b - 1] > vm.node[b]; --b) {
      const int tn = vm.node[b]; vm.node[b] = vm.node[b - 1]; vm.node[b - 1] = tn;
      const double tw = vm.w[b]; vm.w[b] = vm.w[b - 1]; vm.w[b - 1] = tw;
    }
  for (int a = 0; a < vm.n; ++a)
    for (int i = 0; i < 3; ++i) atomicAdd(&g[3 * vm.node[a] + i], vm.w[a] * kappa * bd.db * 2.0 * d * nv[i]);
  const int kbase = koff[pair_base + p];
  for (int a = 0; a < vm.n; ++a)
    for (int b = a; b < vm.n; ++b) {
      const double f = vm.w[a] * vm.w[b] * hc;
      if (f == 0.0) continue;
      T* dst;
      if (a == b) dst = diag + 9 * (size_t)vm.node[a];
      else {
        const int sl = dslot[kbase + pair_rank(a, b, vm.n)];
        if (sl < 0) { dev_flag(status, DEV_BADINDEX); continue; }
        dst = vals + 9 * (size_t)sl;
      }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) atomicAdd(dst + 3 * i + j, (T)(f * nv[i] * nv[j]));
    }
}

// ---------------------------------------------------------------- CCD
__device__ double pair_dist2(int kind, const d3* x) {
  double s;
  if (kind == 0) dist::pt_classify(x[0], x[1], x[2], x[3], &s);
  else dist::ee_classify(x[0], x[1], x[2], x[3], &s);
  return s;
}
// additive CCD along x + t dx, t in [0, tmax]: advance by (1 - gap) d / l_p,
// where l_p bounds the relative motion; stop before the distance falls below
// gap * (starting distance).  Explicitly rounded like the reference arithmetic.
// lp of ACCD (the bound on the pair's relative motion over the step), as accd forms it
__device__ __forceinline__ double accd_motion_bound(int kind, const d3* dx0) {
  using namespace dist;
  double m[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 4; ++i) {
    m[0] = add(m[0], mul(0.25, dx0[i].x));
    m[1] = add(m[1], mul(0.25, dx0[i].y));
    m[2] = add(m[2], mul(0.25, dx0[i].z));
  }
  double nrm[4];
  for (int i = 0; i < 4; ++i) {
    const d3 c = d3{sub(dx0[i].x, m[0]), sub(dx0[i].y, m[1]), sub(dx0[i].z, m[2])};
    nrm[i] = sqrt(vdot(c, c));
  }
  return (kind == 0) ? add(nrm[0], fmax(nrm[1], fmax(nrm[2], nrm[3]))) : add(fmax(nrm[0], nrm[1]), fmax(nrm[2], nrm[3]));
}

__device__ double accd(int kind, d3* x, d3* dx, double gap, double tmax, int max_iter, bool* capped) {
  using namespace dist;
  double m[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 4; ++i) {
    m[0] = add(m[0], mul(0.25, dx[i].x));
    m[1] = add(m[1], mul(0.25, dx[i].y));
    m[2] = add(m[2], mul(0.25, dx[i].z));
  }
  double nrm[4];
  for (int i = 0; i < 4; ++i) {
    dx[i] = d3{sub(dx[i].x, m[0]), sub(dx[i].y, m[1]), sub(dx[i].z, m[2])};
    nrm[i] = sqrt(vdot(dx[i], dx[i]));
  }
  const double lp = (kind == 0) ? add(nrm[0], fmax(nrm[1], fmax(nrm[2], nrm[3])))
                                : add(fmax(nrm[0], nrm[1]), fmax(nrm[2], nrm[3]));
  if (lp == 0.0) return tmax;
  double d = sqrt(pair_dist2(kind, x));
  const double g = mul(gap, d);
  double t = 0.0, tl = dv(mul(sub(1.0, gap), d), lp);
  for (int it = 0; it < max_iter; ++it) {
    for (int i = 0; i < 4; ++i)
      x[i] = d3{add(x[i].x, mul(tl, dx[i].x)), add(x[i].y, mul(tl, dx[i].y)), add(x[i].z, mul(tl, dx[i].z))};
    d = sqrt(pair_dist2(kind, x));
    if (t > 0.0 && d < g) return t;
    t = add(t, tl);
    if (t > tmax) return tmax;
    tl = dv(mul(sub(1.0, gap), d), lp);
  }
  *capped = true;
  return t;
}

__device__ __forceinline__ void atomic_min_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void k_ccd_pg(int nsv, int npl, topo T, const double* __restrict__ P0, const double* __restrict__ D,
                         const double* __restrict__ planes, double gap, double* __restrict__ tmin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsv) return;
  const int v = T.svert[i];
  if (T.vnode[v] < 0) return;
  using namespace dist;
  double best = 1.0;
  const d3 p = ld3(P0, v), dp = ld3(D, v);
  for (int k = 0; k < npl; ++k) {
    const d3 n = d3{planes[4 * k], planes[4 * k + 1], planes[4 * k + 2]};
    const double d0 = sub(vdot(n, p), planes[4 * k + 3]);
    const double vel = vdot(n, dp);
    if (vel >= 0.0) continue;
    const double t = dv(mul(sub(1.0, gap), d0), -vel);
    best = fmin(best, t);
  }
  if (best < 1.0) atomic_min_pos(tmin + (T.vscene ? T.vscene[v] : 0), best);
}

__global__ void k_sub(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}

__global__ void k_reduce_ksum(const ksum* __restrict__ part, int n, double* __restrict__ out) {
  ksum k{0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) kmerge(k, part[i]);
  k = block_ksum(k);
  if (threadIdx.x == 0) *out = k.s + k.c;
}

// ---------------------------------------------------------------- swept candidates
// Candidate pairs of one Newton iteration: query boxes swept over [x, x - p]
// and grown by dhat, against swept (not grown) boxes of the other set.  Every
// pair that comes within dhat anywhere on the segment, and every pair the CCD
// must examine, is in the list.  mode 0: count per query primitive, mode 1:
// write (a, b) sorted by b.
// mode 3: one traversal that counts every candidate of query i into cnt[i]
// and keeps the first kCandSlots partners in tmp[i][.]; k_cand_gather then
// writes the queries that fit, and only overflowing queries run mode 1.
constexpr int kCandSlots = 64;
// A query's grid walk is shared by kQueryLanes lanes (records of each cell
// interleaved over them): the longest walks, of the fastest-moving
// primitives, set the kernel's duration.  The lanes of a query take output
// positions from a shared-memory counter; each query's list is sorted by
// partner afterwards, so the result does not depend on the order they find
// them in.  128 threads per block.
constexpr int kQueryLanes = 4;
constexpr int kQueryThreads = 128;
__global__ void k_cand_query(int total, int kind, int nA, topo T, grid_dev g, boxes A, int mode, int* __restrict__ cnt,
                             const int* __restrict__ off, int* __restrict__ out, int* __restrict__ tmp = nullptr) {
  __shared__ int qc[kQueryThreads / kQueryLanes];
  const int gq = threadIdx.x / kQueryLanes, sub = threadIdx.x % kQueryLanes;
  const int i = blockIdx.x * (kQueryThreads / kQueryLanes) + gq;
  if (sub == 0) qc[gq] = 0;
  __syncwarp();
  if (i >= nA) return;  // the whole group
  if (mode == 1 && tmp && off[i + 1] - off[i] <= kCandSlots) return;  // written by k_cand_gather
  const unsigned gmask = ((1u << kQueryLanes) - 1u) << (threadIdx.x & 31 & ~(kQueryLanes - 1));
  const int base = (mode == 1) ? off[i] : 0;
  const int lim = (mode == 1) ? ((i + 1 < nA) ? off[i + 1] : total) : 0;
  const int a = (kind == 0) ? T.svert[i] : i;
  grid_visit(g, A, i, [&](int j) {
    if (kind == 0) {
      if (pt_excluded(T, a, T.stri[3 * j], T.stri[3 * j + 1], T.stri[3 * j + 2])) return;
    } else {
      if (j <= i) return;
      if (ee_excluded(T, T.sedge[2 * i], T.sedge[2 * i + 1], T.sedge[2 * j], T.sedge[2 * j + 1])) return;
    }
    const int c = atomicAdd(&qc[gq], 1);
    if (mode == 1) {
      if (base + c >= lim) { dev_flag(T.status, DEV_CAPACITY); return; }
      out[2 * (size_t)(base + c)] = a;
      out[2 * (size_t)(base + c) + 1] = j;
    } else if (mode == 3 && c < kCandSlots) {
      tmp[(size_t)i * kCandSlots + c] = j;
    }
  }, kind == 1, sub, kQueryLanes);
  __syncwarp(gmask);  // the group's writes and count are complete
  if (sub != 0) return;
  int c = qc[gq];
  if (mode == 0 || mode == 3) cnt[i] = c;
  if (mode == 1) {
    c = min(c, lim - base);
    int* o = out + 2 * (size_t)base;
    for (int q = 1; q < c; ++q) {
      const int kb = o[2 * q + 1];
      int r = q - 1;
      while (r >= 0 && o[2 * r + 1] > kb) { o[2 * (r + 1) + 1] = o[2 * r + 1]; --r; }
      o[2 * (r + 1) + 1] = kb;
    }
  }
}

// queries whose partners all fit in tmp: sorted by partner id into place
__global__ void k_cand_gather(int kind, int nA, topo T, const int* __restrict__ cnt_off, const int* __restrict__ tmp,
                              int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nA) return;
  const int base = cnt_off[i], c = cnt_off[i + 1] - base;
  if (c == 0 || c > kCandSlots) return;
  int b[kCandSlots];
  for (int q = 0; q < c; ++q) {
    const int kb = tmp[(size_t)i * kCandSlots + q];
    int r = q - 1;
    while (r >= 0 && b[r] > kb) { b[r + 1] = b[r]; --r; }
    b[r + 1] = kb;
  }
  const int a = (kind == 0) ? T.svert[i] : i;
  for (int q = 0; q < c; ++q) {
    out[2 * (size_t)(base + q)] = a;
    out[2 * (size_t)(base + q) + 1] = b[q];
  }
}

__device__ __forceinline__ void cand_vertices(int kind, const int* cand, size_t k, const topo& T, int* ids) {
  const int a = cand[2 * k], b = cand[2 * k + 1];
  if (kind == 0) {
    ids[0] = a; ids[1] = T.stri[3 * b]; ids[2] = T.stri[3 * b + 1]; ids[3] = T.stri[3 * b + 2];
  } else {
    ids[0] = T.sedge[2 * a]; ids[1] = T.sedge[2 * a + 1]; ids[2] = T.sedge[2 * b]; ids[3] = T.sedge[2 * b + 1];
  }
}

__device__ __forceinline__ int cand_first_vertex(int kind, const int* cand, size_t k, const topo& T) {
  const int a = cand[2 * k];
  return kind == 0 ? a : T.sedge[2 * a];
}

// additive CCD over the candidate list; one atomic min per block
__global__ void k_ccd_cand(int kind, int n, const int* __restrict__ cand, topo T, const double* __restrict__ P0,
                           const double* __restrict__ D, const float4* __restrict__ P0f, const float4* __restrict__ Df,
                           double gap, int max_iter, double* __restrict__ tmin, int* status) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double best = 1.0;
  bool capped = false;
  bool todo = k < n;
  int ids[4];
  if (todo) {
    cand_vertices(kind, cand, (size_t)k, T, ids);
    // FP32 first: the full step already holds when (1 - gap)^2 lb^2 > lp^2
    // with the conservative bounds of the copies (a 1e-6 relative margin on
    // top covers ACCD's own FP64 rounding of its first advance)
    float3 df[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) df[q] = ldf3(Df, ids[q]);
    const float mh = motion_hi_f32(df);
    const float om = 1.0f - (float)gap;
    const float g1f = om * om * (1.0f - 8.0f * kU32);
    if (g1f * lb2_f32(kind, P0f, ids) > 4.0f * mh * mh * (1.0f + 1e-6f)) todo = false;
  }
  if (todo) {
    d3 x[4], dx[4];
    for (int q = 0; q < 4; ++q) { x[q] = ld3(P0, ids[q]); dx[q] = ld3(D, ids[q]); }
    // ACCD's first advance is (1 - gap) d0 / lp with lp its bound on the
    // relative motion: when that already exceeds the whole step the answer is
    // the full step, so skip the exact distances
    // Any lower bound lb of d0 will do: lp <= 2 max_k |dx_k - m| (no square
    // roots) decides most pairs, then the separating-axis bound, then lp itself
    double m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 4; ++i) {
      m[0] = dist::add(m[0], dist::mul(0.25, dx[i].x));
      m[1] = dist::add(m[1], dist::mul(0.25, dx[i].y));
      m[2] = dist::add(m[2], dist::mul(0.25, dx[i].z));
    }
    double mx2 = 0.0;
    for (int i = 0; i < 4; ++i) {
      const d3 c = d3{dx[i].x - m[0], dx[i].y - m[1], dx[i].z - m[2]};
      mx2 = fmax(mx2, dot(c, c));
    }
    const double g1 = (1.0 - gap) * (1.0 - gap);
    if (mx2 > 0.0) {  // lp == 0 exactly when every relative motion is 0
      double lb2 = pair_lb2(kind, x[0], x[1], x[2], x[3]);
      if (!(g1 * lb2 > 4.0 * mx2 * (1.0 + 1e-9))) {
        lb2 = fmax(lb2, sat_lb2(kind, x[0], x[1], x[2], x[3]));
        if (!(g1 * lb2 > 4.0 * mx2 * (1.0 + 1e-9))) {
          const double lp = accd_motion_bound(kind, dx);
          if (!(lp == 0.0) && !(g1 * lb2 > lp * lp * (1.0 + 1e-9)))
            best = accd(kind, x, dx, gap, 1.0, max_iter, &capped);
        }
      }
    }
  }
  if (capped) dev_flag(status, DEV_ITERCAP);
  if (T.vscene) {  // batches: one bound per scene
    if (best < 1.0) atomic_min_pos(tmin + T.vscene[cand_first_vertex(kind, cand, (size_t)k, T)], best);
    return;
  }
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = fmin(b, sh[w]);
    if (b < 1.0) atomic_min_pos(tmin, b);
  }
}

// barrier energy over the candidate list at positions P (fixed grid: deterministic)
__global__ void k_energy_cand(int kind, int n, const int* __restrict__ cand, topo T, const double* __restrict__ P,
                              const float4* __restrict__ Pf, double sh, double kappa, int form, ksum* __restrict__ part,
                              double* __restrict__ sacc = nullptr) {
  const float shf = (float)sh * (1.0f + 1e-6f);
  ksum acc{0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < n; base += stride) {
    const long long k = base + lane;
    double e = 0.0;
    int key = -1;
    if (k < n) {
      int ids[4];
      cand_vertices(kind, cand, (size_t)k, T, ids);
      if (!(Pf && lb2_f32(kind, Pf, ids) > shf)) {  // FP32 prefilter, then the FP64 tests
        const d3 y0 = ld3(P, ids[0]), y1 = ld3(P, ids[1]), y2 = ld3(P, ids[2]), y3 = ld3(P, ids[3]);
        if (!surely_apart(pair_lb2(kind, y0, y1, y2, y3), sh) && !sat_apart(kind, y0, y1, y2, y3, sh)) {
          double s;
          if (kind == 0) dist::pt_classify(y0, y1, y2, y3, &s);
          else dist::ee_classify(y0, y1, y2, y3, &s);
          if (s < sh) e = kappa * barrier_fn(s, sh, form).b;
        }
      }
      if (sacc) key = T.vscene[ids[0]];
    }
    // batches: candidates are sorted by their first primitive, so by scene
    if (sacc) seg_add_global(sacc, key, e);
    else kadd(acc, e);
  }
  if (!sacc) {
    acc = block_ksum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
  }
}

// active pairs among the candidates at positions P: flag + subtype
__global__ void k_filter_cand(int kind, int n, const int* __restrict__ cand, topo T, const double* __restrict__ P,
                              const float4* __restrict__ Pf, double sh, int* __restrict__ flag, int* __restrict__ sub) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int ids[4];
  cand_vertices(kind, cand, (size_t)k, T, ids);
  if (Pf && lb2_f32(kind, Pf, ids) > (float)sh * (1.0f + 1e-6f)) {  // FP32 prefilter
    flag[k] = 0;
    sub[k] = 0;
    return;
  }
  const d3 y0 = ld3(P, ids[0]), y1 = ld3(P, ids[1]), y2 = ld3(P, ids[2]), y3 = ld3(P, ids[3]);
  if (surely_apart(pair_lb2(kind, y0, y1, y2, y3), sh) || sat_apart(kind, y0, y1, y2, y3, sh)) {
    flag[k] = 0;
    sub[k] = 0;
    return;
  }
  double s;
  int st;
  if (kind == 0) st = dist::pt_classify(y0, y1, y2, y3, &s);
  else st = dist::ee_classify(y0, y1, y2, y3, &s);
  flag[k] = (s < sh) ? 1 : 0;
  sub[k] = st;
}
__global__ void k_compact_cand(int n, const int* __restrict__ cand, const int* __restrict__ flag,
                               const int* __restrict__ off, const int* __restrict__ sub, int* __restrict__ out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = off[k];
  if (k + 1 < n ? off[k + 1] > i : flag[k]) {
    out[3 * (size_t)i] = cand[2 * k];
    out[3 * (size_t)i + 1] = cand[2 * k + 1];
    out[3 * (size_t)i + 2] = sub[k];
  }
}

// ======================================================================== host
topo make_topo(yasps_system* s) {
  return topo{as<int>(s->vnode),  as<int>(s->vbody),  as<int>(s->stri),
              as<int>(s->sedge),  as<int>(s->svert),  as<int>(s->status),
              s->nscene > 1 ? as<int>(s->vscene) : nullptr, as<int>(s->emb_node), as<double>(s->emb_w)};
}

// Build a grid on boxes (blo, bhi) of n primitives.  Buffers: ws[3] start,
// ws[4] fill, ws[5] items, red for the box reduction.
yasps_status build_grid(yasps_system* s, int n, boxes B, grid_dev* out) {
  const double* blo = B.lo;
  const double* bhi = B.hi;
  const int nblk = std::min(148 * 2, std::max(1, (n + 255) / 256));
  ENSURE(s, s->red, sizeof(double) * 8 * nblk + 64);
  double* part = as<double>(s->red);
  k_box_reduce<<<nblk, 256, 0, s->stream>>>(n, blo, bhi, part);
  LAUNCH_CHECK(s, "k_box_reduce");
  std::vector<double> hp(8 * (size_t)nblk);
  CK(s, cudaMemcpyAsync(hp.data(), part, sizeof(double) * 8 * nblk, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  double r[8] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300, 0.0, 0.0};
  for (int b = 0; b < nblk; ++b)
    for (int q = 0; q < 8; ++q)
      r[q] = (q < 3) ? std::min(r[q], hp[8 * b + q]) : (q < 7 ? std::max(r[q], hp[8 * b + q]) : r[q] + hp[8 * b + q]);
  for (int q = 0; q < 8; ++q)
    if (!std::isfinite(r[q])) SYS_FAIL(s, YASPS_E_NAN, "non-finite primitive box in the broadphase");
  gridp G;
  double span = 0.0;
  for (int c = 0; c < 3; ++c) span = std::max(span, r[3 + c] - r[c]);
  // cells as large as the mean box: a few large (fast, swept) boxes span more
  // cells instead of making every cell crowded
  double cell = std::max(r[7] / std::max(n, 1), 1e-12);
  if (span / cell > 512.0) cell = span / 512.0;
  long long ncell;
  for (;;) {
    ncell = 1;
    // one spare cell on each side: the FP32 origin sits a cell below the boxes
    for (int c = 0; c < 3; ++c) {
      G.dim[c] = (int)((r[3 + c] - r[c]) / cell) + 3;
      ncell *= G.dim[c];
    }
    if (ncell <= (1LL << 23)) break;
    cell *= 1.25;
  }
  for (int c = 0; c < 3; ++c) G.lo[c] = (float)(r[c] - cell);
  G.inv = (float)(1.0 / cell);
  ENSURE(s, s->ws[3], sizeof(int) * (ncell + 1));
  ENSURE(s, s->ws[4], sizeof(int) * (ncell + 1));
  int* start = as<int>(s->ws[3]);
  int* fill = as<int>(s->ws[4]);
  CK(s, cudaMemsetAsync(start, 0, sizeof(int) * (ncell + 1), s->stream));
  k_grid_count<<<blocks_for(n, 256), 256, 0, s->stream>>>(n, B.lof, B.hif, G, start);
  LAUNCH_CHECK(s, "k_grid_count");
  int total = 0;
  RC(scan_exclusive(s, start, start, (int)(ncell + 1), &total));
  ENSURE(s, s->ws[5], sizeof(float4) * 2 * ((size_t)total + 1));
  CK(s, cudaMemsetAsync(fill, 0, sizeof(int) * (ncell + 1), s->stream));
  k_grid_fill<<<blocks_for(n, 256), 256, 0, s->stream>>>(n, B.lof, B.hif, G, start, fill, as<float4>(s->ws[5]));
  LAUNCH_CHECK(s, "k_grid_fill");
  out->G = G;
  out->start = start;
  out->pk = as<float4>(s->ws[5]);
  out->B = B;
  return YASPS_OK;
}

// box buffers: vec slots are not used here; ws[0..2] (A lo/hi, B lo/hi packed)
struct boxbufs {
  boxw a, b;
};
yasps_status alloc_boxes(yasps_system* s, boxbufs* bb) {
  const size_t nmax = std::max({s->nsv, s->nst, s->nse, 1});
  const size_t bytes = (sizeof(double) + sizeof(float)) * 6 * nmax;
  ENSURE(s, s->ws[0], bytes);
  ENSURE(s, s->ws[1], bytes);
  for (int k = 0; k < 2; ++k) {
    boxw& w = k == 0 ? bb->a : bb->b;
    double* d = as<double>(s->ws[k]);
    w.lo = d;
    w.hi = d + 3 * nmax;
    w.lof = reinterpret_cast<float*>(d + 6 * nmax);
    w.hif = w.lof + 3 * nmax;
    w.vscene = s->nscene > 1 ? as<int>(s->vscene) : nullptr;
    w.spacing = s->scene_spacing;
    w.shift = nullptr;
    w.nsc = s->nscene;
  }
  return YASPS_OK;
}

// run a count / write pair (or energy) query of kind 0 (PT) or 1 (EE)
template <typename Launch>
yasps_status two_pass(yasps_system* s, int nA, Launch&& launch, gbuf& outbuf, int* nout) {
  ENSURE(s, s->ws[2], sizeof(int) * (nA + 1));
  int* cnt = as<int>(s->ws[2]);
  RC(launch(0, 0, cnt, (const int*)nullptr, (int*)nullptr));
  int total = 0;
  RC(scan_exclusive(s, cnt, cnt, nA, &total));
  ENSURE(s, outbuf, sizeof(int) * 3 * ((size_t)total + 1));
  if (total > 0) RC(launch(1, total, (int*)nullptr, cnt, as<int>(outbuf)));
  *nout = total;
  return YASPS_OK;
}

// coef, L = chol(coef coef^T) and Q = L^-1 coef of the four distance types
bar_tables make_bar_tables() {
  bar_tables t{};
  const double c[4][3][4] = {{{1, -1, 0, 0}},
                             {{1, -1, 0, 0}, {0, -1, 1, 0}},
                             {{1, -1, 0, 0}, {0, -1, 1, 0}, {0, -1, 0, 1}},
                             {{1, 0, -1, 0}, {-1, 1, 0, 0}, {0, 0, -1, 1}}};
  const int k[4] = {1, 2, 3, 3};
  for (int d = 0; d < 4; ++d) {
    t.k[d] = k[d];
    double G[3][3] = {}, L[3][3] = {};
    for (int r = 0; r < k[d]; ++r)
      for (int q = 0; q < k[d]; ++q)
        for (int v = 0; v < 4; ++v) G[r][q] += c[d][r][v] * c[d][q][v];
    for (int j = 0; j < k[d]; ++j) {
      double sjj = G[j][j];
      for (int m = 0; m < j; ++m) sjj -= L[j][m] * L[j][m];
      L[j][j] = std::sqrt(sjj);
      for (int i = j + 1; i < k[d]; ++i) {
        double sij = G[i][j];
        for (int m = 0; m < j; ++m) sij -= L[i][m] * L[j][m];
        L[i][j] = sij / L[j][j];
      }
    }
    for (int v = 0; v < 4; ++v)
      for (int r = 0; r < k[d]; ++r) {  // forward substitution L Q = coef
        double acc = c[d][r][v];
        for (int m = 0; m < r; ++m) acc -= L[r][m] * t.Q[d][m][v];
        t.Q[d][r][v] = acc / L[r][r];
      }
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) {
        t.L[d][r][q] = L[r][q];
        t.Lf[d][r][q] = (float)L[r][q];
      }
      for (int v = 0; v < 4; ++v) {
        t.coef[d][r][v] = c[d][r][v];
        t.Qf[d][r][v] = (float)t.Q[d][r][v];
      }
    }
  }
  return t;
}

template <typename T>
yasps_status eval_barrier_t(yasps_system* s, int project) {
  static const bar_tables tb = make_bar_tables();
  const topo Tp = make_topo(s);
  const double sh = s->prm.dhat * s->prm.dhat;
  int* st = as<int>(s->status);
  T* diag = as<T>(s->diag);
  T* vals = as<T>(s->Hd.vals);
  double* g = as<double>(s->grad);
  const double* P = as<double>(s->P);
  const int* koff = as<int>(s->pair_key_off);
  const int* dslot = as<int>(s->dyn_slot);
  const int np = s->npt + s->nee;
  if (np) {
    // per-pair classification (a thread per pair), then the derivatives (a warp per pair)
    ENSURE(s, s->bar_prep, (sizeof(double2) + sizeof(int)) * ((size_t)np + 1) + 16);
    double2* bd = as<double2>(s->bar_prep);
    int* info = reinterpret_cast<int*>(bd + np + 1);
    k_barrier_prep<<<blocks_for(np, 128), 128, 0, s->stream>>>(s->npt, s->nee, as<int>(s->pt), as<int>(s->ee), Tp, P,
                                                              sh, s->prm.barrier_form, info, bd);
    LAUNCH_CHECK(s, "k_barrier_prep");
    // A pair per thread has a long latency per pair (one thread's sweeps,
    // ~0.1 ms in FP32 measured) but a high throughput; a warp per pair has
    // half the latency and spreads few pairs over every SM.  Below a few
    // thousand pairs the warp projection is faster.  FP64 Jacobi also runs on
    // the scarce FP64 pipe, where 32 pairs' sweeps on one SM sub-partition pay
    // only once the pairs fill every sub-partition many times over.
    constexpr int kThreadProjMin32 = 8192, kThreadProjMin64 = 16384;
    if (!project || np < (sizeof(T) == 8 ? kThreadProjMin64 : kThreadProjMin32)) {
      k_barrier_pair<T, 0><<<blocks_for(np, 4), 128, 0, s->stream>>>(np, s->npt, as<int>(s->pt), as<int>(s->ee), Tp,
                                                                    as<double>(s->vr), P, info, bd, s->prm.kappa, project, tb,
                                                                    koff, dslot, g, diag, vals, st, nullptr, nullptr);
      LAUNCH_CHECK(s, "k_barrier_pair");
    } else {
      // K of every pair to scratch, projected a pair per thread, then the rest
      ENSURE(s, s->bar_k, (sizeof(T) * 81 + sizeof(double) * 9) * ((size_t)np + 1));
      double* gzb = as<double>(s->bar_k);
      T* kb = reinterpret_cast<T*>(gzb + 9 * ((size_t)np + 1));
      k_barrier_pair<T, 1><<<blocks_for(np, 4), 128, 0, s->stream>>>(np, s->npt, as<int>(s->pt), as<int>(s->ee), Tp,
                                                                    as<double>(s->vr), P, info, bd, s->prm.kappa, 1, tb,
                                                                    koff, dslot, g, diag, vals, st, kb, gzb);
      LAUNCH_CHECK(s, "k_barrier_pair(1)");
      k_project_pairs<T><<<blocks_for(np, 128), 128, 0, s->stream>>>(np, info, tb, kb);
      LAUNCH_CHECK(s, "k_project_pairs");
      k_barrier_pair<T, 2><<<blocks_for(np, 4), 128, 0, s->stream>>>(np, s->npt, as<int>(s->pt), as<int>(s->ee), Tp,
                                                                    as<double>(s->vr), P, info, bd, s->prm.kappa, 1, tb,
                                                                    koff, dslot, g, diag, vals, st, kb, gzb);
      LAUNCH_CHECK(s, "k_barrier_pair(2)");
    }
  }
  if (s->npg) {
    k_barrier_pg<T><<<blocks_for(s->npg, 128), 128, 0, s->stream>>>(s->npg, s->npt + s->nee, as<int>(s->pg), Tp,
                                                                   as<double>(s->vr), P, as<double>(s->planes), sh,
                                                                   s->prm.kappa, s->prm.barrier_form, project, koff,
                                                                   dslot, g, diag, vals, st);
    LAUNCH_CHECK(s, "k_barrier_pg");
  }
  return YASPS_OK;
}

// Projection of a batch of symmetric N x N matrices (row-major), one warp per
// matrix, four per block: the EVD micro-benchmark of the projection sizes
// (yasps_project_batch) with the same warp Jacobi the barrier kernel uses.
template <typename T, int N>
__global__ void __launch_bounds__(128) k_project_batch(int count, const T* __restrict__ in, T* __restrict__ out) {
  constexpr int NP = N + (N & 1);
  __shared__ T A[4][N * N], V[4][N * N];
  __shared__ T cs[4][NP / 2], sn[4][NP / 2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long m = (long long)blockIdx.x * 4 + w;
  if (m >= count) return;  // warp-uniform
  const T* src = in + (size_t)m * N * N;
  for (int e = lane; e < N * N; e += 32) A[w][e] = src[e];
  __syncwarp();
  warp_project<T, N>(A[w], V[w], cs[w], sn[w], lane);
  T* dst = out + (size_t)m * N * N;
  for (int e = lane; e < N * N; e += 32) dst[e] = A[w][e];
}

template <typename T>
yasps_status project_batch_t(int n, int count, const void* in, void* out, cudaStream_t st) {
  const T* I = static_cast<const T*>(in);
  T* O = static_cast<T*>(out);
  const int g = blocks_for(count, 4);
  switch (n) {
    case 3: k_project_batch<T, 3><<<g, 128, 0, st>>>(count, I, O); break;
    case 6: k_project_batch<T, 6><<<g, 128, 0, st>>>(count, I, O); break;
    case 9: k_project_batch<T, 9><<<g, 128, 0, st>>>(count, I, O); break;
    case 12: k_project_batch<T, 12><<<g, 128, 0, st>>>(count, I, O); break;
    case 15: k_project_batch<T, 15><<<g, 128, 0, st>>>(count, I, O); break;
    case 24: k_project_batch<T, 24><<<g, 128, 0, st>>>(count, I, O); break;
    default: return YASPS_E_INVAL;
  }
  return cudaGetLastError() == cudaSuccess ? YASPS_OK : YASPS_E_CUDA;
}

}  // namespace

// ======================================================================== API
yasps_status detect_pairs(yasps_system* s, const double* P) {
  const topo Tp = make_topo(s);
  const double sh = s->prm.dhat * s->prm.dhat;
  s->npt = s->nee = s->npg = 0;
  float4* Pf = nullptr;
  if (s->nv > 0 && (s->nst > 0 || s->nse > 1)) {
    ENSURE(s, s->pf32, sizeof(float4) * (2 * (size_t)s->nv + 1));
    Pf = as<float4>(s->pf32);
    k_f32_copy<<<blocks_for(s->nv, 256), 256, 0, s->stream>>>(s->nv, P, Pf);
    LAUNCH_CHECK(s, "k_f32_copy");
  }
  if (s->nsv > 0 && s->npl > 0) {
    RC(two_pass(s, s->nsv, [&](int mode, int total, int* cnt, const int* off, int* out) -> yasps_status {
      k_pg_query<<<blocks_for(s->nsv, 128), 128, 0, s->stream>>>(total, s->nsv, s->npl, Tp, P, as<double>(s->planes), sh, mode,
                                                                cnt, off, out, 0.0, 0, nullptr);
      LAUNCH_CHECK(s, "k_pg_query");
      return YASPS_OK;
    }, s->pg, &s->npg));
  }
  if (s->nst > 0 && s->nsv > 0) {
    boxbufs bb;
    RC(alloc_boxes(s, &bb));
    k_boxes<<<blocks_for(s->nsv, 256), 256, 0, s->stream>>>(s->nsv, 1, as<int>(s->svert), P, nullptr, s->prm.dhat,
                                                           bb.a);
    LAUNCH_CHECK(s, "k_boxes");
    k_boxes<<<blocks_for(s->nst, 256), 256, 0, s->stream>>>(s->nst, 3, as<int>(s->stri), P, nullptr, 0.0, bb.b);
    LAUNCH_CHECK(s, "k_boxes");
    grid_dev g;
    RC(build_grid(s, s->nst, bb.b, &g));
    RC(two_pass(s, s->nsv, [&](int mode, int total, int* cnt, const int* off, int* out) -> yasps_status {
      k_pt_query<<<blocks_for(s->nsv, 128), 128, 0, s->stream>>>(total, s->nsv, Tp, P, Pf, g, bb.a, sh, mode, cnt, off,
                                                                out, 0.0, 0, nullptr);
      LAUNCH_CHECK(s, "k_pt_query");
      return YASPS_OK;
    }, s->pt, &s->npt));
  }
  if (s->nse > 1) {
    boxbufs bb;
    RC(alloc_boxes(s, &bb));
    k_boxes_self<<<blocks_for(s->nse, 256), 256, 0, s->stream>>>(s->nse, 2, as<int>(s->sedge), P, nullptr,
                                                               s->prm.dhat, bb.a, bb.b);
    LAUNCH_CHECK(s, "k_boxes_self");
    grid_dev g;
    RC(build_grid(s, s->nse, bb.b, &g));
    RC(two_pass(s, s->nse, [&](int mode, int total, int* cnt, const int* off, int* out) -> yasps_status {
      k_ee_query<<<blocks_for(s->nse, 128), 128, 0, s->stream>>>(total, s->nse, Tp, P, Pf, g, bb.a, sh, mode, cnt, off,
                                                                out, 0.0, 0, nullptr);
      LAUNCH_CHECK(s, "k_ee_query");
      return YASPS_OK;
    }, s->ee, &s->nee));
  }
  return build_dynamic_bsr(s);
}

double barrier_db(double s, double sh, int form) { return barrier_fn(s, sh, form).db; }

yasps_status pairs_min_dist2(yasps_system* s, const double* P, double* s_min_host) {
  const int np = s->npt + s->nee + s->npg;
  *s_min_host = __builtin_huge_val();
  if (np == 0) return YASPS_OK;
  ENSURE(s, s->ws[11], sizeof(unsigned long long) * 2);
  unsigned long long* d = as<unsigned long long>(s->ws[11]);
  const double inf = __builtin_huge_val();
  unsigned long long init;
  std::memcpy(&init, &inf, sizeof init);
  CK(s, cudaMemcpyAsync(d, &init, sizeof init, cudaMemcpyHostToDevice, s->stream));
  const topo Tp = make_topo(s);
  k_pairs_min_s<<<blocks_for(np, 128), 128, 0, s->stream>>>(s->npt, s->nee, s->npg, as<int>(s->pt), as<int>(s->ee),
                                                          as<int>(s->pg), Tp, P, as<double>(s->planes), d);
  LAUNCH_CHECK(s, "k_pairs_min_s");
  unsigned long long h = init;
  CK(s, cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  std::memcpy(s_min_host, &h, sizeof h);
  return YASPS_OK;
}

yasps_status build_dynamic_bsr(yasps_system* s) {
  const topo Tp = make_topo(s);
  const int np = s->npt + s->nee + s->npg;
  ENSURE(s, s->pair_key_off, sizeof(int) * (np + 1));
  int* koff = as<int>(s->pair_key_off);
  int nkeys = 0;
  if (np > 0) {
    k_pair_nkeys<<<blocks_for(np, 128), 128, 0, s->stream>>>(s->npt, s->nee, s->npg, as<int>(s->pt), as<int>(s->ee),
                                                            as<int>(s->pg), Tp, as<double>(s->vr), koff);
    LAUNCH_CHECK(s, "k_pair_nkeys");
    RC(scan_exclusive(s, koff, koff, np, &nkeys));
  }
  s->nkeys = nkeys;
  ENSURE(s, s->dyn_slot, sizeof(int) * (nkeys + 1));
  ENSURE(s, s->ws[0], sizeof(uint64_t) * (nkeys + 1));
  ENSURE(s, s->ws[1], sizeof(int) * (nkeys + 1));
  if (nkeys > 0) {
    k_pair_keys<<<blocks_for(np, 128), 128, 0, s->stream>>>(s->npt, s->nee, s->npg, as<int>(s->pt), as<int>(s->ee),
                                                           as<int>(s->pg), Tp, as<double>(s->vr), koff, s->nbits,
                                                           as<uint64_t>(s->ws[0]), as<int>(s->ws[1]));
    LAUNCH_CHECK(s, "k_pair_keys");
  }
  RC(bsr_from_keys(s, as<uint64_t>(s->ws[0]), as<int>(s->ws[1]), nkeys, s->Hd, as<int>(s->dyn_slot), nkeys));
  const size_t es = (s->hess_precision == 1) ? sizeof(float) : sizeof(double);
  ENSURE(s, s->Hd.vals, es * 9 * ((size_t)s->Hd.nnzb + 1));
  return YASPS_OK;
}

yasps_status launch_eval_barrier(yasps_system* s, int project) {
  if (s->hess_precision == 1) return eval_barrier_t<float>(s, project);
  return eval_barrier_t<double>(s, project);
}

yasps_status barrier_energy(yasps_system* s, const double* P, double* E_host) {
  const topo Tp = make_topo(s);
  const double sh = s->prm.dhat * s->prm.dhat;
  const int nblk_v = blocks_for(std::max(s->nsv, 1), 128), nblk_e = blocks_for(std::max(s->nse, 1), 128);
  const int npart = 2 * nblk_v + nblk_e;
  gbuf& pb = s->ws[9];
  ENSURE(s, pb, sizeof(ksum) * (npart + 4));
  ksum* part = as<ksum>(pb);
  CK(s, cudaMemsetAsync(part, 0, sizeof(ksum) * (npart + 4), s->stream));
  float4* Pf = nullptr;
  if (s->nv > 0 && (s->nst > 0 || s->nse > 1)) {
    ENSURE(s, s->pf32, sizeof(float4) * (2 * (size_t)s->nv + 1));
    Pf = as<float4>(s->pf32);
    k_f32_copy<<<blocks_for(s->nv, 256), 256, 0, s->stream>>>(s->nv, P, Pf);
    LAUNCH_CHECK(s, "k_f32_copy");
  }
  if (s->nsv > 0 && s->npl > 0) {
    k_pg_query<<<nblk_v, 128, 0, s->stream>>>(0, s->nsv, s->npl, Tp, P, as<double>(s->planes), sh, 2, nullptr, nullptr,
                                              nullptr, s->prm.kappa, s->prm.barrier_form, part);
    LAUNCH_CHECK(s, "k_pg_query(E)");
  }
  if (s->nst > 0 && s->nsv > 0) {
    boxbufs bb;
    RC(alloc_boxes(s, &bb));
    k_boxes<<<blocks_for(s->nsv, 256), 256, 0, s->stream>>>(s->nsv, 1, as<int>(s->svert), P, nullptr, s->prm.dhat,
                                                           bb.a);
    LAUNCH_CHECK(s, "k_boxes");
    k_boxes<<<blocks_for(s->nst, 256), 256, 0, s->stream>>>(s->nst, 3, as<int>(s->stri), P, nullptr, 0.0, bb.b);
    LAUNCH_CHECK(s, "k_boxes");
    grid_dev g;
    RC(build_grid(s, s->nst, bb.b, &g));
    k_pt_query<<<nblk_v, 128, 0, s->stream>>>(0, s->nsv, Tp, P, Pf, g, bb.a, sh, 2, nullptr, nullptr, nullptr,
                                              s->prm.kappa, s->prm.barrier_form, part + nblk_v);
    LAUNCH_CHECK(s, "k_pt_query(E)");
  }
  if (s->nse > 1) {
    boxbufs bb;
    RC(alloc_boxes(s, &bb));
    k_boxes_self<<<blocks_for(s->nse, 256), 256, 0, s->stream>>>(s->nse, 2, as<int>(s->sedge), P, nullptr,
                                                               s->prm.dhat, bb.a, bb.b);
    LAUNCH_CHECK(s, "k_boxes_self");
    grid_dev g;
    RC(build_grid(s, s->nse, bb.b, &g));
    k_ee_query<<<nblk_e, 128, 0, s->stream>>>(0, s->nse, Tp, P, Pf, g, bb.a, sh, 2, nullptr, nullptr, nullptr,
                                              s->prm.kappa, s->prm.barrier_form, part + 2 * nblk_v);
    LAUNCH_CHECK(s, "k_ee_query(E)");
  }
  double* out = reinterpret_cast<double*>(part + npart + 2);
  k_reduce_ksum<<<1, 256, 0, s->stream>>>(part, npart, out);
  LAUNCH_CHECK(s, "k_reduce_ksum");
  CK(s, cudaMemcpyAsync(E_host, out, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

yasps_status ccd_bound(yasps_system* s, const double* x, const double* p, double* alpha_host) {
  RC(swept_candidates(s, x, p));
  return ccd_candidates(s, alpha_host);
}

// ======================================================================== candidates
yasps_status swept_candidates(yasps_system* s, const double* x, const double* p) {
  const topo Tp = make_topo(s);
  const size_t nv3 = 3 * (size_t)s->nv;
  ENSURE(s, s->stepv[3], sizeof(double) * (3 * (size_t)s->nn + 1));
  const int ns = s->nscene;
  // P1, D, the step bound (one scene: D + nv3), the per-scene displacement sums
  ENSURE(s, s->stepv[4], sizeof(double) * (2 * nv3 + 2 + 4 * (size_t)ns + 2));
  double* x1 = as<double>(s->stepv[3]);
  double* P1 = as<double>(s->stepv[4]);
  double* D = P1 + nv3;
  double* dsum = D + nv3 + 2;
  double* P0 = as<double>(s->P);
  RC(launch_positions(s, x, P0));
  k_sub<<<blocks_for(3LL * s->nn, 256), 256, 0, s->stream>>>(3 * s->nn, x, p, x1);
  LAUNCH_CHECK(s, "k_sub");
  RC(launch_positions(s, x1, P1));
  k_sub<<<blocks_for((long long)nv3, 256), 256, 0, s->stream>>>((int)nv3, P1, P0, D);
  LAUNCH_CHECK(s, "k_sub");
  CK(s, cudaMemsetAsync(dsum, 0, sizeof(double) * 4 * (size_t)ns, s->stream));
  k_disp_sum<<<std::min(148 * 4, std::max(1, blocks_for(s->nv, 256))), 256, 0, s->stream>>>(
      s->nv, D, ns > 1 ? as<int>(s->vscene) : nullptr, ns, dsum);
  LAUNCH_CHECK(s, "k_disp_sum");
  s->ncpt = s->ncee = 0;
  for (int kind = 0; kind < 2; ++kind) {
    const int nA = kind == 0 ? s->nsv : s->nse;
    const int nB = kind == 0 ? s->nst : s->nse;
    if (nA == 0 || nB == 0 || (kind == 1 && nA < 2)) continue;
    boxbufs bb;
    RC(alloc_boxes(s, &bb));
    bb.a.shift = bb.b.shift = dsum;
    if (kind == 0) {
      k_boxes<<<blocks_for(nA, 256), 256, 0, s->stream>>>(nA, 1, as<int>(s->svert), P0, P1, s->prm.dhat, bb.a);
      LAUNCH_CHECK(s, "k_boxes");
      k_boxes<<<blocks_for(nB, 256), 256, 0, s->stream>>>(nB, 3, as<int>(s->stri), P0, P1, 0.0, bb.b);
      LAUNCH_CHECK(s, "k_boxes");
    } else {
      k_boxes_self<<<blocks_for(nA, 256), 256, 0, s->stream>>>(nA, 2, as<int>(s->sedge), P0, P1,
                                                                 s->prm.dhat, bb.a, bb.b);
      LAUNCH_CHECK(s, "k_boxes_self");
    }
    grid_dev g;
    RC(build_grid(s, nB, bb.b, &g));
    ENSURE(s, s->ws[2], sizeof(int) * (nA + 2));
    ENSURE(s, s->ws[10], sizeof(int) * ((size_t)nA * kCandSlots + 1));
    int* cnt = as<int>(s->ws[2]);
    int* tmp = as<int>(s->ws[10]);
    // one traversal: exact counts, the first kCandSlots partners kept
    const int qblk = blocks_for((long long)nA * kQueryLanes, kQueryThreads);
    k_cand_query<<<qblk, kQueryThreads, 0, s->stream>>>(0, kind, nA, Tp, g, bb.a, 3, cnt, nullptr, nullptr, tmp);
    LAUNCH_CHECK(s, "k_cand_query");
    int total = 0;
    RC(scan_exclusive(s, cnt, cnt, nA, &total));
    CK(s, cudaMemcpyAsync(cnt + nA, &total, sizeof(int), cudaMemcpyHostToDevice, s->stream));
    gbuf& out = kind == 0 ? s->cpt : s->cee;
    ENSURE(s, out, sizeof(int) * 2 * ((size_t)total + 1));
    if (total > 0) {
      k_cand_gather<<<blocks_for(nA, 256), 256, 0, s->stream>>>(kind, nA, Tp, cnt, tmp, as<int>(out));
      LAUNCH_CHECK(s, "k_cand_gather");
      // queries with more partners than slots traverse again and write in place
      k_cand_query<<<qblk, kQueryThreads, 0, s->stream>>>(total, kind, nA, Tp, g, bb.a, 1, nullptr, cnt,
                                                               as<int>(out), tmp);
      LAUNCH_CHECK(s, "k_cand_query");
    }
    (kind == 0 ? s->ncpt : s->ncee) = total;
  }
  s->cand_valid = true;
  return YASPS_OK;
}

yasps_status ccd_candidates(yasps_system* s, double* alpha_host) {
  const topo Tp = make_topo(s);
  const size_t nv3 = 3 * (size_t)s->nv;
  double* P0 = as<double>(s->P);
  double* D = as<double>(s->stepv[4]) + nv3;
  // one bound per scene (batches) or one in all
  const int nb_t = s->nscene;
  double* tmin = (nb_t > 1) ? as<double>(s->scene_buf) + 3 * (size_t)nb_t : D + nv3;
  const std::vector<double> ones(nb_t, 1.0);
  CK(s, cudaMemcpyAsync(tmin, ones.data(), sizeof(double) * nb_t, cudaMemcpyHostToDevice, s->stream));
  int* st = as<int>(s->status);
  // FP32 copies of the positions and displacements for the prefilter
  ENSURE(s, s->pf32, sizeof(float4) * (2 * (size_t)s->nv + 1));
  float4* P0f = as<float4>(s->pf32);
  float4* Df = P0f + s->nv;
  if (s->nv > 0 && (s->ncpt > 0 || s->ncee > 0)) {
    k_f32_copy<<<blocks_for(s->nv, 256), 256, 0, s->stream>>>(s->nv, P0, P0f);
    k_f32_copy<<<blocks_for(s->nv, 256), 256, 0, s->stream>>>(s->nv, D, Df);
    LAUNCH_CHECK(s, "k_f32_copy");
  }
  if (s->nsv > 0 && s->npl > 0) {
    k_ccd_pg<<<blocks_for(s->nsv, 128), 128, 0, s->stream>>>(s->nsv, s->npl, Tp, P0, D, as<double>(s->planes),
                                                            s->prm.ccd_gap, tmin);
    LAUNCH_CHECK(s, "k_ccd_pg");
  }
  for (int kind = 0; kind < 2; ++kind) {
    const int n = kind == 0 ? s->ncpt : s->ncee;
    if (n == 0) continue;
    k_ccd_cand<<<blocks_for(n, 128), 128, 0, s->stream>>>(kind, n, as<int>(kind == 0 ? s->cpt : s->cee), Tp, P0, D,
                                                         P0f, Df, s->prm.ccd_gap, s->prm.ccd_max_iter, tmin, st);
    LAUNCH_CHECK(s, "k_ccd_cand");
  }
  CK(s, cudaMemcpyAsync(alpha_host, tmin, sizeof(double) * nb_t, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

yasps_status barrier_energy_candidates(yasps_system* s, const double* P, double* E_host, double* sacc) {
  const topo Tp = make_topo(s);
  const double sh = s->prm.dhat * s->prm.dhat;
  const int nblk_v = blocks_for(std::max(s->nsv, 1), 128);
  const int nblk_c = 148 * 2;
  const int npart = nblk_v + 2 * nblk_c;
  gbuf& pb = s->ws[9];
  ENSURE(s, pb, sizeof(ksum) * (npart + 4));
  ksum* part = as<ksum>(pb);
  CK(s, cudaMemsetAsync(part, 0, sizeof(ksum) * (npart + 4), s->stream));
  if (s->nsv > 0 && s->npl > 0) {
    k_pg_query<<<nblk_v, 128, 0, s->stream>>>(0, s->nsv, s->npl, Tp, P, as<double>(s->planes), sh, 2, nullptr, nullptr,
                                              nullptr, s->prm.kappa, s->prm.barrier_form, part, sacc);
    LAUNCH_CHECK(s, "k_pg_query(E)");
  }
  float4* Pf = as<float4>(s->pf32);
  if (s->ncpt > 0 || s->ncee > 0) {
    ENSURE(s, s->pf32, sizeof(float4) * (2 * (size_t)s->nv + 1));
    Pf = as<float4>(s->pf32);
    k_f32_copy<<<blocks_for(s->nv, 256), 256, 0, s->stream>>>(s->nv, P, Pf);
    LAUNCH_CHECK(s, "k_f32_copy");
  }
  for (int kind = 0; kind < 2; ++kind) {
    const int n = kind == 0 ? s->ncpt : s->ncee;
    if (n == 0) continue;
    k_energy_cand<<<nblk_c, 128, 0, s->stream>>>(kind, n, as<int>(kind == 0 ? s->cpt : s->cee), Tp, P, Pf, sh, s->prm.kappa,
                                                 s->prm.barrier_form, part + nblk_v + kind * nblk_c, sacc);
    LAUNCH_CHECK(s, "k_energy_cand");
  }
  if (sacc) return YASPS_OK;  // batches: the per-scene sums are the result
  double* out = reinterpret_cast<double*>(part + npart + 2);
  k_reduce_ksum<<<1, 256, 0, s->stream>>>(part, npart, out);
  LAUNCH_CHECK(s, "k_reduce_ksum");
  CK(s, cudaMemcpyAsync(E_host, out, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

yasps_status detect_from_candidates(yasps_system* s, const double* P) {
  const topo Tp = make_topo(s);
  const double sh = s->prm.dhat * s->prm.dhat;
  s->npt = s->nee = s->npg = 0;
  if (s->nsv > 0 && s->npl > 0) {
    RC(two_pass(s, s->nsv, [&](int mode, int total, int* cnt, const int* off, int* out) -> yasps_status {
      k_pg_query<<<blocks_for(s->nsv, 128), 128, 0, s->stream>>>(total, s->nsv, s->npl, Tp, P, as<double>(s->planes), sh,
                                                                mode, cnt, off, out, 0.0, 0, nullptr);
      LAUNCH_CHECK(s, "k_pg_query");
      return YASPS_OK;
    }, s->pg, &s->npg));
  }
  float4* Pf = nullptr;
  if (s->ncpt > 0 || s->ncee > 0) {
    ENSURE(s, s->pf32, sizeof(float4) * (2 * (size_t)s->nv + 1));
    Pf = as<float4>(s->pf32);
    k_f32_copy<<<blocks_for(s->nv, 256), 256, 0, s->stream>>>(s->nv, P, Pf);
    LAUNCH_CHECK(s, "k_f32_copy");
  }
  for (int kind = 0; kind < 2; ++kind) {
    const int n = kind == 0 ? s->ncpt : s->ncee;
    int& nout = kind == 0 ? s->npt : s->nee;
    gbuf& outbuf = kind == 0 ? s->pt : s->ee;
    nout = 0;
    if (n == 0) continue;
    ENSURE(s, s->ws[0], sizeof(int) * (n + 1));
    ENSURE(s, s->ws[1], sizeof(int) * (n + 1));
    ENSURE(s, s->ws[2], sizeof(int) * (n + 1));
    int *flag = as<int>(s->ws[0]), *sub = as<int>(s->ws[1]), *off = as<int>(s->ws[2]);
    const int* cand = as<int>(kind == 0 ? s->cpt : s->cee);
    k_filter_cand<<<blocks_for(n, 128), 128, 0, s->stream>>>(kind, n, cand, Tp, P, Pf, sh, flag, sub);
    LAUNCH_CHECK(s, "k_filter_cand");
    int total = 0;
    RC(scan_exclusive(s, flag, off, n, &total));
    ENSURE(s, outbuf, sizeof(int) * 3 * ((size_t)total + 1));
    if (total > 0) {
      k_compact_cand<<<blocks_for(n, 256), 256, 0, s->stream>>>(n, cand, flag, off, sub, as<int>(outbuf));
      LAUNCH_CHECK(s, "k_compact_cand");
    }
    nout = total;
  }
  return build_dynamic_bsr(s);
}

extern "C" yasps_status yasps_project_batch(int n, int count, int precision, const void* in_dev, void* out_dev,
                                            void* cuda_stream) {
  if (count < 0 || (count > 0 && (!in_dev || !out_dev)) || (precision != 0 && precision != 1)) return YASPS_E_INVAL;
  if (count == 0) return YASPS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return precision == 0 ? project_batch_t<double>(n, count, in_dev, out_dev, st)
                        : project_batch_t<float>(n, count, in_dev, out_dev, st);
}
