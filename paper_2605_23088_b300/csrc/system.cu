// system.cu -- the C ABI (include/yasps.h): system build, state helpers, and
// the implicit time step of the incremental potential (Sec. 3 "System
// Overview": collision detection -> minimise (assemble H, g; solve H p = g) ->
// CCD step bound and line search -> update).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

static thread_local std::string g_build_error;

// ---------------------------------------------------------------- memory
void* sys_alloc(yasps_system* s, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (s->have_allocator) return s->allocator.alloc(s->allocator.ctx, bytes, (void*)s->stream);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void sys_free(yasps_system* s, void* p) {
  if (!p) return;
  if (s->have_allocator) s->allocator.free(s->allocator.ctx, p, (void*)s->stream);
  else cudaFreeAsync(p, s->stream);
}
bool ensure(yasps_system* s, gbuf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return true;
  size_t cap = std::max<size_t>(bytes + bytes / 4, 256);
  sys_free(s, b.p);
  b.p = sys_alloc(s, cap);
  b.cap = b.p ? cap : 0;
  return b.p != nullptr;
}
void release(yasps_system* s, gbuf& b) {
  sys_free(s, b.p);
  b.p = nullptr;
  b.cap = 0;
}

yasps_status cuda_check(yasps_system* s, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return YASPS_OK;
  s->err = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? YASPS_E_NOMEM : YASPS_E_CUDA;
}

template <typename T>
static yasps_status upload(yasps_system* s, gbuf& b, const T* host, size_t count) {
  ENSURE(s, b, sizeof(T) * (count + 1));
  if (count) CK(s, cudaMemcpyAsync(b.p, host, sizeof(T) * count, cudaMemcpyHostToDevice, s->stream));
  return YASPS_OK;
}

static void all_bufs(yasps_system* s, std::vector<gbuf*>& v) {
  gbuf* one[] = {&s->vnode, &s->vbody, &s->vr, &s->emb_node, &s->emb_w, &s->vmass, &s->rest, &s->xfix, &s->fixed, &s->fixvel, &s->nodemass,
                 &s->tet_v, &s->tet_n, &s->tet_rest, &s->tet_E, &s->tet_nu, &s->vscene, &s->node_scene, &s->scene_buf, &s->tet_slot, &s->tri_v, &s->tri_n, &s->tri_rest, &s->tri_slot,
                 &s->hinge_v, &s->hinge_n, &s->hinge_rest, &s->hinge_slot, &s->body_kv, &s->body_slot, &s->stri,
                 &s->sedge, &s->svert, &s->planes, &s->Hs.row_ptr, &s->Hs.col, &s->Hs.row, &s->Hs.vals,
                 &s->Hd.row_ptr, &s->Hd.col, &s->Hd.row, &s->Hd.vals, &s->diag, &s->grad, &s->minv, &s->dsym, &s->P, &s->pt,
                 &s->ee, &s->pg, &s->cpt, &s->cee, &s->pair_key_off, &s->dyn_slot, &s->bar_prep, &s->pcg_bt, &s->pf32, &s->bar_k, &s->status, &s->scal, &s->red, &s->scan_tmp};
  for (gbuf* b : one) v.push_back(b);
  for (auto& b : s->ws) v.push_back(&b);
  for (auto& b : s->vec) v.push_back(&b);
  for (auto& b : s->stepv) v.push_back(&b);
}

// ---------------------------------------------------------------- profiler
cudaEvent_t prof_begin(yasps_system* s) {
  if (!s->prof_on) return nullptr;
  cudaEvent_t e;
  if (!s->prof_pool.empty()) {
    e = s->prof_pool.back();
    s->prof_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaEventRecord(e, s->stream);
  return e;
}
void prof_end(yasps_system* s, int stage, cudaEvent_t a, double bytes) {
  if (!a) return;
  cudaEvent_t b = prof_begin(s);
  if (!b) return;
  s->prof_pending.push_back({stage, a, b, bytes});
  if (s->prof_pending.size() >= 256) prof_resolve(s);
}
void prof_resolve(yasps_system* s) {
  if (s->prof_pending.empty()) return;
  cudaStreamSynchronize(s->stream);
  for (auto& p : s->prof_pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto& acc = s->prof_acc[p.stage];
    acc.count += 1;
    acc.ms += ms;
    acc.bytes += p.bytes;
    s->prof_pool.push_back(p.a);
    s->prof_pool.push_back(p.b);
  }
  s->prof_pending.clear();
}

// ======================================================================== ABI
extern "C" {

yasps_status yasps_profile_enable(yasps_system* s, int enable) {
  if (!s) return YASPS_E_INVAL;
  prof_resolve(s);
  s->prof_on = enable != 0;
  if (enable) {
    for (auto& a : s->prof_acc) a = yasps_stage_stats{0, 0.0, 0.0};
    for (auto& t : s->pcg_phase_ms) t = 0.0;
    s->pcg_busy_ns.clear();
    s->pcg_busy_sm.clear();
    s->pcg_busy_iters = 0;
  }
  return YASPS_OK;
}

yasps_status yasps_pcg_block_busy(const yasps_system* s, int capacity, int* n_blocks, double* us_per_iter,
                                  int* sm_ids) {
  if (!s || !n_blocks || capacity < 0) return YASPS_E_INVAL;
  const int G = (int)s->pcg_busy_ns.size();
  *n_blocks = G;
  const double it = s->pcg_busy_iters > 0 ? (double)s->pcg_busy_iters : 1.0;
  for (int b = 0; b < G && b < capacity; ++b) {
    if (us_per_iter) us_per_iter[b] = s->pcg_busy_ns[b] * 1e-3 / it;
    if (sm_ids) sm_ids[b] = s->pcg_busy_sm[b];
  }
  return YASPS_OK;
}

yasps_status yasps_pcg_phase_ms(const yasps_system* s, double* out) {
  if (!s || !out) return YASPS_E_INVAL;
  for (int k = 0; k < 8; ++k) out[k] = s->pcg_phase_ms[k];
  return YASPS_OK;
}

yasps_status yasps_profile_get(yasps_system* s, int stage, yasps_stage_stats* out) {
  if (!s || !out || stage < 0 || stage >= YASPS_NUM_STAGES) return YASPS_E_INVAL;
  prof_resolve(s);
  *out = s->prof_acc[stage];
  return YASPS_OK;
}

void yasps_default_params(yasps_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->precision = 0;
  p->dt = 0.01;
  p->dhat = 1e-3;
  p->kappa = 1e4;
  p->gravity[1] = -9.81;
  p->newton_tol = 1e-6;
  p->pcg_rel_tol = 1e-4;
  p->pcg_max_iter = 0;
  p->newton_max_iter = 100;
  p->ls_max_iter = 30;
  p->barrier_form = 0;
  p->ccd_gap = 0.1;
  p->ccd_max_iter = 100000;
  p->refine_sweeps = 4;
  p->pcg_warm_start = 1;
  p->kappa_adaptive = 0;
  p->kappa_min = 0.0;
  p->kappa_max = 0.0;
  p->kappa_dmin = 0.0;
  p->ls_armijo = 0.0;
}

const char* yasps_build_error(void) { return g_build_error.c_str(); }
const char* yasps_last_error(const yasps_system* s) { return s ? s->err.c_str() : "null system"; }
long long yasps_kernel_launches(const yasps_system* s) { return s ? s->launches : 0; }

static yasps_status build_impl(yasps_system* s, const yasps_scene_desc* d) {
  const int nv = d->n_verts;
  if (nv < 0 || d->n_tets < 0 || d->n_tris < 0 || d->n_hinges < 0 || d->n_bodies < 0 || d->n_fixed < 0 ||
      d->n_surf_tris < 0 || d->n_surf_edges < 0 || d->n_surf_verts < 0 || d->n_planes < 0)
    SYS_FAIL(s, YASPS_E_INVAL, "negative size in the scene");
  if (nv > 0 && (!d->rest_pos || !d->vert_body)) SYS_FAIL(s, YASPS_E_INVAL, "rest_pos / vert_body missing");
  if (d->cloth_model != 0 && d->cloth_model != 1) SYS_FAIL(s, YASPS_E_INVAL, "cloth_model must be 0 or 1");
  if (d->cloth_model == 1 && d->n_tris > 0 && !d->tri_shear)
    SYS_FAIL(s, YASPS_E_INVAL, "tri_shear missing for the Baraff-Witkin cloth");
  auto bad_idx = [&](const int* a, long long n, int hi) {
    for (long long i = 0; i < n; ++i)
      if (a[i] < 0 || a[i] >= hi) return true;
    return false;
  };
  if (bad_idx(d->tet2v, 4LL * d->n_tets, nv) || bad_idx(d->tri2v, 3LL * d->n_tris, nv) ||
      bad_idx(d->hinge2v, 4LL * d->n_hinges, nv) || bad_idx(d->fixed_verts, d->n_fixed, nv) ||
      bad_idx(d->surf_tri2v, 3LL * d->n_surf_tris, nv) || bad_idx(d->surf_edge2v, 2LL * d->n_surf_edges, nv) ||
      bad_idx(d->surf_verts, d->n_surf_verts, nv))
    SYS_FAIL(s, YASPS_E_INVAL, "vertex index out of range in the scene");
  for (int i = 1; i < d->n_surf_verts; ++i)
    if (d->surf_verts[i] <= d->surf_verts[i - 1]) SYS_FAIL(s, YASPS_E_INVAL, "surf_verts must be strictly increasing");
  for (int v = 0; v < nv; ++v)
    if (d->vert_body[v] < -2 || d->vert_body[v] >= d->n_bodies) SYS_FAIL(s, YASPS_E_INVAL, "vert_body out of range");
  // cage-embedded vertices: each listed once, its 8 cage vertices free
  const int ne = d->n_embedded > 0 ? d->n_embedded : 0;
  std::vector<int> emb_row(nv, -1);
  if (ne > 0 && (!d->embed_verts || !d->embed_cage || !d->embed_w))
    SYS_FAIL(s, YASPS_E_INVAL, "embed_verts / embed_cage / embed_w missing");
  if (bad_idx(d->embed_verts, ne, nv) || bad_idx(d->embed_cage, 8LL * ne, nv))
    SYS_FAIL(s, YASPS_E_INVAL, "embedding index out of range");
  for (int e = 0; e < ne; ++e) {
    const int v = d->embed_verts[e];
    if (e > 0 && v <= d->embed_verts[e - 1]) SYS_FAIL(s, YASPS_E_INVAL, "embed_verts must be strictly increasing");
    if (d->vert_body[v] != -2) SYS_FAIL(s, YASPS_E_INVAL, "an embedded vertex must have vert_body -2");
    emb_row[v] = e;
  }
  for (int v = 0; v < nv; ++v)
    if (d->vert_body[v] == -2 && emb_row[v] < 0) SYS_FAIL(s, YASPS_E_INVAL, "vert_body -2 without an embedding");

  // batching: scenes contiguous in vertex order, every element inside one scene
  const int ns = (d->n_scenes > 1) ? d->n_scenes : 1;
  if (ns > 1) {
    if (ns > kMaxScenes) SYS_FAIL(s, YASPS_E_CAPACITY, "more scenes than a batch may hold");
    if (!d->vert_scene) SYS_FAIL(s, YASPS_E_INVAL, "vert_scene missing for a batch");
    for (int v = 0; v < nv; ++v)
      if (d->vert_scene[v] < 0 || d->vert_scene[v] >= ns || (v > 0 && d->vert_scene[v] < d->vert_scene[v - 1]))
        SYS_FAIL(s, YASPS_E_INVAL, "vert_scene must be non-decreasing and in [0, n_scenes)");
    auto mixed = [&](const int* a, int k, long long n) {
      for (long long e = 0; e < n; ++e)
        for (int q = 1; q < k; ++q)
          if (d->vert_scene[a[k * e + q]] != d->vert_scene[a[k * e]]) return true;
      return false;
    };
    if (mixed(d->tet2v, 4, d->n_tets) || mixed(d->tri2v, 3, d->n_tris) || mixed(d->hinge2v, 4, d->n_hinges) ||
        mixed(d->surf_tri2v, 3, d->n_surf_tris) || mixed(d->surf_edge2v, 2, d->n_surf_edges))
      SYS_FAIL(s, YASPS_E_INVAL, "an element spans two scenes");
    std::vector<int> bscene(d->n_bodies, -1);
    for (int v = 0; v < nv; ++v) {
      const int b = d->vert_body[v];
      if (b < 0) continue;
      if (bscene[b] >= 0 && bscene[b] != d->vert_scene[v]) SYS_FAIL(s, YASPS_E_INVAL, "an affine body spans two scenes");
      bscene[b] = d->vert_scene[v];
    }
  }
  s->nscene = ns;
  s->nv = nv; s->nt = d->n_tets; s->nc = d->n_tris; s->nh = d->n_hinges; s->nb = d->n_bodies;
  s->nst = d->n_surf_tris; s->nse = d->n_surf_edges; s->nsv = d->n_surf_verts; s->npl = d->n_planes;
  s->nfix = d->n_fixed;

  // DOF layout (App. A "Gradient Size Computation"): free vertices, then 4 nodes per body
  std::vector<int> isfixed(nv, 0), vnode(nv, -1);
  for (int i = 0; i < d->n_fixed; ++i) isfixed[d->fixed_verts[i]] = 1;
  for (int v = 0; v < nv; ++v)
    if (isfixed[v] && d->vert_body[v] != -1) SYS_FAIL(s, YASPS_E_INVAL, "a fixed vertex must be free (not in a body or a cage)");
  int nf = 0;
  for (int v = 0; v < nv; ++v)
    if (!isfixed[v] && d->vert_body[v] == -1) vnode[v] = nf++;
  s->nfree = nf;
  s->nn = nf + 4 * s->nb;
  for (int v = 0; v < nv; ++v)
    if (d->vert_body[v] >= 0) vnode[v] = nf + 4 * d->vert_body[v];
  // embedded vertices: no node of their own; the node table lists their cage's
  std::vector<int> emb_node(8 * (size_t)ne + 8, 0);
  for (int e = 0; e < ne; ++e)
    for (int k = 0; k < 8; ++k) {
      const int c = d->embed_cage[8 * e + k];
      if (d->vert_body[c] != -1 || isfixed[c]) SYS_FAIL(s, YASPS_E_INVAL, "a cage vertex must be free and not fixed");
      emb_node[8 * e + k] = vnode[c];
    }
  for (int e = 0; e < ne; ++e) vnode[d->embed_verts[e]] = emb_node[8 * e];
  s->ne = ne;
  int nbits = 1;
  while (((1LL << nbits) - 1) < (long long)s->nn + 1) ++nbits;
  if (nbits > 31) SYS_FAIL(s, YASPS_E_INVAL, "too many nodes");
  s->nbits = nbits;
  if (ns > 1) {
    std::vector<int> nscene(s->nn, 0);
    for (int v = 0; v < nv; ++v) {
      if (isfixed[v] || d->vert_body[v] == -2) continue;  // an embedded vertex's nodes are its cage's
      if (d->vert_body[v] < 0) nscene[vnode[v]] = d->vert_scene[v];
      else
        for (int k = 0; k < 4; ++k) nscene[vnode[v] + k] = d->vert_scene[v];
    }
    // broadphase lattice: 1.5 x the largest scene extent plus 0.1 m between scene origins
    std::vector<double> lo(3 * (size_t)ns, 1e300), hi(3 * (size_t)ns, -1e300);
    for (int v = 0; v < nv; ++v)
      for (int c = 0; c < 3; ++c) {
        const int k = d->vert_scene[v];
        lo[3 * k + c] = std::min(lo[3 * k + c], d->rest_pos[3 * v + c]);
        hi[3 * k + c] = std::max(hi[3 * k + c], d->rest_pos[3 * v + c]);
      }
    double ext = 0.0;
    for (int k = 0; k < ns; ++k)
      for (int c = 0; c < 3; ++c)
        if (hi[3 * k + c] >= lo[3 * k + c]) ext = std::max(ext, hi[3 * k + c] - lo[3 * k + c]);
    s->scene_spacing = 1.5 * ext + 0.1;
    RC(upload(s, s->vscene, d->vert_scene, (size_t)nv));
    RC(upload(s, s->node_scene, nscene.data(), (size_t)s->nn));
    ENSURE(s, s->scene_buf, sizeof(double) * 8 * (size_t)ns);
  }

  // affine bodies: body-centred rest coordinates r, uniformly lumped masses,
  // node mass matrix M_ab = sum_v m_v w_a w_b with w = (1, r1, r2, r3)
  std::vector<double> vr(3 * (size_t)nv, 0.0), bcen(3 * (size_t)s->nb, 0.0), bvm(nv, 0.0), Mb(16 * (size_t)s->nb, 0.0);
  std::vector<int> bcnt(s->nb, 0);
  for (int v = 0; v < nv; ++v)
    if (d->vert_body[v] >= 0) {
      const int b = d->vert_body[v];
      bcnt[b]++;
      for (int c = 0; c < 3; ++c) bcen[3 * b + c] += d->rest_pos[3 * v + c];
    }
  for (int b = 0; b < s->nb; ++b) {
    if (bcnt[b] == 0) SYS_FAIL(s, YASPS_E_INVAL, "affine body without vertices");
    for (int c = 0; c < 3; ++c) bcen[3 * b + c] /= bcnt[b];
  }
  for (int v = 0; v < nv; ++v)
    if (d->vert_body[v] >= 0) {
      const int b = d->vert_body[v];
      for (int c = 0; c < 3; ++c) vr[3 * v + c] = d->rest_pos[3 * v + c] - bcen[3 * b + c];
      bvm[v] = d->body_mass[b] / bcnt[b];
      const double w[4] = {1.0, vr[3 * v], vr[3 * v + 1], vr[3 * v + 2]};
      for (int a = 0; a < 4; ++a)
        for (int q = 0; q < 4; ++q) Mb[16 * b + 4 * a + q] += bvm[v] * w[a] * w[q];
    }
  std::vector<double> kv(s->nb);
  for (int b = 0; b < s->nb; ++b) kv[b] = d->body_kappa[b] * d->body_vol[b];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v = 0; v < nv; ++v)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], d->rest_pos[3 * v + c]);
      hi[c] = std::max(hi[c], d->rest_pos[3 * v + c]);
    }
  s->bbox_diag = nv ? std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                (hi[2] - lo[2]) * (hi[2] - lo[2]))
                    : 1.0;

  RC(upload(s, s->rest, d->rest_pos, 3 * (size_t)nv));
  RC(upload(s, s->xfix, d->rest_pos, 3 * (size_t)nv));
  RC(upload(s, s->vnode, vnode.data(), nv));
  // device body codes: -1 free, >= 0 affine body, -2 - e embedded with embedding row e
  std::vector<int> vb(d->vert_body, d->vert_body + nv);
  for (int v = 0; v < nv; ++v)
    if (emb_row[v] >= 0) vb[v] = -2 - emb_row[v];
  RC(upload(s, s->vbody, vb.data(), nv));
  RC(upload(s, s->emb_node, emb_node.data(), 8 * (size_t)ne));
  RC(upload(s, s->emb_w, d->embed_w, 8 * (size_t)ne));
  RC(upload(s, s->vr, vr.data(), 3 * (size_t)nv));
  RC(upload(s, s->vmass, bvm.data(), nv));
  RC(upload(s, s->fixed, d->fixed_verts, d->n_fixed));
  RC(upload(s, s->fixvel, d->fixed_vel, 3 * (size_t)d->n_fixed));
  ENSURE(s, s->nodemass, sizeof(double) * ((size_t)nf + 16 * (size_t)s->nb + 1));
  CK(s, cudaMemsetAsync(s->nodemass.p, 0, sizeof(double) * nf, s->stream));
  if (s->nb)
    CK(s, cudaMemcpyAsync(as<double>(s->nodemass) + nf, Mb.data(), sizeof(double) * 16 * s->nb, cudaMemcpyHostToDevice,
                          s->stream));
  RC(upload(s, s->tet_v, d->tet2v, 4 * (size_t)s->nt));
  ENSURE(s, s->tet_n, sizeof(int) * (4 * (size_t)s->nt + 4));
  ENSURE(s, s->tet_rest, sizeof(double) * (12 * (size_t)s->nt + 1));
  ENSURE(s, s->tet_slot, sizeof(int) * (6 * (size_t)s->nt + 1));
  RC(upload(s, s->tri_v, d->tri2v, 3 * (size_t)s->nc));
  ENSURE(s, s->tri_n, sizeof(int) * (3 * (size_t)s->nc + 1));
  ENSURE(s, s->tri_rest, sizeof(double) * (8 * (size_t)s->nc + 1));
  ENSURE(s, s->tri_slot, sizeof(int) * (3 * (size_t)s->nc + 1));
  RC(upload(s, s->hinge_v, d->hinge2v, 4 * (size_t)s->nh));
  ENSURE(s, s->hinge_n, sizeof(int) * (4 * (size_t)s->nh + 1));
  ENSURE(s, s->hinge_rest, sizeof(double) * (2 * (size_t)s->nh + 1));
  ENSURE(s, s->hinge_slot, sizeof(int) * (6 * (size_t)s->nh + 1));
  RC(upload(s, s->body_kv, kv.data(), s->nb));
  ENSURE(s, s->body_slot, sizeof(int) * (6 * (size_t)s->nb + 1));
  RC(upload(s, s->stri, d->surf_tri2v, 3 * (size_t)s->nst));
  RC(upload(s, s->sedge, d->surf_edge2v, 2 * (size_t)s->nse));
  RC(upload(s, s->svert, d->surf_verts, s->nsv));
  RC(upload(s, s->planes, d->planes, 4 * (size_t)s->npl));
  ENSURE(s, s->status, 64);
  CK(s, cudaMemsetAsync(s->status.p, 0, 64, s->stream));
  ENSURE(s, s->P, sizeof(double) * (3 * (size_t)nv + 1));

  // per-element material inputs (temporaries)
  gbuf tmp[9];
  const bool bw = d->cloth_model == 1;
  // Baraff-Witkin: the second membrane constant is the shear stiffness
  struct { const double* p; size_t n; } mats[9] = {{d->tet_E, (size_t)s->nt},     {d->tet_nu, (size_t)s->nt},
                                                  {d->tet_rho, (size_t)s->nt},   {d->tri_E, (size_t)s->nc},
                                                  {bw ? d->tri_shear : d->tri_nu, (size_t)s->nc},
                                                  {d->tri_thick, (size_t)s->nc}, {d->tri_rho, (size_t)s->nc},
                                                  {d->hinge_kb, (size_t)s->nh},  {nullptr, 0}};
  yasps_status rc = YASPS_OK;
  for (int k = 0; k < 8 && rc == YASPS_OK; ++k) rc = upload(s, tmp[k], mats[k].p, mats[k].n);
  if (rc == YASPS_OK) rc = upload(s, s->tet_E, d->tet_E, (size_t)s->nt);
  if (rc == YASPS_OK) rc = upload(s, s->tet_nu, d->tet_nu, (size_t)s->nt);
  s->cloth_model = bw ? 1 : 0;
  if (rc == YASPS_OK)
    rc = setup_rest(s, as<double>(tmp[0]), as<double>(tmp[1]), as<double>(tmp[2]), as<double>(tmp[3]),
                    as<double>(tmp[4]), as<double>(tmp[5]), as<double>(tmp[6]), as<double>(tmp[7]));
  for (auto& b : tmp) release(s, b);
  RC(rc);
  int bits = 0;
  RC(read_status(s, &bits));
  if (bits) SYS_FAIL(s, YASPS_E_INVAL, "degenerate rest element or elastic element on an affine-body vertex");
  RC(static_sparsity(s));
  RC(alloc_hessian(s));
  // no contact pairs yet
  s->npt = s->nee = s->npg = 0;
  RC(build_dynamic_bsr(s));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

yasps_status yasps_build_system(const yasps_scene_desc* scene, const yasps_params* params,
                                const yasps_allocator* allocator, void* cuda_stream, yasps_system** out) {
  if (!out || !scene || !params) {
    g_build_error = "null argument";
    return YASPS_E_INVAL;
  }
  *out = nullptr;
  yasps_system* s = new yasps_system();
  s->prm = *params;
  s->stream = (cudaStream_t)cuda_stream;
  if (allocator && allocator->alloc && allocator->free) {
    s->allocator = *allocator;
    s->have_allocator = true;
  }
  for (auto& e : s->ev) cudaEventCreate(&e);
  yasps_status rc = build_impl(s, scene);
  if (rc != YASPS_OK) {
    g_build_error = s->err;
    yasps_destroy(s);
    return rc;
  }
  *out = s;
  return YASPS_OK;
}

void yasps_destroy(yasps_system* s) {
  if (!s) return;
  prof_resolve(s);
  for (auto e : s->prof_pool) cudaEventDestroy(e);
  std::vector<gbuf*> bufs;
  all_bufs(s, bufs);
  for (gbuf* b : bufs) release(s, *b);
  cudaStreamSynchronize(s->stream);
  for (auto& e : s->ev)
    if (e) cudaEventDestroy(e);
  delete s;
}

yasps_status yasps_set_params(yasps_system* s, const yasps_params* p) {
  if (!s || !p) return YASPS_E_INVAL;
  const int old = s->hess_precision;
  s->prm = *p;
  if ((p->precision == 1 ? 1 : 0) != old) {
    release(s, s->diag); release(s, s->Hs.vals); release(s, s->Hd.vals); release(s, s->minv);
    RC(alloc_hessian(s));
  }
  return YASPS_OK;
}

yasps_status yasps_get_sizes(const yasps_system* s, int* n_nodes, int* n_free, int* n_verts) {
  if (!s) return YASPS_E_INVAL;
  if (n_nodes) *n_nodes = s->nn;
  if (n_free) *n_free = s->nfree;
  if (n_verts) *n_verts = s->nv;
  return YASPS_OK;
}

yasps_status yasps_initial_state(yasps_system* s, const double* vel0, double* x_dev, double* v_dev) {
  if (!s || !x_dev || !v_dev) return YASPS_E_INVAL;
  std::vector<double> rest(3 * (size_t)s->nv), vr(3 * (size_t)s->nv);
  std::vector<int> vnode(s->nv), vbody(s->nv);
  CK(s, cudaMemcpyAsync(rest.data(), s->rest.p, sizeof(double) * rest.size(), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaMemcpyAsync(vr.data(), s->vr.p, sizeof(double) * vr.size(), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaMemcpyAsync(vnode.data(), s->vnode.p, sizeof(int) * s->nv, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaMemcpyAsync(vbody.data(), s->vbody.p, sizeof(int) * s->nv, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  std::vector<double> x(3 * (size_t)s->nn, 0.0), v(3 * (size_t)s->nn, 0.0);
  std::vector<int> cnt(s->nb, 0);
  for (int i = 0; i < s->nv; ++i) {
    const int n = vnode[i];
    if (n < 0 || vbody[i] <= -2) continue;  // fixed, or embedded (its cage carries the state)
    if (vbody[i] < 0) {
      for (int c = 0; c < 3; ++c) {
        x[3 * n + c] = rest[3 * i + c];
        v[3 * n + c] = vel0 ? vel0[3 * i + c] : 0.0;
      }
    } else {
      const int b = vbody[i];
      for (int c = 0; c < 3; ++c) {
        x[3 * n + c] = rest[3 * i + c] - vr[3 * i + c];  // t = body centre
        if (vel0) v[3 * n + c] += vel0[3 * i + c];
      }
      for (int k = 0; k < 3; ++k) x[3 * (n + 1 + k) + k] = 1.0;  // A = I
      cnt[b]++;
    }
  }
  for (int b = 0; b < s->nb; ++b) {
    const int n = s->nfree + 4 * b;
    for (int c = 0; c < 3; ++c) v[3 * n + c] /= std::max(cnt[b], 1);
  }
  CK(s, cudaMemcpyAsync(x_dev, x.data(), sizeof(double) * x.size(), cudaMemcpyHostToDevice, s->stream));
  CK(s, cudaMemcpyAsync(v_dev, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

yasps_status yasps_vertex_positions(yasps_system* s, const double* x_dev, double* P_dev) {
  if (!s || !x_dev || !P_dev) return YASPS_E_INVAL;
  return launch_positions(s, x_dev, P_dev);
}

yasps_status yasps_xtilde(yasps_system* s, const double* xt, const double* vt, double* xtil) {
  if (!s || !xt || !vt || !xtil) return YASPS_E_INVAL;
  return launch_xtilde(s, xt, vt, xtil);
}

yasps_status yasps_detect_pairs(yasps_system* s, const double* x_dev, int* n_pt, int* n_ee, int* n_pg) {
  if (!s || !x_dev) return YASPS_E_INVAL;
  RC(launch_positions(s, x_dev, as<double>(s->P)));
  RC(detect_pairs(s, as<double>(s->P)));
  if (n_pt) *n_pt = s->npt;
  if (n_ee) *n_ee = s->nee;
  if (n_pg) *n_pg = s->npg;
  return YASPS_OK;
}

yasps_status yasps_export_pairs(yasps_system* s, int* pt, int* ee, int* pg) {
  if (!s) return YASPS_E_INVAL;
  if (pt && s->npt) CK(s, cudaMemcpyAsync(pt, s->pt.p, sizeof(int) * 3 * s->npt, cudaMemcpyDeviceToHost, s->stream));
  if (ee && s->nee) CK(s, cudaMemcpyAsync(ee, s->ee.p, sizeof(int) * 3 * s->nee, cudaMemcpyDeviceToHost, s->stream));
  if (pg && s->npg) CK(s, cudaMemcpyAsync(pg, s->pg.p, sizeof(int) * 3 * s->npg, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

static yasps_status energy_impl(yasps_system* s, const double* x, const double* xtil, double* E, double* terms,
                                bool on_candidates = false) {
  RC(launch_positions(s, x, as<double>(s->P)));
  double t[6] = {0, 0, 0, 0, 0, 0};
  RC(energy_static(s, x, xtil, t));
  if (on_candidates) RC(barrier_energy_candidates(s, as<double>(s->P), &t[5]));
  else RC(barrier_energy(s, as<double>(s->P), &t[5]));
  // compensated total
  ksum k{0.0, 0.0};
  for (int i = 0; i < 6; ++i) kadd(k, t[i]);
  *E = k.s + k.c;
  if (terms) std::memcpy(terms, t, sizeof t);
  if (!std::isfinite(*E)) SYS_FAIL(s, YASPS_E_NAN, "non-finite energy");
  return YASPS_OK;
}

yasps_status yasps_energy(yasps_system* s, const double* x_dev, const double* xtilde_dev, double* E, double* terms) {
  if (!s || !x_dev || !xtilde_dev || !E) return YASPS_E_INVAL;
  return energy_impl(s, x_dev, xtilde_dev, E, terms);
}

yasps_status yasps_assemble(yasps_system* s) {
  if (!s) return YASPS_E_INVAL;
  return build_dynamic_bsr(s);
}

static yasps_status eval_impl(yasps_system* s, const double* x, const double* xtil, int mask, int project) {
  RC(launch_positions(s, x, as<double>(s->P)));
  const size_t es = (s->hess_precision == 1) ? sizeof(float) : sizeof(double);
  ENSURE(s, s->Hd.vals, es * 9 * ((size_t)s->Hd.nnzb + 1));
  RC(zero_system(s));
  RC(launch_eval_static(s, x, xtil, mask, project));
  if (mask & YASPS_TERM_BARRIER) {
    const double es = (s->hess_precision == 1) ? 4.0 : 8.0;
    const double bytes = (double)(s->npt + s->nee + s->npg) * (12.0 + 4 * 24.0) + (double)s->nkeys * 4.0 +
                         es * 9.0 * ((double)s->Hd.nnzb + s->nn) + 24.0 * s->nn;
    cudaEvent_t pa = prof_begin(s);
    RC(launch_eval_barrier(s, project));
    prof_end(s, YASPS_STAGE_BARRIER, pa, bytes);
  }
  // the block-Jacobi preconditioner needs the mass-regularised full Hessian
  if (mask & YASPS_TERM_INERTIA) RC(launch_bjacobi(s));
  return YASPS_OK;
}

yasps_status yasps_eval_local(yasps_system* s, const double* x_dev, const double* xtilde_dev, int mask, int project) {
  if (!s || !x_dev || !xtilde_dev) return YASPS_E_INVAL;
  RC(eval_impl(s, x_dev, xtilde_dev, mask, project));
  int bits = 0;
  RC(read_status(s, &bits));
  if (bits & (DEV_NAN | DEV_BADINDEX)) SYS_FAIL(s, YASPS_E_NAN, "device error during local evaluation");
  // an exact (unprojected) Hessian may have indefinite diagonal blocks: the
  // assembly stands, only the block-Jacobi preconditioner is then not built
  if (project && (bits & DEV_INDEFINITE))
    SYS_FAIL(s, YASPS_E_NAN, "projected Hessian has a diagonal block that is not positive definite");
  return YASPS_OK;
}

yasps_status yasps_export_bsr(yasps_system* s, int which, int* nnzb, int* row_ptr, int* col, double* vals,
                              double* diag) {
  if (!s || !nnzb) return YASPS_E_INVAL;
  bsr_struct& B = which ? s->Hd : s->Hs;
  *nnzb = B.nnzb;
  if (row_ptr) CK(s, cudaMemcpyAsync(row_ptr, B.row_ptr.p, sizeof(int) * (s->nn + 1), cudaMemcpyDeviceToHost, s->stream));
  if (col && B.nnzb) CK(s, cudaMemcpyAsync(col, B.col.p, sizeof(int) * B.nnzb, cudaMemcpyDeviceToHost, s->stream));
  const bool f32 = s->hess_precision == 1;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  std::vector<char> tmpv, tmpd;
  if (vals && B.nnzb) {
    tmpv.resize(es * 9 * B.nnzb);
    CK(s, cudaMemcpyAsync(tmpv.data(), B.vals.p, tmpv.size(), cudaMemcpyDeviceToHost, s->stream));
  }
  if (diag && which == 0) {
    tmpd.resize(es * 9 * s->nn);
    CK(s, cudaMemcpyAsync(tmpd.data(), s->diag.p, tmpd.size(), cudaMemcpyDeviceToHost, s->stream));
  }
  CK(s, cudaStreamSynchronize(s->stream));
  auto conv = [&](const std::vector<char>& src, double* dst, size_t n) {
    for (size_t i = 0; i < n; ++i)
      dst[i] = f32 ? (double)reinterpret_cast<const float*>(src.data())[i] : reinterpret_cast<const double*>(src.data())[i];
  };
  if (vals && B.nnzb) conv(tmpv, vals, 9 * (size_t)B.nnzb);
  if (diag && which == 0) conv(tmpd, diag, 9 * (size_t)s->nn);
  return YASPS_OK;
}

yasps_status yasps_export_gradient(yasps_system* s, double* g_dev) {
  if (!s || !g_dev) return YASPS_E_INVAL;
  CK(s, cudaMemcpyAsync(g_dev, s->grad.p, sizeof(double) * 3 * s->nn, cudaMemcpyDeviceToDevice, s->stream));
  return YASPS_OK;
}

yasps_status yasps_spmv(yasps_system* s, const double* x_dev, double* y_dev) {
  if (!s || !x_dev || !y_dev) return YASPS_E_INVAL;
  return spmv64(s, x_dev, y_dev);
}

yasps_status yasps_pcg_solve(yasps_system* s, const double* rhs, double* p, double tol, int* iters, double* rel) {
  if (!s || !rhs || !p) return YASPS_E_INVAL;
  return pcg_solve(s, rhs, p, tol, s->prm.pcg_max_iter, iters, rel);
}

yasps_status yasps_ccd_bound(yasps_system* s, const double* x_dev, const double* p_dev, double* alpha) {
  if (!s || !x_dev || !p_dev || !alpha) return YASPS_E_INVAL;
  return ccd_bound(s, x_dev, p_dev, alpha);
}

yasps_status yasps_set_fixed_positions(yasps_system* s, const double* P) {
  if (!s || !P) return YASPS_E_INVAL;
  std::vector<int> fx(s->nfix);
  if (s->nfix) {
    CK(s, cudaMemcpyAsync(fx.data(), s->fixed.p, sizeof(int) * s->nfix, cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
  }
  for (int v : fx)
    CK(s, cudaMemcpyAsync(as<double>(s->xfix) + 3 * (size_t)v, P + 3 * (size_t)v, sizeof(double) * 3,
                          cudaMemcpyHostToDevice, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

yasps_status yasps_get_fixed_positions(yasps_system* s, double* P) {
  if (!s || !P) return YASPS_E_INVAL;
  CK(s, cudaMemcpyAsync(P, s->xfix.p, sizeof(double) * 3 * s->nv, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- time step
namespace {
__global__ void k_fixed_advance(int nfix, const int* __restrict__ fixed, const double* __restrict__ fv, double h,
                                double* __restrict__ xfix) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nfix) return;
  const int v = fixed[i];
  for (int c = 0; c < 3; ++c) xfix[3 * v + c] += h * fv[3 * i + c];
}
__global__ void k_axpy_out(int n, const double* __restrict__ x, double a, const double* __restrict__ p,
                           double* __restrict__ out) {  // out = x - a p
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[i] - a * p[i];
}
__global__ void k_scale_out(int n, double c, const double* __restrict__ p, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = c * p[i];
}
__global__ void k_velocity(int n, const double* __restrict__ x, const double* __restrict__ xt, double inv_h,
                           double* __restrict__ v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (x[i] - xt[i]) * inv_h;
}
}  // namespace

static float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

static yasps_status step_batched(yasps_system* s, double* x, double* v, yasps_step_stats* stats);

// Adaptive barrier stiffness at the start of a step (kappa_adaptive): pairs
// and their smallest distance at x; the first step with pairs balances the
// barrier gradient g_B (kappa = 1) against the gradient g_E of the other
// terms, argmin_k |g_E + k g_B| = -g_E.g_B / g_B.g_B, clamped to
// [kappa_min, kappa_max] (kappa_min before that step); later steps double
// kappa, up to kappa_max, when the smallest distance is below kappa_dmin and
// below the previous step's.  kappa is then frozen for the step.
// The bounds of the adaptive stiffness: kappa_min > 0 and kappa_max > 0 as
// given; kappa_min <= 0 takes the stiffness at which the barrier alone holds
// the weight of an average vertex (total mass / vertex count) at half the
// activation distance: the weight enters this potential as m h^2 |g| and the
// barrier as kappa |db/dd| = kappa 2 d |b'(d^2)|, so
// kappa_min = m h^2 |g| / (2 d |b'(d^2)|) at d = dhat / 2 (|g| = 0: standard
// gravity); kappa_max <= 0 takes 1e4 kappa_min.
static yasps_status kappa_bounds(yasps_system* s) {
  double lo = s->prm.kappa_min;
  if (!(lo > 0.0)) {
    std::vector<double> vm(std::max(s->nv, 1), 0.0);
    if (s->nv)
      CK(s, cudaMemcpyAsync(vm.data(), s->vmass.p, sizeof(double) * s->nv, cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    double m = 0.0;
    for (int v = 0; v < s->nv; ++v) m += vm[v];
    m /= std::max(s->nv, 1);
    const double* gv = s->prm.gravity;
    double gn = std::sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
    if (!(gn > 0.0)) gn = 9.80665;
    const double d = 0.5 * s->prm.dhat;
    const double db = barrier_db(d * d, s->prm.dhat * s->prm.dhat, s->prm.barrier_form);
    lo = m * s->prm.dt * s->prm.dt * gn / std::fabs(2.0 * d * db);
  }
  s->kappa_lo = lo;
  s->kappa_hi = s->prm.kappa_max > 0.0 ? s->prm.kappa_max : 1e4 * lo;
  return YASPS_OK;
}

static yasps_status kappa_update(yasps_system* s, const double* x, const double* xtil) {
  RC(launch_positions(s, x, as<double>(s->P)));
  RC(detect_pairs(s, as<double>(s->P)));
  double s2 = 0.0;
  RC(pairs_min_dist2(s, as<double>(s->P), &s2));
  const double dmin = std::sqrt(s2);
  if (!s->kappa_init) {
    RC(kappa_bounds(s));
    if (std::isfinite(dmin)) {
      const int n3 = 3 * s->nn;
      ENSURE(s, s->stepv[5], sizeof(double) * (n3 + 4));
      double* gE = as<double>(s->stepv[5]);
      RC(eval_impl(s, x, xtil, YASPS_TERM_ALL & ~YASPS_TERM_BARRIER, 0));
      CK(s, cudaMemcpyAsync(gE, s->grad.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s->stream));
      const double keep = s->prm.kappa;
      s->prm.kappa = 1.0;
      yasps_status rc = eval_impl(s, x, xtil, YASPS_TERM_BARRIER, 0);
      s->prm.kappa = keep;
      RC(rc);
      double num = 0.0, den = 0.0;
      RC(dot2(s, gE, as<double>(s->grad), n3, &num, &den));
      double k = den > 0.0 ? -num / den : s->kappa_lo;
      if (!(k >= s->kappa_lo)) k = s->kappa_lo;
      if (k > s->kappa_hi) k = s->kappa_hi;
      s->prm.kappa = k;
      s->kappa_init = true;
    } else {
      s->prm.kappa = s->kappa_lo;
    }
  } else if (dmin < (s->prm.kappa_dmin > 0.0 ? s->prm.kappa_dmin : 0.1 * s->prm.dhat) && dmin < s->kappa_dmin_prev) {
    s->prm.kappa = std::min(2.0 * s->prm.kappa, s->kappa_hi);
  }
  s->kappa_dmin_prev = dmin;
  return YASPS_OK;
}

extern "C" yasps_status yasps_get_kappa_state(yasps_system* s, double* kappa, int* initialised, double* dmin_prev,
                                              double* kappa_lo, double* kappa_hi) {
  if (!s) return YASPS_E_INVAL;
  RC(kappa_bounds(s));
  if (kappa) *kappa = s->prm.kappa;
  if (initialised) *initialised = s->kappa_init ? 1 : 0;
  if (dmin_prev) *dmin_prev = s->kappa_dmin_prev;
  if (kappa_lo) *kappa_lo = s->kappa_lo;
  if (kappa_hi) *kappa_hi = s->kappa_hi;
  return YASPS_OK;
}

extern "C" yasps_status yasps_set_kappa_state(yasps_system* s, double kappa, int initialised, double dmin_prev) {
  if (!s || !(kappa >= 0.0) || std::isnan(dmin_prev)) return YASPS_E_INVAL;
  RC(kappa_bounds(s));
  s->prm.kappa = kappa;
  s->kappa_init = initialised != 0;
  s->kappa_dmin_prev = dmin_prev;
  return YASPS_OK;
}

extern "C" yasps_status yasps_newton_trace(const yasps_system* s, int capacity, yasps_newton_record* out, int* count) {
  if (!s || capacity < 0 || (capacity > 0 && !out)) return YASPS_E_INVAL;
  const int n = (int)s->trace.size();
  for (int k = 0; k < std::min(n, capacity); ++k) out[k] = s->trace[k];
  if (count) *count = n;
  return YASPS_OK;
}

extern "C" yasps_status yasps_newton_trace_enable(yasps_system* s, int enable) {
  if (!s) return YASPS_E_INVAL;
  s->trace_smin = enable != 0;
  return YASPS_OK;
}

extern "C" yasps_status yasps_step(yasps_system* s, double* x, double* v, yasps_step_stats* stats) {
  if (!s || !x || !v) return YASPS_E_INVAL;
  if (s->nscene > 1) return step_batched(s, x, v, stats);
  const int n3 = 3 * s->nn;
  const double h = s->prm.dt;
  yasps_step_stats st{};
  for (int k = 0; k < 4; ++k) ENSURE(s, s->stepv[k], sizeof(double) * (n3 + 4));
  double* xt = as<double>(s->stepv[0]);
  double* xtil = as<double>(s->stepv[1]);
  double* p = as<double>(s->stepv[2]);
  gbuf& trial = s->vec[7];
  ENSURE(s, trial, sizeof(double) * (n3 + 4));
  double* xtrial = as<double>(trial);
  ENSURE(s, s->vec[9], sizeof(double) * (n3 + 4));
  double* p0 = as<double>(s->vec[9]);
  if (s->nfix) {
    k_fixed_advance<<<blocks_for(s->nfix, 128), 128, 0, s->stream>>>(s->nfix, as<int>(s->fixed), as<double>(s->fixvel),
                                                                    h, as<double>(s->xfix));
    LAUNCH_CHECK(s, "k_fixed_advance");
  }
  CK(s, cudaMemcpyAsync(xt, x, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s->stream));
  RC(launch_xtilde(s, x, v, xtil));
  s->cand_valid = false;
  s->trace.clear();
  if (s->prm.kappa_adaptive) RC(kappa_update(s, x, xtil));
  st.kappa = s->prm.kappa;
  yasps_status rc = YASPS_OK;
  int it = 0;
  double pinf = 0.0, alpha = 1.0;
  double E_acc = 0.0;  // energy at x after the last accepted line search
  bool have_E = false;
  for (it = 0; it < s->prm.newton_max_iter; ++it) {
    cudaEventRecord(s->ev[0], s->stream);
    cudaEvent_t pd = prof_begin(s);
    RC(launch_positions(s, x, as<double>(s->P)));
    // after the first iteration, x lies on the previous iteration's swept
    // segment, so its active pairs are among that segment's candidates
    if (it > 0 && s->cand_valid) RC(detect_from_candidates(s, as<double>(s->P)));
    else RC(detect_pairs(s, as<double>(s->P)));
    prof_end(s, YASPS_STAGE_DETECT, pd, 0.0);
    cudaEvent_t pe = prof_begin(s);
    RC(eval_impl(s, x, xtil, YASPS_TERM_ALL, 1));
    prof_end(s, YASPS_STAGE_EVAL, pe, 0.0);
    cudaEventRecord(s->ev[1], s->stream);
    int pit = 0;
    double rel = 0.0;
    // warm start from the part of the last direction the line search left
    const double* x0 = nullptr;
    if (s->prm.pcg_warm_start && it > 0 && alpha < 1.0) {
      k_scale_out<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, 1.0 - alpha, p, p0);
      LAUNCH_CHECK(s, "k_scale_out");
      x0 = p0;
    }
    rc = pcg_solve(s, as<double>(s->grad), p, s->prm.pcg_rel_tol, s->prm.pcg_max_iter, &pit, &rel, x0);
    st.pcg_iters_total += pit;
    if (rc == YASPS_E_NOCONV) rc = YASPS_OK;  // inexact Newton: keep the last iterate
    if (rc != YASPS_OK) break;
    cudaEventRecord(s->ev[2], s->stream);
    int bits = 0;
    RC(read_status(s, &bits));
    if (bits & (DEV_NAN | DEV_BADINDEX | DEV_INDEFINITE)) {
      s->err = "device error during evaluation";
      rc = YASPS_E_NAN;
      break;
    }
    yasps_newton_record rec{};
    rec.pcg_iters = pit;
    rec.pcg_rel_res = rel;
    rec.n_pt = s->npt; rec.n_ee = s->nee; rec.n_pg = s->npg;
    rec.s_min = -1.0;
    if (s->trace_smin) RC(pairs_min_dist2(s, as<double>(s->P), &rec.s_min));
    RC(inf_norm(s, p, n3, &pinf, &rec.pinf_node));
    rec.pinf_node /= 3;
    rec.p_inf = pinf;
    double gp = 0.0, pp = 0.0;
    RC(dot2(s, as<double>(s->grad), p, n3, &gp, &pp));
    rec.g_dot_p = gp;
    if (s->trace_smin) {
      CK(s, cudaMemcpyAsync(rec.p_at_max, p + 3 * (size_t)rec.pinf_node, sizeof(double) * 3, cudaMemcpyDeviceToHost,
                            s->stream));
      CK(s, cudaStreamSynchronize(s->stream));
    }
    s->trace.push_back(rec);
    if (!std::isfinite(pinf)) {
      s->err = "non-finite Newton direction";
      rc = YASPS_E_NAN;
      break;
    }
    st.t_eval_ms += elapsed(s->ev[0], s->ev[1]);
    st.t_pcg_ms += elapsed(s->ev[1], s->ev[2]);
    st.n_pt = s->npt; st.n_ee = s->nee; st.n_pg = s->npg;
    if (pinf <= s->prm.newton_tol) break;
    cudaEventRecord(s->ev[3], s->stream);
    cudaEvent_t pc = prof_begin(s);
    RC(ccd_bound(s, x, p, &alpha));
    prof_end(s, YASPS_STAGE_CCD, pc, 0.0);
    s->trace.back().alpha_ccd = alpha;
    s->trace.back().n_cand_pt = s->ncpt;
    s->trace.back().n_cand_ee = s->ncee;
    st.n_cand_pt = s->ncpt;
    st.n_cand_ee = s->ncee;
    cudaEventRecord(s->ev[4], s->stream);
    cudaEvent_t pl = prof_begin(s);
    // E(x) is the energy the previous line search accepted (the same sum over
    // the same active pairs, since both candidate sets hold every pair within
    // dhat of x); only the first iteration evaluates it
    double E0 = E_acc, E1 = 0.0;
    if (!have_E) RC(energy_impl(s, x, xtil, &E0, nullptr, true));
    int ls = 0;
    for (ls = 0; ls < s->prm.ls_max_iter; ++ls) {
      k_axpy_out<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, x, alpha, p, xtrial);
      LAUNCH_CHECK(s, "k_axpy_out");
      RC(energy_impl(s, xtrial, xtil, &E1, nullptr, true));
      // a decrease, up to the rounding of the energy sums: FP64 element
      // energies do not resolve differences below 1e-12 |E0|
      if (E1 <= E0 + 1e-12 * std::fabs(E0) - s->prm.ls_armijo * alpha * gp) break;
      alpha *= 0.5;
    }
    prof_end(s, YASPS_STAGE_LS, pl, 0.0);
    cudaEventRecord(s->ev[5], s->stream);
    cudaEventSynchronize(s->ev[5]);
    st.t_ccd_ms += elapsed(s->ev[3], s->ev[4]);
    st.t_ls_ms += elapsed(s->ev[4], s->ev[5]);
    s->trace.back().ls_halvings = ls;
    s->trace.back().alpha = ls == s->prm.ls_max_iter ? 0.0 : alpha;
    s->trace.back().E0 = E0;
    s->trace.back().E1 = E1;
    if (ls == s->prm.ls_max_iter) {
      s->err = "line search found no decreasing step";
      rc = YASPS_E_LINESEARCH;
      break;
    }
    CK(s, cudaMemcpyAsync(x, xtrial, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s->stream));
    st.alpha_last = alpha;
    E_acc = E1;
    have_E = true;
  }
  if (rc == YASPS_OK && it == s->prm.newton_max_iter) {
    s->err = "Newton hit its iteration cap";
    rc = YASPS_E_NOCONV;
  }
  k_velocity<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, x, xt, 1.0 / h, v);
  LAUNCH_CHECK(s, "k_velocity");
  CK(s, cudaStreamSynchronize(s->stream));
  st.newton_iters = it;
  st.p_inf = pinf;
  st.status = rc;
  if (stats) *stats = st;
  return rc;
}

// ---------------------------------------------------------------- adjoint (form 2)
namespace {
__global__ void k_adj_rhs(int n, const double* __restrict__ xbar, const double* __restrict__ vbar, double inv_h,
                          double* __restrict__ rhs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = xbar[i] + vbar[i] * inv_h;
}
// y = M x: free nodes m I3, bodies their 4x4 mass matrix (x) I3
__global__ void k_mass_apply(int nfree, int nb, const double* __restrict__ nodemass, const double* __restrict__ x,
                             double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nfree) {
    const double m = nodemass[i];
    for (int c = 0; c < 3; ++c) y[3 * (size_t)i + c] = m * x[3 * (size_t)i + c];
  } else if (i < nfree + nb) {
    const int b = i - nfree;
    const double* M = nodemass + nfree + 16 * (size_t)b;
    const size_t o = 3 * ((size_t)nfree + 4 * (size_t)b);
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += M[4 * a + k] * x[o + 3 * k + c];
        y[o + 3 * a + c] = acc;
      }
  }
}
__global__ void k_adj_out(int n, const double* __restrict__ Ml, const double* __restrict__ vbar, double h,
                          double* __restrict__ xbar_prev, double* __restrict__ vbar_prev) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double m = Ml[i];
    xbar_prev[i] = m - vbar[i] / h;
    vbar_prev[i] = h * m;
  }
}
}  // namespace

extern "C" yasps_status yasps_set_tet_young(yasps_system* s, const double* E_dev) {
  if (!s || (!E_dev && s->nt > 0)) return YASPS_E_INVAL;
  RC(launch_set_young(s, E_dev));
  int bits = 0;
  RC(read_status(s, &bits));
  if (bits & DEV_NAN) SYS_FAIL(s, YASPS_E_INVAL, "Young's moduli must be positive and finite");
  return YASPS_OK;
}

extern "C" yasps_status yasps_adjoint_step(yasps_system* s, const double* x_t, const double* v_t, const double* x_next,
                                           const double* xbar, const double* vbar, double* xbar_prev,
                                           double* vbar_prev, double* Ebar, double pcg_rel_tol, int* pcg_iters,
                                           double* rel_res) {
  if (!s || !x_t || !v_t || !x_next || !xbar || !vbar || !xbar_prev || !vbar_prev || (!Ebar && s->nt > 0))
    return YASPS_E_INVAL;
  const int n3 = 3 * s->nn;
  const double h = s->prm.dt;
  ENSURE(s, s->stepv[1], sizeof(double) * (n3 + 4));
  ENSURE(s, s->stepv[2], sizeof(double) * (n3 + 4));
  ENSURE(s, s->stepv[4], sizeof(double) * (n3 + 4));
  ENSURE(s, s->stepv[5], sizeof(double) * (n3 + 4));
  double* xtil = as<double>(s->stepv[1]);
  double* Ml = as<double>(s->stepv[2]);
  double* rhs = as<double>(s->stepv[4]);
  double* lam = as<double>(s->stepv[5]);
  RC(launch_xtilde(s, x_t, v_t, xtil));
  // pairs and the EXACT (unprojected) Hessian at the step's solution
  RC(launch_positions(s, x_next, as<double>(s->P)));
  RC(detect_pairs(s, as<double>(s->P)));
  RC(eval_impl(s, x_next, xtil, YASPS_TERM_ALL, 0));
  int bits = 0;
  RC(read_status(s, &bits));
  if (bits & (DEV_NAN | DEV_BADINDEX | DEV_INDEFINITE))
    SYS_FAIL(s, YASPS_E_NAN, "exact Hessian at the step solution has a non-positive diagonal block");
  k_adj_rhs<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, xbar, vbar, 1.0 / h, rhs);
  LAUNCH_CHECK(s, "k_adj_rhs");
  int it = 0;
  double rel = 0.0;
  RC(pcg_solve(s, rhs, lam, pcg_rel_tol, s->prm.pcg_max_iter, &it, &rel));
  if (pcg_iters) *pcg_iters = it;
  if (rel_res) *rel_res = rel;
  k_mass_apply<<<blocks_for(std::max(s->nfree + s->nb, 1), 256), 256, 0, s->stream>>>(
      s->nfree, s->nb, as<double>(s->nodemass), lam, Ml);
  LAUNCH_CHECK(s, "k_mass_apply");
  k_adj_out<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, Ml, vbar, h, xbar_prev, vbar_prev);
  LAUNCH_CHECK(s, "k_adj_out");
  RC(launch_snh_young_adj(s, as<double>(s->P), lam, h * h, Ebar));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

// ---------------------------------------------------------------- batches
namespace {
// per-scene max |p| over the scene's nodes (bit patterns of non-negative doubles order like the values)
__global__ void k_absmax_scene(int nn, const double* __restrict__ p, const int* __restrict__ node_scene,
                               unsigned long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double m = fmax(fabs(p[3 * (size_t)i]), fmax(fabs(p[3 * (size_t)i + 1]), fabs(p[3 * (size_t)i + 2])));
  atomicMax(&out[node_scene[i]], (unsigned long long)__double_as_longlong(m));
}
// zero the gradient of the scenes whose Newton iteration has finished: their
// PCG then starts converged (r0 = 0) and their step stays 0
__global__ void k_zero_done(int nn, double* __restrict__ g, const int* __restrict__ node_scene,
                            const int* __restrict__ done) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn || !done[node_scene[i]]) return;
  g[3 * (size_t)i] = 0.0;
  g[3 * (size_t)i + 1] = 0.0;
  g[3 * (size_t)i + 2] = 0.0;
}
// out = x - alpha[scene] p
__global__ void k_axpy_scene(int nn, const double* __restrict__ x, const double* __restrict__ alpha,
                             const int* __restrict__ node_scene, const double* __restrict__ p, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double a = alpha[node_scene[i]];
  for (int c = 0; c < 3; ++c) out[3 * (size_t)i + c] = x[3 * (size_t)i + c] - a * p[3 * (size_t)i + c];
}
}  // namespace

// incremental potential per scene at x (swept candidates for the barrier)
static yasps_status energy_scenes(yasps_system* s, const double* x, const double* xtil, std::vector<double>& E) {
  const int ns = s->nscene;
  double* acc = as<double>(s->scene_buf) + 2 * (size_t)ns;
  CK(s, cudaMemsetAsync(acc, 0, sizeof(double) * ns, s->stream));
  RC(launch_positions(s, x, as<double>(s->P)));
  RC(energy_static(s, x, xtil, nullptr, acc));
  RC(barrier_energy_candidates(s, as<double>(s->P), nullptr, acc));
  E.assign(ns, 0.0);
  CK(s, cudaMemcpyAsync(E.data(), acc, sizeof(double) * ns, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return YASPS_OK;
}

// One implicit step of every scene of a batch.  The scenes share the launches
// (detection, evaluation, assembly, one PCG with per-scene alpha / beta /
// stopping test, CCD, energies) but every decision is per scene: a scene whose
// Newton step is below newton_tol stops moving (its step length is 0), each
// scene has its own CCD bound and its own backtracking, so each scene follows
// the trajectory it would follow alone.
static yasps_status step_batched(yasps_system* s, double* x, double* v, yasps_step_stats* stats) {
  const int n3 = 3 * s->nn, ns = s->nscene;
  const double h = s->prm.dt;
  if (s->prm.kappa_adaptive) SYS_FAIL(s, YASPS_E_INVAL, "adaptive kappa is available for single scenes only");
  s->trace.clear();
  yasps_step_stats st{};
  st.kappa = s->prm.kappa;
  for (int k = 0; k < 4; ++k) ENSURE(s, s->stepv[k], sizeof(double) * (n3 + 4));
  double* xt = as<double>(s->stepv[0]);
  double* xtil = as<double>(s->stepv[1]);
  double* p = as<double>(s->stepv[2]);
  gbuf& trial = s->vec[7];
  ENSURE(s, trial, sizeof(double) * (n3 + 4));
  double* xtrial = as<double>(trial);
  double* sb = as<double>(s->scene_buf);
  double* alpha_dev = sb + 5 * (size_t)ns;
  unsigned long long* pmax_dev = reinterpret_cast<unsigned long long*>(sb + 4 * (size_t)ns);
  if (s->nfix) {
    k_fixed_advance<<<blocks_for(s->nfix, 128), 128, 0, s->stream>>>(s->nfix, as<int>(s->fixed), as<double>(s->fixvel),
                                                                    h, as<double>(s->xfix));
    LAUNCH_CHECK(s, "k_fixed_advance");
  }
  CK(s, cudaMemcpyAsync(xt, x, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s->stream));
  RC(launch_xtilde(s, x, v, xtil));
  s->cand_valid = false;
  s->scene_newton.assign(ns, 0);
  s->scene_status.assign(ns, YASPS_OK);
  std::vector<int> pcg_tot(ns, 0);
  std::vector<char> done(ns, 0);
  std::vector<double> pinf(ns), alpha(ns), E0, E1;
  std::vector<unsigned long long> pbits(ns);
  yasps_status rc = YASPS_OK;
  int it = 0;
  for (it = 0; it < s->prm.newton_max_iter; ++it) {
    cudaEvent_t pd = prof_begin(s);
    RC(launch_positions(s, x, as<double>(s->P)));
    if (it > 0 && s->cand_valid) RC(detect_from_candidates(s, as<double>(s->P)));
    else RC(detect_pairs(s, as<double>(s->P)));
    prof_end(s, YASPS_STAGE_DETECT, pd, 0.0);
    cudaEvent_t pe = prof_begin(s);
    RC(eval_impl(s, x, xtil, YASPS_TERM_ALL, 1));
    prof_end(s, YASPS_STAGE_EVAL, pe, 0.0);
    if (it > 0) {
      std::vector<int> dm(done.begin(), done.end());
      int* done_dev = reinterpret_cast<int*>(sb + 6 * (size_t)ns);
      CK(s, cudaMemcpyAsync(done_dev, dm.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s->stream));
      k_zero_done<<<blocks_for(s->nn, 256), 256, 0, s->stream>>>(s->nn, as<double>(s->grad), as<int>(s->node_scene),
                                                                done_dev);
      LAUNCH_CHECK(s, "k_zero_done");
    }
    int pit = 0;
    double rel = 0.0;
    rc = pcg_solve(s, as<double>(s->grad), p, s->prm.pcg_rel_tol, s->prm.pcg_max_iter, &pit, &rel);
    st.pcg_iters_total += pit;
    for (int k = 0; k < ns; ++k)
      if (!done[k] && (int)s->scene_pcg.size() == ns) pcg_tot[k] += s->scene_pcg[k];
    if (rc == YASPS_E_NOCONV) rc = YASPS_OK;  // inexact Newton: keep the last iterate
    if (rc != YASPS_OK) break;
    int bits = 0;
    RC(read_status(s, &bits));
    if (bits & (DEV_NAN | DEV_BADINDEX | DEV_INDEFINITE)) {
      s->err = "device error during evaluation";
      rc = YASPS_E_NAN;
      break;
    }
    // per-scene Newton convergence
    CK(s, cudaMemsetAsync(pmax_dev, 0, sizeof(double) * ns, s->stream));
    k_absmax_scene<<<blocks_for(s->nn, 256), 256, 0, s->stream>>>(s->nn, p, as<int>(s->node_scene), pmax_dev);
    LAUNCH_CHECK(s, "k_absmax_scene");
    CK(s, cudaMemcpyAsync(pbits.data(), pmax_dev, sizeof(double) * ns, cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    bool any = false;
    for (int k = 0; k < ns; ++k) {
      std::memcpy(&pinf[k], &pbits[k], sizeof(double));
      if (!std::isfinite(pinf[k])) {
        s->err = "non-finite Newton direction";
        return YASPS_E_NAN;
      }
      if (!done[k] && pinf[k] <= s->prm.newton_tol) {
        done[k] = 1;
        s->scene_newton[k] = it;
      }
      any |= !done[k];
    }
    st.p_inf = *std::max_element(pinf.begin(), pinf.end());
    st.n_pt = s->npt; st.n_ee = s->nee; st.n_pg = s->npg;
    if (!any) break;
    // per-scene CCD bound, then per-scene backtracking from it
    cudaEvent_t pc = prof_begin(s);
    RC(swept_candidates(s, x, p));
    RC(ccd_candidates(s, alpha.data()));
    prof_end(s, YASPS_STAGE_CCD, pc, 0.0);
    for (int k = 0; k < ns; ++k)
      if (done[k]) alpha[k] = 0.0;
    cudaEvent_t pl = prof_begin(s);
    if (it == 0) RC(energy_scenes(s, x, xtil, E0));  // later: the energies the last line search accepted
    std::vector<char> acc(ns, 0);
    for (int k = 0; k < ns; ++k) acc[k] = done[k];
    int ls = 0;
    for (ls = 0; ls < s->prm.ls_max_iter; ++ls) {
      CK(s, cudaMemcpyAsync(alpha_dev, alpha.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s->stream));
      k_axpy_scene<<<blocks_for(s->nn, 256), 256, 0, s->stream>>>(s->nn, x, alpha_dev, as<int>(s->node_scene), p,
                                                                 xtrial);
      LAUNCH_CHECK(s, "k_axpy_scene");
      RC(energy_scenes(s, xtrial, xtil, E1));
      bool all = true;
      for (int k = 0; k < ns; ++k) {
        if (acc[k]) continue;
        // a decrease, up to the rounding of the energy sums
        if (E1[k] <= E0[k] + 1e-12 * std::fabs(E0[k])) acc[k] = 1;
        else alpha[k] *= 0.5;
        all &= acc[k] != 0;
      }
      if (all) break;
    }
    if (ls == s->prm.ls_max_iter) {
      // scenes whose line search found no decreasing step stop where they are
      for (int k = 0; k < ns; ++k)
        if (!acc[k]) {
          alpha[k] = 0.0;
          done[k] = 1;
          s->scene_newton[k] = it;
          s->scene_status[k] = YASPS_E_LINESEARCH;
        }
      CK(s, cudaMemcpyAsync(alpha_dev, alpha.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s->stream));
      k_axpy_scene<<<blocks_for(s->nn, 256), 256, 0, s->stream>>>(s->nn, x, alpha_dev, as<int>(s->node_scene), p,
                                                                 xtrial);
      LAUNCH_CHECK(s, "k_axpy_scene");
    }
    prof_end(s, YASPS_STAGE_LS, pl, 0.0);
    st.n_cand_pt = s->ncpt;
    st.n_cand_ee = s->ncee;
    // energies at the new x: accepted trials; scenes that did not move keep E0
    for (int k = 0; k < ns; ++k)
      if (alpha[k] != 0.0) E0[k] = E1[k];
    CK(s, cudaMemcpyAsync(x, xtrial, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s->stream));
    st.alpha_last = *std::max_element(alpha.begin(), alpha.end());
  }
  for (int k = 0; k < ns; ++k)
    if (!done[k]) {
      s->scene_newton[k] = it;
      if (rc == YASPS_OK) s->scene_status[k] = YASPS_E_NOCONV;
    }
  s->scene_pcg = pcg_tot;
  if (rc == YASPS_OK)
    for (int k = 0; k < ns; ++k)
      if (s->scene_status[k] != YASPS_OK) {
        rc = s->scene_status[k];
        s->err = rc == YASPS_E_LINESEARCH ? "line search found no decreasing step in a scene"
                                          : "Newton hit its iteration cap in a scene";
        break;
      }
  k_velocity<<<blocks_for(n3, 256), 256, 0, s->stream>>>(n3, x, xt, 1.0 / h, v);
  LAUNCH_CHECK(s, "k_velocity");
  CK(s, cudaStreamSynchronize(s->stream));
  st.newton_iters = it;
  st.status = rc;
  if (stats) *stats = st;
  return rc;
}

extern "C" yasps_status yasps_scene_stats(const yasps_system* s, int* newton_iters, int* pcg_iters, int* status) {
  if (!s) return YASPS_E_INVAL;
  for (int k = 0; k < s->nscene; ++k) {
    const bool have = (int)s->scene_newton.size() == s->nscene;
    if (newton_iters) newton_iters[k] = have ? s->scene_newton[k] : 0;
    if (pcg_iters) pcg_iters[k] = (int)s->scene_pcg.size() == s->nscene ? s->scene_pcg[k] : 0;
    if (status) status[k] = (int)s->scene_status.size() == s->nscene ? s->scene_status[k] : 0;
  }
  return YASPS_OK;
}

extern "C" yasps_status yasps_autotune_pcg(yasps_system* s, int iters, int* variant, double* us_per_iter) {
  if (!s) return YASPS_E_INVAL;
  if (s->hess_precision < 0) SYS_FAIL(s, YASPS_E_INVAL, "nothing assembled yet");
  return autotune_pcg(s, iters, variant, us_per_iter);
}

extern "C" yasps_status yasps_set_wait_limit(yasps_system* s, long long polls, int unmet_next) {
  if (!s || polls < 0) return YASPS_E_INVAL;
  s->wait_limit = polls;
  s->wait_unmet = unmet_next != 0;
  return YASPS_OK;
}

extern "C" yasps_status yasps_set_pcg_variant(yasps_system* s, int variant) {
  if (!s || variant < 0 || variant >= YASPS_PCG_VARIANTS) return YASPS_E_INVAL;
  s->pcg_variant = variant;
  return YASPS_OK;
}
