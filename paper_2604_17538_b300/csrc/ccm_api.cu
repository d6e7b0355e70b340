// Host side of the C ABI declared in include/ccm.h: contexts, resident
// geometry, batches (pair plans) and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ccm.h"
#include "ccm_device.cuh"
#include "ccm_host.h"
#include "ccm_launch.h"

namespace ccm {

std::atomic<long long> g_kernel_launches{0};


// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

ccm_status fail(ccm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

ccm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CCM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
template <class T>
static ccm_status upload(DevBuf& b, const std::vector<T>& h, const char* what) {
  const size_t bytes = h.size() * sizeof(T);
  if (bytes > b.bytes) {
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.ptr, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) return fail(CCM_ERR_OOM, "%s: cudaMalloc(%zu): %s", what, bytes,
                                      cudaGetErrorString(e));
    b.bytes = std::max<size_t>(bytes, 256);
  }
  if (bytes) CCM_CUDA(cudaMemcpy(b.ptr, h.data(), bytes, cudaMemcpyHostToDevice), what);
  return CCM_OK;
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

DevGeom Context::dev_geom() const {
  DevGeom g;
  g.pieces = static_cast<const PieceRec*>(d_pieces.ptr);
  g.bodies = static_cast<const BodyRec*>(d_bodies.ptr);
  g.verts = static_cast<const float4*>(d_verts.ptr);
  g.planes = static_cast<const float4*>(d_planes.ptr);
  g.edges = static_cast<const uint32_t*>(d_edges.ptr);
  g.voxels = static_cast<const VoxelRec*>(d_voxels.ptr);
  g.voxel_vals = static_cast<const float*>(d_voxel_vals.ptr);
  g.n_voxels = (int32_t)n_voxels;
  return g;
}

ccm_status Context::body_of(ccm_geom h, int32_t* idx) const {
  if (h == 0 || h > bodies.size()) return fail(CCM_ERR_INVALID, "unknown geometry handle %llu",
                                               (unsigned long long)h);
  if (!alive[h - 1]) return fail(CCM_ERR_INVALID, "geometry handle %llu was released",
                                 (unsigned long long)h);
  *idx = (int32_t)(h - 1);
  return CCM_OK;
}

ccm_status make_kparams(const ccm_params* p, KParams* k) {
  if (!p) return fail(CCM_ERR_INVALID, "params is NULL");
  const float taus[4] = {p->tau_sdf, p->tau_trace, p->tau_clip, p->tau_blend};
  for (float t : taus)
    if (!(t > 0.f) || !std::isfinite(t)) return fail(CCM_ERR_INVALID, "softness must be > 0");
  if (!(p->gate_width > 0.f) || !std::isfinite(p->gate_width) || !std::isfinite(p->d_max))
    return fail(CCM_ERR_INVALID, "gate_width must be > 0 and d_max finite");
  if (p->trace_iters < 0 || p->trace_iters > 16)
    return fail(CCM_ERR_INVALID, "trace_iters must be in [0, 16]");
  k->tau_sdf = p->tau_sdf;
  k->tau_trace = p->tau_trace;
  k->tau_clip = p->tau_clip;
  k->tau_blend = p->tau_blend;
  k->d_max = p->d_max;
  k->gate_width = p->gate_width;
  k->trace_iters = p->trace_iters;
  k->flags = p->flags;
  k->c_sdf = (float)(1.4426950408889634 / p->tau_sdf);
  k->ic_sdf = 1.0f / k->c_sdf;
  k->c_trace = (float)(1.4426950408889634 / p->tau_trace);
  k->c_clip = (float)(1.4426950408889634 / p->tau_clip);
  k->c_blend = (float)(1.4426950408889634 / p->tau_blend);
  k->inv_gate = (float)(1.0 / p->gate_width);
  return CCM_OK;
}

}  // namespace ccm

using namespace ccm;

extern "C" {

const char* ccm_last_error(void) { return g_err.c_str(); }

void ccm_default_params(ccm_params* p) {
  if (!p) return;
  p->tau_sdf = p->tau_trace = p->tau_clip = p->tau_blend = 5e-3f;
  p->d_max = 0.01f;
  p->gate_width = 0.01f;
  p->trace_iters = 3;
  p->flags = 0;
}

ccm_status ccm_create(int device, size_t hbm_budget_bytes, ccm_ctx* out) {
  if (!out) return fail(CCM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(CCM_ERR_INVALID, "no CUDA device %d", device);
  CCM_CUDA(cudaSetDevice(device), "cudaSetDevice");
  Context* c = new Context();
  c->device = device;
  c->budget = hbm_budget_bytes;
  cudaDeviceProp prop;
  CCM_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
  c->n_sm = prop.multiProcessorCount;
  c->smem_optin = (int)prop.sharedMemPerBlockOptin;
  *out = reinterpret_cast<ccm_ctx>(c);
  return CCM_OK;
}

void ccm_destroy(ccm_ctx ctx) {
  if (!ctx) return;
  Context* c = reinterpret_cast<Context*>(ctx);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  c->shutdown_serving();
  c->d_pieces.release();
  c->d_bodies.release();
  c->d_verts.release();
  c->d_planes.release();
  c->d_edges.release();
  c->d_splines.release();
  c->d_spline_coef.release();
  c->d_voxels.release();
  c->d_voxel_vals.release();
  delete c;
}

ccm_status ccm_build_voxel_grids(ccm_ctx ctx, int voxels) {
  if (!ctx || voxels < 1 || voxels > 64) return fail(CCM_ERR_INVALID, "voxels must be in [1, 64]");
  Context* c = reinterpret_cast<Context*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  CCM_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
  std::vector<VoxelRec> recs(c->pieces.size());
  std::vector<float> vals;
  for (size_t p = 0; p < c->pieces.size(); ++p) {
    const PieceRec& pr = c->pieces[p];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < pr.nv; ++i) {
      const float4 v = c->verts[pr.v0 + i];
      const double xs[3] = {v.x, v.y, v.z};
      for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], xs[a]); hi[a] = std::max(hi[a], xs[a]); }
    }
    double ext = 0;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, hi[a] - lo[a]);
    const double h = std::max(ext, 1e-6) / voxels;
    int dims[3];
    for (int a = 0; a < 3; ++a)
      dims[a] = std::max(1, (int)std::ceil((hi[a] - lo[a]) / h - 1e-9));
    const double r = 0.5 * h * std::sqrt(3.0);
    VoxelRec vr;
    vr.grid = make_float4((float)lo[0], (float)lo[1], (float)lo[2], (float)h);
    vr.dims = make_int4(dims[0], dims[1], dims[2], (int)vals.size());
    // the grid as the kernels see it (float origin and size): a voxel's
    // points lie within its circumradius (plus rounding) of its centre
    const double fo[3] = {vr.grid.x, vr.grid.y, vr.grid.z}, fh = vr.grid.w;
    for (int ix = 0; ix < dims[0]; ++ix)
      for (int iy = 0; iy < dims[1]; ++iy)
        for (int iz = 0; iz < dims[2]; ++iz) {
          const double cx = fo[0] + (ix + 0.5) * fh, cy = fo[1] + (iy + 0.5) * fh,
                       cz = fo[2] + (iz + 0.5) * fh;
          double m = -INFINITY;
          for (int k = 0; k < pr.nf; ++k) {
            const float4 q = c->planes[pr.f0 + k];
            m = std::max(m, q.x * cx + q.y * cy + q.z * cz + (double)q.w);
          }
          // the largest plane value is 1-Lipschitz and below the piece's SDF
          vals.push_back((float)(m - r * (1.0 + 1e-6) - 1e-6));
        }
    recs[p] = vr;
  }
  if ((int64_t)vals.size() >= ((int64_t)1 << 31)) return fail(CCM_ERR_INVALID, "grids too large");
  CCM_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  ccm_status s;
  if ((s = upload(c->d_voxels, recs, "voxel grids")) != CCM_OK) return s;
  if (vals.empty()) vals.push_back(0.f);
  if ((s = upload(c->d_voxel_vals, vals, "voxel grids")) != CCM_OK) return s;
  c->n_voxels = (int64_t)recs.size();
  return CCM_OK;
}

ccm_status ccm_attach_splines(ccm_ctx ctx, ccm_geom body, const ccm_spline_desc* desc) {
  if (!ctx || !desc || !desc->grid || !desc->dims || !desc->coef)
    return fail(CCM_ERR_INVALID, "bad arguments");
  Context* c = reinterpret_cast<Context*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  int32_t bi;
  ccm_status s = c->body_of(body, &bi);
  if (s != CCM_OK) return s;
  const BodyRec br = c->bodies[bi];
  // validate before touching the context
  int64_t rows = 0;
  for (int p = 0; p < br.np; ++p) {
    const float* gq = desc->grid + 4 * p;
    const int32_t* d = desc->dims + 3 * p;
    for (int a = 0; a < 4; ++a)
      if (!std::isfinite(gq[a])) return fail(CCM_ERR_INVALID, "piece %d: non-finite grid", p);
    if (!(gq[3] > 0.f)) return fail(CCM_ERR_INVALID, "piece %d: voxel size must be > 0", p);
    for (int a = 0; a < 3; ++a)
      if (d[a] < 1 || d[a] > 256)
        return fail(CCM_ERR_INVALID, "piece %d: voxel counts out of [1, 256]", p);
    rows += (int64_t)(d[0] + 3) * (d[1] + 3) * (d[2] + 3);
  }
  if ((int64_t)c->spline_coef.size() + rows >= ((int64_t)1 << 31))
    return fail(CCM_ERR_INVALID, "too many spline coefficients");
  for (int64_t i = 0; i < 4 * rows; ++i)
    if (!std::isfinite(desc->coef[i])) return fail(CCM_ERR_INVALID, "non-finite coefficient");
  CCM_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
  if (c->splines.size() < c->pieces.size()) c->splines.resize(c->pieces.size(), SplineRec{});
  int64_t r0 = 0;
  for (int p = 0; p < br.np; ++p) {
    const float* gq = desc->grid + 4 * p;
    const int32_t* d = desc->dims + 3 * p;
    const int64_t n = (int64_t)(d[0] + 3) * (d[1] + 3) * (d[2] + 3);
    SplineRec sr;
    sr.grid = make_float4(gq[0], gq[1], gq[2], gq[3]);
    sr.dims = make_int4(d[0], d[1], d[2], (int)c->spline_coef.size());
    for (int64_t i = 0; i < n; ++i) {
      const float* q = desc->coef + 4 * (r0 + i);
      c->spline_coef.push_back(make_float4(q[0], q[1], q[2], q[3]));
    }
    c->splines[br.p0 + p] = sr;
    r0 += n;
  }
  CCM_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  if ((s = upload(c->d_splines, c->splines, "splines")) != CCM_OK) return s;
  return upload(c->d_spline_coef, c->spline_coef, "spline coefficients");
}

// Morton (Z-order) key of a point quantised to 10 bits per axis in a box
static uint32_t zorder_key(const float* v, const float lo[3], const float inv[3]) {
  uint32_t key = 0;
  uint32_t q[3];
  for (int a = 0; a < 3; ++a) {
    const float t = (v[a] - lo[a]) * inv[a];
    q[a] = (uint32_t)std::min(1023.0f, std::max(0.0f, t * 1023.0f));
  }
  for (int bit = 9; bit >= 0; --bit)
    for (int a = 0; a < 3; ++a) key = (key << 1) | ((q[a] >> bit) & 1u);
  return key;
}

// Sec. 4.3 serialisation: the order in which a piece's vertices and edges are
// stored, along a Z-order curve through the piece's bounding box, so that
// features with neighbouring indices are near each other and the lanes of a
// warp that take them in order tend to agree on a cull.  perm_v[new] = old
// vertex, perm_e[new] = old edge (ties keep the caller's order).
static void serialise_piece(const float* verts, int nv, const int32_t* edges, int ne,
                            std::vector<int>* perm_v, std::vector<int>* perm_e) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = 0; i < nv; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], verts[3 * i + a]);
      hi[a] = std::max(hi[a], verts[3 * i + a]);
    }
  float inv[3];
  for (int a = 0; a < 3; ++a) inv[a] = hi[a] > lo[a] ? 1.0f / (hi[a] - lo[a]) : 0.f;
  std::vector<uint32_t> kv(nv), ke(ne);
  for (int i = 0; i < nv; ++i) kv[i] = zorder_key(verts + 3 * i, lo, inv);
  for (int j = 0; j < ne; ++j) {
    const float* a = verts + 3 * edges[2 * j];
    const float* b = verts + 3 * edges[2 * j + 1];
    const float m[3] = {0.5f * (a[0] + b[0]), 0.5f * (a[1] + b[1]), 0.5f * (a[2] + b[2])};
    ke[j] = zorder_key(m, lo, inv);
  }
  perm_v->resize(nv);
  perm_e->resize(ne);
  for (int i = 0; i < nv; ++i) (*perm_v)[i] = i;
  for (int j = 0; j < ne; ++j) (*perm_e)[j] = j;
  std::stable_sort(perm_v->begin(), perm_v->end(), [&](int x, int y) { return kv[x] < kv[y]; });
  std::stable_sort(perm_e->begin(), perm_e->end(), [&](int x, int y) { return ke[x] < ke[y]; });
}

ccm_status ccm_load_geometry(ccm_ctx ctx, const ccm_body_desc* bodies, int n_bodies,
                             ccm_geom* out) {
  if (!ctx || !bodies || !out || n_bodies < 0) return fail(CCM_ERR_INVALID, "bad arguments");
  Context* c = reinterpret_cast<Context*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  CCM_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
  // validate everything before touching the context
  for (int b = 0; b < n_bodies; ++b) {
    const ccm_body_desc& d = bodies[b];
    if (d.n_pieces < 1 || d.n_pieces > 4096)
      return fail(CCM_ERR_INVALID, "body %d: n_pieces=%d outside [1, 4096]", b, d.n_pieces);
    if (!d.nv || !d.nf || !d.ne || !d.verts || !d.planes || (!d.edges))
      return fail(CCM_ERR_INVALID, "body %d: NULL array", b);
    int64_t vo = 0, eo = 0, fo = 0;
    for (int p = 0; p < d.n_pieces; ++p) {
      const int nv = d.nv[p], nf = d.nf[p], ne = d.ne[p];
      if (nv < 1 || nv > 1024 || nf < 1 || nf > 1024 || ne < 0 || ne > 3072)
        return fail(CCM_ERR_INVALID, "body %d piece %d: sizes (%d, %d, %d) out of range", b, p,
                    nv, nf, ne);
      for (int64_t i = 0; i < 3 * (int64_t)nv; ++i)
        if (!std::isfinite(d.verts[3 * vo + i]))
          return fail(CCM_ERR_INVALID, "body %d piece %d: non-finite vertex", b, p);
      for (int64_t i = 0; i < 4 * (int64_t)nf; ++i)
        if (!std::isfinite(d.planes[4 * fo + i]))
          return fail(CCM_ERR_INVALID, "body %d piece %d: non-finite plane", b, p);
      for (int j = 0; j < ne; ++j) {
        const int i0 = d.edges[2 * (eo + j)], i1 = d.edges[2 * (eo + j) + 1];
        if (i0 < 0 || i1 < 0 || i0 >= nv || i1 >= nv || i0 == i1)
          return fail(CCM_ERR_INVALID, "body %d piece %d edge %d: bad indices", b, p, j);
        const float* a = d.verts + 3 * (vo + i0);
        const float* q = d.verts + 3 * (vo + i1);
        const double L = std::sqrt((double)(q[0] - a[0]) * (q[0] - a[0]) +
                                   (double)(q[1] - a[1]) * (q[1] - a[1]) +
                                   (double)(q[2] - a[2]) * (q[2] - a[2]));
        if (!(L > 1e-12)) return fail(CCM_ERR_INVALID, "body %d piece %d edge %d: zero length", b, p, j);
      }
      vo += nv; fo += nf; eo += ne;
    }
  }
  for (int b = 0; b < n_bodies; ++b) {
    const ccm_body_desc& d = bodies[b];
    BodyRec br;
    br.p0 = (int32_t)c->pieces.size();
    br.np = d.n_pieces;
    int64_t vo = 0, eo = 0, fo = 0;
    for (int p = 0; p < d.n_pieces; ++p) {
      const int nv = d.nv[p], nf = d.nf[p], ne = d.ne[p];
      PieceRec pr;
      pr.v0 = (int32_t)c->verts.size();
      pr.nv = nv;
      pr.f0 = (int32_t)c->planes.size();
      pr.nf = nf;
      pr.e0 = (int32_t)c->edges.size();
      pr.ne = ne;
      pr.body = (int32_t)c->bodies.size();
      pr.pad = 0;
      std::vector<int> pv, pe, rank(nv);
      serialise_piece(d.verts + 3 * vo, nv, d.edges + 2 * eo, ne, &pv, &pe);
      for (int i = 0; i < nv; ++i) rank[pv[i]] = i;
      double cx = 0, cy = 0, cz = 0;
      for (int i = 0; i < nv; ++i) {
        const float* v = d.verts + 3 * (vo + pv[i]);
        c->verts.push_back(make_float4(v[0], v[1], v[2], 0.f));
        cx += v[0]; cy += v[1]; cz += v[2];
      }
      cx /= nv; cy /= nv; cz /= nv;
      const float fcx = (float)cx, fcy = (float)cy, fcz = (float)cz;
      double r = 0;
      for (int i = 0; i < nv; ++i) {
        const float* v = d.verts + 3 * (vo + i);
        const double dx = v[0] - (double)fcx, dy = v[1] - (double)fcy, dz = v[2] - (double)fcz;
        r = std::max(r, std::sqrt(dx * dx + dy * dy + dz * dz));
      }
      // a slightly inflated radius keeps the float32 gate conservative
      pr.sphere = make_float4(fcx, fcy, fcz, (float)(r * (1.0 + 1e-5) + 1e-7));
      for (int k = 0; k < nf; ++k) {
        const float* q = d.planes + 4 * (fo + k);
        c->planes.push_back(make_float4(q[0], q[1], q[2], q[3]));
      }
      for (int j = 0; j < ne; ++j) {
        const int o = pe[j];
        const uint32_t i0 = (uint32_t)rank[d.edges[2 * (eo + o)]],
                       i1 = (uint32_t)rank[d.edges[2 * (eo + o) + 1]];
        c->edges.push_back(i0 | (i1 << 16));
      }
      c->pieces.push_back(pr);
      vo += nv; fo += nf; eo += ne;
    }
    c->bodies.push_back(br);
    c->alive.push_back(1);
    out[b] = (ccm_geom)c->bodies.size();
  }
  // resident copy (uploads happen while no batch kernel can be in flight:
  // loads are synchronous with the device)
  CCM_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  ccm_status s;
  if ((s = upload(c->d_pieces, c->pieces, "pieces")) != CCM_OK) return s;
  if ((s = upload(c->d_bodies, c->bodies, "bodies")) != CCM_OK) return s;
  if ((s = upload(c->d_verts, c->verts, "verts")) != CCM_OK) return s;
  if ((s = upload(c->d_planes, c->planes, "planes")) != CCM_OK) return s;
  if ((s = upload(c->d_edges, c->edges, "edges")) != CCM_OK) return s;
  return CCM_OK;
}

ccm_status ccm_free_geometry(ccm_ctx ctx, const ccm_geom* handles, int n) {
  if (!ctx || (!handles && n > 0)) return fail(CCM_ERR_INVALID, "bad arguments");
  Context* c = reinterpret_cast<Context*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  for (int i = 0; i < n; ++i) {
    int32_t b;
    ccm_status s = c->body_of(handles[i], &b);
    if (s != CCM_OK) return s;
  }
  for (int i = 0; i < n; ++i) c->alive[handles[i] - 1] = 0;
  return CCM_OK;
}

ccm_status ccm_output_size(ccm_ctx ctx, int64_t n, const ccm_geom* A, const ccm_geom* B,
                           int64_t* groups) {
  if (!ctx || n < 0 || (n > 0 && (!A || !B)) || !groups) return fail(CCM_ERR_INVALID, "bad arguments");
  Context* c = reinterpret_cast<Context*>(ctx);
  std::lock_guard<std::mutex> lk(c->mu);
  int64_t G = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t a, b;
    ccm_status s;
    if ((s = c->body_of(A[i], &a)) != CCM_OK || (s = c->body_of(B[i], &b)) != CCM_OK) return s;
    G += c->bodies[a].np + c->bodies[b].np;
  }
  *groups = G;
  return CCM_OK;
}

ccm_status ccm_batch_create(ccm_ctx ctx, int64_t n, const ccm_geom* A, const ccm_geom* B,
                            ccm_batch* out) {
  if (!ctx || n < 0 || (n > 0 && (!A || !B)) || !out) return fail(CCM_ERR_INVALID, "bad arguments");
  if (n > (int64_t)1 << 30) return fail(CCM_ERR_INVALID, "too many pairs");
  Context* c = reinterpret_cast<Context*>(ctx);
  *out = nullptr;
  Batch* bt = new Batch();
  bt->ctx = c;
  bt->n = n;
  ccm_status s = build_batch(c, n, A, B, bt);
  if (s != CCM_OK) {
    bt->release();
    delete bt;
    return s;
  }
  *out = reinterpret_cast<ccm_batch>(bt);
  return CCM_OK;
}

void ccm_batch_destroy(ccm_batch batch) {
  if (!batch) return;
  Batch* b = reinterpret_cast<Batch*>(batch);
  cudaSetDevice(b->ctx->device);
  b->release();
  delete b;
}

ccm_status ccm_batch_info(ccm_batch batch, int64_t* n_pairs, int64_t* n_groups, int64_t* off) {
  if (!batch) return fail(CCM_ERR_INVALID, "batch is NULL");
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (n_pairs) *n_pairs = b->n;
  if (n_groups) *n_groups = b->G;
  if (off) std::memcpy(off, b->goff.data(), sizeof(int64_t) * (b->n + 1));
  return CCM_OK;
}

ccm_status ccm_batch_get_tuning(ccm_batch batch, ccm_tuning* out) {
  if (!batch || !out) return fail(CCM_ERR_INVALID, "bad arguments");
  *out = reinterpret_cast<Batch*>(batch)->tuning;
  return CCM_OK;
}

ccm_status ccm_batch_set_tuning(ccm_batch batch, const ccm_tuning* t) {
  if (!batch || !t) return fail(CCM_ERR_INVALID, "bad arguments");
  Batch* b = reinterpret_cast<Batch*>(batch);
  std::lock_guard<std::mutex> lk(b->ctx->mu);
  const ccm_status s = apply_tuning(b->ctx, b, *t);
  if (s != CCM_OK) return s;
  return setup_flat(b->ctx, b);
}

ccm_status ccm_kernel_launches(int64_t* n) {
  if (!n) return fail(CCM_ERR_INVALID, "n is NULL");
  *n = g_kernel_launches.load(std::memory_order_relaxed);
  return CCM_OK;
}

ccm_status ccm_batch_check(ccm_batch batch, ccm_stream stream) {
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (!b) return fail(CCM_ERR_INVALID, "batch is NULL");
  CCM_CUDA(cudaSetDevice(b->ctx->device), "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t status = 0;
  CCM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  CCM_CUDA(cudaMemcpy(&status, b->d_status.ptr, sizeof(status), cudaMemcpyDeviceToHost),
           "cudaMemcpy");
  if (status == 0) return CCM_OK;
  const int32_t zero = 0;
  CCM_CUDA(cudaMemcpy(b->d_status.ptr, &zero, sizeof(zero), cudaMemcpyHostToDevice), "cudaMemcpy");
  return fail((ccm_status)status, "a kernel of the batch stopped on a bounded device-side wait");
}

ccm_status ccm_contacts(ccm_batch batch, const float* pose_a, const float* pose_b,
                        const ccm_params* prm, float* y, ccm_stream stream) {
  return run_forward(reinterpret_cast<Batch*>(batch), pose_a, pose_b, prm, y, nullptr, nullptr,
                     static_cast<cudaStream_t>(stream));
}

ccm_status ccm_contacts_backward(ccm_batch batch, const float* pose_a, const float* pose_b,
                                 const ccm_params* prm, const float* ybar, const float* dir,
                                 float* grad, float* hvp, float* jvp, ccm_stream stream) {
  return run_backward(reinterpret_cast<Batch*>(batch), pose_a, pose_b, prm, nullptr, ybar, dir, grad, hvp,
                      jvp, nullptr, static_cast<cudaStream_t>(stream));
}

ccm_status ccm_contacts_save(ccm_batch batch, const float* pose_a, const float* pose_b,
                             const ccm_params* prm, float* y, float* saved, ccm_stream stream) {
  if (!saved) return fail(CCM_ERR_INVALID, "saved is NULL");
  return run_forward(reinterpret_cast<Batch*>(batch), pose_a, pose_b, prm, y, saved, nullptr,
                     static_cast<cudaStream_t>(stream));
}

ccm_status ccm_contacts_backward_saved(ccm_batch batch, const float* pose_a, const float* pose_b,
                                       const ccm_params* prm, const float* saved,
                                       const float* ybar, const float* dir, float* grad,
                                       float* hvp, float* jvp, ccm_stream stream) {
  if (!saved) return fail(CCM_ERR_INVALID, "saved is NULL");
  return run_backward(reinterpret_cast<Batch*>(batch), pose_a, pose_b, prm, saved, ybar, dir,
                      grad, hvp, jvp, nullptr, static_cast<cudaStream_t>(stream));
}

ccm_status ccm_contacts_backward_counted(ccm_batch batch, const float* pose_a,
                                         const float* pose_b, const ccm_params* prm,
                                         const float* saved, const float* ybar, const float* dir,
                                         float* grad, float* hvp, float* jvp, int64_t* counters,
                                         ccm_stream stream) {
  if (!counters) return fail(CCM_ERR_INVALID, "counters is NULL");
  return run_backward(reinterpret_cast<Batch*>(batch), pose_a, pose_b, prm, saved, ybar, dir,
                      grad, hvp, jvp, reinterpret_cast<unsigned long long*>(counters),
                      static_cast<cudaStream_t>(stream));
}

static ccm_status reserve(DevBuf& b, size_t bytes, const char* what) {
  if (bytes <= b.bytes) return CCM_OK;
  b.release();
  cudaError_t e = cudaMalloc(&b.ptr, std::max<size_t>(bytes, 256));
  if (e != cudaSuccess)
    return fail(CCM_ERR_OOM, "%s: cudaMalloc(%zu): %s", what, bytes, cudaGetErrorString(e));
  b.bytes = std::max<size_t>(bytes, 256);
  return CCM_OK;
}

static ccm_status host_step_state(Batch* b) {
  if (!b->hs) b->hs = new HostStep();
  HostStep& h = *b->hs;
  const size_t P = sizeof(float) * 12 * (size_t)b->n, G = sizeof(float) * (size_t)b->G;
  struct { DevBuf* buf; size_t bytes; const char* what; } bufs[] = {
      {&h.pa, P, "step poses"}, {&h.pb, P, "step poses"}, {&h.y, 8 * G, "step outputs"},
      {&h.saved, CCM_SAVED_FLOATS * G, "step record"}, {&h.ybar, 8 * G, "step cotangents"},
      {&h.grad, P, "step gradient"}, {&h.grad2, P, "step gradient"}, {&h.hvp, P, "step hvp"},
      {&h.dir, P, "step direction"}, {&h.jvp, 8 * G, "step jvp"}};
  for (auto& x : bufs) {
    const ccm_status s = reserve(*x.buf, x.bytes, x.what);
    if (s != CCM_OK) return s;
  }
  if (!h.cin) CCM_CUDA(cudaStreamCreateWithFlags(&h.cin, cudaStreamNonBlocking), "stream");
  if (!h.cout) CCM_CUDA(cudaStreamCreateWithFlags(&h.cout, cudaStreamNonBlocking), "stream");
  for (cudaEvent_t& e : h.ev)
    if (!e) CCM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
  return CCM_OK;
}

ccm_status ccm_contacts_step_host(ccm_batch batch, const float* pose_a, const float* pose_b,
                                  const ccm_params* prm, const float* ybar, const float* dir,
                                  float* y, float* grad, float* hvp, float* jvp,
                                  ccm_stream stream) {
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (!b) return fail(CCM_ERR_INVALID, "batch is NULL");
  if (!pose_a || !pose_b || !y) return fail(CCM_ERR_INVALID, "NULL pose or output pointer");
  if (ybar && !grad) return fail(CCM_ERR_INVALID, "ybar given without grad");
  if (dir && (!ybar || !hvp)) return fail(CCM_ERR_INVALID, "dir needs ybar, grad and hvp");
  if (b->n == 0) return CCM_OK;
  CCM_CUDA(cudaSetDevice(b->ctx->device), "cudaSetDevice");
  ccm_status s = host_step_state(b);
  if (s != CCM_OK) return s;
  HostStep& h = *b->hs;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t P = sizeof(float) * 12 * (size_t)b->n, G8 = sizeof(float) * 8 * (size_t)b->G;
  const cudaMemcpyKind in = cudaMemcpyHostToDevice, out = cudaMemcpyDeviceToHost;
  float* pa = static_cast<float*>(h.pa.ptr);
  float* pb = static_cast<float*>(h.pb.ptr);
  float* yd = static_cast<float*>(h.y.ptr);
  float* sv = static_cast<float*>(h.saved.ptr);
  float* yb = static_cast<float*>(h.ybar.ptr);
  float* gd = static_cast<float*>(h.grad.ptr);
  // the side streams start behind the work already queued on `stream` (an
  // earlier step's kernels still read the buffers they overwrite) and behind
  // the pose copies, which the forward waits for: sharing the link with the
  // cotangent copy would delay it
  CCM_CUDA(cudaMemcpyAsync(pa, pose_a, P, in, st), "pose copy");
  CCM_CUDA(cudaMemcpyAsync(pb, pose_b, P, in, st), "pose copy");
  CCM_CUDA(cudaEventRecord(h.ev[0], st), "event");
  if (ybar) {
    CCM_CUDA(cudaStreamWaitEvent(h.cin, h.ev[0], 0), "wait");
    CCM_CUDA(cudaMemcpyAsync(yb, ybar, G8, in, h.cin), "cotangent copy");
    if (dir) CCM_CUDA(cudaMemcpyAsync(h.dir.ptr, dir, P, in, h.cin), "direction copy");
    CCM_CUDA(cudaEventRecord(h.ev[1], h.cin), "event");
  }
  if ((s = run_forward(b, pa, pb, prm, yd, sv, nullptr, st)) != CCM_OK) return s;
  CCM_CUDA(cudaEventRecord(h.ev[2], st), "event");
  CCM_CUDA(cudaStreamWaitEvent(h.cout, h.ev[2], 0), "wait");
  CCM_CUDA(cudaMemcpyAsync(y, yd, G8, out, h.cout), "output copy");
  // With dir, one forward-over-reverse pass gives the gradient (its primal
  // part) with H u and J u (its tangents); without, the gradient pass.
  if (ybar) {
    CCM_CUDA(cudaStreamWaitEvent(st, h.ev[1], 0), "wait");
    float* hd = dir ? static_cast<float*>(h.hvp.ptr) : nullptr;
    float* jd = dir && jvp ? static_cast<float*>(h.jvp.ptr) : nullptr;
    if ((s = run_backward(b, pa, pb, prm, sv, yb,
                          dir ? static_cast<const float*>(h.dir.ptr) : nullptr, gd, hd, jd,
                          nullptr, st)) != CCM_OK)
      return s;
    CCM_CUDA(cudaEventRecord(h.ev[3], st), "event");
    CCM_CUDA(cudaStreamWaitEvent(h.cout, h.ev[3], 0), "wait");
    CCM_CUDA(cudaMemcpyAsync(grad, gd, P, out, h.cout), "gradient copy");
    if (dir) CCM_CUDA(cudaMemcpyAsync(hvp, hd, P, out, h.cout), "hvp copy");
    if (jd) CCM_CUDA(cudaMemcpyAsync(jvp, jd, G8, out, h.cout), "jvp copy");
  }
  // later work on `stream` waits for the copies of the side streams
  CCM_CUDA(cudaEventRecord(h.ev[0], h.cout), "event");
  CCM_CUDA(cudaStreamWaitEvent(st, h.ev[0], 0), "wait");
  return CCM_OK;
}

// Blocks of the reverse kernels for a batch: one per unit of work (item or
// pair) at most, and no more than stay resident.
static void set_bwd_grids(const Batch& b, const KParams& kp, bool dual, BwdLaunch* L) {
  const int d = dual ? 1 : 0, k = kp.trace_iters == 3 ? 1 : 0;
  const int64_t n_sm = b.ctx->n_sm;
  L->grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(b.n_items, n_sm * std::max(1, b.bwd_occ.unit[d][k])));
  L->pair_grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(b.n, n_sm * std::max(1, b.bwd_occ.pair[d][k])));
}

ccm_status ccm_contacts_backward_noalloc(ccm_batch batch, const float* pose_a,
                                         const float* pose_b, const ccm_params* prm,
                                         const float* ybar, const float* dir, float* grad,
                                         float* hvp, float* jvp, ccm_stream stream) {
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (!b) return fail(CCM_ERR_INVALID, "batch is NULL");
  if (b->n == 0) return CCM_OK;
  if (b->n_items > noalloc_max_items())
    return fail(CCM_ERR_INVALID,
                "ccm_contacts_backward_noalloc: %lld work items exceed its fixed scratch of %lld",
                (long long)b->n_items, (long long)noalloc_max_items());
  if (!pose_a || !pose_b || !ybar || !grad) return fail(CCM_ERR_INVALID, "NULL pointer");
  if (dir && !hvp) return fail(CCM_ERR_INVALID, "dir given without hvp");
  KParams kp;
  ccm_status s = make_kparams(prm, &kp);
  if (s != CCM_OK) return s;
  if (kp.flags & CCM_FLAG_NO_CULL) return fail(CCM_ERR_INVALID, "the reverse pass always culls");
  if (kp.flags & (CCM_FLAG_BODY_UNION | CCM_FLAG_PROJECT | CCM_FLAG_SPLINE))
    return fail(CCM_ERR_INVALID,
                "the body-union, projection and spline variants are forward only");
  CCM_CUDA(cudaSetDevice(b->ctx->device), "cudaSetDevice");
  BwdLaunch L;
  L.g = b->ctx->dev_geom();
  L.pairs = static_cast<const PairRec*>(b->d_pairs.ptr);
  L.items = static_cast<const WorkItem*>(b->d_items.ptr);
  L.order = static_cast<const int32_t*>(b->d_item_order.ptr);
  L.n_items = b->n_items;
  L.item_off = static_cast<const int64_t*>(b->d_item_off.ptr);
  L.dev_items = nullptr;
  L.n_pairs = b->n;
  L.pose_a = pose_a;
  L.pose_b = pose_b;
  L.ybar = ybar;
  L.dir = dir;
  L.saved = nullptr;
  L.pair_order = nullptr;
  L.counters = nullptr;
  L.sched = nullptr;   // no workspace: units dealt round-robin
  L.kp = kp;
  L.us = b->us;
  L.part = nullptr;
  L.grad = grad;
  L.dev_pairs = nullptr;
  L.hvp = hvp;
  L.jvp = dir ? jvp : nullptr;
  set_bwd_grids(*b, kp, dir != nullptr, &L);
  const cudaError_t e =
      launch_backward_noalloc(L, b->ctx->device, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "backward (no-alloc) launch");
  return CCM_OK;
}

ccm_status ccm_contacts_counted(ccm_batch batch, const float* pose_a, const float* pose_b,
                                const ccm_params* prm, float* y, int64_t* counters,
                                ccm_stream stream) {
  if (!counters) return fail(CCM_ERR_INVALID, "counters is NULL");
  return run_forward(reinterpret_cast<Batch*>(batch), pose_a, pose_b, prm, y, nullptr,
                     reinterpret_cast<unsigned long long*>(counters),
                     static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace ccm {

static_assert(kSavedFloats == CCM_SAVED_FLOATS, "saved record layout");

BatchMaxima body_maxima(const Context& c, int32_t body) {
  BatchMaxima m;
  const BodyRec& br = c.bodies[body];
  int sp = 0, cv = 0, ce = 0;
  for (int p = 0; p < br.np; ++p) {
    const PieceRec& pr = c.pieces[br.p0 + p];
    m.vmax = std::max(m.vmax, pr.nv);
    m.fmax = std::max(m.fmax, pr.nf);
    m.emax = std::max(m.emax, pr.ne);
    sp += pr.nf;
    if (p < kGroupsPerChunk) { cv += pr.nv; ce += pr.ne; }
  }
  m.s_planes = std::max(1, sp);
  m.s_pieces = std::max(1, br.np);
  m.pieces_any = m.s_pieces;
  m.f_verts = std::max(1, cv);
  m.f_edges = std::max(1, ce);
  return m;
}

void merge_maxima(BatchMaxima* m, const BatchMaxima& b) {
  m->vmax = std::max(m->vmax, b.vmax);
  m->fmax = std::max(m->fmax, b.fmax);
  m->emax = std::max(m->emax, b.emax);
  m->s_planes = std::max(m->s_planes, b.s_planes);
  m->s_pieces = std::max(m->s_pieces, b.s_pieces);
  m->pieces_any = std::max(m->pieces_any, b.pieces_any);
  m->f_verts = std::max(m->f_verts, b.f_verts);
  m->f_edges = std::max(m->f_edges, b.f_edges);
}

void body_chunks(const Context& c, int32_t body, const UnitShape& us,
                 std::vector<PieceChunk>* out) {
  const BodyRec& F = c.bodies[body];
  // the kernels' chunking: at most us.groups pieces within the budgets
  for (int fc0 = 0; fc0 < F.np;) {
    int fc1 = fc0, V = 0, E = 0;
    int64_t feats = 0;
    while (fc1 < F.np && fc1 - fc0 < us.groups) {
      const PieceRec& p = c.pieces[F.p0 + fc1];
      if (V + p.nv > us.vert_budget || E + p.ne > us.edge_budget) break;
      V += p.nv;
      E += p.ne;
      feats += p.nv + p.ne;
      ++fc1;
    }
    out->push_back(PieceChunk{(uint16_t)fc0, (uint16_t)fc1, feats});
    fc0 = fc1;
  }
}

void push_items(const std::vector<PieceChunk>& chunks, int32_t unit, int32_t s_np,
                std::vector<WorkItem>* items, std::vector<int64_t>* cost) {
  for (const PieceChunk& ch : chunks) {
    items->push_back(WorkItem{unit, ch.fc0, ch.fc1});
    // directions, plus features times SDF pieces, plus staging S
    cost->push_back((int64_t)(ch.fc1 - ch.fc0) * s_np + ch.feats * s_np / 8 + s_np);
  }
}

void make_items(const Context& c, const PairRec* pairs, int64_t n, int64_t unit_pair0,
                const UnitShape& us, std::vector<WorkItem>* items, std::vector<int64_t>* cost,
                std::vector<int64_t>* item_off) {
  std::vector<PieceChunk> ch;
  for (int64_t i = 0; i < n; ++i) {
    for (int side = 0; side < 2; ++side) {
      const int32_t f = side == 0 ? pairs[i].bodyA : pairs[i].bodyB;
      const int32_t s = side == 0 ? pairs[i].bodyB : pairs[i].bodyA;
      ch.clear();
      body_chunks(c, f, us, &ch);
      push_items(ch, (int32_t)(2 * (unit_pair0 + i) + side), c.bodies[s].np, items, cost);
    }
    if (item_off) item_off->push_back((int64_t)items->size());
  }
}

std::vector<int32_t> items_by_cost(const std::vector<int64_t>& cost) {
  std::vector<int32_t> order(cost.size());
  for (size_t k = 0; k < cost.size(); ++k) order[k] = (int32_t)k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  return order;
}

ccm_status build_batch(Context* c, int64_t n, const ccm_geom* A, const ccm_geom* B, Batch* bt) {
  std::lock_guard<std::mutex> lk(c->mu);
  CCM_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
  std::vector<PairRec> pairs(n);
  bt->goff.assign(n + 1, 0);
  int64_t G = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t a, b;
    ccm_status s;
    if ((s = c->body_of(A[i], &a)) != CCM_OK || (s = c->body_of(B[i], &b)) != CCM_OK) return s;
    pairs[i].bodyA = a;
    pairs[i].bodyB = b;
    pairs[i].goff = G;
    bt->goff[i] = G;
    G += c->bodies[a].np + c->bodies[b].np;
  }
  bt->goff[n] = G;
  bt->G = G;
  // budgets of the per-warp shared-memory slice, from the bodies in the batch
  std::vector<uint8_t> seen(c->bodies.size(), 0);
  BatchMaxima mx;
  for (int64_t i = 0; i < n; ++i) {
    for (int32_t bi : {pairs[i].bodyA, pairs[i].bodyB}) {
      if (seen[bi]) continue;
      seen[bi] = 1;
      merge_maxima(&mx, body_maxima(*c, bi));
    }
  }
  bt->mx = mx;
  ccm_status s;
  if ((s = upload(bt->d_pairs, pairs, "pairs")) != CCM_OK) return s;
  {   // pair and side of every output group
    std::vector<int32_t> rp((size_t)std::max<int64_t>(1, G));
    for (int64_t i = 0; i < n; ++i) {
      const int npA = c->bodies[pairs[i].bodyA].np, npB = c->bodies[pairs[i].bodyB].np;
      for (int q = 0; q < npA + npB; ++q)
        rp[pairs[i].goff + q] = (int32_t)((i << 1) | (q < npA ? 0 : 1));
    }
    if ((s = upload(bt->d_row_pair, rp, "group pairs")) != CCM_OK) return s;
  }
  bt->pairs = std::move(pairs);
  ccm_tuning t;
  default_tuning(&t);
  if ((s = apply_tuning(c, bt, t)) != CCM_OK) return s;
  return setup_flat(c, bt);
}

ContactList Batch::contact_list() const {
  ContactList cl{};
  if (!flat_cap) return cl;
  cl.recs = static_cast<int4*>(d_frecs.ptr);
  cl.sorted = static_cast<int4*>(d_fsorted.ptr);
  cl.cap = flat_cap;
  cl.ctl = static_cast<unsigned long long*>(d_fctl.ptr);
  cl.cnt_v = static_cast<int32_t*>(d_fcnt.ptr);
  cl.cnt_e = cl.cnt_v + G;
  cl.off_v = static_cast<int32_t*>(d_foff.ptr);
  cl.off_e = cl.off_v + (G + 1);
  cl.live_g = cl.off_e + (G + 1);
  cl.tile_sum = static_cast<long long*>(d_ftiles.ptr);
  return cl;
}

FlatPass Batch::flat_pass(bool dual) const {
  const DevBuf* b = d_fpass[dual ? 1 : 0];
  FlatPass f;
  f.cval = b[0].ptr;
  f.force = b[1].ptr;
  f.coef = b[2].ptr;
  f.oterm = b[3].ptr;
  f.sched = static_cast<int*>(b[4].ptr);
  return f;
}

ccm_status setup_flat(Context* c, Batch* bt) {
  const int fr = bt->tuning.flat_records;
  int64_t cap = 0;
  if (bt->per_pair && bt->G > 0 && fr >= 0)
    cap = fr > 0 ? fr * bt->G
                 : std::min<int64_t>(std::max<int64_t>(16 * bt->G, 4096), (int64_t)1 << 24);
  if (cap == bt->flat_cap) return CCM_OK;
  for (DevBuf* b : {&bt->d_fctl, &bt->d_fcnt, &bt->d_foff, &bt->d_frecs, &bt->d_fsorted,
                   &bt->d_ftiles, &bt->d_unit_dir_off, &bt->d_rel, &bt->d_live, &bt->d_cand,
                   &bt->d_cand_m, &bt->d_cval, &bt->d_sval, &bt->d_skey, &bt->d_ffctl,
                   &bt->d_ffhits})
    b->release();
  for (auto& pass : bt->d_fpass)
    for (DevBuf& b : pass) b.release();
  bt->flat_cap = 0;
  if (cap == 0) return CCM_OK;
  CCM_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
  auto alloc = [&](DevBuf& b, size_t bytes, const char* what) -> ccm_status {
    const cudaError_t e = cudaMalloc(&b.ptr, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess)
      return fail(CCM_ERR_OOM, "%s: cudaMalloc(%zu): %s", what, bytes, cudaGetErrorString(e));
    b.bytes = std::max<size_t>(bytes, 256);
    return CCM_OK;
  };
  const size_t G = (size_t)bt->G;
  ccm_status s;
  if ((s = alloc(bt->d_fctl, kCtlWords * sizeof(unsigned long long), "contact list")) != CCM_OK ||
      (s = alloc(bt->d_fcnt, 2 * G * sizeof(int32_t), "contact counts")) != CCM_OK ||
      (s = alloc(bt->d_foff, (3 * G + 2) * sizeof(int32_t), "contact offsets")) != CCM_OK ||
      (s = alloc(bt->d_frecs, (size_t)cap * sizeof(int4), "contact list")) != CCM_OK ||
      (s = alloc(bt->d_fsorted, (size_t)cap * sizeof(int4), "contact list")) != CCM_OK ||
      (s = alloc(bt->d_ftiles, 2 * (size_t)flat_scan_tiles(bt->G) * sizeof(long long),
                 "contact list scan")) != CCM_OK)
    return s;
  for (int d = 0; d < 2; ++d) {
    size_t sz[4];
    flat_pass_bytes(d == 1, cap, bt->G, &sz[0], &sz[1], &sz[2], &sz[3]);
    for (int q = 0; q < 4; ++q)
      if ((s = alloc(bt->d_fpass[d][q], sz[q], "per-contact pass")) != CCM_OK) return s;
    if ((s = alloc(bt->d_fpass[d][4], 3 * sizeof(int), "per-contact pass")) != CCM_OK) return s;
  }
  {   // the flat forward: directions per unit (u = 2 pair + side), candidates
    std::vector<int64_t> off(2 * (size_t)bt->n + 1, 0);
    for (int64_t i = 0; i < bt->n; ++i) {
      const int64_t d = (int64_t)c->bodies[bt->pairs[i].bodyA].np * c->bodies[bt->pairs[i].bodyB].np;
      off[2 * i + 1] = off[2 * i] + d;
      off[2 * i + 2] = off[2 * i + 1] + d;
    }
    bt->n_dirs = off.back();
    bt->cand_cap = std::min<int64_t>(std::max<int64_t>(64 * bt->G, (int64_t)1 << 14),
                                     (int64_t)1 << 25);
    if ((s = upload(bt->d_unit_dir_off, off, "direction offsets")) != CCM_OK ||
        (s = alloc(bt->d_rel, 12 * sizeof(float) * 2 * (size_t)bt->n, "relative poses")) != CCM_OK ||
        (s = alloc(bt->d_live, (size_t)bt->n_dirs * sizeof(int4), "live directions")) != CCM_OK ||
        (s = alloc(bt->d_cand, (size_t)bt->cand_cap * sizeof(int4), "candidates")) != CCM_OK ||
        (s = alloc(bt->d_cand_m, (size_t)bt->cand_cap * sizeof(float2), "candidates")) != CCM_OK ||
        (s = alloc(bt->d_cval, (size_t)bt->cand_cap * 8 * sizeof(float), "candidates")) != CCM_OK ||
        (s = alloc(bt->d_sval, (size_t)cap * 8 * sizeof(float), "contact values")) != CCM_OK ||
        (s = alloc(bt->d_skey, (size_t)cap * sizeof(long long), "contact keys")) != CCM_OK ||
        (s = alloc(bt->d_ffctl, kFfWords * sizeof(unsigned long long), "flat forward")) != CCM_OK ||
        (s = alloc(bt->d_ffhits, (size_t)bt->G * kHitWords * sizeof(uint32_t), "hit words")) != CCM_OK)
      return s;
  }
  // a list that no forward filled yet reads as overflowed (the per-pair path)
  unsigned long long init[kCtlWords] = {};
  init[kCtlOverflow] = 1ull;
  CCM_CUDA(cudaMemcpy(bt->d_fctl.ptr, init, sizeof(init), cudaMemcpyHostToDevice), "cudaMemcpy");
  bt->flat_cap = cap;
  return CCM_OK;
}

void default_tuning(ccm_tuning* t) {
  std::memset(t, 0, sizeof(*t));
  t->item_v = 256;
  t->item_e = 512;
  t->item_vb = 256;
  t->item_eb = 512;
  t->fwd_warps = 2;
  t->groups = 16;
}

// Shared-memory budgets and launch shapes of a batch for the tuning `t`
// (budgets are raised to hold the largest piece of the batch).
ccm_status apply_tuning(Context* c, Batch* bt, const ccm_tuning& t) {
  if (t.item_v < 1 || t.item_e < 1 || t.item_vb < 1 || t.item_eb < 1 || t.item_v > 8192 ||
      t.item_e > 16384 || t.item_vb > 8192 || t.item_eb > 16384 || t.fwd_warps < 1 ||
      t.fwd_warps > 4 || t.groups < 1 || t.groups > kGroupsPerChunk ||
      (t.stage_planes != 0 && (t.stage_planes < 16 || t.stage_planes > 4096)) ||
      (t.stage_verts != 0 && (t.stage_verts < 16 || t.stage_verts > 4096)) ||
      t.groups_b < 0 || t.groups_b > kGroupsPerChunk || t.flat_records < -1 ||
      t.flat_records > 4096 || t.stage_tma < -1 || t.stage_tma > 0 || t.stage_wait < -1 ||
      t.stage_wait > (1 << 30) || t.flat_forward < -1 || t.flat_forward > 0 || t.pdl < -1 ||
      t.pdl > 0)
    return fail(CCM_ERR_INVALID, "tuning out of range");
  const BatchMaxima& mx = bt->mx;
  UnitShape us{};
  const int cap_p = t.stage_planes ? t.stage_planes : 1024;
  const int cap_v = t.stage_verts ? t.stage_verts : 512;
  us.plane_budget = std::max(mx.fmax, std::min(mx.s_planes, cap_p));
  us.spiece_budget = std::min(mx.s_pieces, 256);
  us.vert_budget = std::max(mx.vmax, std::min(mx.f_verts, cap_v));
  us.edge_budget = std::max(mx.emax, std::min(mx.f_edges, 3 * cap_v));
  us.item_v = std::max(mx.vmax, t.item_v);
  us.item_e = std::max(mx.emax, t.item_e);
  us.item_vb = std::max(mx.vmax, t.item_vb);
  us.item_eb = std::max(mx.emax, t.item_eb);
  us.groups = std::min(t.groups, mx.pieces_any);
  // the reverse pass's chunks: a handful of (marked) groups keeps a chunk's
  // directions in one list, which its adjoint sweep then reuses
  us.groups_b = std::min(us.groups, t.groups_b ? t.groups_b : 4);
  us.hit_words = std::min(kHitWords, (mx.s_pieces + 31) / 32);
  us.stage_tma = t.stage_tma == 0 ? 1 : 0;
  us.wait_limit = t.stage_wait == 0 ? (1ll << 22) : (t.stage_wait < 0 ? 0 : t.stage_wait);
  us.slice_bytes = unit_slice_bytes(us);
  us.warps = t.fwd_warps;
  while (us.warps > 1 && us.warps * us.slice_bytes > c->smem_optin) --us.warps;
  if (us.slice_bytes > c->smem_optin)
    return fail(CCM_ERR_INVALID, "pieces too large: %d bytes of shared memory per warp",
                us.slice_bytes);
  if (backward_slice_bytes(us, true) > c->smem_optin)
    return fail(CCM_ERR_INVALID, "pieces too large for the reverse pass");
  CCM_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
  int per_sm = 1;
  cudaError_t e = configure_forward(us, c->smem_optin, &per_sm);
  if (e != cudaSuccess) return cuda_fail(e, "configure_forward");
  BwdOccupancy occ{};
  e = configure_backward(us, c->smem_optin, &occ);
  if (e != cudaSuccess) return cuda_fail(e, "configure_backward");
  // work items of the pairs for this shape, heaviest first
  std::vector<WorkItem> items;
  std::vector<int64_t> cost, item_off(1, 0);
  items.reserve(2 * bt->pairs.size());
  make_items(*c, bt->pairs.data(), (int64_t)bt->pairs.size(), 0, us, &items, &cost, &item_off);
  if ((int64_t)items.size() >= ((int64_t)1 << 31))
    return fail(CCM_ERR_INVALID, "too many work items (%zu)", items.size());
  ccm_status st;
  if ((st = upload(bt->d_items, items, "work items")) != CCM_OK) return st;
  if ((st = upload(bt->d_item_order, items_by_cost(cost), "item order")) != CCM_OK) return st;
  if ((st = upload(bt->d_item_off, item_off, "item offsets")) != CCM_OK) return st;
  {   // pairs by decreasing cost (the sum of their items'), for the per-pair reverse pass
    std::vector<int64_t> pcost(bt->pairs.size(), 0);
    for (size_t i = 0; i < bt->pairs.size(); ++i)
      for (int64_t j = item_off[i]; j < item_off[i + 1]; ++j) pcost[i] += cost[j];
    if ((st = upload(bt->d_pair_order, items_by_cost(pcost), "pair order")) != CCM_OK) return st;
  }
  bt->per_pair = bt->mx.s_pieces <= kHitS;
  if (!bt->d_sched.ptr) {   // forward, gradient pass, H u pass
    std::vector<int32_t> zeros(3, 0);
    if ((st = upload(bt->d_sched, zeros, "work counters")) != CCM_OK) return st;
  }
  if (!bt->d_status.ptr) {
    std::vector<int32_t> zeros(1, 0);
    if ((st = upload(bt->d_status, zeros, "status word")) != CCM_OK) return st;
  }
  if ((int64_t)items.size() != bt->n_items || !bt->d_part.ptr) {
    bt->d_part.release();
    std::vector<float> zeros((size_t)std::max<size_t>(1, items.size()) * 24, 0.f);
    if ((st = upload(bt->d_part, zeros, "reverse-pass slots")) != CCM_OK) return st;
  }
  bt->n_items = (int64_t)items.size();
  const int64_t units = bt->n_items;
  bt->us = us;
  bt->tuning = t;
  bt->grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((units + us.warps - 1) / us.warps, (int64_t)c->n_sm * std::max(1, per_sm)));
  bt->bwd_occ = occ;
  return CCM_OK;
}

ccm_status run_backward(Batch* b, const float* pose_a, const float* pose_b, const ccm_params* prm,
                        const float* saved, const float* ybar, const float* dir, float* grad,
                        float* hvp, float* jvp, unsigned long long* counters,
                        cudaStream_t stream) {
  if (!b) return fail(CCM_ERR_INVALID, "batch is NULL");
  if (b->n == 0) return CCM_OK;
  if (!pose_a || !pose_b || !ybar || !grad) return fail(CCM_ERR_INVALID, "NULL pointer");
  if (dir && !hvp) return fail(CCM_ERR_INVALID, "dir given without hvp");
  KParams kp;
  ccm_status s = make_kparams(prm, &kp);
  if (s != CCM_OK) return s;
  if (kp.flags & CCM_FLAG_NO_CULL) return fail(CCM_ERR_INVALID, "the reverse pass always culls");
  if (kp.flags & (CCM_FLAG_BODY_UNION | CCM_FLAG_PROJECT | CCM_FLAG_SPLINE))
    return fail(CCM_ERR_INVALID,
                "the body-union, projection and spline variants are forward only");
  CCM_CUDA(cudaSetDevice(b->ctx->device), "cudaSetDevice");
  BwdLaunch L;
  L.g = b->ctx->dev_geom();
  L.pairs = static_cast<const PairRec*>(b->d_pairs.ptr);
  L.items = static_cast<const WorkItem*>(b->d_items.ptr);
  L.order = static_cast<const int32_t*>(b->d_item_order.ptr);
  L.n_items = b->n_items;
  L.item_off = static_cast<const int64_t*>(b->d_item_off.ptr);
  L.dev_items = nullptr;
  L.n_pairs = b->n;
  L.pose_a = pose_a;
  L.pose_b = pose_b;
  L.ybar = ybar;
  L.dir = dir;
  L.saved = saved;
  L.pair_order = saved && b->per_pair ? static_cast<const int32_t*>(b->d_pair_order.ptr) : nullptr;
  L.counters = counters;
  // the gradient and the H u pass count on separate words: with a saved record
  // they may run concurrently on two streams
  L.sched = static_cast<int*>(b->d_sched.ptr) + (dir ? 2 : 1);
  L.kp = kp;
  L.us = b->us;
  L.part = static_cast<float*>(b->d_part.ptr);
  L.grad = grad;
  L.dev_pairs = nullptr;
  L.hvp = hvp;
  L.jvp = dir ? jvp : nullptr;
  set_bwd_grids(*b, kp, dir != nullptr, &L);
  if (saved && b->per_pair && b->flat_cap > 0) {
    // the per-contact passes from the forward's contact list; the per-pair
    // kernel runs only if that list overflowed
    FlatLaunch F;
    F.g = L.g;
    F.pairs = L.pairs;
    F.row_pair = static_cast<const int32_t*>(b->d_row_pair.ptr);
    F.n_pairs = b->n;
    F.G = b->G;
    F.pose_a = pose_a;
    F.pose_b = pose_b;
    F.ybar = ybar;
    F.dir = dir;
    F.saved = saved;
    F.kp = kp;
    F.cl = b->contact_list();
    F.fp = b->flat_pass(dir != nullptr);
    F.grad = grad;
    F.hvp = hvp;
    F.jvp = dir ? jvp : nullptr;
    F.counters = counters;
    F.n_sm = b->ctx->n_sm;
    F.pdl = b->tuning.pdl == 0 ? 1 : 0;
    F.fallback_sched = L.sched;
    cudaError_t e = launch_flat_backward(F, stream);
    if (e != cudaSuccess) return cuda_fail(e, "per-contact backward launch");
    L.only_if = F.fp.sched + 2;
    L.after_chain = F.pdl != 0;
  }
  cudaError_t e = launch_backward(L, stream);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return CCM_OK;
}

void HostStep::release() {
  for (DevBuf* b : {&pa, &pb, &y, &saved, &ybar, &grad, &grad2, &hvp, &dir, &jvp}) b->release();
  if (cin) cudaStreamDestroy(cin);
  if (cout) cudaStreamDestroy(cout);
  for (cudaEvent_t& e : ev)
    if (e) cudaEventDestroy(e);
  cin = cout = nullptr;
}

void Batch::release() {
  if (hs) {
    hs->release();
    delete hs;
    hs = nullptr;
  }
  d_pairs.release();
  d_items.release();
  d_item_order.release();
  d_item_off.release();
  d_pair_order.release();
  d_sched.release();
  d_status.release();
  d_part.release();
  d_row_pair.release();
  for (DevBuf* b : {&d_fctl, &d_fcnt, &d_foff, &d_frecs, &d_fsorted, &d_ftiles, &d_unit_dir_off,
                    &d_rel, &d_live, &d_cand, &d_cand_m, &d_cval, &d_sval, &d_skey, &d_ffctl})
    b->release();
  for (auto& pass : d_fpass)
    for (DevBuf& b : pass) b.release();
  flat_cap = 0;
}

ccm_status run_forward(Batch* b, const float* pose_a, const float* pose_b, const ccm_params* prm,
                       float* y, float* saved, unsigned long long* counters, cudaStream_t stream) {
  if (!b) return fail(CCM_ERR_INVALID, "batch is NULL");
  if (b->n == 0) return CCM_OK;
  if (!pose_a || !pose_b || !y) return fail(CCM_ERR_INVALID, "NULL pose or output pointer");
  KParams kp;
  ccm_status s = make_kparams(prm, &kp);
  if (s != CCM_OK) return s;
  CCM_CUDA(cudaSetDevice(b->ctx->device), "cudaSetDevice");
  if ((kp.flags & (CCM_FLAG_BODY_UNION | CCM_FLAG_PROJECT | CCM_FLAG_SPLINE)) &&
      (saved || counters))
    return fail(CCM_ERR_INVALID,
                "the body-union, projection and spline variants keep no record and count no work");
  if (kp.flags & CCM_FLAG_SPLINE) {
    if (kp.flags & CCM_FLAG_BODY_UNION)
      return fail(CCM_ERR_INVALID, "the spline variant has no body union");
    {   // every piece of every body of the batch needs its spline
      std::lock_guard<std::mutex> lk(b->ctx->mu);
      const Context& c = *b->ctx;
      for (const PairRec& pr : b->pairs)
        for (int32_t bi : {pr.bodyA, pr.bodyB}) {
          const BodyRec& br = c.bodies[bi];
          if ((int64_t)c.splines.size() < (int64_t)br.p0 + br.np)
            return fail(CCM_ERR_INVALID, "body %d has no spline SDF", bi);
          for (int p = 0; p < br.np; ++p)
            if (c.splines[br.p0 + p].dims.x == 0)
              return fail(CCM_ERR_INVALID, "body %d has no spline SDF", bi);
        }
    }
    SplineLaunch Sp;
    Sp.g = b->ctx->dev_geom();
    Sp.splines = static_cast<const SplineRec*>(b->ctx->d_splines.ptr);
    Sp.coef = static_cast<const float4*>(b->ctx->d_spline_coef.ptr);
    Sp.pairs = static_cast<const PairRec*>(b->d_pairs.ptr);
    Sp.row_pair = static_cast<const int32_t*>(b->d_row_pair.ptr);
    Sp.G = b->G;
    Sp.pose_a = pose_a;
    Sp.pose_b = pose_b;
    Sp.kp = kp;
    Sp.y = y;
    Sp.n_sm = b->ctx->n_sm;
    const cudaError_t e = launch_spline_forward(Sp, stream);
    if (e != cudaSuccess) return cuda_fail(e, "spline forward launch");
    return CCM_OK;
  }
  if (kp.flags & CCM_FLAG_BODY_UNION) {
    UnionLaunch U;
    U.g = b->ctx->dev_geom();
    U.pairs = static_cast<const PairRec*>(b->d_pairs.ptr);
    U.row_pair = static_cast<const int32_t*>(b->d_row_pair.ptr);
    U.G = b->G;
    U.pose_a = pose_a;
    U.pose_b = pose_b;
    U.kp = kp;
    U.y = y;
    U.n_sm = b->ctx->n_sm;
    const cudaError_t e = launch_union_forward(U, stream);
    if (e != cudaSuccess) return cuda_fail(e, "body-union forward launch");
    return CCM_OK;
  }
  FwdLaunch L;
  L.g = b->ctx->dev_geom();
  L.pairs = static_cast<const PairRec*>(b->d_pairs.ptr);
  L.items = static_cast<const WorkItem*>(b->d_items.ptr);
  L.order = static_cast<const int32_t*>(b->d_item_order.ptr);
  L.n_items = b->n_items;
  L.dev_items = nullptr;
  L.pose_a = pose_a;
  L.pose_b = pose_b;
  L.kp = kp;
  L.us = b->us;
  L.y = y;
  L.saved = saved;
  L.counters = counters;
  L.sched = static_cast<int*>(b->d_sched.ptr);
  L.grid = b->grid;
  L.status = static_cast<int*>(b->d_status.ptr);
  const bool staged = b->flat_cap > 0 && b->tuning.flat_forward == 0 &&
                      !(kp.flags & CCM_FLAG_NO_CULL) && flat_forward_fits(b->mx.vmax, b->mx.fmax);
  const bool flat = saved && b->flat_cap > 0;
  if (flat || staged) {
    if (++b->list_tag == 0u) b->list_tag = 1u;   // a new tag per list (0: none)
  }
  if (staged) {
    // the flat forward; the per-item kernel below runs only if it overflowed
    // (then without a contact list: the reverse passes run per pair)
    FlatFwdLaunch F;
    F.g = L.g;
    F.pairs = L.pairs;
    F.row_pair = static_cast<const int32_t*>(b->d_row_pair.ptr);
    F.unit_dir_off = static_cast<const int64_t*>(b->d_unit_dir_off.ptr);
    F.n_pairs = b->n;
    F.G = b->G;
    F.n_dirs = b->n_dirs;
    F.pose_a = pose_a;
    F.pose_b = pose_b;
    F.kp = kp;
    F.y = y;
    F.saved = saved;
    F.hits = static_cast<uint32_t*>(b->d_ffhits.ptr);
    F.cl = b->contact_list();
    F.cl.tag = b->list_tag;
    F.sval = static_cast<float*>(b->d_sval.ptr);
    F.sval_key = static_cast<long long*>(b->d_skey.ptr);
    F.rel = static_cast<float*>(b->d_rel.ptr);
    F.live = static_cast<int4*>(b->d_live.ptr);
    F.cand_cap = b->cand_cap;
    F.cand = static_cast<int4*>(b->d_cand.ptr);
    F.cand_m = static_cast<float2*>(b->d_cand_m.ptr);
    F.cval = static_cast<float*>(b->d_cval.ptr);
    F.ctl = static_cast<unsigned long long*>(b->d_ffctl.ptr);
    F.counters = counters;
    F.vmax = b->mx.vmax;
    F.fmax = b->mx.fmax;
    // the gate stages the SDF body's planes per chunk (4 warps in 48 KB) unless a
    // piece is so large that a warp's chunk would hold few directions' planes
    // for a lot of shared memory; then it reads them from global memory
    // (tuning stage_planes bounds the chunk, as for the per-item kernel)
    // (512 by default: on the uneven batch 2.37 ms against 2.51 ms with 760)
    const int gate_cap = b->tuning.stage_planes ? std::min(b->tuning.stage_planes, 760) : 512;
    F.gate_planes = b->mx.fmax > kGateStageMaxPlanes
                        ? 0
                        : std::max(b->mx.fmax, std::min(b->mx.s_planes, gate_cap));
    F.stage_tma = b->us.stage_tma;
    F.wait_limit = b->us.wait_limit;
    F.status = static_cast<int*>(b->d_status.ptr);
    F.n_sm = b->ctx->n_sm;
    F.pdl = b->tuning.pdl == 0 ? 1 : 0;
    F.fallback_sched = L.sched;
    cudaError_t e = launch_flat_forward(F, stream);
    if (e != cudaSuccess) return cuda_fail(e, "flat forward launch");
    L.only_if = F.ctl + kFfOverflow;
    L.after_chain = F.pdl != 0;   // then launched behind the chain, which zeroed its counter
    e = launch_forward(L, stream);
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
    return CCM_OK;
  }
  if (flat) {
    L.cl = b->contact_list();
    L.cl.tag = b->list_tag;
  }
  cudaError_t e = launch_forward(L, stream);
  if (e != cudaSuccess) return cuda_fail(e, "forward launch");
  if (flat) {
    e = launch_flat_prep(L.cl, b->G, b->ctx->n_sm, stream);
    if (e != cudaSuccess) return cuda_fail(e, "contact list launch");
  }
  return CCM_OK;
}

}  // namespace ccm
