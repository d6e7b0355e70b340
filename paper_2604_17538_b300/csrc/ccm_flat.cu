// Per-contact reverse passes (the derivatives of Sec. 4.2-4.4 of arxiv
// 2604.17538) driven by the forward's contact list (ccm_clist.cuh).
//
// The per-warp reverse kernels (ccm_bwd.cu) re-gate piece pairs, re-cull
// features and build lists before they reach the few contacts of non-zero
// weight; most of their lanes idle on short lists.  Here the forward has
// already named those contacts, so every stage is a flat loop with one
// contact (or one group, or one pair) per thread and every lane busy:
//   eval     recomputes each contact (SDF, sphere trace, mollifier) on T;
//   fold     blends each group's contacts in their fixed order (online
//            softmax, Sec. 4.4) and forms its adjoint coefficients, J u row
//            and output-transform terms (four lanes per group with contacts);
//   adjoint  recomputes each contact with its group's coefficients and
//            back-propagates into its feature points: a force and a torque;
//   reduce   sums a pair's forces, torques and output terms (one warp per
//            pair, fixed lane order) into its 12 twist components.
// Nothing is stored between the eval and adjoint kernels but the contact
// values the fold needs: the SDF is recomputed.  A pair's results depend only
// on its own contacts and their order, so they are the same in any batch.
#include <algorithm>

#include "ccm_adjoint.cuh"
#include "ccm_clist.cuh"
#include "ccm_flat.h"
#include "ccm_launch.h"

namespace ccm {

// ---------------------------------------------------------------------------
// fixed order of the list
// ---------------------------------------------------------------------------
// Exclusive prefixes of the per-group counts in two kernels over tiles of
// 4096 groups (1024 threads x 4): the tile totals, then per tile the sum of
// the totals before it plus the tile's own block scan.  The last tile writes
// the totals NV, NE and the list's tag.
constexpr int kScanTile = 4096;

__device__ __forceinline__ void block_scan2(long long& v, long long& e, long long* wv,
                                            long long* we) {
  // inclusive block-wide scan of (v, e) over 1024 threads
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long a = __shfl_up_sync(kFull, v, o), b = __shfl_up_sync(kFull, e, o);
    if (lane >= o) { v += a; e += b; }
  }
  if (lane == 31) { wv[w] = v; we[w] = e; }
  __syncthreads();
  if (w == 0) {
    long long x = wv[lane], y = we[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long a = __shfl_up_sync(kFull, x, o), b = __shfl_up_sync(kFull, y, o);
      if (lane >= o) { x += a; y += b; }
    }
    wv[lane] = x;
    we[lane] = y;
  }
  __syncthreads();
  if (w > 0) { v += wv[w - 1]; e += we[w - 1]; }
}

// Counts of a tile: the vertex and edge contacts packed into one word (low
// and high 32 bits; a list's counts fit 31 bits, so the low half never
// carries) and the number of groups with contacts.
__global__ void __launch_bounds__(1024) clist_tile_sum_kernel(ContactList cl, int64_t G,
                                                              long long* tile_sum) {
  pdl_wait();
  __shared__ long long wv[32], we[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
  long long sp = 0, sl = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (base + q < G) {
      const long long v = cl.cnt_v[base + q], e = cl.cnt_e[base + q];
      sp += v | (e << 32);
      sl += (v + e) > 0;
    }
  block_scan2(sp, sl, wv, we);
  if (threadIdx.x == 1023) {
    tile_sum[2 * blockIdx.x] = sp;
    tile_sum[2 * blockIdx.x + 1] = sl;
  }
}

__global__ void __launch_bounds__(1024) clist_scan_kernel(ContactList cl, int64_t G,
                                                          const long long* tile_sum) {
  pdl_wait();
  __shared__ long long wv[32], we[32], pre[2];
  const int t = threadIdx.x;
  // totals of the tiles before this one
  long long pp = 0, pl = 0;
  for (int b = t; b < (int)blockIdx.x; b += 1024) { pp += tile_sum[2 * b]; pl += tile_sum[2 * b + 1]; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pp += __shfl_xor_sync(kFull, pp, o);
    pl += __shfl_xor_sync(kFull, pl, o);
  }
  if ((t & 31) == 0) { wv[t >> 5] = pp; we[t >> 5] = pl; }
  __syncthreads();
  if (t == 0) {
    long long a = 0, b = 0;
    for (int w = 0; w < 32; ++w) { a += wv[w]; b += we[w]; }
    pre[0] = a;
    pre[1] = b;
  }
  __syncthreads();
  const long long p0 = pre[0], p0l = pre[1];
  __syncthreads();   // wv / we are reused by the scan
  const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * t;
  int cv[4], ce[4];
  long long sp = 0, sl = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    cv[q] = base + q < G ? cl.cnt_v[base + q] : 0;
    ce[q] = base + q < G ? cl.cnt_e[base + q] : 0;
    sp += (long long)cv[q] | ((long long)ce[q] << 32);
    sl += (cv[q] + ce[q]) > 0;
  }
  long long ip = sp, il = sl;
  block_scan2(ip, il, wv, we);
  const long long op = p0 + ip - sp;
  long long ov = op & 0xffffffffll, oe = op >> 32, ol = p0l + il - sl;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (base + q < G) {
      cl.off_v[base + q] = (int32_t)ov;
      cl.off_e[base + q] = (int32_t)oe;
      cl.cnt_v[base + q] = 0;   // the counts become the scatter's cursors
      cl.cnt_e[base + q] = 0;
      if (cv[q] + ce[q] > 0) cl.live_g[ol++] = (int32_t)(base + q);
    }
    ov += cv[q];
    oe += ce[q];
  }
  if (blockIdx.x == gridDim.x - 1 && t == 1023) {
    const long long tp = p0 + ip;
    cl.off_v[G] = (int32_t)(tp & 0xffffffffll);
    cl.off_e[G] = (int32_t)(tp >> 32);
    cl.ctl[kCtlNV] = (unsigned long long)(tp & 0xffffffffll);
    cl.ctl[kCtlNE] = (unsigned long long)(tp >> 32);
    cl.ctl[kCtlNG] = (unsigned long long)(p0l + il);
    cl.ctl[kCtlTag] = cl.tag;
  }
}

// Every record to its place: vertex contacts in [0, NV) by group and rank,
// then edge contacts in [NV, NV + NE).
__global__ void clist_scatter_kernel(ContactList cl) {
  pdl_wait();
  if (cl.ctl[kCtlOverflow]) return;
  const int64_t n = (int64_t)cl.ctl[kCtlCursor];
  const int64_t NV = (int64_t)cl.ctl[kCtlNV];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int4 r = cl.recs[i];
    const uint32_t w = (uint32_t)r.w;
    const uint32_t kind = w >> 31;
    const int feat = (int)((w >> kRankBits) & ((1u << kFeatBits) - 1u));
    const int seq = (int)(w & ((1u << kRankBits) - 1u));
    const int64_t dest = kind ? NV + cl.off_e[r.x] + seq : (int64_t)cl.off_v[r.x] + seq;
    cl.sorted[dest] = make_int4(r.x, r.y, r.z, (int)((kind << 31) | (uint32_t)feat));
  }
}

int64_t flat_scan_tiles(int64_t G) { return std::max<int64_t>(1, (G + kScanTile - 1) / kScanTile); }

cudaError_t launch_flat_prep_scan(const ContactList& cl, int64_t G, cudaStream_t stream,
                                  bool pdl) {
  const int64_t tiles = flat_scan_tiles(G);
  cudaError_t e = launch_k(pdl, clist_tile_sum_kernel, (int)tiles, 1024, 0, stream, cl, G,
                           cl.tile_sum);
  if (e != cudaSuccess) return e;
  return launch_k(pdl, clist_scan_kernel, (int)tiles, 1024, 0, stream, cl, G, cl.tile_sum);
}

cudaError_t launch_flat_prep(const ContactList& cl, int64_t G, int n_sm, cudaStream_t stream) {
  cudaError_t e = launch_flat_prep_scan(cl, G, stream);
  if (e != cudaSuccess) return e;
  clist_scatter_kernel<<<4 * n_sm, 256, 0, stream>>>(cl);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// one contact on T
// ---------------------------------------------------------------------------
template <class T> struct RecGeom {
  const float4* pl;   // planes of the SDF piece
  int nf;
  int side;           // 0: F = A, S = B; 1: F = B, S = A
  int64_t pair;
  PoseT<T> PS;        // pose of the SDF body
  T Rr[9], tr[3];     // relative pose S <- F
  V3T<T> tba;         // t_B - t_A
};

// Poses of a record's pair side on T (with the direction's tangents for
// Dual) and its relative pose, in the arithmetic of the per-pair kernel.
template <class T>
__device__ __forceinline__ void rec_geom(const FlatLaunch& L, int4 rec, RecGeom<T>& G) {
  const int rp = L.row_pair[rec.x];
  G.pair = rp >> 1;
  G.side = rp & 1;
  const PieceRec sp = L.g.pieces[rec.y];
  G.pl = L.g.planes + sp.f0;
  G.nf = sp.nf;
  const float* pF = (G.side == 0 ? L.pose_a : L.pose_b) + 12 * G.pair;
  const float* pS = (G.side == 0 ? L.pose_b : L.pose_a) + 12 * G.pair;
  const float* uF = L.dir ? L.dir + 12 * G.pair + (G.side == 0 ? 0 : 6) : nullptr;
  const float* uS = L.dir ? L.dir + 12 * G.pair + (G.side == 0 ? 6 : 0) : nullptr;
  PoseT<T> PF;
  load_pose_t(pF, uF, PF);
  load_pose_t(pS, uS, G.PS);
  const PoseT<T>& S = G.PS;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      G.Rr[3 * i + j] = fma_t(S.R[i], PF.R[j], fma_t(S.R[3 + i], PF.R[3 + j], S.R[6 + i] * PF.R[6 + j]));
  const V3T<T> q = rotT(S.R, v3(PF.t[0] - S.t[0], PF.t[1] - S.t[1], PF.t[2] - S.t[2]));
  G.tr[0] = q.x;
  G.tr[1] = q.y;
  G.tr[2] = q.z;
  G.tba = G.side == 0 ? v3(S.t[0] - PF.t[0], S.t[1] - PF.t[1], S.t[2] - PF.t[2])
                      : v3(PF.t[0] - S.t[0], PF.t[1] - S.t[1], PF.t[2] - S.t[2]);
}

template <class T>
__device__ __forceinline__ V3T<T> to_sdf_frame(const RecGeom<T>& G, float4 v) {
  const V3T<T> x = rot(G.Rr, v3(T(v.x), T(v.y), T(v.z)));
  return v3(x.x + G.tr[0], x.y + G.tr[1], x.z + G.tr[2]);
}

// Force and torque (about t_A, world frame) of a contact-point adjoint xb at
// x (SDF frame): +(f, p x f) when A carries the features, -(...) otherwise.
template <class T>
__device__ __forceinline__ void add_point_force(const RecGeom<T>& G, V3T<T> x, V3T<T> xb,
                                                V3T<T>& F, V3T<T>& M) {
  const V3T<T> f = rot(G.PS.R, xb);
  V3T<T> p = rot(G.PS.R, x);
  if (G.side == 0) p = v3(p.x + G.tba.x, p.y + G.tba.y, p.z + G.tba.z);
  const V3T<T> m = cross3(p, f);
  if (G.side == 0) {
    F = v3(F.x + f.x, F.y + f.y, F.z + f.z);
    M = v3(M.x + m.x, M.y + m.y, M.z + m.z);
  } else {
    F = v3(F.x - f.x, F.y - f.y, F.z - f.z);
    M = v3(M.x - m.x, M.y - m.y, M.z - m.z);
  }
}

template <class T> __device__ __forceinline__ void store_t(T* p, T v) { *p = v; }

// next 32 records of a warp: edge contacts first (the long ones), then vertex
// contacts; returns the record index of this lane or -1
__device__ __forceinline__ int64_t grab(int* sched, int64_t NV, int64_t NE, int lane,
                                        int64_t& base) {
  int b = 0;
  if (lane == 0) b = atomicAdd(sched, 32);
  base = __shfl_sync(kFull, b, 0);
  const int64_t k = base + lane;
  if (k >= NV + NE) return -1;
  return k < NE ? NV + k : k - NE;
}

struct FlatCounts {
  unsigned long long recs = 0, live = 0, maxp = 0, g1 = 0, v1 = 0, h2 = 0, g2 = 0;
};

__device__ __forceinline__ void flush_counts(const FlatCounts& c, unsigned long long* out,
                                             int lane) {
  const unsigned long long v[8] = {c.recs, c.live, c.maxp, 0ull, c.g1, c.v1, c.h2, c.g2};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    unsigned long long x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (lane == 0 && x) atomicAdd(out + q, x);
  }
}

// ---------------------------------------------------------------------------
// eval: contact values for the fold
// ---------------------------------------------------------------------------
template <class T, bool kCount>
__global__ void __launch_bounds__(128) flat_eval_kernel(FlatLaunch L) {
  pdl_wait();
  if (L.fp.sched[2]) return;
  const int lane = threadIdx.x & 31;
  const int64_t NV = (int64_t)L.cl.ctl[kCtlNV], NE = (int64_t)L.cl.ctl[kCtlNE];
  const KParams& kp = L.kp;
  T* cval = static_cast<T*>(L.fp.cval);
  FlatCounts cnt;
  const int K = kp.trace_iters;
  for (;;) {
    int64_t base;
    const int64_t k = grab(L.fp.sched, NV, NE, lane, base);
    if (base >= NV + NE) break;
    if (k < 0) continue;
    const int4 rec = L.cl.sorted[k];
    RecGeom<T> G;
    rec_geom(L, rec, G);
    const PieceRec fpc = L.g.pieces[rec.z];
    const bool edge = ((uint32_t)rec.w >> 31) != 0u;
    const int feat = rec.w & ((1 << kFeatBits) - 1);
    SdfT<T> c;
    V3T<T> p;
    if (!edge) {
      p = to_sdf_frame(G, L.g.verts[fpc.v0 + feat]);
      const float m = max_plane(G.pl, G.nf, val(p.x), val(p.y), val(p.z));
      c = sdf_t<T, 1>(G.pl, G.nf, p, m, p, kp);
      if (kCount) { cnt.maxp += G.nf; cnt.g1 += G.nf; }
    } else {
      const uint32_t e = L.g.edges[fpc.e0 + feat];
      const V3T<T> a = to_sdf_frame(G, L.g.verts[fpc.v0 + (e & 0xffff)]);
      const V3T<T> b = to_sdf_frame(G, L.g.verts[fpc.v0 + (e >> 16)]);
      const float mI = max_plane(G.pl, G.nf, val(a.x), val(a.y), val(a.z));
      const float mII = max_plane(G.pl, G.nf, val(b.x), val(b.y), val(b.z));
      const SdfT<T> ca = sdf_t<T, 1>(G.pl, G.nf, a, mI, a, kp);
      const SdfT<T> cb = sdf_t<T, 1>(G.pl, G.nf, b, mII, b, kp);
      Coef<T> none{};
      V3T<T> xbI, xbII;
      edge_t<T, false, 0>(G.pl, G.nf, a, b, mI, mII, ca.phi, cb.phi, ca.g, cb.g, none, kp, c, p,
                          xbI, xbII);
      if (kCount) {
        cnt.maxp += 2ull * G.nf;
        cnt.g1 += 3ull * G.nf;
        cnt.v1 += (unsigned long long)G.nf * 2 * (K > 0 ? K - 1 : 0);
      }
    }
    T f, fpr;
    transition_t(c.phi, kp, f, fpr);
    const T dc = fma_t(f, c.phi - kp.d_max, T(kp.d_max));
    T* o = cval + 8 * k;
    store_t(o + 0, f);
    store_t(o + 1, dc);
    store_t(o + 2, p.x);
    store_t(o + 3, p.y);
    store_t(o + 4, p.z);
    store_t(o + 5, c.g.x);
    store_t(o + 6, c.g.y);
    store_t(o + 7, c.g.z);
    if (kCount) cnt.recs += 1;
  }
  if (kCount && L.counters) flush_counts(cnt, L.counters, lane);
}

// ---------------------------------------------------------------------------
// fold: one group with contacts per kFoldSplit lanes (the scan's list of
// them; fold_split); the groups without contacts have no adjoint, and the
// reduce kernel gives them zero output terms and tangent rows
// ---------------------------------------------------------------------------
constexpr int kFoldSplit = 4;   // lanes per group in the folds

template <class T>
__global__ void __launch_bounds__(128) flat_fold_kernel(FlatLaunch L) {
  pdl_wait();
  if (L.fp.sched[2]) return;
  const int64_t NV = (int64_t)L.cl.ctl[kCtlNV], NG = (int64_t)L.cl.ctl[kCtlNG];
  const T* cval = static_cast<const T*>(L.fp.cval);
  Coef<T>* coef = static_cast<Coef<T>*>(L.fp.coef);
  T* ot = static_cast<T*>(L.fp.oterm);
  const int sub = threadIdx.x & (kFoldSplit - 1);
  const int64_t per_block = blockDim.x / kFoldSplit;
  // block-uniform loop: every lane takes part in the fold's shuffles
  for (int64_t base = (int64_t)blockIdx.x * per_block; base < NG;
       base += (int64_t)gridDim.x * per_block) {
    const int64_t i = base + threadIdx.x / kFoldSplit;
    const bool valid = i < NG;
    const int64_t g = valid ? L.cl.live_g[i] : 0;
    int64_t v0 = 0, v1 = 0, e0 = 0, e1 = 0;
    PoseT<T> PS;
    if (valid) {
      v0 = L.cl.off_v[g]; v1 = L.cl.off_v[g + 1];
      e0 = NV + L.cl.off_e[g]; e1 = NV + L.cl.off_e[g + 1];
      if (sub == 0) {   // the pose's loads overlap the fold
        const int rp = L.row_pair[g];
        const int64_t pair = rp >> 1;
        const int side = rp & 1;
        load_pose_t((side == 0 ? L.pose_b : L.pose_a) + 12 * pair,
                    L.dir ? L.dir + 12 * pair + (side == 0 ? 6 : 0) : nullptr, PS);
      }
    }
    PartT<T> acc;
    fold_split<T, kFoldSplit>(cval, v0, v1, e0, e1, L.kp.c_blend, sub, acc);
    if (valid && sub == 0) {
      Coef<T> cf;
      V3T<T> ow, ov;
      form_coef(acc, L.ybar + 8 * g, PS, L.jvp ? L.jvp + 8 * g : nullptr, cf, ow, ov);
      coef[g] = cf;
      T* o = ot + 6 * g;
      o[0] = ow.x; o[1] = ow.y; o[2] = ow.z;
      o[3] = ov.x; o[4] = ov.y; o[5] = ov.z;
    }
  }
}

// ---------------------------------------------------------------------------
// adjoint: force and torque of each contact
// ---------------------------------------------------------------------------
template <class T, bool kCount>
__global__ void __launch_bounds__(128) flat_adjoint_kernel(FlatLaunch L) {
  pdl_wait();
  if (L.fp.sched[2]) return;
  const int lane = threadIdx.x & 31;
  const int64_t NV = (int64_t)L.cl.ctl[kCtlNV], NE = (int64_t)L.cl.ctl[kCtlNE];
  const KParams& kp = L.kp;
  const Coef<T>* coef = static_cast<const Coef<T>*>(L.fp.coef);
  T* force = static_cast<T*>(L.fp.force);
  FlatCounts cnt;
  const int K = kp.trace_iters;
  for (;;) {
    int64_t base;
    const int64_t k = grab(L.fp.sched + 1, NV, NE, lane, base);
    if (base >= NV + NE) break;
    if (k < 0) continue;
    const int4 rec = L.cl.sorted[k];
    const Coef<T> cf = coef[rec.x];
    V3T<T> F = zero3t<T>(), M = zero3t<T>();
    if (cf.live) {
      RecGeom<T> G;
      rec_geom(L, rec, G);
      const PieceRec fpc = L.g.pieces[rec.z];
      const bool edge = ((uint32_t)rec.w >> 31) != 0u;
      const int feat = rec.w & ((1 << kFeatBits) - 1);
      if (!edge) {
        const V3T<T> x = to_sdf_frame(G, L.g.verts[fpc.v0 + feat]);
        const float m = max_plane(G.pl, G.nf, val(x.x), val(x.y), val(x.z));
        const SdfT<T> c = sdf_t<T, 2>(G.pl, G.nf, x, m, cf.nb, kp);
        add_point_force(G, x, contact_adjoint(c, x, cf, kp), F, M);
        if (kCount) { cnt.maxp += G.nf; cnt.h2 += G.nf; }
      } else {
        const uint32_t e = L.g.edges[fpc.e0 + feat];
        const V3T<T> a = to_sdf_frame(G, L.g.verts[fpc.v0 + (e & 0xffff)]);
        const V3T<T> b = to_sdf_frame(G, L.g.verts[fpc.v0 + (e >> 16)]);
        const float mI = max_plane(G.pl, G.nf, val(a.x), val(a.y), val(a.z));
        const float mII = max_plane(G.pl, G.nf, val(b.x), val(b.y), val(b.z));
        const SdfT<T> ca = sdf_t<T, 1>(G.pl, G.nf, a, mI, a, kp);
        const SdfT<T> cb = sdf_t<T, 1>(G.pl, G.nf, b, mII, b, kp);
        SdfT<T> c;
        V3T<T> pe, xbI, xbII;
        edge_t<T, true, 0>(G.pl, G.nf, a, b, mI, mII, ca.phi, cb.phi, ca.g, cb.g, cf, kp, c, pe,
                           xbI, xbII);
        add_point_force(G, a, xbI, F, M);
        add_point_force(G, b, xbII, F, M);
        if (kCount) {
          cnt.maxp += 2ull * G.nf;
          cnt.g2 += (unsigned long long)G.nf * (2 + 2 * (K > 0 ? K - 1 : 0));
          cnt.h2 += G.nf;
        }
      }
      if (kCount) cnt.live += 1;
    }
    T* o = force + 6 * k;
    o[0] = F.x; o[1] = F.y; o[2] = F.z;
    o[3] = M.x; o[4] = M.y; o[5] = M.z;
  }
  if (kCount && L.counters) flush_counts(cnt, L.counters, lane);
}

// ---------------------------------------------------------------------------
// reduce: one warp per pair
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void add3(V3T<T>& a, const T* p) {
  a = v3(a.x + p[0], a.y + p[1], a.z + p[2]);
}
template <class T> __device__ __forceinline__ V3T<T> warp_sum3(V3T<T> a) {
  return v3(warp_sum_t(a.x), warp_sum_t(a.y), warp_sum_t(a.z));
}

template <class T>
__global__ void __launch_bounds__(128) flat_reduce_kernel(FlatLaunch L) {
  pdl_wait();
  if (L.fp.sched[2]) return;
  const int lane = threadIdx.x & 31;
  const int64_t NV = (int64_t)L.cl.ctl[kCtlNV];
  const T* force = static_cast<const T*>(L.fp.force);
  const T* ot = static_cast<const T*>(L.fp.oterm);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < L.n_pairs;
       p += warps) {
    const PairRec pr = L.pairs[p];
    const int64_t g0 = pr.goff, g1 = p + 1 < L.n_pairs ? L.pairs[p + 1].goff : L.G;
    const int npA = L.g.bodies[pr.bodyA].np;
    V3T<T> F = zero3t<T>(), M = F, oAw = F, oAv = F, oBw = F, oBv = F;
    for (int64_t k = L.cl.off_v[g0] + lane; k < L.cl.off_v[g1]; k += 32) {
      add3(F, force + 6 * k);
      add3(M, force + 6 * k + 3);
    }
    for (int64_t k = NV + L.cl.off_e[g0] + lane; k < NV + L.cl.off_e[g1]; k += 32) {
      add3(F, force + 6 * k);
      add3(M, force + 6 * k + 3);
    }
    for (int64_t g = g0 + lane; g < g1; g += 32) {
      if (L.cl.off_v[g + 1] == L.cl.off_v[g] && L.cl.off_e[g + 1] == L.cl.off_e[g]) {
        // no contact: no output terms, a zero tangent row
        if (L.jvp) {
          float4* jr = reinterpret_cast<float4*>(L.jvp + 8 * g);
          jr[0] = make_float4(0.f, 0.f, 0.f, 0.f);
          jr[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      } else if (g - g0 < npA) {   // side 0: the SDF body is B
        add3(oBw, ot + 6 * g);
        add3(oBv, ot + 6 * g + 3);
      } else {
        add3(oAw, ot + 6 * g);
        add3(oAv, ot + 6 * g + 3);
      }
    }
    F = warp_sum3(F);
    M = warp_sum3(M);
    oAw = warp_sum3(oAw);
    oAv = warp_sum3(oAv);
    oBw = warp_sum3(oBw);
    oBv = warp_sum3(oBv);
    if (lane == 0) {
      const float* uA = L.dir ? L.dir + 12 * p : nullptr;
      const float* uB = L.dir ? L.dir + 12 * p + 6 : nullptr;
      PoseT<T> PA, PB;
      load_pose_t(L.pose_a + 12 * p, uA, PA);
      load_pose_t(L.pose_b + 12 * p, uB, PB);
      const V3T<T> tba = v3(PB.t[0] - PA.t[0], PB.t[1] - PA.t[1], PB.t[2] - PA.t[2]);
      write_twists(F, M, oAw, oAv, oBw, oBv, tba, uA, uB, L.grad + 12 * p,
                   L.hvp ? L.hvp + 12 * p : nullptr);
    }
  }
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
void flat_pass_bytes(bool dual, int64_t cap, int64_t G, size_t* cval, size_t* force,
                     size_t* coef, size_t* oterm) {
  const size_t t = dual ? sizeof(Dual) : sizeof(float);
  *cval = t * 8 * (size_t)cap;
  *force = t * 6 * (size_t)cap;
  *coef = (dual ? sizeof(Coef<Dual>) : sizeof(Coef<float>)) * (size_t)G;
  *oterm = t * 6 * (size_t)G;
}

// The pass uses the list only if it did not overflow and the saved record
// carries its tag (the record and the list come from the same forward).
__global__ void flat_gate_kernel(ContactList cl, const float* __restrict__ saved, int* sched,
                                 int* fallback_sched) {
  pdl_wait();
  const uint32_t tag = reinterpret_cast<const uint32_t*>(saved)[kSavedTag];
  sched[0] = 0;
  sched[1] = 0;
  if (fallback_sched) *fallback_sched = 0;
  sched[2] = (cl.ctl[kCtlOverflow] != 0ull || tag == 0u ||
              (unsigned long long)tag != cl.ctl[kCtlTag]) ? 1 : 0;
}

template <class T>
static cudaError_t launch_flat_t(const FlatLaunch& L, cudaStream_t stream) {
  const bool pdl = L.pdl != 0;
  cudaError_t e = launch_k(pdl, flat_gate_kernel, 1, 1, 0, stream, L.cl, L.saved, L.fp.sched,
                           L.fallback_sched);
  if (e != cudaSuccess) return e;
  const int rec_blocks = 16 * L.n_sm;   // persistent: warps draw 32 contacts at a time
  e = launch_k(pdl, L.counters ? flat_eval_kernel<T, true> : flat_eval_kernel<T, false>,
               rec_blocks, 128, 0, stream, L);
  if (e != cudaSuccess) return e;
  // groups with contacts: at most G, kFoldSplit lanes each
  const int gb = (int)std::max<int64_t>(
      1, std::min<int64_t>((kFoldSplit * L.G + 127) / 128, 16 * L.n_sm));
  if ((e = launch_k(pdl, flat_fold_kernel<T>, gb, 128, 0, stream, L)) != cudaSuccess) return e;
  e = launch_k(pdl, L.counters ? flat_adjoint_kernel<T, true> : flat_adjoint_kernel<T, false>,
               rec_blocks, 128, 0, stream, L);
  if (e != cudaSuccess) return e;
  const int pb = (int)std::max<int64_t>(1, std::min<int64_t>((L.n_pairs + 3) / 4, 64 * L.n_sm));
  return launch_k(pdl, flat_reduce_kernel<T>, pb, 128, 0, stream, L);
}

cudaError_t launch_flat_backward(const FlatLaunch& L, cudaStream_t stream) {
  if (L.dir) return launch_flat_t<Dual>(L, stream);
  FlatLaunch M = L;
  M.hvp = nullptr;
  M.jvp = nullptr;
  return launch_flat_t<float>(M, stream);
}

}  // namespace ccm
