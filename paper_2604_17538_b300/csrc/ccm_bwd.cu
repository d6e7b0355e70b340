// Reverse pass of the contact manifold (Sec. 4.2-4.4 of arxiv 2604.17538):
// a hand-written adjoint, templated on the scalar type.  With T = float it
// gives the gradient of L = <ybar, y> with respect to the twists of the two
// poses; with T = Dual (poses seeded with the tangent of a direction u) the
// same code yields, forward-over-reverse, H u and the output tangents J u.
//
// One warp runs one work item (a unit (pair, side) or a slice of its feature
// pieces) like the forward kernel and re-derives everything it needs -- the
// per-vertex SDF is recomputed, never stored:
//   pass 1  recomputes the blends of the unit's groups (online softmax);
//   then    each group's adjoint coefficients are formed from ybar;
//   pass 2  recomputes every contact and back-propagates through the blend,
//           the mollifier (Sec. 4.3), the LSE SDF (its gradient and the
//           Hessian-vector product (sum_k w_k n_k n_k^T - g g^T) v / tau),
//           the soft clip, midpoint and sphere-trace steps of an edge
//           (Sec. 4.2) into the feature points, whose adjoints x_bar are
//           summed as sum x_bar and sum x cross x_bar in the SDF frame.
// The item's 12 twist components are written to a per-item slot; a second
// kernel adds the slots of each pair in a fixed order (deterministic).
#include <algorithm>
#include <mutex>

#include "ccm_adjoint.cuh"
#include "ccm_unit.cuh"
#include "ccm_bwd.h"
#include "ccm_launch.h"

namespace ccm {


// List memo of the per-pair reverse pass: when a chunk of groups fits one
// S chunk and one list, the adjoint sweep reuses the recompute sweep's lists
// (same directions, same budgets, so the same lists) instead of rebuilding
// them, and visits only the vertices and edges whose contact had f > 0 (plus
// the corners such edges start their traces from): the others have a zero
// adjoint.  Layout (ints): S chunks, lists, nd, TV, TE, n_v, n_e, unused,
// then the vertex-item bits, then the edge-item bits.
constexpr int kMemoHead = 8;

// ---------------------------------------------------------------------------
// slice of the backward kernel (per warp)
// ---------------------------------------------------------------------------
template <class T> struct BwdSlice {
  float4* planes;     // [plane_budget]
  int2* sp;           // [2 spiece_budget] (both bodies in the per-pair pass)
  V3T<T>* xs;         // [vert_budget] F vertices in the S frame
  uint32_t* edges;    // [edge_budget]
  int4* fp;           // [32]
  float4* fs;         // [32]
  PartT<T>* acc;      // [32]
  Coef<T>* coef;      // [32], the same slots as acc
  int* dir;           // [32]
  int* dsub;          // [32]
  int* pv;            // [33]
  int* pe;            // [33]
  float* m;           // [item_v]
  T* phi;             // [item_v]
  V3T<T>* grad;       // [item_v]
  uint16_t* vlist;    // [item_v]
  uint16_t* elist;    // [item_e]
  uint8_t* need;      // [item_v]
  uint16_t* am;       // [item_v] a plane attaining the max-plane value (in grad's space)
  int* gside;         // [groups] side of each group: 0 (F = A, S = B) or 1 (F = B, S = A)
  PoseT<T>* spose;    // [2] pose of the SDF body of side 0 (B) and side 1 (A)
  V3T<T>* tba;        // [1] t_B - t_A
  T* pacc;            // [18] pair totals: F, M (about t_A), output terms of A and B
  PoseT<T>* rel;      // [2] relative pose S <- F of side 0 and side 1
  int* memo;          // list memo of the per-pair pass (see kMemoHead)
  uint32_t* hit;      // [groups * hw] directions that gave a contact in pass 1
  int hw;             // hit words per group (UnitShape::hit_words)
};


template <class T> __host__ __device__ constexpr int group_table_bytes() {
  return (int)(sizeof(PartT<T>) > sizeof(Coef<T>) ? sizeof(PartT<T>) : sizeof(Coef<T>));
}

template <class T> __host__ __device__ inline int bwd_slice_bytes(const UnitShape& u) {
  int b = 0;
  b += align16i(4 * u.groups_b);
  b += align16i((int)sizeof(PoseT<T>) * 2);
  b += align16i((int)sizeof(V3T<T>));
  b += align16i((int)sizeof(T) * 18);
  b += align16i((int)sizeof(PoseT<T>) * 2);
  b += align16i(4 * (kMemoHead + (u.item_vb + 31) / 32 + (u.item_eb + 31) / 32));
  b += align16i(4 * u.hit_words * u.groups_b);
  b += 16 * u.plane_budget;
  b += align16i(8 * 2 * u.spiece_budget);
  b += align16i((int)sizeof(V3T<T>) * u.vert_budget);
  b += align16i(4 * u.edge_budget);
  b += 16 * u.groups_b * 2;
  b += align16i(group_table_bytes<T>() * u.groups_b);
  b += align16i(4 * kPending) * 2;
  b += align16i(4 * (kPending + 1)) * 2;
  b += align16i(4 * u.item_vb);
  b += align16i((int)sizeof(T) * u.item_vb);
  b += align16i((int)sizeof(V3T<T>) * u.item_vb);
  b += align16i(2 * u.item_vb);
  b += align16i(2 * u.item_eb);
  b += align16i(u.item_vb);
  return b;
}

template <class T> __device__ inline BwdSlice<T> bwd_slice(unsigned char* p, const UnitShape& u) {
  BwdSlice<T> s;
  s.gside = reinterpret_cast<int*>(p);          p += align16i(4 * u.groups_b);
  s.spose = reinterpret_cast<PoseT<T>*>(p);     p += align16i((int)sizeof(PoseT<T>) * 2);
  s.tba = reinterpret_cast<V3T<T>*>(p);         p += align16i((int)sizeof(V3T<T>));
  s.pacc = reinterpret_cast<T*>(p);             p += align16i((int)sizeof(T) * 18);
  s.rel = reinterpret_cast<PoseT<T>*>(p);       p += align16i((int)sizeof(PoseT<T>) * 2);
  s.memo = reinterpret_cast<int*>(p);
  p += align16i(4 * (kMemoHead + (u.item_vb + 31) / 32 + (u.item_eb + 31) / 32));
  s.hit = reinterpret_cast<uint32_t*>(p);       p += align16i(4 * u.hit_words * u.groups_b);
  s.hw = u.hit_words;
  s.planes = reinterpret_cast<float4*>(p);     p += 16 * u.plane_budget;
  s.sp = reinterpret_cast<int2*>(p);           p += align16i(8 * 2 * u.spiece_budget);
  s.xs = reinterpret_cast<V3T<T>*>(p);         p += align16i((int)sizeof(V3T<T>) * u.vert_budget);
  s.edges = reinterpret_cast<uint32_t*>(p);    p += align16i(4 * u.edge_budget);
  s.fp = reinterpret_cast<int4*>(p);           p += 16 * u.groups_b;
  s.fs = reinterpret_cast<float4*>(p);         p += 16 * u.groups_b;
  // a group's blend partial (sweep 1) and its adjoint coefficients (sweep 2)
  // share one slot: the coefficients are formed from the partial in registers
  s.acc = reinterpret_cast<PartT<T>*>(p);
  s.coef = reinterpret_cast<Coef<T>*>(p);      p += align16i(group_table_bytes<T>() * u.groups_b);
  s.dir = reinterpret_cast<int*>(p);           p += align16i(4 * kPending);
  s.dsub = reinterpret_cast<int*>(p);          p += align16i(4 * kPending);
  s.pv = reinterpret_cast<int*>(p);            p += align16i(4 * (kPending + 1));
  s.pe = reinterpret_cast<int*>(p);            p += align16i(4 * (kPending + 1));
  s.m = reinterpret_cast<float*>(p);           p += align16i(4 * u.item_vb);
  s.phi = reinterpret_cast<T*>(p);             p += align16i((int)sizeof(T) * u.item_vb);
  s.grad = reinterpret_cast<V3T<T>*>(p);       p += align16i((int)sizeof(V3T<T>) * u.item_vb);
  s.vlist = reinterpret_cast<uint16_t*>(p);    p += align16i(2 * u.item_vb);
  s.elist = reinterpret_cast<uint16_t*>(p);    p += align16i(2 * u.item_eb);
  s.need = reinterpret_cast<uint8_t*>(p);
  // the attaining planes live only from the max-plane pass to the edge cull,
  // before the vertex gradients of the same list are written
  s.am = reinterpret_cast<uint16_t*>(s.grad);
  return s;
}

// ---------------------------------------------------------------------------
// one list of live directions: pass 1 (fold) or pass 2 (adjoint)
// ---------------------------------------------------------------------------
// Per-lane sums of the contact-point adjoints as forces on the bodies:
// F = sum sigma f and M = sum sigma (p - t_A) x f, where f = R_S x_bar is the
// world-frame adjoint of a contact point p (world) of a group whose feature
// body is A (sigma = +1, side 0) or B (sigma = -1, side 1).  Body A receives
// the force F and the torque M about t_A; body B receives -F and
// -M + (t_B - t_A) x F about t_B.
template <class T> struct Accum {
  V3T<T> F, M;
};

template <class T>
__device__ __forceinline__ void add_force(Accum<T>& ac, const BwdSlice<T>& sl, int grp, V3T<T> x,
                                          V3T<T> xb) {
  const int side = sl.gside[grp];
  const PoseT<T>& P = sl.spose[side];
  const V3T<T> f = rot(P.R, xb);
  V3T<T> p = rot(P.R, x);
  if (side == 0) {
    const V3T<T> t = sl.tba[0];
    p = v3(p.x + t.x, p.y + t.y, p.z + t.z);
  }
  const V3T<T> m = cross3(p, f);
  if (side == 0) {
    ac.F = v3(ac.F.x + f.x, ac.F.y + f.y, ac.F.z + f.z);
    ac.M = v3(ac.M.x + m.x, ac.M.y + m.y, ac.M.z + m.z);
  } else {
    ac.F = v3(ac.F.x - f.x, ac.F.y - f.y, ac.F.z - f.z);
    ac.M = v3(ac.M.x - m.x, ac.M.y - m.y, ac.M.z - m.z);
  }
}

// Work counters of a counted reverse pass (CCM_BWD_CNT_* of ccm.h): plane
// evaluations by kind and pass, per lane, summed at the end of the kernel.
struct BwdCounts {
  unsigned long long dirs = 0, live = 0, maxp = 0, gate = 0, g1 = 0, v1 = 0, h2 = 0, g2 = 0;
};

template <class T, int kPass, int kK, bool kCount>
__device__ void bwd_run_list(const BwdSlice<T>& sl, int nd, int TV, int TE, int sc0,
                             const KParams& kp, int lane, Accum<T>& ac, BwdCounts& cnt,
                             int* memo, bool reuse) {
  const int* dsub = sl.dsub;
  uint32_t* vbits = memo ? reinterpret_cast<uint32_t*>(memo + kMemoHead) : nullptr;
  uint32_t* ebits = nullptr;
  int n_e = 0, n_v = 0;
  const uint16_t* vl = sl.vlist;
  if (memo) ebits = vbits + memo[7];
  if (reuse) {
    // the recompute sweep's single list: keep the contributing edges (in
    // place, in order) and the vertices that contributed or start a kept trace
    nd = memo[2];
    TV = memo[3];
    TE = memo[4];
    const int nv0 = memo[5], ne0 = memo[6];
    for (int t = lane; t < TV; t += 32) sl.need[t] = 0;
    __syncwarp();
    for (int k0 = 0; k0 < ne0; k0 += 32) {
      const int k = k0 + lane;
      bool keep = false;
      int t = 0;
      if (k < ne0) {
        t = sl.elist[k];
        keep = (ebits[k >> 5] >> (k & 31)) & 1u;
        if (keep) {
          const int r = find_dir(sl.pe, nd, t);
          const int4 f = sl.fp[dsub[r] >> 16];
          const uint32_t e = sl.edges[f.z + t - sl.pe[r]];
          sl.need[sl.pv[r] + (e & 0xffff)] = 1;
          sl.need[sl.pv[r] + (e >> 16)] = 1;
        }
      }
      const unsigned bal = __ballot_sync(kFull, keep);
      if (keep) sl.elist[n_e + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
      n_e += __popc(bal);
    }
    __syncwarp();
    for (int k0 = 0; k0 < nv0; k0 += 32) {
      const int k = k0 + lane;
      bool keep = false;
      int t = 0;
      if (k < nv0) {
        t = sl.vlist[k];
        keep = ((vbits[k >> 5] >> (k & 31)) & 1u) || sl.need[t];
      }
      const unsigned bal = __ballot_sync(kFull, keep);
      if (keep) sl.vlist[n_v + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
      n_v += __popc(bal);
    }
    __syncwarp();
  } else {
  for (int t = lane; t < TV; t += 32) {
    const int r = find_dir(sl.pv, nd, t);
    const int code = dsub[r];
    const int4 f = sl.fp[code >> 16];
    const int2 s = sl.sp[code & 0xffff];
    const V3T<T> x = sl.xs[f.x + t - sl.pv[r]];
    int arg;
    sl.m[t] = max_plane_arg(sl.planes + s.x, s.y, val(x.x), val(x.y), val(x.z), arg);
    sl.am[t] = (uint16_t)arg;
    sl.need[t] = 0;
    if (kCount) cnt.maxp += s.y;
  }
  __syncwarp();
  for (int t0 = 0; t0 < TE; t0 += 32) {
    const int t = t0 + lane;
    bool live = false;
    if (t < TE) {
      const int r = find_dir(sl.pe, nd, t);
      const int4 f = sl.fp[dsub[r] >> 16];
      const int2 s = sl.sp[dsub[r] & 0xffff];
      const uint32_t e = sl.edges[f.z + t - sl.pe[r]];
      const int i0 = e & 0xffff, i1 = e >> 16;
      const int t0v = sl.pv[r] + i0, t1v = sl.pv[r] + i1;
      const V3T<T> a = sl.xs[f.x + i0], b = sl.xs[f.x + i1];
      const float lb = edge_plane_bound(sl.planes[s.x + sl.am[t0v]], sl.planes[s.x + sl.am[t1v]],
                                        val(b.x) - val(a.x), val(b.y) - val(a.y),
                                        val(b.z) - val(a.z), sl.m[t0v], sl.m[t1v]);
      live = lb - kEdgeTol < kp.d_max;
      if (live) { sl.need[t0v] = 1; sl.need[t1v] = 1; }
    }
    const unsigned bal = __ballot_sync(kFull, live);
    if (live) sl.elist[n_e + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
    n_e += __popc(bal);
  }
  __syncwarp();
  for (int t0 = 0; t0 < TV; t0 += 32) {
    const int t = t0 + lane;
    const bool live = t < TV && (sl.m[t] < kp.d_max || sl.need[t]);
    const unsigned bal = __ballot_sync(kFull, live);
    if (live) sl.vlist[n_v + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
    n_v += __popc(bal);
  }
  __syncwarp();
  if (memo && kPass == 1 && lane == 0) {
    memo[1] += 1;
    memo[2] = nd; memo[3] = TV; memo[4] = TE; memo[5] = n_v; memo[6] = n_e;
  }
  }
  // vertices
  for (int k0 = 0; k0 < n_v; k0 += 32) {
    const int k = k0 + lane;
    PartT<T> c;
    part_zero(c);
    int key = 0xffff;
    bool contrib = false;
    if (k < n_v) {
      const int t = vl[k];
      const int r = find_dir(sl.pv, nd, t);
      const int code = dsub[r];
      const int g = code >> 16;
      const int4 f = sl.fp[g];
      const int2 s = sl.sp[code & 0xffff];
      const V3T<T> x = sl.xs[f.x + t - sl.pv[r]];
      const float m = sl.m[t];
      key = g;
      if (kCount) { if (kPass == 1) cnt.g1 += s.y; else cnt.h2 += s.y; }
      if (kPass == 1) {
        const SdfT<T> e = sdf_t<T, 1>(sl.planes + s.x, s.y, x, m, x, kp);
        sl.phi[t] = e.phi;
        if (m < kp.d_max) {
          T w, wp;
          transition_t(e.phi, kp, w, wp);
          const T dc = fma_t(w, e.phi - kp.d_max, T(kp.d_max));
          part_from_contact(c, w, dc, x, e.g, kp.c_blend);
          mark_hit(sl.hit, sl.hw, g, sc0 + (code & 0xffff), val(w));
          contrib = val(w) > 0.f;
        }
      } else {
        const Coef<T>& cf = sl.coef[g];
        const SdfT<T> e = sdf_t<T, 2>(sl.planes + s.x, s.y, x, m, cf.nb, kp);
        sl.phi[t] = e.phi;
        sl.grad[t] = e.g;
        if (m < kp.d_max && cf.live) add_force(ac, sl, g, x, contact_adjoint(e, x, cf, kp));
      }
    }
    if (kPass == 1) {
      if (memo) {
        const unsigned cb = __ballot_sync(kFull, contrib);
        if (lane == 0) vbits[k0 >> 5] = cb;
      }
      fold_t(c, key, sl.acc, lane);
    }
  }
  __syncwarp();
  // edges
  for (int k0 = 0; k0 < n_e; k0 += 32) {
    const int k = k0 + lane;
    PartT<T> c;
    part_zero(c);
    int key = 0xffff;
    bool contrib = false;
    if (k < n_e) {
      const int t = sl.elist[k];
      const int r = find_dir(sl.pe, nd, t);
      const int code = dsub[r];
      const int g = code >> 16;
      const int4 f = sl.fp[g];
      const int2 s = sl.sp[code & 0xffff];
      const uint32_t e = sl.edges[f.z + t - sl.pe[r]];
      const int i0 = e & 0xffff, i1 = e >> 16;
      const int t0v = sl.pv[r] + i0, t1v = sl.pv[r] + i1;
      const V3T<T> a = sl.xs[f.x + i0], b = sl.xs[f.x + i1];
      key = g;
      SdfT<T> sc;
      V3T<T> pe, xbI, xbII;
      const Coef<T>& cf = sl.coef[g];
      const int steps = 2 * ((kK > 0 ? kK : kp.trace_iters) - 1);
      if (kPass == 1) {
        if (kCount) { cnt.g1 += s.y; cnt.v1 += (unsigned long long)steps * s.y; }
        const V3T<T> z = v3(T(0.f), T(0.f), T(0.f));
        edge_t<T, false, kK>(sl.planes + s.x, s.y, a, b, sl.m[t0v], sl.m[t1v], sl.phi[t0v],
                         sl.phi[t1v], z, z, cf, kp, sc, pe, xbI, xbII);
        T w, wp;
        transition_t(sc.phi, kp, w, wp);
        const T dc = fma_t(w, sc.phi - kp.d_max, T(kp.d_max));
        part_from_contact(c, w, dc, pe, sc.g, kp.c_blend);
        mark_hit(sl.hit, sl.hw, g, sc0 + (code & 0xffff), val(w));
        contrib = val(w) > 0.f;
      } else if (cf.live) {
        if (kCount) { cnt.h2 += s.y; cnt.g2 += (unsigned long long)steps * s.y; }
        edge_t<T, true, kK>(sl.planes + s.x, s.y, a, b, sl.m[t0v], sl.m[t1v], sl.phi[t0v],
                        sl.phi[t1v], sl.grad[t0v], sl.grad[t1v], cf, kp, sc, pe, xbI, xbII);
        add_force(ac, sl, g, a, xbI);
        add_force(ac, sl, g, b, xbII);
      }
    }
    if (kPass == 1) {
      if (memo) {
        const unsigned cb = __ballot_sync(kFull, contrib);
        if (lane == 0) ebits[k0 >> 5] = cb;
      }
      fold_t(c, key, sl.acc, lane);
    }
  }
  __syncwarp();
}

template <class T, int kPass, int kK, bool kCount>
__device__ void bwd_run_pending(const BwdSlice<T>& sl, int np, int sc0, const UnitShape& us,
                                const KParams& kp, int lane, Accum<T>& ac, BwdCounts& cnt,
                                int* memo = nullptr) {
  int start = 0;
  while (start < np) {
    const int r = start + lane;
    int nvr = 0, ner = 0, code = 0;
    if (r < np) {
      code = sl.dir[r];
      const int4 f = sl.fp[code >> 16];
      nvr = f.y;
      ner = f.w;
    }
    int iv = nvr, ie = ner;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(kFull, iv, o), b = __shfl_up_sync(kFull, ie, o);
      if (lane >= o) { iv += a; ie += b; }
    }
    const bool fits = r < np && iv <= us.item_vb && ie <= us.item_eb;
    const int nd = __popc(__ballot_sync(kFull, fits));
    if (lane < nd) {
      sl.dsub[lane] = code;
      sl.pv[lane] = iv - nvr;
      sl.pe[lane] = ie - ner;
    }
    const int TV = __shfl_sync(kFull, iv, nd - 1), TE = __shfl_sync(kFull, ie, nd - 1);
    __syncwarp();
    if (kCount && lane == 0) cnt.live += nd;
    bwd_run_list<T, kPass, kK, kCount>(sl, nd, TV, TE, sc0, kp, lane, ac, cnt, memo, false);
    start += nd;
  }
}

// all live directions of the staged F chunk against S, chunk by chunk
template <class T, int kPass, int kK, bool kCount>
__device__ void bwd_sweep(const DevGeom& g, const BwdSlice<T>& sl, const BodyRec& S, int nfc,
                          float margin, bool by_hits, const UnitShape& us, const KParams& kp,
                          int lane, Accum<T>& ac, BwdCounts& cnt) {
  for (int sc0 = 0; sc0 < S.np;) {
    int sc1 = sc0, P = 0;
    while (sc1 < S.np && sc1 - sc0 < us.spiece_budget) {
      const int nf = g.pieces[S.p0 + sc1].nf;
      if (P + nf > us.plane_budget) break;
      P += nf;
      ++sc1;
    }
    const int nsc = sc1 - sc0;
    if (nsc == 0) break;   // unreachable: budgets hold every piece
    __syncwarp();
    if (by_hits && S.np <= kHitS) {
      // only the pieces some direction of the chunk is marked with are
      // visited: stage just their planes, packed
      int base = 0;
      for (int q0 = 0; q0 < nsc; q0 += 32) {
        const int q = q0 + lane;
        int nf = 0, f0 = 0;
        bool need = false;
        if (q < nsc) {
          const int sg = sc0 + q;
          uint32_t any = 0;
          for (int f = 0; f < nfc; ++f) any |= sl.hit[f * sl.hw + (sg >> 5)];
          need = (any >> (sg & 31)) & 1u;
          if (need) {
            const PieceRec p = g.pieces[S.p0 + sg];
            nf = p.nf;
            f0 = p.f0;
          }
        }
        int incl = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += t;
        }
        const int off = base + incl - nf;
        if (q < nsc) sl.sp[q] = make_int2(off, nf);
        unsigned m = __ballot_sync(kFull, need);
        while (m) {
          const int l = __ffs(m) - 1;
          m &= m - 1;
          const int o_l = __shfl_sync(kFull, off, l), n_l = __shfl_sync(kFull, nf, l),
                    f_l = __shfl_sync(kFull, f0, l);
          stage_copy(sl.planes + o_l, g.planes + f_l, n_l, lane);
        }
        base += __shfl_sync(kFull, incl, 31);
      }
      __syncwarp();
      if (base == 0) {   // no marked direction in this chunk
        sc0 = sc1;
        continue;
      }
    } else {
      const int f_first = g.pieces[S.p0 + sc0].f0;
      for (int q = lane; q < nsc; q += 32) {
        const PieceRec p = g.pieces[S.p0 + sc0 + q];
        sl.sp[q] = make_int2(p.f0 - f_first, p.nf);
      }
      stage_copy(sl.planes, g.planes + f_first, P, lane);
      __syncwarp();
    }
    int np = 0;
    const int ndir = nfc * nsc;
    for (int d0 = 0; d0 < ndir; d0 += 32) {
      const int d = d0 + lane;
      bool live = false;
      int code = 0;
      if (d < ndir) {
        const int fcd = d / nsc, scd = d - fcd * nsc;
        const int sg = sc0 + scd;
        if (by_hits && sg < kHitS) {
          live = (sl.hit[fcd * sl.hw + (sg >> 5)] >> (sg & 31)) & 1u;
        } else {
          const float4 c = sl.fs[fcd];
          const int2 s = sl.sp[scd];
          const float mc = max_plane(sl.planes + s.x, s.y, c.x, c.y, c.z);
          live = mc - c.w - margin < kp.d_max;
          if (kCount) cnt.gate += s.y;
        }
        if (kCount) cnt.dirs += 1;
        code = (fcd << 16) | scd;
      }
      const unsigned bal = __ballot_sync(kFull, live);
      const int nl = __popc(bal);
      if (np + nl > kPending) {
        bwd_run_pending<T, kPass, kK, kCount>(sl, np, sc0, us, kp, lane, ac, cnt);
        np = 0;
      }
      if (live) sl.dir[np + __popc(bal & ((1u << lane) - 1u))] = code;
      np += nl;
      __syncwarp();
    }
    if (np > 0) bwd_run_pending<T, kPass, kK, kCount>(sl, np, sc0, us, kp, lane, ac, cnt);
    sc0 = sc1;
  }
}


// A group's adjoint coefficients (Coef) from its blend partial A and its

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <class T, int kK, bool kCount>
__global__ void __launch_bounds__(32, 1)
bwd_unit_kernel(DevGeom g, const PairRec* __restrict__ pairs,
                const WorkItem* __restrict__ items, const int32_t* __restrict__ order,
                int64_t n_items, const int64_t* __restrict__ dev_items,
                const float* __restrict__ pose_a, const float* __restrict__ pose_b,
                const float* __restrict__ ybar, const float* __restrict__ dir,
                const float* __restrict__ saved, KParams kp, UnitShape us,
                float* __restrict__ part, float* __restrict__ jvp,
                unsigned long long* __restrict__ counters, int* __restrict__ sched) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  BwdCounts cnt;
  const BwdSlice<T> sl = bwd_slice<T>(smem_raw, us);
  const int64_t n_run = dev_items ? *dev_items : n_items;
  for (int64_t k = first_unit(sched, blockIdx.x); k < n_run;
       k = next_unit(sched, k, gridDim.x)) {
    const int32_t item = order[k];   // heaviest items first, round-robin
    const WorkItem it = items[item];
    const int64_t u = it.unit;
    const int64_t pi = u >> 1;
    const int side = (int)(u & 1);
    const PairRec pr = pairs[pi];
    const BodyRec bA = g.bodies[pr.bodyA], bB = g.bodies[pr.bodyB];
    const BodyRec F = side == 0 ? bA : bB, S = side == 0 ? bB : bA;
    const int64_t row0 = pr.goff + (side == 0 ? 0 : bA.np);
    const float* pF = (side == 0 ? pose_a : pose_b) + 12 * pi;
    const float* pS = (side == 0 ? pose_b : pose_a) + 12 * pi;
    const float* uF = dir ? dir + 12 * pi + (side == 0 ? 0 : 6) : nullptr;
    const float* uS = dir ? dir + 12 * pi + (side == 0 ? 6 : 0) : nullptr;
    PoseT<T> PF, PS;
    load_pose_t(pF, uF, PF);
    load_pose_t(pS, uS, PS);
    // relative pose S <- F
    T Rr[9], tr[3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Rr[3 * i + j] = fma_t(PS.R[i], PF.R[j], fma_t(PS.R[3 + i], PF.R[3 + j], PS.R[6 + i] * PF.R[6 + j]));
    {
      const V3T<T> dt = v3(PF.t[0] - PS.t[0], PF.t[1] - PS.t[1], PF.t[2] - PS.t[2]);
      const V3T<T> q = rotT(PS.R, dt);
      tr[0] = q.x; tr[1] = q.y; tr[2] = q.z;
    }
    const float margin = 1e-6f * (1.0f + fabsf(val(tr[0])) + fabsf(val(tr[1])) + fabsf(val(tr[2])));
    Accum<T> ac;
    ac.F = v3(T(0.f), T(0.f), T(0.f));
    ac.M = ac.F;
    V3T<T> gws = ac.F, gvs = ac.F;   // output-transform terms of this lane's groups
    if (lane == 0) {
      sl.spose[side] = PS;
      sl.tba[0] = side == 0 ? v3(PS.t[0] - PF.t[0], PS.t[1] - PF.t[1], PS.t[2] - PF.t[2])
                            : v3(PF.t[0] - PS.t[0], PF.t[1] - PS.t[1], PF.t[2] - PS.t[2]);
    }

    for (int fc0 = it.fc0; fc0 < it.fc1;) {
      int fc1 = fc0, V = 0, E = 0;
      while (fc1 < it.fc1 && fc1 - fc0 < us.groups_b) {
        const PieceRec p = g.pieces[F.p0 + fc1];
        if (V + p.nv > us.vert_budget || E + p.ne > us.edge_budget) break;
        V += p.nv;
        E += p.ne;
        ++fc1;
      }
      const int nfc = fc1 - fc0;
      if (nfc == 0) break;   // unreachable: budgets hold every piece
      const PieceRec pfirst = g.pieces[F.p0 + fc0];
      __syncwarp();
      PieceRec p{};
      if (lane < nfc) p = g.pieces[F.p0 + fc0 + lane];
      if (lane < nfc) {
        sl.fp[lane] = make_int4(p.v0 - pfirst.v0, p.nv, p.e0 - pfirst.e0, p.ne);
        const float4 c = p.sphere;
        const float cx = val(Rr[0]) * c.x + val(Rr[1]) * c.y + val(Rr[2]) * c.z + val(tr[0]);
        const float cy = val(Rr[3]) * c.x + val(Rr[4]) * c.y + val(Rr[5]) * c.z + val(tr[1]);
        const float cz = val(Rr[6]) * c.x + val(Rr[7]) * c.y + val(Rr[8]) * c.z + val(tr[2]);
        sl.fs[lane] = make_float4(cx, cy, cz, c.w);
        sl.gside[lane] = side;
        PartT<T> z;
        part_zero(z);
        sl.acc[lane] = z;
        if (saved) {   // the forward's hits: pass 1 visits only those directions
          const uint32_t* h =
              reinterpret_cast<const uint32_t*>(saved + (int64_t)kSavedFloats * (row0 + fc0 + lane) + 18);
          for (int q = 0; q < sl.hw; ++q) sl.hit[lane * sl.hw + q] = h[q];
        } else {
          for (int q = 0; q < sl.hw; ++q) sl.hit[lane * sl.hw + q] = 0u;
        }
      }
      if (saved && S.np <= kHitS) {
        // with the forward's hits known, only the pieces with a marked
        // direction are visited: stage just their vertices and edges, packed
        __syncwarp();
        bool need = false;
        if (lane < nfc)
          for (int q = 0; q < sl.hw; ++q) need |= sl.hit[lane * sl.hw + q] != 0u;
        const int nv = need ? p.nv : 0, ne = need ? p.ne : 0;
        int iv = nv, ie = ne;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int a = __shfl_up_sync(kFull, iv, o), b = __shfl_up_sync(kFull, ie, o);
          if (lane >= o) { iv += a; ie += b; }
        }
        if (lane < nfc) sl.fp[lane] = make_int4(iv - nv, p.nv, ie - ne, p.ne);
        unsigned m = __ballot_sync(kFull, need);
        while (m) {
          const int l = __ffs(m) - 1;
          m &= m - 1;
          const int vo = __shfl_sync(kFull, iv - nv, l), vn = __shfl_sync(kFull, nv, l),
                    v0 = __shfl_sync(kFull, p.v0, l);
          const int eo = __shfl_sync(kFull, ie - ne, l), en = __shfl_sync(kFull, ne, l),
                    e0 = __shfl_sync(kFull, p.e0, l);
          for (int i = lane; i < vn; i += 32) {
            const float4 v = g.verts[v0 + i];
            const V3T<T> x = rot(Rr, v3(T(v.x), T(v.y), T(v.z)));
            sl.xs[vo + i] = v3(x.x + tr[0], x.y + tr[1], x.z + tr[2]);
          }
          stage_copy(sl.edges + eo, g.edges + e0, en, lane);
        }
      } else {
        for (int i = lane; i < V; i += 32) {
          const float4 v = g.verts[pfirst.v0 + i];
          const V3T<T> vv = v3(T(v.x), T(v.y), T(v.z));
          const V3T<T> x = rot(Rr, vv);
          sl.xs[i] = v3(x.x + tr[0], x.y + tr[1], x.z + tr[2]);
        }
        stage_copy(sl.edges, g.edges + pfirst.e0, E, lane);
      }
      __syncwarp();

      bwd_sweep<T, 1, kK, kCount>(g, sl, S, nfc, margin, saved != nullptr, us, kp, lane, ac, cnt);
      __syncwarp();

      // group outputs, adjoint coefficients and output-transform terms
      if (lane < nfc) {
        Coef<T> cf;
        V3T<T> ow, ov;
        form_coef(sl.acc[lane], ybar + 8 * (row0 + fc0 + lane), PS,
                  jvp ? jvp + 8 * (row0 + fc0 + lane) : nullptr, cf, ow, ov);
        gws = v3(gws.x + ow.x, gws.y + ow.y, gws.z + ow.z);
        gvs = v3(gvs.x + ov.x, gvs.y + ov.y, gvs.z + ov.z);
        sl.coef[lane] = cf;
      }
      __syncwarp();
      bwd_sweep<T, 2, kK, kCount>(g, sl, S, nfc, margin, true, us, kp, lane, ac, cnt);
      fc0 = fc1;
    }

    // reduce the lanes; the item's forces and its groups' output terms (on
    // the SDF body) give its share of the pair's 12 twist components
    const V3T<T> Fs = v3(warp_sum_t(ac.F.x), warp_sum_t(ac.F.y), warp_sum_t(ac.F.z));
    const V3T<T> Ms = v3(warp_sum_t(ac.M.x), warp_sum_t(ac.M.y), warp_sum_t(ac.M.z));
    gws = v3(warp_sum_t(gws.x), warp_sum_t(gws.y), warp_sum_t(gws.z));
    gvs = v3(warp_sum_t(gvs.x), warp_sum_t(gvs.y), warp_sum_t(gvs.z));
    if (lane == 0) {
      const V3T<T> z = zero3t<T>();
      // slot layout per item: [grad (w_A, v_A, w_B, v_B) | H u (same layout)]
      float* o = part + 24 * (int64_t)item;
      write_twists(Fs, Ms, side == 1 ? gws : z, side == 1 ? gvs : z, side == 0 ? gws : z,
                   side == 0 ? gvs : z, sl.tba[0], dir ? dir + 12 * pi : nullptr,
                   dir ? dir + 12 * pi + 6 : nullptr, o, dir ? o + 12 : nullptr);
    }
    __syncwarp();
  }
  if (kCount) {
    const unsigned long long v[8] = {cnt.dirs, cnt.live, cnt.maxp, cnt.gate,
                                     cnt.g1, cnt.v1, cnt.h2, cnt.g2};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      unsigned long long x = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (lane == 0) atomicAdd(counters + q, x);
    }
  }
}

// grad / hvp of pair i = the two units' slots, side 0 then side 1
// ---------------------------------------------------------------------------
// Reverse pass per body pair, given the forward's saved record.  Only the
// groups the forward found contacts in (a non-zero hit word) are visited,
// those of both sides of the pair in the same lists: every group carries its
// side, so the contacts of A's vertices and edges in B's frame and of B's in
// A's frame share a warp's lanes.  The SDF pieces of the marked directions of
// both bodies are staged packed in one index space, [0, npB) for B's pieces
// and [npB, npB + npA) for A's.  The pair's 12 gradient (and H u) components
// are written directly; a pair without marked groups gets zeros.  Every SDF
// body must have at most kHitS pieces (the host checks).
// ---------------------------------------------------------------------------
constexpr int kNoMark = -(1 << 30);   // run_list offset that disables hit marks

template <class T, int kPass, int kK, bool kCount>
__device__ void pair_sweep(const DevGeom& g, const BwdSlice<T>& sl, const BodyRec& bA,
                           const BodyRec& bB, int nfc, const UnitShape& us, const KParams& kp,
                           int lane, Accum<T>& ac, BwdCounts& cnt) {
  const int npB = bB.np, nS = bA.np + bB.np;
  int* memo = sl.memo;
  if (kPass == 2 && memo[0] == 1 && memo[1] == 1) {
    // one S chunk and one list in the recompute sweep: its planes and its
    // list are still staged; visit only the contributing contacts
    bwd_run_list<T, 2, kK, kCount>(sl, 0, 0, 0, kNoMark, kp, lane, ac, cnt, memo, true);
    return;
  }
  if (kPass == 1) {
    if (lane == 0) { memo[0] = 0; memo[1] = 0; memo[7] = (us.item_vb + 31) / 32; }
    __syncwarp();
  }
  // does some group of the matching side mark S index si?
  auto needed = [&](int si) {
    const int side = si < npB ? 0 : 1;
    const int b = side == 0 ? si : si - npB;
    uint32_t any = 0;
    for (int f = 0; f < nfc; ++f)
      if (sl.gside[f] == side) any |= sl.hit[f * sl.hw + (b >> 5)];
    return ((any >> (b & 31)) & 1u) != 0u;
  };
  for (int sc0 = 0; sc0 < nS;) {
    // the chunk [sc0, sc1): at most 2 spiece_budget indices (a piece budget
    // for each body) whose needed pieces' planes fit plane_budget; stage
    // those planes, packed
    int sc1 = sc0, P = 0;
    __syncwarp();
    while (sc1 < nS && sc1 - sc0 < 2 * us.spiece_budget) {
      const int si = sc1 + lane;
      const bool valid = si < nS && si - sc0 < 2 * us.spiece_budget;
      int nf = 0, f0 = 0;
      if (valid && needed(si)) {
        const PieceRec p = g.pieces[si < npB ? bB.p0 + si : bA.p0 + (si - npB)];
        nf = p.nf;
        f0 = p.f0;
      }
      int incl = nf;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
      }
      const bool fits = valid && P + incl <= us.plane_budget;
      const unsigned fb = __ballot_sync(kFull, fits);
      const int take = __popc(fb);   // a prefix of the lanes: incl grows with the lane
      if (valid && fits) sl.sp[si - sc0] = make_int2(P + incl - nf, nf);
      unsigned m = __ballot_sync(kFull, fits && nf > 0);
      while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1;
        const int o_l = P + __shfl_sync(kFull, incl - nf, l), n_l = __shfl_sync(kFull, nf, l),
                  f_l = __shfl_sync(kFull, f0, l);
        stage_copy(sl.planes + o_l, g.planes + f_l, n_l, lane);
      }
      if (take > 0) P += __shfl_sync(kFull, incl, take - 1);
      sc1 += take;
      if (take < 32) break;
    }
    __syncwarp();
    if (kPass == 1 && lane == 0) memo[0] += 1;
    if (sc1 == sc0) break;   // unreachable: every piece fits the plane budget
    if (P == 0) {            // no marked direction in this chunk
      sc0 = sc1;
      continue;
    }
    const int nsc = sc1 - sc0;
    int np = 0;
    const int ndir = nfc * nsc;
    for (int d0 = 0; d0 < ndir; d0 += 32) {
      const int d = d0 + lane;
      bool live = false;
      int code = 0;
      if (d < ndir) {
        const int fcd = d / nsc, scd = d - fcd * nsc;
        const int si = sc0 + scd;
        const int side = si < npB ? 0 : 1;
        if (sl.gside[fcd] == side) {
          const int b = side == 0 ? si : si - npB;
          live = (sl.hit[fcd * sl.hw + (b >> 5)] >> (b & 31)) & 1u;
        }
        code = (fcd << 16) | scd;
        if (kCount) cnt.dirs += 1;
      }
      const unsigned bal = __ballot_sync(kFull, live);
      const int nl = __popc(bal);
      if (np + nl > kPending) {
        bwd_run_pending<T, kPass, kK, kCount>(sl, np, kNoMark, us, kp, lane, ac, cnt, memo);
        np = 0;
      }
      if (live) sl.dir[np + __popc(bal & ((1u << lane) - 1u))] = code;
      np += nl;
      __syncwarp();
    }
    if (np > 0) bwd_run_pending<T, kPass, kK, kCount>(sl, np, kNoMark, us, kp, lane, ac, cnt, memo);
    sc0 = sc1;
  }
}

template <class T>
__device__ __forceinline__ bool any_hit(const float* saved, int64_t row, int hw) {
  const uint32_t* h = reinterpret_cast<const uint32_t*>(saved + (int64_t)kSavedFloats * row + 18);
  uint32_t a = 0;
  for (int q = 0; q < hw; ++q) a |= h[q];   // the record's words past hw are zero
  return a != 0u;
}

template <class T, int kK, bool kCount>
__global__ void __launch_bounds__(32, 1)
bwd_pair_kernel(DevGeom g, const PairRec* __restrict__ pairs, const int32_t* __restrict__ porder,
                int64_t n_pairs, const int64_t* __restrict__ dev_pairs,
                const float* __restrict__ pose_a, const float* __restrict__ pose_b,
                const float* __restrict__ ybar, const float* __restrict__ dir,
                const float* __restrict__ saved, KParams kp, UnitShape us,
                float* __restrict__ grad, float* __restrict__ hvp, float* __restrict__ jvp,
                unsigned long long* __restrict__ counters, int* __restrict__ sched,
                const int* __restrict__ only_if) {
  pdl_wait();   // launched behind the per-contact pass: its flag and buffers first
  if (only_if && *only_if == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  BwdCounts cnt;
  const BwdSlice<T> sl = bwd_slice<T>(smem_raw, us);
  PoseT<T>* rel = sl.rel;
  const int64_t n_run = dev_pairs ? *dev_pairs : n_pairs;
  for (int64_t k = first_unit(sched, blockIdx.x); k < n_run;
       k = next_unit(sched, k, gridDim.x)) {
    const int64_t pi = porder[k];   // heaviest pairs first, round-robin
    const PairRec pr = pairs[pi];
    const BodyRec bA = g.bodies[pr.bodyA], bB = g.bodies[pr.bodyB];
    const float* uA = dir ? dir + 12 * pi : nullptr;
    const float* uB = dir ? dir + 12 * pi + 6 : nullptr;
    __syncwarp();
    if (lane == 0) {
      PoseT<T> PA, PB;
      load_pose_t(pose_a + 12 * pi, uA, PA);
      load_pose_t(pose_b + 12 * pi, uB, PB);
      sl.spose[0] = PB;
      sl.spose[1] = PA;
      sl.tba[0] = v3(PB.t[0] - PA.t[0], PB.t[1] - PA.t[1], PB.t[2] - PA.t[2]);
      for (int side = 0; side < 2; ++side) {   // relative pose S <- F
        const PoseT<T>& F = side == 0 ? PA : PB;
        const PoseT<T>& S = side == 0 ? PB : PA;
        PoseT<T> r;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            r.R[3 * i + j] = fma_t(S.R[i], F.R[j], fma_t(S.R[3 + i], F.R[3 + j], S.R[6 + i] * F.R[6 + j]));
        const V3T<T> q = rotT(S.R, v3(F.t[0] - S.t[0], F.t[1] - S.t[1], F.t[2] - S.t[2]));
        r.t[0] = q.x; r.t[1] = q.y; r.t[2] = q.z;
        rel[side] = r;
      }
      for (int q = 0; q < 18; ++q) sl.pacc[q] = T(0.f);
    }
    __syncwarp();
    Accum<T> ac;
    ac.F = v3(T(0.f), T(0.f), T(0.f));
    ac.M = ac.F;
    const int ncand = bA.np + bB.np;   // group rows goff + c; c < npA: A's pieces (side 0)
    int cand = 0;
    for (;;) {
      // the next chunk: up to us.groups_b marked groups within the budgets
      int nfc = 0, V = 0, E = 0;
      while (cand < ncand && nfc < us.groups_b) {
        const int c = cand + lane;
        bool live = false;
        int nv = 0, ne = 0;
        if (c < ncand) {
          live = any_hit<T>(saved, pr.goff + c, sl.hw);
          if (live) {
            const PieceRec p = g.pieces[c < bA.np ? bA.p0 + c : bB.p0 + (c - bA.np)];
            nv = p.nv;
            ne = p.ne;
          }
        }
        unsigned m = __ballot_sync(kFull, live);
        int next = min(ncand, cand + 32);
        while (m) {
          const int l = __ffs(m) - 1;
          const int nv_l = __shfl_sync(kFull, nv, l), ne_l = __shfl_sync(kFull, ne, l);
          if (nfc == us.groups_b || V + nv_l > us.vert_budget || E + ne_l > us.edge_budget) {
            next = cand + l;   // starts the next chunk
            break;
          }
          if (lane == 0) sl.gside[nfc] = cand + l;   // candidate index for now
          V += nv_l;
          E += ne_l;
          ++nfc;
          m &= m - 1;
        }
        cand = next;
        if (m) break;
      }
      if (nfc == 0) break;
      __syncwarp();
      // stage the chunk's groups: side, packed vertices (moved into the SDF
      // frame of their side) and edges, hits, zero partials
      int c = 0, side = 0;
      PieceRec p{};
      if (lane < nfc) {
        c = sl.gside[lane];
        side = c < bA.np ? 0 : 1;
        p = g.pieces[side == 0 ? bA.p0 + c : bB.p0 + (c - bA.np)];
      }
      const int nv = lane < nfc ? p.nv : 0, ne = lane < nfc ? p.ne : 0;
      int iv = nv, ie = ne;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(kFull, iv, o), b = __shfl_up_sync(kFull, ie, o);
        if (lane >= o) { iv += a; ie += b; }
      }
      __syncwarp();
      if (lane < nfc) {
        sl.gside[lane] = side;
        sl.fp[lane] = make_int4(iv - nv, p.nv, ie - ne, p.ne);
        const PoseT<T>& r = rel[side];
        const float4 s4 = p.sphere;
        const float cx = val(r.R[0]) * s4.x + val(r.R[1]) * s4.y + val(r.R[2]) * s4.z + val(r.t[0]);
        const float cy = val(r.R[3]) * s4.x + val(r.R[4]) * s4.y + val(r.R[5]) * s4.z + val(r.t[1]);
        const float cz = val(r.R[6]) * s4.x + val(r.R[7]) * s4.y + val(r.R[8]) * s4.z + val(r.t[2]);
        sl.fs[lane] = make_float4(cx, cy, cz, s4.w);
        PartT<T> z;
        part_zero(z);
        sl.acc[lane] = z;
        const uint32_t* h =
            reinterpret_cast<const uint32_t*>(saved + (int64_t)kSavedFloats * (pr.goff + c) + 18);
        for (int q = 0; q < sl.hw; ++q) sl.hit[lane * sl.hw + q] = h[q];
      }
      for (int l = 0; l < nfc; ++l) {
        const int vo = __shfl_sync(kFull, iv - nv, l), vn = __shfl_sync(kFull, nv, l),
                  v0 = __shfl_sync(kFull, p.v0, l), sd = __shfl_sync(kFull, side, l);
        const int eo = __shfl_sync(kFull, ie - ne, l), en = __shfl_sync(kFull, ne, l),
                  e0 = __shfl_sync(kFull, p.e0, l);
        const PoseT<T>& r = rel[sd];
        for (int i = lane; i < vn; i += 32) {
          const float4 v = g.verts[v0 + i];
          const V3T<T> x = rot(r.R, v3(T(v.x), T(v.y), T(v.z)));
          sl.xs[vo + i] = v3(x.x + r.t[0], x.y + r.t[1], x.z + r.t[2]);
        }
        stage_copy(sl.edges + eo, g.edges + e0, en, lane);
      }
      __syncwarp();

      pair_sweep<T, 1, kK, kCount>(g, sl, bA, bB, nfc, us, kp, lane, ac, cnt);
      __syncwarp();

      // coefficients; the output terms go to the SDF body of each group
      V3T<T> oAw = zero3t<T>(), oAv = oAw, oBw = oAw, oBv = oAw;
      if (lane < nfc) {
        Coef<T> cf;
        V3T<T> ow, ov;
        const int64_t row = pr.goff + c;
        form_coef(sl.acc[lane], ybar + 8 * row, sl.spose[side], jvp ? jvp + 8 * row : nullptr, cf,
                  ow, ov);
        if (side == 0) { oBw = ow; oBv = ov; } else { oAw = ow; oAv = ov; }
        sl.coef[lane] = cf;
      }
      __syncwarp();
      pair_sweep<T, 2, kK, kCount>(g, sl, bA, bB, nfc, us, kp, lane, ac, cnt);

      // chunk totals into the pair's accumulators
      const T s[12] = {oAw.x, oAw.y, oAw.z, oAv.x, oAv.y, oAv.z,
                       oBw.x, oBw.y, oBw.z, oBv.x, oBv.y, oBv.z};
      for (int q = 0; q < 12; ++q) {
        const T t = warp_sum_t(s[q]);
        if (lane == 0) sl.pacc[6 + q] += t;
      }
      __syncwarp();
    }
    const V3T<T> Fs = v3(warp_sum_t(ac.F.x), warp_sum_t(ac.F.y), warp_sum_t(ac.F.z));
    const V3T<T> Ms = v3(warp_sum_t(ac.M.x), warp_sum_t(ac.M.y), warp_sum_t(ac.M.z));
    // groups without marks: zero output tangents
    if (jvp)
      for (int c0 = lane; c0 < ncand; c0 += 32)
        if (!any_hit<T>(saved, pr.goff + c0, sl.hw)) {
          float* o = jvp + 8 * (pr.goff + c0);
          for (int q = 0; q < 8; ++q) o[q] = 0.f;
        }
    if (lane == 0) {
      const T* a = sl.pacc;
      write_twists(Fs, Ms, v3(a[6], a[7], a[8]), v3(a[9], a[10], a[11]), v3(a[12], a[13], a[14]),
                   v3(a[15], a[16], a[17]), sl.tba[0], uA, uB, grad + 12 * pi,
                   hvp ? hvp + 12 * pi : nullptr);
    }
  }
  if (kCount) {
    const unsigned long long v[8] = {cnt.dirs, cnt.live, cnt.maxp, cnt.gate,
                                     cnt.g1, cnt.v1, cnt.h2, cnt.g2};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      unsigned long long x = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (lane == 0) atomicAdd(counters + q, x);
    }
  }
}

// grad / hvp of pair p: the sum of its items' slots [item_off[p], item_off[p+1])
// in index order.
__global__ void bwd_reduce_kernel(const float* __restrict__ part,
                                  const int64_t* __restrict__ item_off, int64_t n_pairs,
                                  const int64_t* __restrict__ dev_pairs,
                                  float* __restrict__ grad, float* __restrict__ hvp) {
  const int64_t n = (dev_pairs ? *dev_pairs : n_pairs) * 12;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / 12;
    const int q = (int)(i - p * 12);
    const int64_t i0 = item_off[p], i1 = item_off[p + 1];
    float g = 0.f, h = 0.f;
    for (int64_t j = i0; j < i1; ++j) {
      g += part[24 * j + q];
      if (hvp) h += part[24 * j + 12 + q];
    }
    grad[i] = g;
    if (hvp) hvp[i] = h;
  }
}

// The per-pair pass keeps the trace-step loop (kK = 0) for every step count:
// its code is smaller and it needs fewer registers than the unrolled three
// steps, so more warps stay resident without thrashing the instruction cache
// (measured faster on both float and Dual).
template <class T, int kK>
static void launch_pair(const BwdLaunch& L, cudaStream_t stream) {
  const int smem = bwd_slice_bytes<T>(L.us);
  // (a launch error surfaces through cudaGetLastError in launch_backward)
  launch_k(L.after_chain, L.counters ? bwd_pair_kernel<T, kK, true> : bwd_pair_kernel<T, kK, false>,
           L.pair_grid, 32, smem, stream, L.g, L.pairs, L.pair_order, L.n_pairs, L.dev_pairs,
           L.pose_a, L.pose_b, L.ybar, L.dir, L.saved, L.kp, L.us, L.grad, L.hvp, L.jvp,
           L.counters, L.sched, L.only_if);
}

template <class T, int kK>
static void launch_unit(const BwdLaunch& L, cudaStream_t stream) {
  const int smem = bwd_slice_bytes<T>(L.us);
  if (L.counters)
    bwd_unit_kernel<T, kK, true><<<L.grid, 32, smem, stream>>>(
        L.g, L.pairs, L.items, L.order, L.n_items, L.dev_items, L.pose_a, L.pose_b, L.ybar, L.dir,
        L.saved, L.kp, L.us, L.part, L.jvp, L.counters, L.sched);
  else
    bwd_unit_kernel<T, kK, false><<<L.grid, 32, smem, stream>>>(
        L.g, L.pairs, L.items, L.order, L.n_items, L.dev_items, L.pose_a, L.pose_b, L.ybar, L.dir,
        L.saved, L.kp, L.us, L.part, L.jvp, nullptr, L.sched);
  count_launch();
}

cudaError_t launch_backward(const BwdLaunch& L, cudaStream_t stream) {
  const bool small_k = L.kp.trace_iters == 3;   // the paper's three steps: unrolled
  if (L.sched && !L.after_chain) {
    const cudaError_t e = cudaMemsetAsync(L.sched, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
  }
  if (L.saved && L.pair_order) {   // per pair, from the forward's record
    if (L.dir) {
      launch_pair<Dual, 0>(L, stream);
    } else {
      BwdLaunch M = L;
      M.hvp = nullptr;
      M.jvp = nullptr;
      launch_pair<float, 0>(M, stream);
    }
    return cudaGetLastError();
  }
  if (L.dir) {
    if (small_k) launch_unit<Dual, 3>(L, stream); else launch_unit<Dual, 0>(L, stream);
  } else {
    BwdLaunch M = L;
    M.dir = nullptr;
    M.jvp = nullptr;
    if (small_k) launch_unit<float, 3>(M, stream); else launch_unit<float, 0>(M, stream);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = L.n_pairs * 12;
  const int blocks = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (n + 255) / 256));
  bwd_reduce_kernel<<<blocks, 256, 0, stream>>>(L.part, L.item_off, L.n_pairs, L.dev_pairs, L.grad,
                                                L.dir ? L.hvp : nullptr);
  count_launch();
  return cudaGetLastError();
}

// The limit is raised to the device's opt-in maximum, not to this shape's size:
// the attribute is shared by every batch and captured graph of the process.
template <class T, int kK>
static cudaError_t configure_pair(int bytes, int smem_limit, int* per_sm) {
  cudaError_t e = cudaSuccess;
  if (bytes > 48 * 1024) {
    e = cudaFuncSetAttribute(bwd_pair_kernel<T, kK, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bwd_pair_kernel<T, kK, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  }
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, bwd_pair_kernel<T, kK, false>, 32,
                                                       bytes);
}

template <class T, int kK>
static cudaError_t configure_unit(int bytes, int smem_limit, int* per_sm) {
  cudaError_t e = cudaSuccess;
  if (bytes > 48 * 1024)
    e = cudaFuncSetAttribute(bwd_unit_kernel<T, kK, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  if (e == cudaSuccess && bytes > 48 * 1024)
    e = cudaFuncSetAttribute(bwd_unit_kernel<T, kK, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, bwd_unit_kernel<T, kK, false>, 32,
                                                       bytes);
}

cudaError_t configure_backward(const UnitShape& us, int smem_limit, BwdOccupancy* occ) {
  const int sf = bwd_slice_bytes<float>(us), sd = bwd_slice_bytes<Dual>(us);
  int pf = 1, pd = 1;
  cudaError_t e;
  if ((e = configure_unit<float, 0>(sf, smem_limit, &occ->unit[0][0])) != cudaSuccess) return e;
  if ((e = configure_unit<Dual, 0>(sd, smem_limit, &occ->unit[1][0])) != cudaSuccess) return e;
  if ((e = configure_unit<float, 3>(sf, smem_limit, &occ->unit[0][1])) != cudaSuccess) return e;
  if ((e = configure_unit<Dual, 3>(sd, smem_limit, &occ->unit[1][1])) != cudaSuccess) return e;
  if ((e = configure_pair<float, 0>(sf, smem_limit, &pf)) != cudaSuccess) return e;
  if ((e = configure_pair<Dual, 0>(sd, smem_limit, &pd)) != cudaSuccess) return e;
  occ->pair[0][0] = occ->pair[0][1] = pf;
  occ->pair[1][0] = occ->pair[1][1] = pd;
  return cudaSuccess;
}

int backward_slice_bytes(const UnitShape& us, bool dual) {
  return dual ? bwd_slice_bytes<Dual>(us) : bwd_slice_bytes<float>(us);
}

}  // namespace ccm

// ---------------------------------------------------------------------------
// Scratch for ccm_contacts_backward_noalloc: the per-item slots of the reverse
// pass live in this fixed array instead of the batch's workspace, so that the
// call needs no device memory of its own.  Every GPU that loads the library
// holds the array (4 MiB) until the process exits.
// ---------------------------------------------------------------------------
namespace ccm {

constexpr int64_t kNoAllocSlotFloats = (int64_t)1 << 20;   // 24 floats per work item
static __device__ __align__(256) float g_noalloc_slots[kNoAllocSlotFloats];

// Device address of g_noalloc_slots on `device`, looked up once per device
// with that device current (the symbol name is only a host-side stand-in).
static cudaError_t noalloc_slots(int device, float** out) {
  static std::mutex mu;
  static float* addr[256] = {nullptr};
  if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_slots);
    if (e != cudaSuccess) return e;
    addr[device] = static_cast<float*>(p);
  }
  *out = addr[device];
  return cudaSuccess;
}

int64_t noalloc_max_items() { return kNoAllocSlotFloats / 24; }

cudaError_t launch_backward_noalloc(BwdLaunch L, int device, cudaStream_t stream) {
  float* slots = nullptr;
  const cudaError_t e = noalloc_slots(device, &slots);
  if (e != cudaSuccess) return e;
  L.part = slots;
  return launch_backward(L, stream);
}

}  // namespace ccm
