// Forward contact-manifold kernel (Sec. 4.2-4.4 of arxiv 2604.17538).
//
// One warp computes one unit (pair, side): the blend groups of every convex
// piece f of the feature body F against the SDF pieces s of the other body S
// (side 0: F = A, S = B; side 1: F = B, S = A).  See ccm_unit.cuh for how the
// work is flattened over directions (s, f).
//
// Exact culls (every culled contact has transition weight 0, Sec. 4.3):
//   * piece pair: max_k phi_k(c_f) - r_f >= d_max proves phi_s >= d_max on
//     all of f (phi >= max-plane and both are 1-Lipschitz);
//   * vertex: max-plane value m >= d_max;
//   * edge: a lower bound of the max-plane value along the edge >= d_max,
//     from the planes attaining it at the two corners (edge_plane_bound).
// A pair's outputs depend only on that pair: bit-identical in any batch.
#include "ccm_narrow.cuh"
#include "ccm_unit.cuh"
#include "ccm_fwd.h"
#include "ccm_launch.h"

namespace ccm {

// Where the records of a list's contacts point: the global output row and
// piece index of the F chunk's first group, and the first piece of body S.
struct ChunkRef {
  int64_t row;
  int32_t fpiece;
  int32_t spiece;
};

// Appends this round's contacts of non-zero weight (lane's `contrib`: group
// `key` of the F chunk, SDF piece `s_glob` (global index), piece-local
// feature `feat` of kind `kind`, 0 vertex / 1 edge) to the contact list.  A
// contact's rank among its group's contacts of its kind follows the lane
// order, so it does not depend on where the round's records land.  Records
// that do not fit set the overflow flag.
__device__ __forceinline__ void append_contacts(const ContactList& cl, int* gcnt, bool contrib,
                                                int key, int kind, int feat, int s_glob,
                                                const ChunkRef& cr, int lane) {
  const unsigned cm = __ballot_sync(kFull, contrib);
  if (cm == 0u) return;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned same = __match_any_sync(kFull, contrib ? key : 0x10000 + lane) & cm;
  int base = 0;
  if (contrib) base = gcnt[2 * key + kind];
  __syncwarp();
  const int rank = __popc(same & lt);
  if (contrib && rank == 0) gcnt[2 * key + kind] = base + __popc(same);
  unsigned long long at = 0;
  if (lane == 0) at = atomicAdd(cl.ctl + kCtlCursor, (unsigned long long)__popc(cm));
  at = __shfl_sync(kFull, at, 0) + __popc(cm & lt);
  if (contrib) {
    const int seq = base + rank;
    if ((long long)at < cl.cap && seq < (1 << kRankBits) && feat < (1 << kFeatBits)) {
      const uint32_t w = ((uint32_t)kind << 31) | ((uint32_t)feat << kRankBits) | (uint32_t)seq;
      cl.recs[at] = make_int4((int)(cr.row + key), s_glob, cr.fpiece + key, (int)w);
    } else {
      cl.ctl[kCtlOverflow] = 1ull;   // the reverse passes fall back to re-gating
    }
  }
  __syncwarp();
}

struct FwdCounts {
  unsigned long long dirs = 0, gate = 0, live = 0, maxp = 0, eg = 0, ev = 0, con = 0, feat = 0;
};

// Narrow phase of the live directions sl.dsub[0..nd) whose vertex / edge items
// are numbered by the exclusive prefixes sl.pv / sl.pe (totals TV, TE).
template <bool kCount>
__device__ void run_list(const DevGeom& g, const UnitSlice& sl, const int* dsub, int nd, int TV,
                         int TE, int sc0, const KParams& kp, bool no_cull, int lane,
                         FwdCounts& cnt, const ContactList& cl, const ChunkRef& cr) {
  const bool project = (kp.flags & CCM_FLAG_PROJECT) != 0u;
  const bool voxel = (kp.flags & CCM_FLAG_VOXEL_CULL) != 0u && !no_cull;
  // Sec. 4.3 voxel-grid broad phase (with CCM_FLAG_VOXEL_CULL): a vertex whose
  // voxel's lower bound of the SDF is >= d_max is culled without a plane
  // scan; it keeps the one plane value below as its (valid, lower) max-plane
  // bound for the edge cull and marks its plane index with kVoxCulled.
  // max-plane value of every (direction, vertex) item.  First one plane: the
  // plane attaining the max at the feature piece's centre (from the gate) is
  // far above d_max at the vertices on the far side of the piece, and its
  // value is a lower bound of the max-plane value, so those vertices are
  // culled exactly; the others (packed into vlist, used here as scratch) get
  // the exact max over all planes
  int nfull = 0;
  for (int t0 = 0; t0 < TV; t0 += 32) {
    const int t = t0 + lane;
    bool full = false;
    if (t < TV) {
      const int r = find_dir(sl.pv, nd, t);
      const int code = dsub[r];
      const int4 f = sl.fp[code >> 16];
      const int2 s = sl.sp[code & 0xffff];
      const float4 x = sl.xs[f.x + t - sl.pv[r]];
      const int j = sl.dsubpl[r];
      const float4 pj = sl.planes[s.x + j];
      const float vj = fmaf(pj.x, x.x, fmaf(pj.y, x.y, fmaf(pj.z, x.z, pj.w)));
      sl.need[t] = 0;
      const float vb = voxel ? voxel_bound(g, cr.spiece + sc0 + (code & 0xffff), x.x, x.y, x.z)
                             : -INFINITY;
      sl.vb[t] = vb;
      if (!no_cull && vj >= kp.d_max) {
        sl.m[t] = vj;
        sl.am[t] = (uint16_t)j;
        if (kCount) cnt.maxp += 1;
      } else if (vb - kVoxTol >= kp.d_max) {
        sl.m[t] = vj;
        sl.am[t] = (uint16_t)(j | kVoxCulled);
        if (kCount) cnt.maxp += 1;
      } else {
        full = true;
      }
    }
    const unsigned bal = __ballot_sync(kFull, full);
    if (full) sl.vlist[nfull + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
    nfull += __popc(bal);
  }
  __syncwarp();
  for (int k = lane; k < nfull; k += 32) {
    const int t = sl.vlist[k];
    const int r = find_dir(sl.pv, nd, t);
    const int code = dsub[r];
    const int4 f = sl.fp[code >> 16];
    const int2 s = sl.sp[code & 0xffff];
    const float4 x = sl.xs[f.x + t - sl.pv[r]];
    int arg;
    sl.m[t] = max_plane_arg(sl.planes + s.x, s.y, x.x, x.y, x.z, arg);
    sl.am[t] = (uint16_t)arg;
    if (kCount) cnt.maxp += s.y;
  }
  __syncwarp();
  // edge cull: the max-plane value along the edge is bounded below by the
  // two planes that attain it at the corners (edge_plane_bound)
  int n_e = 0;
  for (int t0 = 0; t0 < TE; t0 += 32) {
    const int t = t0 + lane;
    bool live = false;
    if (t < TE) {
      const int r = find_dir(sl.pe, nd, t);
      const int code = dsub[r];
      const int4 f = sl.fp[code >> 16];
      const int2 s = sl.sp[code & 0xffff];
      const uint32_t e = sl.edges[f.z + t - sl.pe[r]];
      const int i0 = e & 0xffff, i1 = e >> 16;
      const int t0v = sl.pv[r] + i0, t1v = sl.pv[r] + i1;
      const float4 a = sl.xs[f.x + i0], b = sl.xs[f.x + i1];
      const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
      const float lb = edge_plane_bound(sl.planes[s.x + (sl.am[t0v] & kPlaneMask)],
                                        sl.planes[s.x + (sl.am[t1v] & kPlaneMask)], dx, dy, dz,
                                        sl.m[t0v], sl.m[t1v]);
      // Sec. 4.3 voxel edge bound: min(phi_1, phi_2) - r - l (r inside vb)
      // 1-Lipschitz max-plane value: above (b_I + b_II - L) / 2 along the edge
      const float vlb = 0.5f * (sl.vb[t0v] + sl.vb[t1v] - sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))));
      live = no_cull || (lb - kEdgeTol < kp.d_max && vlb - kVoxTol < kp.d_max);
      if (live) { sl.need[t0v] = 1; sl.need[t1v] = 1; }
    }
    const unsigned bal = __ballot_sync(kFull, live);
    if (live) sl.elist[n_e + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
    n_e += __popc(bal);
  }
  __syncwarp();
  int n_v = 0;
  for (int t0 = 0; t0 < TV; t0 += 32) {
    const int t = t0 + lane;
    bool live = false;
    if (t < TV) {
      if (sl.am[t] & kVoxCulled) {
        // from here on m is only a lower bound (the SDF shift and the contact
        // test): the voxel bound lifts it to >= d_max, so no contact is made
        sl.m[t] = fmaxf(sl.m[t], sl.vb[t]);
      }
      live = no_cull || sl.m[t] < kp.d_max || sl.need[t];
    }
    const unsigned bal = __ballot_sync(kFull, live);
    if (live) sl.vlist[n_v + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
    n_v += __popc(bal);
  }
  __syncwarp();
  // V-SDF contacts (and the SDF at vertices that start a sphere trace)
  for (int k0 = 0; k0 < n_v; k0 += 32) {
    const int k = k0 + lane;
    PartT<float> c;
    part_zero(c);
    int key = 0xffff;
    bool contrib = false;
    int feat = 0, s_glob = 0;
    if (k < n_v) {
      const int t = sl.vlist[k];
      const int r = find_dir(sl.pv, nd, t);
      const int code = dsub[r];
      const int4 f = sl.fp[code >> 16];
      const int2 s = sl.sp[code & 0xffff];
      feat = t - sl.pv[r];
      const float4 x = sl.xs[f.x + feat];
      const float m = sl.m[t];
      const SdfGrad sg = sdf_grad(sl.planes + s.x, s.y, x.x, x.y, x.z, m, kp);
      sl.phi[t] = sg.phi;
      key = code >> 16;
      s_glob = cr.spiece + sc0 + (code & 0xffff);
      if (no_cull || m < kp.d_max) {
        const float w = transition(sg.phi, kp);
        const float dc = fmaf(w, sg.phi - kp.d_max, kp.d_max);   // f phi + (1 - f) d_max
        float3 p = make_float3(x.x, x.y, x.z);
        if (project) p = make_float3(fmaf(-sg.phi, sg.gx, p.x), fmaf(-sg.phi, sg.gy, p.y),
                                     fmaf(-sg.phi, sg.gz, p.z));   // Sec. 4.1 projection
        part_from_contact(c, w, dc, v3(p.x, p.y, p.z), v3(sg.gx, sg.gy, sg.gz), kp.c_blend);
        mark_hit(sl.hit, sl.hw, code >> 16, sc0 + (code & 0xffff), w);
        contrib = w > 0.f;
        if (kCount) cnt.con += w > 0.f;
      }
      if (kCount) cnt.eg += s.y;
    }
    if (cl.recs) append_contacts(cl, sl.gcnt, contrib, key, 0, feat, s_glob, cr, lane);
    fold_t(c, key, sl.acc, lane);
  }
  __syncwarp();
  // E-SDF contacts: sphere trace from both corners, soft clip, midpoint
  for (int k0 = 0; k0 < n_e; k0 += 32) {
    const int k = k0 + lane;
    PartT<float> c;
    part_zero(c);
    int key = 0xffff;
    bool contrib = false;
    int feat = 0, s_glob = 0;
    if (k < n_e) {
      const int t = sl.elist[k];
      const int r = find_dir(sl.pe, nd, t);
      const int code = dsub[r];
      const int4 f = sl.fp[code >> 16];
      const int2 s = sl.sp[code & 0xffff];
      feat = t - sl.pe[r];
      s_glob = cr.spiece + sc0 + (code & 0xffff);
      const uint32_t e = sl.edges[f.z + feat];
      const int i0 = e & 0xffff, i1 = e >> 16;
      const int t0v = sl.pv[r] + i0, t1v = sl.pv[r] + i1;
      const EdgeContact ec = edge_contact(sl.planes + s.x, s.y, sl.xs[f.x + i0], sl.xs[f.x + i1],
                                          sl.m[t0v], sl.m[t1v], sl.phi[t0v], sl.phi[t1v], kp);
      const float w = transition(ec.phi, kp);
      const float dc = fmaf(w, ec.phi - kp.d_max, kp.d_max);
      float3 p = make_float3(ec.px, ec.py, ec.pz);
      if (project) p = make_float3(fmaf(-ec.phi, ec.gx, p.x), fmaf(-ec.phi, ec.gy, p.y),
                                   fmaf(-ec.phi, ec.gz, p.z));   // Sec. 4.1 projection
      part_from_contact(c, w, dc, v3(p.x, p.y, p.z), v3(ec.gx, ec.gy, ec.gz), kp.c_blend);
      mark_hit(sl.hit, sl.hw, code >> 16, sc0 + (code & 0xffff), w);
      key = code >> 16;
      contrib = w > 0.f;
      if (kCount) {
        cnt.con += w > 0.f;
        cnt.eg += s.y;
        cnt.ev += (unsigned long long)s.y * 2 * (kp.trace_iters > 0 ? kp.trace_iters - 1 : 0);
      }
    }
    if (cl.recs) append_contacts(cl, sl.gcnt, contrib, key, 1, feat, s_glob, cr, lane);
    fold_t(c, key, sl.acc, lane);
  }
  __syncwarp();
}

// Splits the pending directions sl.dir[0..np) into lists that fit the item
// budgets and runs each.
template <bool kCount>
__device__ void run_pending(const DevGeom& g, const UnitSlice& sl, int* dsub, int np, int sc0,
                           const UnitShape& us, const KParams& kp, bool no_cull, int lane,
                           FwdCounts& cnt, const ContactList& cl, const ChunkRef& cr) {
  int start = 0;
  while (start < np) {
    const int r = start + lane;
    int nvr = 0, ner = 0, code = 0, pl = 0;
    if (r < np) {
      code = sl.dir[r];
      pl = sl.dpl[r];
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
    const bool fits = r < np && iv <= us.item_v && ie <= us.item_e;
    const int nd = __popc(__ballot_sync(kFull, fits));   // >= 1: budgets hold any one piece
    if (lane < nd) {
      dsub[lane] = code;
      sl.dsubpl[lane] = pl;
      sl.pv[lane] = iv - nvr;
      sl.pe[lane] = ie - ner;
      if (kCount) { cnt.live += 1; cnt.feat += nvr + ner; }
    }
    const int TV = __shfl_sync(kFull, iv, nd - 1), TE = __shfl_sync(kFull, ie, nd - 1);
    __syncwarp();
    run_list<kCount>(g, sl, dsub, nd, TV, TE, sc0, kp, no_cull, lane, cnt, cl, cr);
    start += nd;
  }
}

template <bool kCount>
__global__ void __launch_bounds__(128)
unit_fwd_kernel(DevGeom g, const PairRec* __restrict__ pairs,
                const WorkItem* __restrict__ items, const int32_t* __restrict__ order,
                int64_t n_items, const int64_t* __restrict__ dev_items,
                const float* __restrict__ pose_a, const float* __restrict__ pose_b, KParams kp,
                UnitShape us, float* __restrict__ y, float* __restrict__ saved,
                unsigned long long* __restrict__ counters, int* __restrict__ sched,
                ContactList cl, int* __restrict__ status,
                const unsigned long long* __restrict__ only_if) {
  pdl_wait();   // launched behind the flat chain: its flag and buffers first
  if (only_if && *only_if == 0ull) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const UnitSlice sl = unit_slice(smem_raw + (size_t)warp * us.slice_bytes, us);
  uint32_t phase = 0;   // parity of the warp's next bulk-copy barrier phase
  if (us.stage_tma && lane == 0) mbar_init(sl.mbar, 1);
  __syncwarp();
  int* dsub = sl.dsub;
  const bool no_cull = (kp.flags & 1u) != 0;
  const int64_t n_run = dev_items ? *dev_items : n_items;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  FwdCounts cnt;

  // heaviest items first, dealt round-robin to the warps (balanced, no atomics)
  for (int64_t k = first_unit(sched, (int64_t)blockIdx.x * (blockDim.x >> 5) + warp); k < n_run;
       k = next_unit(sched, k, nwarps)) {
    const WorkItem it = items[order[k]];
    const int64_t u = it.unit;
    const int64_t pi = u >> 1;
    const int side = (int)(u & 1);
    const PairRec pr = pairs[pi];
    const BodyRec bA = g.bodies[pr.bodyA], bB = g.bodies[pr.bodyB];
    const BodyRec F = side == 0 ? bA : bB, S = side == 0 ? bB : bA;
    const int64_t row0 = pr.goff + (side == 0 ? 0 : bA.np);
    const float* pF = (side == 0 ? pose_a : pose_b) + 12 * pi;
    const float* pS = (side == 0 ? pose_b : pose_a) + 12 * pi;
    float Rr[9], tr[3];
    rel_pose_f64(pF, pS, lane, Rr, tr);
    const float margin = 1e-6f * (1.0f + fabsf(tr[0]) + fabsf(tr[1]) + fabsf(tr[2]));

    for (int fc0 = it.fc0; fc0 < it.fc1;) {
      // F chunk [fc0, fc1): up to us.groups (<= 32) pieces within the vertex /
      // edge budgets (the host cut the item to one such chunk), read one per
      // lane: the chunk is the prefix of lanes whose running sums fit
      PieceRec p{};
      const bool valid = fc0 + lane < it.fc1 && lane < us.groups;
      if (valid) p = g.pieces[F.p0 + fc0 + lane];
      int iv = valid ? p.nv : 0, ie = valid ? p.ne : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(kFull, iv, o), b = __shfl_up_sync(kFull, ie, o);
        if (lane >= o) { iv += a; ie += b; }
      }
      const bool in_chunk = valid && iv <= us.vert_budget && ie <= us.edge_budget;
      const int nfc = __popc(__ballot_sync(kFull, in_chunk));   // a prefix of the lanes
      if (nfc == 0) break;   // unreachable: the host sizes the budgets >= every piece
      const int fc1 = fc0 + nfc;
      const int V = __shfl_sync(kFull, iv, nfc - 1), E = __shfl_sync(kFull, ie, nfc - 1);
      const int pv0 = __shfl_sync(kFull, p.v0, 0), pe0 = __shfl_sync(kFull, p.e0, 0);
      __syncwarp();   // the previous chunk's data is no longer read
      if (lane < nfc) {
        sl.fp[lane] = make_int4(p.v0 - pv0, p.nv, p.e0 - pe0, p.ne);
        const float3 c = xform(Rr, tr, p.sphere);
        sl.fs[lane] = make_float4(c.x, c.y, c.z, p.sphere.w);
        part_zero(sl.acc[lane]);
        for (int q = 0; q < sl.hw; ++q) sl.hit[lane * sl.hw + q] = 0u;
        sl.gcnt[2 * lane] = 0;
        sl.gcnt[2 * lane + 1] = 0;
      }
      const ChunkRef cr{row0 + fc0, F.p0 + fc0, S.p0};
      for (int i = lane; i < V; i += 64) {   // two loads in flight per lane
        const bool two = i + 32 < V;
        const float4 v0 = __ldg(g.verts + pv0 + i);
        const float4 v1 = two ? __ldg(g.verts + pv0 + i + 32) : v0;
        const float3 x0 = xform(Rr, tr, v0), x1 = xform(Rr, tr, v1);
        sl.xs[i] = make_float4(x0.x, x0.y, x0.z, 0.f);
        if (two) sl.xs[i + 32] = make_float4(x1.x, x1.y, x1.z, 0.f);
      }
      stage_copy(sl.edges, g.edges + pe0, E, lane);

      for (int sc0 = 0; sc0 < S.np;) {
        // S chunk [sc0, sc1) within the plane / piece budgets: pieces read 32
        // at a time (one per lane); the chunk ends before the first piece whose
        // planes overflow.  A body's planes are contiguous, piece after piece.
        int sc1 = sc0, P = 0;
        __syncwarp();   // the previous S chunk's planes are no longer read
        while (sc1 < S.np && sc1 - sc0 < us.spiece_budget) {
          const int si = sc1 + lane;
          const int nf = si < S.np && si - sc0 < us.spiece_budget ? g.pieces[S.p0 + si].nf : 0;
          int incl = nf;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
          }
          const bool fits = nf > 0 && P + incl <= us.plane_budget;
          const int take = __popc(__ballot_sync(kFull, fits));   // a prefix of the lanes
          if (fits) sl.sp[si - sc0] = make_int2(P + incl - nf, nf);
          if (take > 0) P += __shfl_sync(kFull, incl, take - 1);
          sc1 += take;
          if (take < 32) break;
        }
        const int nsc = sc1 - sc0;
        if (nsc == 0) break;   // unreachable, as above
        if (us.stage_tma) {
          // the chunk's planes (contiguous, 16 B each) in one bulk copy; the
          // lanes' earlier reads of the slice precede it (syncwarp above)
          if (lane == 0) {
            fence_proxy_async_smem();
            bulk_copy_g2s(sl.planes, g.planes + g.pieces[S.p0 + sc0].f0, 16u * (uint32_t)P,
                          sl.mbar);
          }
          // the whole warp gives up together (a lane may see the phase
          // complete on the poll after another lane's last one)
          const bool ok = __all_sync(kFull, mbar_wait_bounded(sl.mbar, phase, us.wait_limit));
          if (!ok) {
            // record the timeout, let the copy land, and stop this warp
            if (lane == 0 && status) atomicExch(status, (int)CCM_ERR_TIMEOUT);
            mbar_wait_bounded(sl.mbar, phase, kDrainLimit);
            return;
          }
          phase ^= 1u;
        } else {
          stage_copy(sl.planes, g.planes + g.pieces[S.p0 + sc0].f0, P, lane);
        }
        __syncwarp();

        // gate the directions (fc, sc), 32 at a time, collecting live ones
        int np = 0;
        const int ndir = nfc * nsc;
        for (int d0 = 0; d0 < ndir; d0 += 32) {
          const int d = d0 + lane;
          bool live = false;
          int code = 0, pl = 0;
          if (d < ndir) {
            const int fcd = d / nsc, scd = d - fcd * nsc;
            const float4 c = sl.fs[fcd];
            const int2 s = sl.sp[scd];
            const float mc = max_plane_arg(sl.planes + s.x, s.y, c.x, c.y, c.z, pl);
            live = no_cull || mc - c.w - margin < kp.d_max;
            code = (fcd << 16) | scd;
            if (kCount) { cnt.dirs += 1; cnt.gate += s.y; }
          }
          const unsigned bal = __ballot_sync(kFull, live);
          const int nl = __popc(bal);
          if (np + nl > kPending) {
            run_pending<kCount>(g, sl, dsub, np, sc0, us, kp, no_cull, lane, cnt, cl, cr);
            np = 0;
          }
          if (live) {
            const int at = np + __popc(bal & ((1u << lane) - 1u));
            sl.dir[at] = code;
            sl.dpl[at] = pl;
          }
          np += nl;
          __syncwarp();
        }
        if (np > 0) run_pending<kCount>(g, sl, dsub, np, sc0, us, kp, no_cull, lane, cnt, cl, cr);
        sc0 = sc1;
      }
      __syncwarp();
      if (lane < nfc) {
        const PartT<float> acc = sl.acc[lane];
        float RS[9], tS[3];
        load_pose(pS, RS, tS);
        write_group(y + 8 * (row0 + fc0 + lane), acc, RS, tS, kp);
        if (saved)
          save_group(saved + (int64_t)kSavedFloats * (row0 + fc0 + lane), acc,
                     sl.hit + lane * sl.hw, sl.hw, cl.recs ? cl.tag : 0u);
        if (cl.recs) {
          cl.cnt_v[row0 + fc0 + lane] = sl.gcnt[2 * lane];
          cl.cnt_e[row0 + fc0 + lane] = sl.gcnt[2 * lane + 1];
        }
      }
      fc0 = fc1;
    }
  }

  if (kCount) {
    unsigned long long v[8] = {cnt.dirs, cnt.live, cnt.maxp, cnt.gate, cnt.eg, cnt.ev, cnt.con,
                               cnt.feat};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      unsigned long long x = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (lane == 0) atomicAdd(counters + q, x);
    }
  }
}

cudaError_t launch_forward(const FwdLaunch& L, cudaStream_t stream) {
  if (L.sched && !L.after_chain) {
    const cudaError_t e = cudaMemsetAsync(L.sched, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
  }
  const size_t smem = (size_t)L.us.warps * L.us.slice_bytes;
  const int threads = 32 * L.us.warps;
  ContactList cl = L.cl;
  if (!L.saved) cl.recs = nullptr;   // the list goes with the saved record
  if (cl.recs) {
    const cudaError_t e = cudaMemsetAsync(cl.ctl, 0, kCtlWords * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = launch_k(L.after_chain, L.counters ? unit_fwd_kernel<true> : unit_fwd_kernel<false>,
                                 L.grid, threads, smem, stream, L.g, L.pairs, L.items, L.order,
                                 L.n_items, L.dev_items, L.pose_a, L.pose_b, L.kp, L.us, L.y,
                                 L.saved, L.counters, L.sched, cl, L.status, L.only_if);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t configure_forward(const UnitShape& us, int smem_limit, int* blocks_per_sm) {
  const int smem = us.warps * us.slice_bytes;
  cudaError_t e;
  // The limit is raised to the device's opt-in maximum (not to this shape's
  // size): the attribute is shared by every batch and captured graph of the
  // process, and lowering it would invalidate their larger launches.
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(unit_fwd_kernel<false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(unit_fwd_kernel<true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit)) != cudaSuccess)
      return e;
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, unit_fwd_kernel<false>,
                                                32 * us.warps, smem);
  return cudaGetLastError();
}

}  // namespace ccm
