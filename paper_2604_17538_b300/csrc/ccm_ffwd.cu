// Flat forward (Sec. 4.2-4.4): the per-item forward kernel (ccm_fwd.cu) split
// into stages that each run flat over the whole batch, so that the lanes of a
// warp take independent work instead of one unit's short lists:
//   setup    per unit the relative pose S <- F (FP64, rounded once), and the
//            per-call counters cleared;
//   gate     one direction (unit, F piece f, S piece s) per thread: the exact
//            piece-pair cull of Sec. 4.3 (the largest plane value of s at the
//            centre of f's bounding sphere, minus its radius, >= d_max);
//   feature  one live direction per warp, lanes over f's vertices and edges:
//            the exact vertex cull (largest plane value >= d_max), the
//            two-plane edge bound and, with CCM_FLAG_VOXEL_CULL, the voxel
//            bounds; survivors become candidate contacts;
//   eval     one candidate per thread: V-SDF (the vertex) or E-SDF (sphere
//            trace of both corners, soft clip, midpoint), mollified; contacts
//            of non-zero weight are counted per output group and mark their
//            direction in the saved record's hit words;
//   scan     the counts to offsets (ccm_flat.cu), then scatter: the contacts
//            of non-zero weight to their group's segment of the contact list;
//   rank     one contact per thread: its place in the segment's (SDF piece,
//            feature) order, where it and its values are written; and every
//            group's outputs and record written as if it had no contact;
//   fold     one group with contacts per four lanes: its vertex contacts,
//            then its edge contacts, blended (online softmax, Sec. 4.4) in a
//            fixed order into the group's outputs and saved record.
// The contact list it leaves is the one the per-contact reverse passes read
// (ccm_flat.cu).  The fixed order of the fold makes a pair's outputs depend
// on the pair alone.  Culls are those of the per-item kernel, so the set of
// contacts with non-zero weight is the same; a candidate or contact list that
// overflows its capacity sets a flag, the later stages do nothing, and the
// caller runs the per-item kernel instead.
#include <algorithm>

#include "ccm_narrow.cuh"
#include "ccm_unit.cuh"
#include "ccm_ffwd.h"
#include "ccm_launch.h"

namespace ccm {

// ---------------------------------------------------------------------------
// setup: relative poses per unit; counters (the per-item fallback's too),
// group counts and hit words zeroed
// ---------------------------------------------------------------------------
__global__ void ff_setup_kernel(FlatFwdLaunch L) {
  pdl_wait();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (tid < kFfWords) L.ctl[tid] = 0ull;
  if (tid < kCtlWords) L.cl.ctl[tid] = 0ull;
  if (tid == 0 && L.fallback_sched) *L.fallback_sched = 0;
  for (int64_t i = tid; i < L.G; i += stride) {
    L.cl.cnt_v[i] = 0;
    L.cl.cnt_e[i] = 0;
  }
  if (L.saved) {
    uint4* h = reinterpret_cast<uint4*>(L.hits);
    for (int64_t i = tid; i < L.G * (kHitWords / 4); i += stride) h[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int64_t u = tid; u < 2 * L.n_pairs; u += stride) {
    const int64_t p = u >> 1;
    const int side = (int)(u & 1);
    const float* pF = (side == 0 ? L.pose_a : L.pose_b) + 12 * p;
    const float* pS = (side == 0 ? L.pose_b : L.pose_a) + 12 * p;
    float* r = L.rel + 12 * u;
    // Rr = R_S^T R_F, tr = R_S^T (t_F - t_S), accumulated in double
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += (double)__ldg(pS + 3 * k + i) * (double)__ldg(pF + 3 * k + j);
        r[3 * i + j] = (float)acc;
      }
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k)
        acc += (double)__ldg(pS + 3 * k + i) * ((double)__ldg(pF + 9 + k) - (double)__ldg(pS + 9 + k));
      r[9 + i] = (float)acc;
    }
  }
}

__device__ __forceinline__ void load_rel(const float* r, float R[9], float t[3]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = r[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i] = r[9 + i];
}

// sort key of a contact within its group and kind: (SDF piece, feature)
__device__ __forceinline__ long long ff_key(int4 r) {
  return ((long long)r.y << 12) | (r.w & 0xfff);
}

// warp-aggregated append of the lanes with `want` to a counter-indexed array
__device__ __forceinline__ int64_t ff_slot(unsigned long long* counter, bool want, int lane) {
  const unsigned m = __ballot_sync(kFull, want);
  if (m == 0u) return -1;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, 0);
  return want ? (int64_t)(base + __popc(m & ((1u << lane) - 1u))) : -1;
}

// Copies n planes to a warp's shared memory: one bulk copy completed on the
// warp's mbarrier, or the lanes' loads.  A bulk copy whose wait runs out
// records CCM_ERR_TIMEOUT, waits (bounded) for the copy to land and returns
// false: the warp then stops.  The caller's syncwarp before the call orders
// the lanes' earlier reads of dst before the copy.
__device__ __forceinline__ bool ff_stage(const FlatFwdLaunch& L, float4* dst, const float4* src,
                                         int n, uint64_t* bar, uint32_t& phase, int lane) {
  if (!L.stage_tma) {
    stage_copy(dst, src, n, lane);
    return true;
  }
  if (lane == 0) {
    fence_proxy_async_smem();
    bulk_copy_g2s(dst, src, 16u * (uint32_t)n, bar);
  }
  const bool ok = __all_sync(kFull, mbar_wait_bounded(bar, phase, L.wait_limit));
  if (!ok) {
    if (lane == 0 && L.status) atomicExch(L.status, (int)CCM_ERR_TIMEOUT);
    mbar_wait_bounded(bar, phase, kDrainLimit);
  }
  phase ^= 1u;
  return ok;
}

// ---------------------------------------------------------------------------
// gate: one unit per warp, lanes over its directions (f, s); the SDF body's
// planes staged in the warp's shared memory, a chunk of pieces at a time
// ---------------------------------------------------------------------------
constexpr int kGateWarps = 4;

template <bool kCount>
__global__ void __launch_bounds__(128) ff_gate_kernel(FlatFwdLaunch L) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* pl_s = reinterpret_cast<float4*>(smem_raw) + (size_t)warp * L.gate_planes;
  __shared__ uint64_t bar_s[kGateWarps];
  uint64_t* bar = bar_s + warp;
  if (L.stage_tma && lane == 0) mbar_init(bar, 1);
  __syncwarp();
  uint32_t phase = 0;
  const bool no_cull = (L.kp.flags & CCM_FLAG_NO_CULL) != 0u;
  const int64_t nu = 2 * L.n_pairs;
  unsigned long long c_dirs = 0, c_gate = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; u < nu; u += warps) {
    const PairRec pr = L.pairs[u >> 1];
    const int side = (int)(u & 1);
    const BodyRec bA = L.g.bodies[pr.bodyA], bB = L.g.bodies[pr.bodyB];
    const BodyRec F = side == 0 ? bA : bB, S = side == 0 ? bB : bA;
    const int64_t row0 = pr.goff + (side == 0 ? 0 : bA.np);
    float R[9], tr[3];
    load_rel(L.rel + 12 * u, R, tr);
    const float margin = 1e-6f * (1.0f + fabsf(tr[0]) + fabsf(tr[1]) + fabsf(tr[2]));
    const int f_base = L.g.pieces[S.p0].f0;   // a body's planes are contiguous
    for (int s0 = 0; s0 < S.np;) {
      // the chunk [s0, s1): whole pieces (at most 32) whose planes fit the
      // warp's budget, from a prefix sum of the pieces' plane counts
      const PieceRec mine = s0 + lane < S.np ? L.g.pieces[S.p0 + s0 + lane] : PieceRec{};
      int pre = s0 + lane < S.np ? mine.nf : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, pre, o);
        if (lane >= o) pre += t;
      }
      const unsigned fit = __ballot_sync(
          kFull, s0 + lane < S.np && (L.gate_planes == 0 || pre <= L.gate_planes));
      const int ns = max(1, __popc(fit));            // the prefix sums grow with the lane
      const int P = __shfl_sync(kFull, pre, ns - 1);
      const int p0 = __shfl_sync(kFull, mine.f0, 0) - f_base;
      if (L.gate_planes > 0) {
        __syncwarp();   // the previous chunk is no longer read
        if (!ff_stage(L, pl_s, L.g.planes + f_base + p0, P, bar, phase, lane)) return;
        __syncwarp();
      }
      // directions f fastest: lanes that share an SDF piece read the same
      // plane (a broadcast) and run the same number of steps
      const int nd = F.np * ns;
      for (int d0 = 0; d0 < nd; d0 += 32) {
        const int d = d0 + lane;
        const int s = d / F.np, f = d - s * F.np;
        const int sf0 = __shfl_sync(kFull, mine.f0, min(s, 31));
        const int snf = __shfl_sync(kFull, mine.nf, min(s, 31));
        bool live = false;
        int4 rec = make_int4(0, 0, 0, 0);
        if (d < nd) {
          const float4 sph = L.g.pieces[F.p0 + f].sphere;
          const float3 c = xform(R, tr, sph);
          int pl = 0;
          // staged planes, or (gate_planes = 0, pieces too large to stage
          // without starving the SM of warps) the planes in global memory
          const float4* spl = L.gate_planes > 0 ? pl_s + (sf0 - f_base - p0) : L.g.planes + sf0;
          const float mc = max_plane_arg(spl, snf, c.x, c.y, c.z, pl);
          live = no_cull || mc - sph.w - margin < L.kp.d_max;
          // (output row, F piece, S piece, a plane attaining the max at the centre)
          rec = make_int4((int)(row0 + f), F.p0 + f, S.p0 + s0 + s, pl);
          if (kCount) { c_dirs += 1; c_gate += snf; }
        }
        const int64_t at = ff_slot(L.ctl + kFfLive, live, lane);
        if (live) L.live[at] = rec;   // capacity: every direction
      }
      s0 += ns;
    }
  }
  if (kCount && L.counters) {
    unsigned long long v[2] = {c_dirs, c_gate};
    for (int q = 0; q < 2; ++q) {
      unsigned long long x = v[q];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (lane == 0 && x) atomicAdd(L.counters + (q == 0 ? CCM_CNT_DIRS : CCM_CNT_GATEPASS), x);
    }
  }
}

// ---------------------------------------------------------------------------
// feature: one live direction per warp
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t ff_feature_warp_bytes(int vmax, int fmax) {
  return (size_t)align16i(16 * vmax) + align16i(4 * vmax) * 2 + align16i(2 * vmax) +
         (size_t)16 * fmax;
}

// dynamic shared memory of a block: the default 48 KB less the static
// mbarrier words of the gate and feature kernels
constexpr int kDynSmem = 48 * 1024 - 256;

bool flat_forward_fits(int vmax, int fmax) {
  return 16 * fmax <= kDynSmem && ff_feature_warp_bytes(vmax, fmax) <= (size_t)kDynSmem;
}

size_t flat_forward_feature_smem(int vmax, int fmax, int* warps_per_block) {
  const size_t per_warp = ff_feature_warp_bytes(vmax, fmax);
  int w = 4;
  while (w > 1 && (size_t)w * per_warp > (size_t)kDynSmem) --w;
  *warps_per_block = w;
  return (size_t)w * per_warp;
}

// candidate index of the t-th candidate of the eval order: the nv vertex
// candidates, then the edge candidates from the middle of the arrays
__device__ __forceinline__ int64_t ff_cand_index(const FlatFwdLaunch& L, int64_t t, int64_t nv) {
  return t < nv ? t : L.cand_cap / 2 + (t - nv);
}

__device__ __forceinline__ void ff_push(const FlatFwdLaunch& L, bool want, int4 rec, float2 mm,
                                        int lane, bool edge) {
  const int64_t at = ff_slot(L.ctl + (edge ? kFfCandE : kFfCand), want, lane);
  if (want) {
    const int64_t half = L.cand_cap / 2;
    if (at < half) {
      const int64_t k = edge ? half + at : at;
      L.cand[k] = rec;
      L.cand_m[k] = mm;
    } else {
      L.ctl[kFfOverflow] = 1ull;
    }
  }
}

template <bool kCount>
__global__ void __launch_bounds__(128, 8) ff_feature_kernel(FlatFwdLaunch L) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int vmax = L.vmax;
  unsigned char* base = smem_raw + (size_t)warp * ff_feature_warp_bytes(vmax, L.fmax);
  float4* xs = reinterpret_cast<float4*>(base);
  float* m = reinterpret_cast<float*>(base + align16i(16 * vmax));
  float* vb = reinterpret_cast<float*>(base + align16i(16 * vmax) + align16i(4 * vmax));
  uint16_t* am = reinterpret_cast<uint16_t*>(base + align16i(16 * vmax) + 2 * align16i(4 * vmax));
  float4* planes = reinterpret_cast<float4*>(base + align16i(16 * vmax) + 2 * align16i(4 * vmax) +
                                             align16i(2 * vmax));
  __shared__ uint64_t bar_s[4];
  uint64_t* bar = bar_s + warp;
  if (L.stage_tma && lane == 0) mbar_init(bar, 1);
  __syncwarp();
  uint32_t phase = 0;
  const bool no_cull = (L.kp.flags & CCM_FLAG_NO_CULL) != 0u;
  const bool voxel = (L.kp.flags & CCM_FLAG_VOXEL_CULL) != 0u && !no_cull;
  const float d_max = L.kp.d_max;
  const int64_t n_live = (int64_t)L.ctl[kFfLive];
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long c_live = 0, c_maxp = 0, c_feat = 0;
  // a persistent grid: each warp takes every warps-th live direction, and the
  // next one's record is loaded while the current one is processed
  int64_t d = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  int4 lv_next = d < n_live ? L.live[d] : make_int4(0, 0, 0, 0);
  for (; d < n_live; d += warps) {
    const int4 lv = lv_next;
    if (d + warps < n_live) lv_next = L.live[d + warps];
    const int row = lv.x, f_glob = lv.y, s_glob = lv.z, pl = lv.w;
    const int64_t u = L.row_pair[row];   // unit = 2 pair + side
    const PieceRec fp = L.g.pieces[f_glob], sp = L.g.pieces[s_glob];
    // the SDF piece's planes in the warp's shared memory (the previous
    // direction's are no longer read: syncwarp at the end of the loop)
    float R[9], tr[3];
    load_rel(L.rel + 12 * u, R, tr);
    if (!ff_stage(L, planes, L.g.planes + sp.f0, sp.nf, bar, phase, lane)) return;
    __syncwarp();
    if (kCount && lane == 0) { c_live += 1; c_feat += fp.nv + fp.ne; }
    // vertices: exact max-plane value (or a one-plane / voxel cull)
    const float4 pj = planes[pl];
    for (int i0 = 0; i0 < fp.nv; i0 += 32) {
      const int i = i0 + lane;
      bool scan = false;
      float3 x = make_float3(0.f, 0.f, 0.f);
      if (i < fp.nv) {
        x = xform(R, tr, L.g.verts[fp.v0 + i]);
        xs[i] = make_float4(x.x, x.y, x.z, 0.f);
        const float vj = fmaf(pj.x, x.x, fmaf(pj.y, x.y, fmaf(pj.z, x.z, pj.w)));
        const float b = voxel ? voxel_bound(L.g, s_glob, x.x, x.y, x.z) : -INFINITY;
        vb[i] = b;
        if (!no_cull && vj >= d_max) {
          m[i] = vj;
          am[i] = (uint16_t)pl;
          if (kCount) c_maxp += 1;
        } else if (b - kVoxTol >= d_max) {
          m[i] = vj;
          am[i] = (uint16_t)(pl | kVoxCulled);
          if (kCount) c_maxp += 1;
        } else {
          scan = true;
          if (kCount) c_maxp += sp.nf;
        }
      }
      // the exact maxima of the few vertices left, one at a time with the
      // planes over the lanes (the lowest index attaining the maximum, as a
      // serial scan would keep)
      unsigned todo = __ballot_sync(kFull, scan);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const float px = __shfl_sync(kFull, x.x, src), py = __shfl_sync(kFull, x.y, src),
                    pz = __shfl_sync(kFull, x.z, src);
        float best = -INFINITY;
        int barg = 0x7fffffff;
        for (int k = lane; k < sp.nf; k += 32) {
          const float4 p = planes[k];
          const float v = fmaf(p.x, px, fmaf(p.y, py, fmaf(p.z, pz, p.w)));
          if (v > best) { best = v; barg = k; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ov = __shfl_xor_sync(kFull, best, o);
          const int oa = __shfl_xor_sync(kFull, barg, o);
          if (ov > best || (ov == best && oa < barg)) { best = ov; barg = oa; }
        }
        if (lane == src) {
          m[i] = best;
          am[i] = (uint16_t)barg;
        }
      }
    }
    __syncwarp();
    // edges: the two-plane bound of the max-plane value along the edge (and
    // the voxel edge bound); survivors carry their corners' lower bounds
    for (int k0 = 0; k0 < fp.ne; k0 += 32) {
      const int k = k0 + lane;
      bool live = false;
      int4 rec = make_int4(0, 0, 0, 0);
      float2 mm = make_float2(0.f, 0.f);
      if (k < fp.ne) {
        const uint32_t e = L.g.edges[fp.e0 + k];
        const int i0 = e & 0xffff, i1 = e >> 16;
        const float4 a = xs[i0], b = xs[i1];
        const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
        const float lb = edge_plane_bound(planes[am[i0] & kPlaneMask], planes[am[i1] & kPlaneMask],
                                          dx, dy, dz, m[i0], m[i1]);
        // the max-plane value is 1-Lipschitz: along the edge it stays above
        // (b_I + b_II - L) / 2 for lower bounds b at the corners
        const float vlb = 0.5f * (vb[i0] + vb[i1] - sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))));
        live = no_cull || (lb - kEdgeTol < d_max && vlb - kVoxTol < d_max);
        rec = make_int4(row, s_glob, f_glob, (int)((1u << 31) | (uint32_t)k));
        mm = make_float2(m[i0], m[i1]);
      }
      ff_push(L, live, rec, mm, lane, true);
    }
    // vertices below d_max (not culled by a voxel)
    for (int i0 = 0; i0 < fp.nv; i0 += 32) {
      const int i = i0 + lane;
      const bool live = i < fp.nv && (no_cull || (m[i] < d_max && !(am[i] & kVoxCulled)));
      ff_push(L, live, make_int4(row, s_glob, f_glob, i), make_float2(i < fp.nv ? m[i] : 0.f, 0.f),
              lane, false);
    }
    __syncwarp();   // the next direction overwrites the slice
  }
  if (kCount && L.counters) {
    unsigned long long v[3] = {c_live, c_maxp, c_feat};
    const int idx[3] = {CCM_CNT_DIRS_LIVE, CCM_CNT_MAXPASS, CCM_CNT_FEATURES};
    for (int q = 0; q < 3; ++q) {
      unsigned long long x = v[q];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (lane == 0 && x) atomicAdd(L.counters + idx[q], x);
    }
  }
}

// ---------------------------------------------------------------------------
// eval: one candidate per thread
// ---------------------------------------------------------------------------
template <bool kCount>
__global__ void __launch_bounds__(128) ff_eval_kernel(FlatFwdLaunch L) {
  pdl_wait();
  if (L.ctl[kFfOverflow]) return;
  const int lane = threadIdx.x & 31;
  const KParams& kp = L.kp;
  const bool project = (kp.flags & CCM_FLAG_PROJECT) != 0u;
  // (an overflow stops this stage above; the clamps keep every index in range)
  const int64_t half = L.cand_cap / 2;
  const int64_t nv = min((int64_t)L.ctl[kFfCand], half);
  const int64_t n = nv + min((int64_t)L.ctl[kFfCandE], half);
  unsigned long long c_eg = 0, c_ev = 0, c_con = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = ff_cand_index(L, t, nv);
    const int4 rec = L.cand[k];
    const float2 mm = L.cand_m[k];
    const int row = rec.x;
    const int rp = L.row_pair[row];
    const int64_t u = rp;   // unit = 2 pair + side
    float R[9], tr[3];
    load_rel(L.rel + 12 * u, R, tr);
    const PieceRec fp = L.g.pieces[rec.z], sp = L.g.pieces[rec.y];
    const float4* planes = L.g.planes + sp.f0;
    const bool edge = ((uint32_t)rec.w >> 31) != 0u;
    const int feat = rec.w & 0xfff;
    float phi, gx, gy, gz, px, py, pz;
    if (!edge) {
      const float3 x = xform(R, tr, L.g.verts[fp.v0 + feat]);
      const SdfGrad sg = sdf_grad(planes, sp.nf, x.x, x.y, x.z, mm.x, kp);
      phi = sg.phi; gx = sg.gx; gy = sg.gy; gz = sg.gz;
      px = x.x; py = x.y; pz = x.z;
      if (kCount) c_eg += sp.nf;
    } else {
      const uint32_t e = L.g.edges[fp.e0 + feat];
      const float3 a = xform(R, tr, L.g.verts[fp.v0 + (e & 0xffff)]);
      const float3 b = xform(R, tr, L.g.verts[fp.v0 + (e >> 16)]);
      float phA, phB, mxA, mxB;
      sdf_val2(planes, sp.nf, a.x, a.y, a.z, mm.x, b.x, b.y, b.z, mm.y, kp, phA, mxA, phB, mxB);
      const EdgeContact ec = edge_contact(planes, sp.nf, make_float4(a.x, a.y, a.z, 0.f),
                                          make_float4(b.x, b.y, b.z, 0.f), mm.x, mm.y, phA, phB, kp);
      phi = ec.phi; gx = ec.gx; gy = ec.gy; gz = ec.gz;
      px = ec.px; py = ec.py; pz = ec.pz;
      if (kCount) {
        c_eg += sp.nf;
        c_ev += (unsigned long long)sp.nf * (2 + 2 * (kp.trace_iters > 0 ? kp.trace_iters - 1 : 0));
      }
    }
    const float w = transition(phi, kp);
    const float dc = fmaf(w, phi - kp.d_max, kp.d_max);   // f phi + (1 - f) d_max
    if (project) {                                          // Sec. 4.1 projection
      px = fmaf(-phi, gx, px);
      py = fmaf(-phi, gy, py);
      pz = fmaf(-phi, gz, pz);
    }
    float* o = L.cval + 8 * k;
    o[0] = w; o[1] = dc; o[2] = px; o[3] = py; o[4] = pz; o[5] = gx; o[6] = gy; o[7] = gz;
    if (w > 0.f) {
      atomicAdd(edge ? L.cl.cnt_e + row : L.cl.cnt_v + row, 1);
      if (L.saved) {   // the direction's hit bit (SDF pieces < 256)
        const PairRec pr = L.pairs[rp >> 1];
        const int sp0 = L.g.bodies[(rp & 1) == 0 ? pr.bodyB : pr.bodyA].p0;
        const int sl = rec.y - sp0;
        if (sl < kHitS)
          atomicOr(L.hits + (int64_t)kHitWords * row + (sl >> 5), 1u << (sl & 31));
      }
      if (kCount) c_con += 1;
    }
  }
  if (kCount && L.counters) {
    unsigned long long v[3] = {c_eg, c_ev, c_con};
    const int idx[3] = {CCM_CNT_EVAL_GRAD, CCM_CNT_EVAL_VAL, CCM_CNT_CONTACTS};
    for (int q = 0; q < 3; ++q) {
      unsigned long long x = v[q];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (lane == 0 && x) atomicAdd(L.counters + idx[q], x);
    }
  }
}

// ---------------------------------------------------------------------------
// scatter: contacts of non-zero weight to their group's segment
// ---------------------------------------------------------------------------
__global__ void ff_scatter_kernel(FlatFwdLaunch L) {
  pdl_wait();
  if (L.ctl[kFfOverflow]) return;
  const int64_t NV = (int64_t)L.cl.ctl[kCtlNV], NE = (int64_t)L.cl.ctl[kCtlNE];
  if (NV + NE > L.cl.cap) {          // the contact list cannot hold them
    if (blockIdx.x == 0 && threadIdx.x == 0) L.ctl[kFfOverflow] = 1ull;
    return;
  }
  // (an overflow stops this stage above; the clamps keep every index in range)
  const int64_t half = L.cand_cap / 2;
  const int64_t nv = min((int64_t)L.ctl[kFfCand], half);
  const int64_t n = nv + min((int64_t)L.ctl[kFfCandE], half);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = ff_cand_index(L, t, nv);
    const float* c = L.cval + 8 * k;
    if (!(c[0] > 0.f)) continue;
    const int4 rec = L.cand[k];
    const bool edge = ((uint32_t)rec.w >> 31) != 0u;
    const int row = rec.x;
    // the scan zeroed the counts, which now serve as cursors
    const int64_t pos = edge ? NV + L.cl.off_e[row] + atomicAdd(L.cl.cnt_e + row, 1)
                             : (int64_t)L.cl.off_v[row] + atomicAdd(L.cl.cnt_v + row, 1);
    L.cl.recs[pos].x = (int)k;          // the candidate, in arrival order
    L.sval_key[pos] = ff_key(rec);
  }
}

// ---------------------------------------------------------------------------
// rank: each contact to its place in its segment's (SDF piece, feature)
// order -- the keys are distinct within a segment -- with its values
// ---------------------------------------------------------------------------
constexpr int64_t kRankCap = 4096;   // longer segments: the per-item forward runs instead

__global__ void __launch_bounds__(256) ff_rank_kernel(FlatFwdLaunch L) {
  pdl_wait();
  if (L.ctl[kFfOverflow]) return;
  const int64_t NV = (int64_t)L.cl.ctl[kCtlNV], NE = (int64_t)L.cl.ctl[kCtlNE];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < NV + NE;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = L.cl.recs[j].x;
    const int4 rec = L.cand[k];
    const bool edge = j >= NV;
    const int row = rec.x;
    const int64_t a = edge ? NV + L.cl.off_e[row] : L.cl.off_v[row];
    const int64_t b = edge ? NV + L.cl.off_e[row + 1] : L.cl.off_v[row + 1];
    if (b - a > kRankCap) {
      L.ctl[kFfOverflow] = 1ull;
      continue;
    }
    const long long key = L.sval_key[j];
    int64_t r = 0;
    for (int64_t i = a; i < b; ++i) r += L.sval_key[i] < key;
    L.cl.sorted[a + r] = rec;
    const float4* c = reinterpret_cast<const float4*>(L.cval + 8 * k);
    float4* o = reinterpret_cast<float4*>(L.sval + 8 * (a + r));
    o[0] = c[0];
    o[1] = c[1];
  }
  // every group's outputs and record as if it had no contact (the fold
  // then rewrites the groups that have some), 32 groups per warp staged in
  // shared memory and written as contiguous float4 rows
  __shared__ __align__(16) float y_s[8][32 * 8];
  __shared__ __align__(16) float r_s[8][32 * kSavedFloats];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 32; g0 < L.G;
       g0 += warps * 32) {
    const int64_t g = g0 + lane;
    const int n_here = (int)(L.G - g0 < 32 ? L.G - g0 : 32);
    if (g < L.G) {
      write_empty(y_s[warp] + 8 * lane, L.kp);
      if (L.saved) {
        PartT<float> z;
        part_zero(z);
        float* o = r_s[warp] + kSavedFloats * lane;
        o[0] = z.M;
        for (int q = 1; q < 18; ++q) o[q] = 0.f;
        const uint4* hs = reinterpret_cast<const uint4*>(L.hits + (int64_t)kHitWords * g);
        uint32_t* h = reinterpret_cast<uint32_t*>(o + 18);
#pragma unroll
        for (int q = 0; q < kHitWords / 4; ++q) {
          const uint4 w = hs[q];
          h[4 * q] = w.x; h[4 * q + 1] = w.y; h[4 * q + 2] = w.z; h[4 * q + 3] = w.w;
        }
        h[kHitWords] = L.cl.tag;
        h[kHitWords + 1] = 0u;
      }
    }
    __syncwarp();
    {
      const float4* src = reinterpret_cast<const float4*>(y_s[warp]);
      float4* dst = reinterpret_cast<float4*>(L.y + 8 * g0);
      for (int i = lane; i < 2 * n_here; i += 32) dst[i] = src[i];
    }
    if (L.saved) {
      const float4* src = reinterpret_cast<const float4*>(r_s[warp]);
      float4* dst = reinterpret_cast<float4*>(L.saved + (int64_t)kSavedFloats * g0);
      for (int i = lane; i < (kSavedFloats / 4) * n_here; i += 32) dst[i] = src[i];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// fold: one group with contacts (the list of such groups from the scan) per
// four lanes, its vertex contacts then its edge contacts in list order split
// over the lanes (fold_split) -- the order and arithmetic of the per-contact
// reverse passes' own fold (ccm_flat.cu) over the same list
// ---------------------------------------------------------------------------
constexpr int kFoldSplit = 4;   // lanes per group in the fold

__global__ void __launch_bounds__(128) ff_fold_kernel(FlatFwdLaunch L) {
  pdl_wait();
  if (L.ctl[kFfOverflow]) return;
  const int64_t NV = (int64_t)L.cl.ctl[kCtlNV], NG = (int64_t)L.cl.ctl[kCtlNG];
  const int sub = threadIdx.x & (kFoldSplit - 1);
  const int64_t per_block = blockDim.x / kFoldSplit;
  // block-uniform loop: every lane takes part in the fold's shuffles
  for (int64_t base = (int64_t)blockIdx.x * per_block; base < NG;
       base += (int64_t)gridDim.x * per_block) {
    const int64_t i = base + threadIdx.x / kFoldSplit;
    const bool valid = i < NG;
    const int64_t g = valid ? L.cl.live_g[i] : 0;
    int64_t v0 = 0, v1 = 0, e0 = 0, e1 = 0;
    float RS[9], tS[3];
    if (valid) {
      v0 = L.cl.off_v[g]; v1 = L.cl.off_v[g + 1];
      e0 = NV + L.cl.off_e[g]; e1 = NV + L.cl.off_e[g + 1];
      if (sub == 0) {   // the pose's loads overlap the fold
        const int rp = L.row_pair[g];
        load_pose(((rp & 1) == 0 ? L.pose_b : L.pose_a) + 12 * (int64_t)(rp >> 1), RS, tS);
      }
    }
    PartT<float> A;
    fold_split<float, kFoldSplit>(L.sval, v0, v1, e0, e1, L.kp.c_blend, sub, A);
    if (valid && sub == 0) {
      float yo[8];
      write_group(yo, A, RS, tS, L.kp);
      float4* yd = reinterpret_cast<float4*>(L.y + 8 * g);
      yd[0] = make_float4(yo[0], yo[1], yo[2], yo[3]);
      yd[1] = make_float4(yo[4], yo[5], yo[6], yo[7]);
      if (L.saved) {   // the partial (hit words and tag are in place)
        float* o = L.saved + (int64_t)kSavedFloats * g;
        o[0] = A.M; o[1] = A.U; o[2] = A.rd; o[3] = A.rf;
        o[4] = A.rp.x; o[5] = A.rp.y; o[6] = A.rp.z;
        o[7] = A.rn.x; o[8] = A.rn.y; o[9] = A.rn.z;
        o[10] = A.Dd; o[11] = A.Da;
        o[12] = A.Dp.x; o[13] = A.Dp.y; o[14] = A.Dp.z;
        o[15] = A.Dn.x; o[16] = A.Dn.y; o[17] = A.Dn.z;
      }
    }
  }
}

// ---------------------------------------------------------------------------
cudaError_t launch_flat_forward(const FlatFwdLaunch& L, cudaStream_t stream) {
  cudaError_t e;
  const bool pdl = L.pdl != 0;
  const int sb = (int)std::max<int64_t>(1, std::min<int64_t>((std::max(L.G, 2 * L.n_pairs) + 255) / 256,
                                                             8 * L.n_sm));
  if ((e = launch_k(pdl, ff_setup_kernel, sb, 256, 0, stream, L)) != cudaSuccess) return e;
  const int gw = L.gate_planes > 0
                     ? std::max(1, std::min(kGateWarps, kDynSmem / (16 * L.gate_planes)))
                     : kGateWarps;
  const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((2 * L.n_pairs + gw - 1) / gw,
                                                             32 * L.n_sm));
  const size_t gsm = (size_t)gw * 16 * L.gate_planes;
  e = launch_k(pdl, L.counters ? ff_gate_kernel<true> : ff_gate_kernel<false>, gb, 32 * gw, gsm,
               stream, L);
  if (e != cudaSuccess) return e;
  int wpb = 1;
  const size_t smem = flat_forward_feature_smem(L.vmax, L.fmax, &wpb);
  // persistent: the blocks that stay resident (64 registers: 8 blocks of 4 warps per SM)
  const int fb = std::max(1, (8 * 4 / wpb)) * L.n_sm;
  e = launch_k(pdl, L.counters ? ff_feature_kernel<true> : ff_feature_kernel<false>, fb, 32 * wpb,
               smem, stream, L);
  if (e != cudaSuccess) return e;
  const int eb = 32 * L.n_sm;
  e = launch_k(pdl, L.counters ? ff_eval_kernel<true> : ff_eval_kernel<false>, eb, 128, 0, stream,
               L);
  if (e != cudaSuccess) return e;
  if ((e = launch_flat_prep_scan(L.cl, L.G, stream, pdl)) != cudaSuccess) return e;
  if ((e = launch_k(pdl, ff_scatter_kernel, 8 * L.n_sm, 256, 0, stream, L)) != cudaSuccess) return e;
  if ((e = launch_k(pdl, ff_rank_kernel, 8 * L.n_sm, 256, 0, stream, L)) != cudaSuccess) return e;
  // groups with contacts: at most G, kFoldSplit lanes each
  const int fo = (int)std::max<int64_t>(
      1, std::min<int64_t>((kFoldSplit * L.G + 127) / 128, 16 * L.n_sm));
  return launch_k(pdl, ff_fold_kernel, fo, 128, 0, stream, L);
}

}  // namespace ccm
