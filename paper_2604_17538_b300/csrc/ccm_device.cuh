// Device-side data layout and math shared by the contact kernels.
//
// Geometry is resident structure-of-arrays: one float4 per vertex (x, y, z, 0),
// one float4 per face plane (n_x, n_y, n_z, h) -- the half-space SDF
// phi_k(x) = n_k . x + h_k of Sec. 3 -- and one packed uint32 per edge
// (i | j << 16, piece-local vertex indices).  Piece and body records index
// into those arrays.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ccm {

struct __align__(16) PieceRec {
  int32_t v0, nv, f0, nf;   // first vertex / count, first plane / count
  int32_t e0, ne, body, pad;
  float4 sphere;            // bounding sphere centre (body frame) and radius
};

struct BodyRec {
  int32_t p0, np;           // first piece, piece count
};

struct PairRec {
  int32_t bodyA, bodyB;
  int64_t goff;
};

// One warp's task: the feature pieces [fc0, fc1) of body F of unit
// `unit` = 2 pair + side (side 0: F = A, S = B) against every piece of S.  A
// unit is split into items of at most UnitShape::groups pieces so that large
// bodies spread over many warps; items never share an output group.
struct WorkItem {
  int32_t unit;
  uint16_t fc0, fc1;
};

// Voxel grid of a piece for the broad phase (Sec. 4.3): origin and voxel
// size, voxel counts and the offset of its values; every value is a lower
// bound of the piece's SDF anywhere in that voxel (the largest plane value at
// the voxel's centre minus the voxel's circumradius).  dims.x = 0: no grid.
struct VoxelRec {
  float4 grid;
  int4 dims;
};

struct DevGeom {
  const PieceRec* __restrict__ pieces;
  const BodyRec* __restrict__ bodies;
  const float4* __restrict__ verts;
  const float4* __restrict__ planes;
  const uint32_t* __restrict__ edges;
  const VoxelRec* __restrict__ voxels = nullptr;    // [n_voxels] or NULL
  const float* __restrict__ voxel_vals = nullptr;
  int32_t n_voxels = 0;                             // pieces with a record
};

// the voxel grid's lower bound of piece p's SDF at x (piece / body frame),
// -inf outside its grid or without one
__device__ __forceinline__ float voxel_bound(const DevGeom& g, int p, float x, float y,
                                             float z) {
  if (!g.voxels || p >= g.n_voxels) return -INFINITY;
  const VoxelRec v = g.voxels[p];
  if (v.dims.x == 0) return -INFINITY;
  const float ih = 1.0f / v.grid.w;
  const float tx = (x - v.grid.x) * ih, ty = (y - v.grid.y) * ih, tz = (z - v.grid.z) * ih;
  if (!(tx >= 0.f && ty >= 0.f && tz >= 0.f && tx < (float)v.dims.x && ty < (float)v.dims.y &&
        tz < (float)v.dims.z))
    return -INFINITY;
  const int ix = (int)tx, iy = (int)ty, iz = (int)tz;
  return __ldg(g.voxel_vals + v.dims.w + (ix * v.dims.y + iy) * v.dims.z + iz);
}

// Tricubic spline SDF of a piece (Sec. 3.2): grid origin and voxel size, and
// the voxel counts with the first of its (nx+3)(ny+3)(nz+3) coefficient rows
// (float4: SDF, normal x, y, z); nx = 0 for a piece without one.
struct SplineRec {
  float4 grid;
  int4 dims;
};

// Method constants with the derived factors the kernels use.
struct KParams {
  float tau_sdf, tau_trace, tau_clip, tau_blend, d_max, gate_width;
  int32_t trace_iters;
  uint32_t flags;
  float c_sdf;      // log2(e) / tau_sdf
  float ic_sdf;     // tau_sdf * ln(2) = 1 / c_sdf
  float c_trace;    // log2(e) / tau_trace
  float c_clip;     // log2(e) / tau_clip
  float c_blend;    // log2(e) / tau_blend
  float inv_gate;   // 1 / gate_width
};

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr unsigned kFull = 0xffffffffu;

// Next work unit of a warp: a shared counter (zeroed before the launch) hands
// out units in order, so warps that drew light units take more of them and
// the heaviest-first order finishes together; without a counter the units are
// dealt round-robin from `first` in steps of `stride`.
__device__ __forceinline__ int64_t next_unit(int* sched, int64_t prev, int64_t stride) {
  if (!sched) return prev + stride;
  int v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(sched, 1);
  return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ int64_t first_unit(int* sched, int64_t first) {
  if (!sched) return first;
  int v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(sched, 1);
  return __shfl_sync(0xffffffffu, v, 0);
}

// 2^x on the SFU (hand-written PTX; flushes denormal results to zero).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Sec. 2 smooth operators on the device
// ---------------------------------------------------------------------------
// sigmoid(x / tau) with c = log2(e) / tau
__device__ __forceinline__ float sigmoid_c(float x, float c) {
  return __frcp_rn(1.0f + ex2(-x * c));
}
// softplus s+(x) = tau log(1 + e^{x/tau}) = max(x, 0) + tau log1p(e^{-|x|/tau})
__device__ __forceinline__ float softplus_c(float x, float tau, float c) {
  return fmaxf(x, 0.0f) + tau * log1pf(ex2(-fabsf(x) * c));
}
// softclip(x, 0, L) = s+(x) - s+(x - L)
__device__ __forceinline__ float softclip0(float x, float L, float tau, float c) {
  return softplus_c(x, tau, c) - softplus_c(x - L, tau, c);
}
// Sec. 4.3 transition: quintic smoothstep of s = (d_max - d) / eps on [0, 1]
__device__ __forceinline__ float transition(float d, const KParams& kp) {
  float s = __saturatef((kp.d_max - d) * kp.inv_gate);
  return s * s * s * fmaf(s, fmaf(s, 6.0f, -15.0f), 10.0f);
}

// ---------------------------------------------------------------------------
// Sec. 3 piece SDF: phi = LSE_tau(n_k . x + h_k), evaluated in one pass over
// the planes with a shift `s` that is a lower bound of the largest plane
// value (so the largest term is >= 1 and nothing underflows to an empty
// sum).  The exact largest value is tracked; if the bound was loose enough to
// risk overflow, the pass is repeated with the exact maximum.
// ---------------------------------------------------------------------------
struct SdfGrad {
  float phi, gx, gy, gz, mx;
};

__device__ __forceinline__ SdfGrad sdf_grad(const float4* __restrict__ pl, int nf, float x, float y,
                                            float z, float s, const KParams& kp) {
  SdfGrad r;
  for (int pass = 0; pass < 2; ++pass) {
    const float sc = s * kp.c_sdf;
    float S = 0.f, gx = 0.f, gy = 0.f, gz = 0.f, mx = -INFINITY;
#pragma unroll 4
    for (int k = 0; k < nf; ++k) {
      const float4 p = pl[k];
      const float v = fmaf(p.x, x, fmaf(p.y, y, fmaf(p.z, z, p.w)));
      mx = fmaxf(mx, v);
      const float e = ex2(fmaf(v, kp.c_sdf, -sc));
      S += e;
      gx = fmaf(e, p.x, gx);
      gy = fmaf(e, p.y, gy);
      gz = fmaf(e, p.z, gz);
    }
    if (pass == 0 && (mx - s) * kp.c_sdf > 64.0f) { s = mx; continue; }
    const float inv = __frcp_rn(S);
    r.phi = fmaf(kp.ic_sdf, __log2f(S), s);
    r.gx = gx * inv;
    r.gy = gy * inv;
    r.gz = gz * inv;
    r.mx = mx;
    break;
  }
  return r;
}

// value-only SDF at two points at once (the two sphere-trace chains of an edge)
__device__ __forceinline__ void sdf_val2(const float4* __restrict__ pl, int nf, float x1, float y1,
                                         float z1, float s1, float x2, float y2, float z2, float s2,
                                         const KParams& kp, float& phi1, float& mx1, float& phi2,
                                         float& mx2) {
  for (int pass = 0; pass < 2; ++pass) {
    const float sc1 = s1 * kp.c_sdf, sc2 = s2 * kp.c_sdf;
    float S1 = 0.f, S2 = 0.f, m1 = -INFINITY, m2 = -INFINITY;
#pragma unroll 4
    for (int k = 0; k < nf; ++k) {
      const float4 p = pl[k];
      const float v1 = fmaf(p.x, x1, fmaf(p.y, y1, fmaf(p.z, z1, p.w)));
      const float v2 = fmaf(p.x, x2, fmaf(p.y, y2, fmaf(p.z, z2, p.w)));
      m1 = fmaxf(m1, v1);
      m2 = fmaxf(m2, v2);
      S1 += ex2(fmaf(v1, kp.c_sdf, -sc1));
      S2 += ex2(fmaf(v2, kp.c_sdf, -sc2));
    }
    const bool bad1 = (m1 - s1) * kp.c_sdf > 64.0f, bad2 = (m2 - s2) * kp.c_sdf > 64.0f;
    if (pass == 0 && (bad1 || bad2)) {
      if (bad1) s1 = m1;
      if (bad2) s2 = m2;
      continue;
    }
    phi1 = fmaf(kp.ic_sdf, __log2f(S1), s1);
    phi2 = fmaf(kp.ic_sdf, __log2f(S2), s2);
    mx1 = m1;
    mx2 = m2;
    break;
  }
}

// exact largest plane value at x (the hard polytope "depth" max_k phi_k)
__device__ __forceinline__ float max_plane(const float4* __restrict__ pl, int nf, float x, float y,
                                           float z) {
  // two running maxima (even / odd planes) halve the dependency chain
  float m0 = -INFINITY, m1 = -INFINITY;
  int k = 0;
#pragma unroll 2
  for (; k + 1 < nf; k += 2) {
    const float4 p = pl[k], q = pl[k + 1];
    m0 = fmaxf(m0, fmaf(p.x, x, fmaf(p.y, y, fmaf(p.z, z, p.w))));
    m1 = fmaxf(m1, fmaf(q.x, x, fmaf(q.y, y, fmaf(q.z, z, q.w))));
  }
  if (k < nf) {
    const float4 p = pl[k];
    m0 = fmaxf(m0, fmaf(p.x, x, fmaf(p.y, y, fmaf(p.z, z, p.w))));
  }
  return fmaxf(m0, m1);
}

// largest plane value at x and the lowest index of a plane attaining it
__device__ __forceinline__ float max_plane_arg(const float4* __restrict__ pl, int nf, float x,
                                               float y, float z, int& arg) {
  float m0 = -INFINITY, m1 = -INFINITY;
  int a0 = 0, a1 = 1;
  int k = 0;
#pragma unroll 2
  for (; k + 1 < nf; k += 2) {
    const float4 p = pl[k], q = pl[k + 1];
    const float v0 = fmaf(p.x, x, fmaf(p.y, y, fmaf(p.z, z, p.w)));
    const float v1 = fmaf(q.x, x, fmaf(q.y, y, fmaf(q.z, z, q.w)));
    if (v0 > m0) { m0 = v0; a0 = k; }
    if (v1 > m1) { m1 = v1; a1 = k + 1; }
  }
  if (k < nf) {
    const float4 p = pl[k];
    const float v0 = fmaf(p.x, x, fmaf(p.y, y, fmaf(p.z, z, p.w)));
    if (v0 > m0) { m0 = v0; a0 = k; }
  }
  const bool second = m1 > m0 || (m1 == m0 && a1 < a0);
  arg = second ? a1 : a0;
  return second ? m1 : m0;
}

// ---------------------------------------------------------------------------
// Bulk (TMA) copies from global to shared memory, completed on an mbarrier
// (hand-written PTX).  Both addresses 16-byte aligned, size a multiple of 16;
// no multicast.  Waits are bounded by an iteration count.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier generic accesses to shared memory before
// later async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// One poll: returns when the phase completes or after a suspend of at most
// kPollHintNs (the hint keeps a waiting warp from spinning through issue
// slots while a copy is in flight).
constexpr uint32_t kPollHintNs = 1000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kPollHintNs)
      : "memory");
  return ok != 0u;
}
// Waits for the mbarrier phase `parity` at most `limit` times; returns false
// if it did not complete.  The caller then drains with a much larger bound so
// that no copy is left in flight into shared memory it gives up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit) {
  for (long long it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
constexpr long long kDrainLimit = 1ll << 24;

// Waits, in a kernel launched with programmatic dependent launch, until the
// previous kernel of the stream has completed and its writes are visible
// (ccm_launch.h); returns at once in a kernel launched without it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Copies n elements from global to shared memory, four loads in flight per
// lane (the staging of a work item's geometry is latency-bound otherwise).
template <class U>
__device__ __forceinline__ void stage_copy(U* __restrict__ dst, const U* __restrict__ src, int n,
                                           int lane) {
  int k = lane;
  for (; k + 96 < n; k += 128) {
    const U a = __ldg(src + k), b = __ldg(src + k + 32), c = __ldg(src + k + 64),
            d = __ldg(src + k + 96);
    dst[k] = a;
    dst[k + 32] = b;
    dst[k + 64] = c;
    dst[k + 96] = d;
  }
  for (; k < n; k += 32) dst[k] = __ldg(src + k);
}

// Lower bound of the max-plane value over the edge x(t) = xI + t (xII - xI),
// t in [0, 1], from the planes a and b that attain it at the two corners
// (values mI and mII): max_k phi_k(x(t)) >= max(phi_a(x(t)), phi_b(x(t))),
// two linear functions whose maximum is convex in t, so its minimum is at a
// corner or where they cross.  Every unit-normal plane changes by at most the
// edge length L along it, so the bound is never below (mI + mII - L) / 2.
__device__ __forceinline__ float edge_plane_bound(float4 pa, float4 pb, float dx, float dy,
                                                  float dz, float mI, float mII) {
  const float A0 = mI, A1 = fmaf(pa.x, dx, fmaf(pa.y, dy, fmaf(pa.z, dz, mI)));
  const float B1 = mII, B0 = mII - fmaf(pb.x, dx, fmaf(pb.y, dy, pb.z * dz));
  float lb = fminf(fmaxf(A0, B0), fmaxf(A1, B1));
  const float g0 = A0 - B0, g1 = A1 - B1;
  if ((g0 < 0.f) != (g1 < 0.f)) {   // the lines cross inside the edge
    const float t = g0 / (g0 - g1);
    lb = fminf(lb, fmaf(t, A1 - A0, A0));
  }
  return lb;
}

__device__ __forceinline__ void write_empty(float* out, const KParams& kp) {
  out[0] = kp.d_max;
#pragma unroll
  for (int k = 1; k < 8; ++k) out[k] = 0.f;
}

__device__ __forceinline__ void load_pose(const float* __restrict__ p, float R[9], float t[3]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = __ldg(p + i);
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i] = __ldg(p + 9 + i);
}

// relative pose mapping feature-body coordinates into the SDF body frame:
// Rr = R_S^T R_F, tr = R_S^T (t_F - t_S)
__device__ __forceinline__ void relative_pose(const float RS[9], const float tS[3], const float RF[9],
                                              const float tF[3], float Rr[9], float tr[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Rr[3 * i + j] = RS[i] * RF[j] + RS[3 + i] * RF[3 + j] + RS[6 + i] * RF[6 + j];
  }
  const float d0 = tF[0] - tS[0], d1 = tF[1] - tS[1], d2 = tF[2] - tS[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) tr[i] = RS[i] * d0 + RS[3 + i] * d1 + RS[6 + i] * d2;
}

// relative pose S <- F in double precision, computed by lanes 0..11 and
// broadcast: Rr = R_S^T R_F, tr = R_S^T (t_F - t_S)
__device__ __forceinline__ void rel_pose_f64(const float* pF, const float* pS, int lane,
                                             float Rr[9], float tr[3]) {
  float v = 0.f;
  if (lane < 9) {
    const int i = lane / 3, j = lane % 3;
    double acc = 0.0;
    for (int k = 0; k < 3; ++k) acc += (double)__ldg(pS + 3 * k + i) * (double)__ldg(pF + 3 * k + j);
    v = (float)acc;
  } else if (lane < 12) {
    const int i = lane - 9;
    double acc = 0.0;
    for (int k = 0; k < 3; ++k)
      acc += (double)__ldg(pS + 3 * k + i) * ((double)__ldg(pF + 9 + k) - (double)__ldg(pS + 9 + k));
    v = (float)acc;
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) Rr[q] = __shfl_sync(kFull, v, q);
#pragma unroll
  for (int q = 0; q < 3; ++q) tr[q] = __shfl_sync(kFull, v, 9 + q);
}

__device__ __forceinline__ float3 xform(const float R[9], const float t[3], float4 v) {
  return make_float3(fmaf(R[0], v.x, fmaf(R[1], v.y, fmaf(R[2], v.z, t[0]))),
                     fmaf(R[3], v.x, fmaf(R[4], v.y, fmaf(R[5], v.z, t[1]))),
                     fmaf(R[6], v.x, fmaf(R[7], v.y, fmaf(R[8], v.z, t[2]))));
}

}  // namespace ccm
