// Forward variant with a body-level SDF: the smooth union of the SDFs of the
// other body's convex pieces (Sec. 3.1, Eq. soft_union),
//   phi_S(x) = -tau log sum_s exp(-phi_s(x) / tau),
// each phi_s the smooth intersection of piece s's half-spaces (Sec. 3), with
// the same softness tau = tau_sdf.  Every vertex and edge of a group's convex
// piece gives one contact against the whole body (Sec. 4.2: V-SDF, and E-SDF
// by sphere tracing), mollified (Sec. 4.3) and blended per group (Sec. 4.4).
// With CCM_FLAG_PROJECT every contact point is moved onto the isosurface,
// p - phi(p) grad phi(p) (Sec. 4.1), after its depth and normal were taken.
//
// One warp per output group; lanes run over the group's features, 32 at a
// time, and fold their contacts in feature order (deterministic).  Culls are
// exact: phi_S >= min_s maxplane_s - tau log N_S (the union lies at most
// tau log N below its smallest term, and every piece SDF lies above its
// largest plane value), so a vertex whose bound is >= d_max has f = 0, and
// phi_S is 1-Lipschitz (its gradient is a convex mix of unit-bounded ones),
// so an edge whose corners satisfy (phi_a + phi_b - L) / 2 >= d_max has no
// point below d_max.
#include <algorithm>

#include "ccm_narrow.cuh"
#include "ccm_union.h"
#include "ccm_launch.h"

namespace ccm {

// phi_S and (if grad) grad phi_S at x: online softmin over the pieces, each
// piece's LSE shifted by its exact largest plane value
template <bool kGrad>
__device__ float union_sdf(const DevGeom& g, const BodyRec& S, float x, float y, float z,
                           const KParams& kp, float* grad) {
  float M = INFINITY, Z = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  for (int s = 0; s < S.np; ++s) {
    const PieceRec p = g.pieces[S.p0 + s];
    const float4* pl = g.planes + p.f0;
    const float m = max_plane(pl, p.nf, x, y, z);
    const SdfGrad r = sdf_grad(pl, p.nf, x, y, z, m, kp);
    float w;
    if (r.phi < M) {           // new smallest term: rescale the sums to it
      const float sc = ex2((r.phi - M) * kp.c_sdf);   // e^{-(M - phi)/tau}, 0 when M = inf
      Z *= sc;
      gx *= sc;
      gy *= sc;
      gz *= sc;
      M = r.phi;
      w = 1.f;
    } else {
      w = ex2((M - r.phi) * kp.c_sdf);
    }
    Z += w;
    if (kGrad) {
      gx = fmaf(w, r.gx, gx);
      gy = fmaf(w, r.gy, gy);
      gz = fmaf(w, r.gz, gz);
    }
  }
  if (kGrad) {
    const float iz = __frcp_rn(Z);
    grad[0] = gx * iz;
    grad[1] = gy * iz;
    grad[2] = gz * iz;
  }
  return M - kp.ic_sdf * __log2f(Z);
}

// exact lower bound of phi_S at x: min_s maxplane_s(x) - tau log N_S
__device__ float union_lower_bound(const DevGeom& g, const BodyRec& S, float x, float y, float z,
                                   const KParams& kp) {
  float lo = INFINITY;
  for (int s = 0; s < S.np; ++s) {
    const PieceRec p = g.pieces[S.p0 + s];
    lo = fminf(lo, max_plane(g.planes + p.f0, p.nf, x, y, z));
  }
  return lo - kp.tau_sdf * logf((float)S.np);
}

__global__ void __launch_bounds__(128)
union_fwd_kernel(DevGeom g, const PairRec* __restrict__ pairs, const int32_t* __restrict__ row_pair,
                 int64_t G, const float* __restrict__ pose_a, const float* __restrict__ pose_b,
                 KParams kp, float* __restrict__ y) {
  __shared__ PartT<float> acc_s[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  PartT<float>* acc = acc_s + warp;
  const bool project = (kp.flags & CCM_FLAG_PROJECT) != 0u;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; row < G; row += nwarps) {
    const int rp = row_pair[row];
    const int64_t pi = rp >> 1;
    const int side = rp & 1;
    const PairRec pr = pairs[pi];
    const BodyRec bA = g.bodies[pr.bodyA], bB = g.bodies[pr.bodyB];
    const BodyRec F = side == 0 ? bA : bB, S = side == 0 ? bB : bA;
    const int fc = (int)(row - pr.goff - (side == 0 ? 0 : bA.np));
    const PieceRec fp = g.pieces[F.p0 + fc];
    const float* pF = (side == 0 ? pose_a : pose_b) + 12 * pi;
    const float* pS = (side == 0 ? pose_b : pose_a) + 12 * pi;
    float Rr[9], tr[3];
    rel_pose_f64(pF, pS, lane, Rr, tr);
    if (lane == 0) part_zero(*acc);
    __syncwarp();
    const int nfeat = fp.nv + fp.ne;
    for (int k0 = 0; k0 < nfeat; k0 += 32) {
      const int k = k0 + lane;
      PartT<float> c;
      part_zero(c);
      if (k < nfeat) {
        float phi, gr[3], px, py, pz;
        bool live;
        if (k < fp.nv) {            // V-SDF: the vertex is the contact point
          const float3 x = xform(Rr, tr, g.verts[fp.v0 + k]);
          px = x.x; py = x.y; pz = x.z;
          live = union_lower_bound(g, S, px, py, pz, kp) - 1e-5f < kp.d_max;
          if (live) phi = union_sdf<true>(g, S, px, py, pz, kp, gr);
        } else {                    // E-SDF: sphere trace from both corners
          const uint32_t e = g.edges[fp.e0 + (k - fp.nv)];
          const float3 a = xform(Rr, tr, g.verts[fp.v0 + (e & 0xffff)]);
          const float3 b = xform(Rr, tr, g.verts[fp.v0 + (e >> 16)]);
          float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
          const float L = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
          const float iL = 1.0f / L;
          ex *= iL; ey *= iL; ez *= iL;
          float phI = union_sdf<false>(g, S, a.x, a.y, a.z, kp, nullptr);
          float phII = union_sdf<false>(g, S, b.x, b.y, b.z, kp, nullptr);
          live = 0.5f * (phI + phII - L) - 1e-5f < kp.d_max;
          if (live) {
            float aI = 0.f, aII = L;
            for (int s = 0; s < kp.trace_iters; ++s) {
              aI += sigmoid_c(phI, kp.c_trace) * phI;
              aII -= sigmoid_c(phII, kp.c_trace) * phII;
              if (s + 1 == kp.trace_iters) break;
              phI = union_sdf<false>(g, S, fmaf(aI, ex, a.x), fmaf(aI, ey, a.y),
                                     fmaf(aI, ez, a.z), kp, nullptr);
              phII = union_sdf<false>(g, S, fmaf(aII, ex, a.x), fmaf(aII, ey, a.y),
                                      fmaf(aII, ez, a.z), kp, nullptr);
            }
            const float am = 0.5f * (softclip0(aI, L, kp.tau_clip, kp.c_clip) +
                                     softclip0(aII, L, kp.tau_clip, kp.c_clip));
            px = fmaf(am, ex, a.x);
            py = fmaf(am, ey, a.y);
            pz = fmaf(am, ez, a.z);
            phi = union_sdf<true>(g, S, px, py, pz, kp, gr);
          }
        }
        if (live) {
          const float w = transition(phi, kp);
          const float dc = fmaf(w, phi - kp.d_max, kp.d_max);   // f phi + (1 - f) d_max
          if (project) {
            px = fmaf(-phi, gr[0], px);
            py = fmaf(-phi, gr[1], py);
            pz = fmaf(-phi, gr[2], pz);
          }
          part_from_contact(c, w, dc, v3(px, py, pz), v3(gr[0], gr[1], gr[2]), kp.c_blend);
        }
      }
      fold_t(c, 0, acc, lane);
      __syncwarp();
    }
    if (lane == 0) {
      float RS[9], tS[3];
      load_pose(pS, RS, tS);
      write_group(y + 8 * row, *acc, RS, tS, kp);
    }
    __syncwarp();
  }
}

cudaError_t launch_union_forward(const UnionLaunch& L, cudaStream_t stream) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((L.G + 3) / 4, 64 * L.n_sm));
  union_fwd_kernel<<<(int)blocks, 128, 0, stream>>>(L.g, L.pairs, L.row_pair, L.G, L.pose_a,
                                                     L.pose_b, L.kp, L.y);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ccm
