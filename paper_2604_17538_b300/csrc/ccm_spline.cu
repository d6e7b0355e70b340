// Forward variant with tricubic spline SDFs (Sec. 3.2): every convex piece of
// the other body is represented by a cubic spline on its own voxel grid,
//   s(x) = sum_{kx,ky,kz} c_k u(tx - kx + 1) u(ty - ky + 1) u(tz - kz + 1),
// t = (x - origin) / h, with the paper's basis u (4 - 6|t|^2 + 3|t|^3 on
// |t| <= 1, (2 - |t|)^3 on 1 <= |t| <= 2, 0 beyond), so 64 coefficients reach
// any point.  The SDF and the three components of the contact normal are four
// such splines sharing the grid (one float4 per coefficient); the normal is
// the normal spline, not the SDF's gradient.  Outside the grid box the SDF is
// the spline at the nearest box point plus the distance to the box.
//
// Contacts are those of Sec. 4.2 (every vertex; every edge sphere traced from
// both corners, soft clipped, midpoint), mollified (Sec. 4.3) and blended per
// group (Sec. 4.4); with CCM_FLAG_PROJECT each contact point moves to
// p - phi(p) n(p) (Sec. 4.1).  One warp per output group; lanes run over the
// (SDF piece, feature) pairs in order, 32 at a time, and fold their contacts
// in that order (deterministic).  No culls: a spline carries no bound.
#include <algorithm>

#include "ccm_narrow.cuh"
#include "ccm_spline.h"
#include "ccm_launch.h"

namespace ccm {

// the four weights u(r + 1), u(r), u(r - 1), u(r - 2) of r in [0, 1]
__device__ __forceinline__ void spline_weights(float r, float w[4]) {
  const float q = 1.0f - r;
  w[0] = q * q * q;
  w[1] = fmaf(r * r, fmaf(3.0f, r, -6.0f), 4.0f);
  w[2] = fmaf(q * q, fmaf(3.0f, q, -6.0f), 4.0f);
  w[3] = r * r * r;
}

// SDF (and, with kNormal, the normal splines) of one piece's spline at x
template <bool kNormal>
__device__ float spline_sdf(const SplineRec& sp, const float4* __restrict__ coef, float x,
                            float y, float z, float* normal) {
  const float h = sp.grid.w, ih = 1.0f / h;
  const float xs[3] = {x, y, z}, org[3] = {sp.grid.x, sp.grid.y, sp.grid.z};
  const int dims[3] = {sp.dims.x, sp.dims.y, sp.dims.z};
  float out2 = 0.f, w[3][4];
  int i0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float t = (xs[a] - org[a]) * ih;
    const float hi = (float)dims[a];
    if (t < 0.f) { out2 = fmaf(t, t, out2); t = 0.f; }
    else if (t > hi) { out2 = fmaf(t - hi, t - hi, out2); t = hi; }
    const int i = min(max((int)floorf(t), 0), dims[a] - 1);
    i0[a] = i;
    spline_weights(t - (float)i, w[a]);
  }
  const int ny = dims[1] + 3, nz = dims[2] + 3;
  float s = 0.f, nx = 0.f, nyv = 0.f, nzv = 0.f;
  for (int a = 0; a < 4; ++a) {
    for (int b = 0; b < 4; ++b) {
      const float wab = w[0][a] * w[1][b];
      const float4* c = coef + sp.dims.w + ((i0[0] + a) * ny + (i0[1] + b)) * nz + i0[2];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 v = __ldg(c + k);
        const float wk = wab * w[2][k];
        s = fmaf(wk, v.x, s);
        if (kNormal) {
          nx = fmaf(wk, v.y, nx);
          nyv = fmaf(wk, v.z, nyv);
          nzv = fmaf(wk, v.w, nzv);
        }
      }
    }
  }
  if (kNormal) {
    normal[0] = nx;
    normal[1] = nyv;
    normal[2] = nzv;
  }
  return out2 > 0.f ? fmaf(h, sqrtf(out2), s) : s;
}

__global__ void __launch_bounds__(128)
spline_fwd_kernel(DevGeom g, const SplineRec* __restrict__ splines,
                  const float4* __restrict__ coef, const PairRec* __restrict__ pairs,
                  const int32_t* __restrict__ row_pair, int64_t G,
                  const float* __restrict__ pose_a, const float* __restrict__ pose_b,
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
    const int total = nfeat * S.np;
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      PartT<float> c;
      part_zero(c);
      if (t < total) {
        const int s = t / nfeat, k = t - s * nfeat;
        const SplineRec sp = splines[S.p0 + s];
        float phi, gr[3], px, py, pz;
        if (k < fp.nv) {            // V-SDF: the vertex is the contact point
          const float3 x = xform(Rr, tr, g.verts[fp.v0 + k]);
          px = x.x; py = x.y; pz = x.z;
          phi = spline_sdf<true>(sp, coef, px, py, pz, gr);
        } else {                    // E-SDF: sphere trace from both corners
          const uint32_t e = g.edges[fp.e0 + (k - fp.nv)];
          const float3 a = xform(Rr, tr, g.verts[fp.v0 + (e & 0xffff)]);
          const float3 b = xform(Rr, tr, g.verts[fp.v0 + (e >> 16)]);
          float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
          const float L = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
          const float iL = 1.0f / L;
          ex *= iL; ey *= iL; ez *= iL;
          float phI = spline_sdf<false>(sp, coef, a.x, a.y, a.z, nullptr);
          float phII = spline_sdf<false>(sp, coef, b.x, b.y, b.z, nullptr);
          float aI = 0.f, aII = L;
          for (int q = 0; q < kp.trace_iters; ++q) {
            aI += sigmoid_c(phI, kp.c_trace) * phI;
            aII -= sigmoid_c(phII, kp.c_trace) * phII;
            if (q + 1 == kp.trace_iters) break;
            phI = spline_sdf<false>(sp, coef, fmaf(aI, ex, a.x), fmaf(aI, ey, a.y),
                                    fmaf(aI, ez, a.z), nullptr);
            phII = spline_sdf<false>(sp, coef, fmaf(aII, ex, a.x), fmaf(aII, ey, a.y),
                                     fmaf(aII, ez, a.z), nullptr);
          }
          const float am = 0.5f * (softclip0(aI, L, kp.tau_clip, kp.c_clip) +
                                   softclip0(aII, L, kp.tau_clip, kp.c_clip));
          px = fmaf(am, ex, a.x);
          py = fmaf(am, ey, a.y);
          pz = fmaf(am, ez, a.z);
          phi = spline_sdf<true>(sp, coef, px, py, pz, gr);
        }
        const float w = transition(phi, kp);
        const float dc = fmaf(w, phi - kp.d_max, kp.d_max);   // f phi + (1 - f) d_max
        if (project) {
          px = fmaf(-phi, gr[0], px);
          py = fmaf(-phi, gr[1], py);
          pz = fmaf(-phi, gr[2], pz);
        }
        part_from_contact(c, w, dc, v3(px, py, pz), v3(gr[0], gr[1], gr[2]), kp.c_blend);
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

cudaError_t launch_spline_forward(const SplineLaunch& L, cudaStream_t stream) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((L.G + 3) / 4, 64 * L.n_sm));
  spline_fwd_kernel<<<(int)blocks, 128, 0, stream>>>(L.g, L.splines, L.coef, L.pairs, L.row_pair,
                                                      L.G, L.pose_a, L.pose_b, L.kp, L.y);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ccm
