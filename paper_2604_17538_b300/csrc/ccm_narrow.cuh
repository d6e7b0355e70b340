// Narrow-phase pieces shared by the kernels: the E-SDF contact of one edge
// (Sec. 4.2) and the normalised, world-frame output of a blend (Sec. 4.4).
#pragma once
#include "ccm_blend.cuh"

namespace ccm {

struct EdgeContact {
  float phi, px, py, pz, gx, gy, gz;
};

// Sec. 4.2 E-SDF contact of the edge (a, b): both corners are sphere traced
// towards each other, alpha_I from 0 along +e_t and alpha_II from L along
// -e_t, with steps sigmoid(phi / tau_trace) phi; the traced edge parameters
// are soft clipped to [0, L] and the contact is their midpoint.  m_a, m_b are
// the exact max-plane values and phi_a, phi_b the SDF at the corners.
__device__ inline EdgeContact edge_contact(const float4* __restrict__ pl, int nf, float4 a,
                                           float4 b, float m_a, float m_b, float phi_a,
                                           float phi_b, const KParams& kp) {
  float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
  const float L = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
  const float iL = 1.0f / L;
  ex *= iL; ey *= iL; ez *= iL;
  float phI = phi_a, phII = phi_b, mI = m_a, mII = m_b;
  float aI = 0.f, aII = L;
  for (int k = 0; k < kp.trace_iters; ++k) {
    const float stI = sigmoid_c(phI, kp.c_trace) * phI;
    const float stII = sigmoid_c(phII, kp.c_trace) * phII;
    aI += stI;
    aII -= stII;
    if (k + 1 == kp.trace_iters) break;
    // 1-Lipschitz lower bounds of the max-plane value at the new points
    const float sI = mI - fabsf(stI), sII = mII - fabsf(stII);
    sdf_val2(pl, nf, fmaf(aI, ex, a.x), fmaf(aI, ey, a.y), fmaf(aI, ez, a.z), sI,
             fmaf(aII, ex, a.x), fmaf(aII, ey, a.y), fmaf(aII, ez, a.z), sII, kp, phI, mI, phII,
             mII);
  }
  const float cI = softclip0(aI, L, kp.tau_clip, kp.c_clip);
  const float cII = softclip0(aII, L, kp.tau_clip, kp.c_clip);
  const float am = 0.5f * (cI + cII);
  EdgeContact c;
  c.px = fmaf(am, ex, a.x);
  c.py = fmaf(am, ey, a.y);
  c.pz = fmaf(am, ez, a.z);
  const float lb = fmaxf(m_a - am, m_b - (L - am));
  const SdfGrad r = sdf_grad(pl, nf, c.px, c.py, c.pz, lb, kp);
  c.phi = r.phi;
  c.gx = r.gx;
  c.gy = r.gy;
  c.gz = r.gz;
  return c;
}

// Normalised blend of a group's partial (Sec. 4.4), rotated into world frame:
// d = rd + Dd / U, a = rf + Da / U, q = rp + Dp / U, n = R_S nu / |R_S nu| with
// nu = rn + Dn / U; an empty group is (d_max, 0, 0, 0).
__device__ inline void write_group(float* out, const PartT<float>& acc, const float* RS,
                                   const float* tS, const KParams& kp) {
  if (acc.U > 0.f) {
    const float iU = __frcp_rn(acc.U);
    const float qx = fmaf(acc.Dp.x, iU, acc.rp.x), qy = fmaf(acc.Dp.y, iU, acc.rp.y),
                qz = fmaf(acc.Dp.z, iU, acc.rp.z);
    const float mx = fmaf(acc.Dn.x, iU, acc.rn.x), my = fmaf(acc.Dn.y, iU, acc.rn.y),
                mz = fmaf(acc.Dn.z, iU, acc.rn.z);
    const float wx = RS[0] * mx + RS[1] * my + RS[2] * mz;
    const float wy = RS[3] * mx + RS[4] * my + RS[5] * mz;
    const float wz = RS[6] * mx + RS[7] * my + RS[8] * mz;
    const float nn = sqrtf(wx * wx + wy * wy + wz * wz);
    const float in = nn > 0.f ? 1.0f / nn : 0.f;
    out[0] = fmaf(acc.Dd, iU, acc.rd);
    out[1] = fmaf(acc.Da, iU, acc.rf);
    out[2] = RS[0] * qx + RS[1] * qy + RS[2] * qz + tS[0];
    out[3] = RS[3] * qx + RS[4] * qy + RS[5] * qz + tS[1];
    out[4] = RS[6] * qx + RS[7] * qy + RS[8] * qz + tS[2];
    out[5] = wx * in;
    out[6] = wy * in;
    out[7] = wz * in;
  } else {
    write_empty(out, kp);
  }
}

}  // namespace ccm
