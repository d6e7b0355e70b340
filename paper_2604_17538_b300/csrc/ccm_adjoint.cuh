// Scalar-generic pieces of the reverse pass (Sec. 2-4 of arxiv 2604.17538),
// on T = float (gradient) or Dual (forward-over-reverse: H u, J u): the smooth
// operators and the transition, the piece SDF with its gradient and
// Hessian-vector product, the sphere-traced edge contact with its adjoint,
// the contact adjoint through the mollifier and the blend, a group's adjoint
// coefficients and the pair's twist components.  Shared by the per-warp
// reverse kernels (ccm_bwd.cu) and the per-contact ones (ccm_flat.cu).
#pragma once
#include "ccm_blend.cuh"

namespace ccm {

// ---------------------------------------------------------------------------
// scalar-generic smooth operators (Sec. 2) and transition (Sec. 4.3)
// ---------------------------------------------------------------------------
// sigmoid(x / tau), c = log2(e) / tau, without overflow on either side
template <class T> __device__ __forceinline__ T sigmoid_t(T x, float c) {
  if (val(x) >= 0.f) return rcp_t(1.0f + ex2_t(x * (-c)));
  const T e = ex2_t(x * c);
  return e * rcp_t(1.0f + e);
}
template <class T> __device__ __forceinline__ T softplus_t(T x, float tau, float c) {
  return max_t(x, T(0.f)) + tau * log1p_t(ex2_t(abs_t(x) * (-c)));
}
template <class T> __device__ __forceinline__ T softclip0_t(T x, T L, float tau, float c) {
  return softplus_t(x, tau, c) - softplus_t(x - L, tau, c);
}
// f_t and its derivative: quintic smoothstep of s = (d_max - d) / eps
template <class T>
__device__ __forceinline__ void transition_t(T d, const KParams& kp, T& f, T& fp) {
  const float sv = (kp.d_max - val(d)) * kp.inv_gate;
  if (sv <= 0.f) { f = T(0.f); fp = T(0.f); return; }
  if (sv >= 1.f) { f = T(1.f); fp = T(0.f); return; }
  const T s = (kp.d_max - d) * kp.inv_gate;
  const T s2 = s * s;
  f = s2 * s * fma_t(s, fma_t(s, T(6.f), T(-15.f)), T(10.f));
  const T om = 1.0f - s;
  fp = s2 * om * om * (-30.f * kp.inv_gate);
}

// ---------------------------------------------------------------------------
// Sec. 3 piece SDF, value + gradient (+ Hessian-vector product) on T
// ---------------------------------------------------------------------------
template <class T> struct SdfT {
  T phi;
  V3T<T> g, hv;
};

// Dual-number version, one pass over the planes.  With unnormalised weights
// e_k = 2^((phi_k - s) c), S = sum e_k, w_k = e_k / S and plane-value tangents
// dphi_k = n_k . x':  phi' = sum w_k dphi_k,  g' = (D / S - phi' g) / tau with
// D = sum e_k dphi_k n_k, and for the Hessian-vector product
// H v = (A / S - g (g . v)) / tau with A = sum e_k (n_k . v) n_k, whose tangent
// (w_k' = w_k (dphi_k - phi') / tau) is
// (H v)' = [(B - phi' A) / (S tau) + C / S - g' (g . v) - g (g' . v + g . v')] / tau,
// B = sum e_k dphi_k (n_k . v) n_k, C = sum e_k (n_k . v') n_k.  The sums
// cancel to rounding where one plane dominates (absolute error ~1e-7 |x'| / tau),
// far inside the reverse pass's tolerance.
// kMode: 0 value, 1 value + gradient, 2 value + gradient + Hessian-vector product
template <int kMode>
__device__ SdfT<Dual> sdf_dual(const float4* __restrict__ pl, int nf, V3T<Dual> x, float s,
                               V3T<Dual> v, const KParams& kp) {
  constexpr bool kHv = kMode == 2;
  constexpr bool kGrad = kMode >= 1;
  const float xv = x.x.v, yv = x.y.v, zv = x.z.v;
  const float xd = x.x.d, yd = x.y.d, zd = x.z.d;
  float S, Gx, Gy, Gz, Pd, Dx, Dy, Dz, Ax, Ay, Az, Bx, By, Bz, Cx, Cy, Cz;
  for (int pass = 0; pass < 2; ++pass) {
    const float sc = s * kp.c_sdf;
    S = Gx = Gy = Gz = Pd = Dx = Dy = Dz = 0.f;
    Ax = Ay = Az = Bx = By = Bz = Cx = Cy = Cz = 0.f;
    float mx = -INFINITY;
#pragma unroll 4
    for (int k = 0; k < nf; ++k) {
      const float4 p = pl[k];
      const float ph = fmaf(p.x, xv, fmaf(p.y, yv, fmaf(p.z, zv, p.w)));
      mx = fmaxf(mx, ph);
      const float e = ex2(fmaf(ph, kp.c_sdf, -sc));
      const float dp = fmaf(p.x, xd, fmaf(p.y, yd, p.z * zd));
      S += e;
      Gx = fmaf(e, p.x, Gx);
      Gy = fmaf(e, p.y, Gy);
      Gz = fmaf(e, p.z, Gz);
      Pd = fmaf(e, dp, Pd);
      if (kGrad) {
        const float ed = e * dp;
        Dx = fmaf(ed, p.x, Dx);
        Dy = fmaf(ed, p.y, Dy);
        Dz = fmaf(ed, p.z, Dz);
      }
      if (kHv) {
        const float q = fmaf(p.x, v.x.v, fmaf(p.y, v.y.v, p.z * v.z.v));
        const float qd = fmaf(p.x, v.x.d, fmaf(p.y, v.y.d, p.z * v.z.d));
        const float eq = e * q, eqd = eq * dp, ew = e * qd;
        Ax = fmaf(eq, p.x, Ax); Ay = fmaf(eq, p.y, Ay); Az = fmaf(eq, p.z, Az);
        Bx = fmaf(eqd, p.x, Bx); By = fmaf(eqd, p.y, By); Bz = fmaf(eqd, p.z, Bz);
        Cx = fmaf(ew, p.x, Cx); Cy = fmaf(ew, p.y, Cy); Cz = fmaf(ew, p.z, Cz);
      }
    }
    if (pass == 0 && (mx - s) * kp.c_sdf > 64.0f) { s = mx; continue; }
    break;
  }
  const float iS = __frcp_rn(S);
  const float it = 1.0f / kp.tau_sdf;
  SdfT<Dual> r;
  r.phi = Dual(fmaf(kp.ic_sdf, __log2f(S), s), Pd * iS);
  if (kMode == 0) return r;
  const float gx = Gx * iS, gy = Gy * iS, gz = Gz * iS;
  const float phd = r.phi.d;
  const float gdx = fmaf(Dx, iS, -phd * gx) * it, gdy = fmaf(Dy, iS, -phd * gy) * it,
              gdz = fmaf(Dz, iS, -phd * gz) * it;
  r.g = v3(Dual(gx, gdx), Dual(gy, gdy), Dual(gz, gdz));
  if (!kHv) return r;
  const float gv = fmaf(gx, v.x.v, fmaf(gy, v.y.v, gz * v.z.v));
  const float gdv = fmaf(gdx, v.x.v, fmaf(gdy, v.y.v, gdz * v.z.v)) +
                    fmaf(gx, v.x.d, fmaf(gy, v.y.d, gz * v.z.d));
  const float iSt = iS * it;
  r.hv = v3(Dual(fmaf(Ax, iS, -gx * gv) * it,
                 (fmaf(fmaf(-phd, Ax, Bx), iSt, fmaf(Cx, iS, -fmaf(gdx, gv, gx * gdv)))) * it),
            Dual(fmaf(Ay, iS, -gy * gv) * it,
                 (fmaf(fmaf(-phd, Ay, By), iSt, fmaf(Cy, iS, -fmaf(gdy, gv, gy * gdv)))) * it),
            Dual(fmaf(Az, iS, -gz * gv) * it,
                 (fmaf(fmaf(-phd, Az, Bz), iSt, fmaf(Cz, iS, -fmaf(gdz, gv, gz * gdv)))) * it));
  return r;
}

template <class T, int kMode>
__device__ SdfT<T> sdf_t(const float4* __restrict__ pl, int nf, V3T<T> x, float s, V3T<T> v,
                         const KParams& kp) {
  if constexpr (sizeof(T) == sizeof(Dual)) {
    return sdf_dual<kMode>(pl, nf, x, s, v, kp);
  }
  constexpr bool kHv = kMode == 2;
  constexpr bool kGrad = kMode >= 1;
  SdfT<T> r;
  for (int pass = 0; pass < 2; ++pass) {
    const float sc = s * kp.c_sdf;
    T S(0.f), gx(0.f), gy(0.f), gz(0.f), hx(0.f), hy(0.f), hz(0.f);
    float mx = -INFINITY;
#pragma unroll 4
    for (int k = 0; k < nf; ++k) {
      const float4 p = pl[k];
      const T ph = fma_t(p.x, x.x, fma_t(p.y, x.y, fma_t(p.z, x.z, T(p.w))));
      mx = fmaxf(mx, val(ph));
      const T e = ex2_t(fma_t(ph, kp.c_sdf, T(-sc)));
      S += e;
      if (kGrad) {
        gx = fma_t(e, p.x, gx);
        gy = fma_t(e, p.y, gy);
        gz = fma_t(e, p.z, gz);
      }
      if (kHv) {
        const T en = e * fma_t(p.x, v.x, fma_t(p.y, v.y, p.z * v.z));
        hx = fma_t(en, p.x, hx);
        hy = fma_t(en, p.y, hy);
        hz = fma_t(en, p.z, hz);
      }
    }
    if (pass == 0 && (mx - s) * kp.c_sdf > 64.0f) { s = mx; continue; }
    const T inv = rcp_t(S);
    r.phi = fma_t(T(kp.ic_sdf), log2_t(S), T(s));
    if (!kGrad) break;
    r.g = v3(gx * inv, gy * inv, gz * inv);
    if (kHv) {
      const T gv = dot3(r.g, v);
      const float it = 1.0f / kp.tau_sdf;
      r.hv = v3((hx * inv - r.g.x * gv) * it, (hy * inv - r.g.y * gv) * it,
                (hz * inv - r.g.z * gv) * it);
    }
    break;
  }
  return r;
}


// Two points at once (the two sphere-trace chains of an edge), kMode 0 or 1:
// one loop over the planes for both, so the two independent dependency
// chains overlap.  Each point's arithmetic is exactly that of sdf_t /
// sdf_dual (same operations in the same order), so its results are bitwise
// those of a single-point call with the same shift.
template <int kMode>
__device__ void sdf_dual2(const float4* __restrict__ pl, int nf, V3T<Dual> xa, float sa,
                          V3T<Dual> xb, float sb, const KParams& kp, SdfT<Dual>& ra,
                          SdfT<Dual>& rb) {
  static_assert(kMode <= 1, "two-point evaluation has no Hessian-vector product");
  constexpr bool kGrad = kMode >= 1;
  const float xav = xa.x.v, yav = xa.y.v, zav = xa.z.v, xad = xa.x.d, yad = xa.y.d, zad = xa.z.d;
  const float xbv = xb.x.v, ybv = xb.y.v, zbv = xb.z.v, xbd = xb.x.d, ybd = xb.y.d, zbd = xb.z.d;
  float Sa, Gxa, Gya, Gza, Pda, Dxa, Dya, Dza, Sb, Gxb, Gyb, Gzb, Pdb, Dxb, Dyb, Dzb;
  for (int pass = 0; pass < 2; ++pass) {
    const float sca = sa * kp.c_sdf, scb = sb * kp.c_sdf;
    Sa = Gxa = Gya = Gza = Pda = Dxa = Dya = Dza = 0.f;
    Sb = Gxb = Gyb = Gzb = Pdb = Dxb = Dyb = Dzb = 0.f;
    float mxa = -INFINITY, mxb = -INFINITY;
#pragma unroll 4
    for (int k = 0; k < nf; ++k) {
      const float4 p = pl[k];
      const float pha = fmaf(p.x, xav, fmaf(p.y, yav, fmaf(p.z, zav, p.w)));
      const float phb = fmaf(p.x, xbv, fmaf(p.y, ybv, fmaf(p.z, zbv, p.w)));
      mxa = fmaxf(mxa, pha);
      mxb = fmaxf(mxb, phb);
      const float ea = ex2(fmaf(pha, kp.c_sdf, -sca));
      const float eb = ex2(fmaf(phb, kp.c_sdf, -scb));
      const float dpa = fmaf(p.x, xad, fmaf(p.y, yad, p.z * zad));
      const float dpb = fmaf(p.x, xbd, fmaf(p.y, ybd, p.z * zbd));
      Sa += ea;
      Sb += eb;
      Gxa = fmaf(ea, p.x, Gxa); Gya = fmaf(ea, p.y, Gya); Gza = fmaf(ea, p.z, Gza);
      Gxb = fmaf(eb, p.x, Gxb); Gyb = fmaf(eb, p.y, Gyb); Gzb = fmaf(eb, p.z, Gzb);
      Pda = fmaf(ea, dpa, Pda);
      Pdb = fmaf(eb, dpb, Pdb);
      if (kGrad) {
        const float eda = ea * dpa, edb = eb * dpb;
        Dxa = fmaf(eda, p.x, Dxa); Dya = fmaf(eda, p.y, Dya); Dza = fmaf(eda, p.z, Dza);
        Dxb = fmaf(edb, p.x, Dxb); Dyb = fmaf(edb, p.y, Dyb); Dzb = fmaf(edb, p.z, Dzb);
      }
    }
    const bool bada = (mxa - sa) * kp.c_sdf > 64.0f, badb = (mxb - sb) * kp.c_sdf > 64.0f;
    if (pass == 0 && (bada || badb)) {
      if (bada) sa = mxa;
      if (badb) sb = mxb;
      continue;
    }
    break;
  }
  const float iSa = __frcp_rn(Sa), iSb = __frcp_rn(Sb);
  const float it = 1.0f / kp.tau_sdf;
  ra.phi = Dual(fmaf(kp.ic_sdf, __log2f(Sa), sa), Pda * iSa);
  rb.phi = Dual(fmaf(kp.ic_sdf, __log2f(Sb), sb), Pdb * iSb);
  if (kMode == 0) return;
  const float gxa = Gxa * iSa, gya = Gya * iSa, gza = Gza * iSa;
  const float gxb = Gxb * iSb, gyb = Gyb * iSb, gzb = Gzb * iSb;
  const float phda = ra.phi.d, phdb = rb.phi.d;
  ra.g = v3(Dual(gxa, fmaf(Dxa, iSa, -phda * gxa) * it), Dual(gya, fmaf(Dya, iSa, -phda * gya) * it),
            Dual(gza, fmaf(Dza, iSa, -phda * gza) * it));
  rb.g = v3(Dual(gxb, fmaf(Dxb, iSb, -phdb * gxb) * it), Dual(gyb, fmaf(Dyb, iSb, -phdb * gyb) * it),
            Dual(gzb, fmaf(Dzb, iSb, -phdb * gzb) * it));
}

template <class T, int kMode>
__device__ void sdf_t2(const float4* __restrict__ pl, int nf, V3T<T> xa, float sa, V3T<T> xb,
                       float sb, const KParams& kp, SdfT<T>& ra, SdfT<T>& rb) {
  if constexpr (sizeof(T) == sizeof(Dual)) {
    sdf_dual2<kMode>(pl, nf, xa, sa, xb, sb, kp, ra, rb);
  } else {
    static_assert(kMode <= 1, "two-point evaluation has no Hessian-vector product");
    constexpr bool kGrad = kMode >= 1;
    for (int pass = 0; pass < 2; ++pass) {
      const float sca = sa * kp.c_sdf, scb = sb * kp.c_sdf;
      T Sa(0.f), gxa(0.f), gya(0.f), gza(0.f), Sb(0.f), gxb(0.f), gyb(0.f), gzb(0.f);
      float mxa = -INFINITY, mxb = -INFINITY;
#pragma unroll 4
      for (int k = 0; k < nf; ++k) {
        const float4 p = pl[k];
        const T pha = fma_t(p.x, xa.x, fma_t(p.y, xa.y, fma_t(p.z, xa.z, T(p.w))));
        const T phb = fma_t(p.x, xb.x, fma_t(p.y, xb.y, fma_t(p.z, xb.z, T(p.w))));
        mxa = fmaxf(mxa, val(pha));
        mxb = fmaxf(mxb, val(phb));
        const T ea = ex2_t(fma_t(pha, kp.c_sdf, T(-sca)));
        const T eb = ex2_t(fma_t(phb, kp.c_sdf, T(-scb)));
        Sa += ea;
        Sb += eb;
        if (kGrad) {
          gxa = fma_t(ea, p.x, gxa); gya = fma_t(ea, p.y, gya); gza = fma_t(ea, p.z, gza);
          gxb = fma_t(eb, p.x, gxb); gyb = fma_t(eb, p.y, gyb); gzb = fma_t(eb, p.z, gzb);
        }
      }
      const bool bada = (mxa - sa) * kp.c_sdf > 64.0f, badb = (mxb - sb) * kp.c_sdf > 64.0f;
      if (pass == 0 && (bada || badb)) {
        if (bada) sa = mxa;
        if (badb) sb = mxb;
        continue;
      }
      ra.phi = fma_t(T(kp.ic_sdf), log2_t(Sa), T(sa));
      rb.phi = fma_t(T(kp.ic_sdf), log2_t(Sb), T(sb));
      if (kGrad) {
        const T ia = rcp_t(Sa), ib = rcp_t(Sb);
        ra.g = v3(gxa * ia, gya * ia, gza * ia);
        rb.g = v3(gxb * ib, gyb * ib, gzb * ib);
      }
      break;
    }
  }
}

// ---------------------------------------------------------------------------
// per-group adjoint coefficients and the contact adjoint
// ---------------------------------------------------------------------------
template <class T> struct Coef {
  T M, invU;           // log2 max logit, 1/U
  T gdel;              // gbar - g_r: ybar . (group values - reference contact values)
  T rd, rf;            // reference contact (see PartT)
  V3T<T> rp, rn;
  V3T<T> qb, nb;       // adjoints of the blended point q and of nu = N / U (S frame)
  float db, ab;        // adjoints of the blended depth and weight (= ybar)
  int live;
};

// Contact adjoint: given the contact's SDF value, gradient and H nu_bar at
// point p, returns x_bar (adjoint of p) -- Sec. 4.3 mollifier and Sec. 4.4
// blend differentiated by hand; see the derivation in the file header of
// ccm_bwd.h.
template <class T>
__device__ __forceinline__ V3T<T> contact_adjoint(const SdfT<T>& c, V3T<T> p, const Coef<T>& k,
                                                  const KParams& kp) {
  T f, fp;
  transition_t(c.phi, kp, f, fp);
  if (val(f) <= 0.f) return v3(T(0.f), T(0.f), T(0.f));
  const T dc = fma_t(f, c.phi - kp.d_max, T(kp.d_max));
  const T om = ex2_t(dc * (-kp.c_blend) - k.M) * k.invU;   // weight per unit f
  const T w = f * om;
  // g_c - gbar = (g_c - g_r) - (gbar - g_r), both from direct differences
  const T gcr = k.db * (dc - k.rd) + k.ab * (f - k.rf) + dot3(k.qb, sub3(p, k.rp)) +
                dot3(k.nb, sub3(c.g, k.rn));
  const T kk = gcr - k.gdel;
  const T fb = fma_t(w, T(k.ab), kk * om);
  const T dcb = w * (k.db - kk * (1.0f / kp.tau_blend));
  const T phib = fma_t(dcb, fma_t(fp, c.phi - kp.d_max, f), fb * fp);
  return v3(fma_t(w, k.qb.x, fma_t(phib, c.g.x, w * c.hv.x)),
            fma_t(w, k.qb.y, fma_t(phib, c.g.y, w * c.hv.y)),
            fma_t(w, k.qb.z, fma_t(phib, c.g.z, w * c.hv.z)));
}

// ---------------------------------------------------------------------------
// poses on T: the tangent of R is [w]x R and of t is v when differentiating
// along a twist direction (w, v)
// ---------------------------------------------------------------------------
template <class T> struct PoseT {
  T R[9];
  T t[3];
};

__device__ inline void load_pose_t(const float* p, const float* u, PoseT<float>& P) {
  (void)u;
  for (int i = 0; i < 9; ++i) P.R[i] = __ldg(p + i);
  for (int i = 0; i < 3; ++i) P.t[i] = __ldg(p + 9 + i);
}
__device__ inline void load_pose_t(const float* p, const float* u, PoseT<Dual>& P) {
  float R[9];
  for (int i = 0; i < 9; ++i) R[i] = __ldg(p + i);
  const float w0 = __ldg(u + 0), w1 = __ldg(u + 1), w2 = __ldg(u + 2);
  const float W[9] = {0.f, -w2, w1, w2, 0.f, -w0, -w1, w0, 0.f};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      P.R[3 * i + j] = Dual(R[3 * i + j], W[3 * i] * R[j] + W[3 * i + 1] * R[3 + j] +
                                              W[3 * i + 2] * R[6 + j]);
  for (int i = 0; i < 3; ++i) P.t[i] = Dual(__ldg(p + 9 + i), __ldg(u + 3 + i));
}

template <class T> __device__ __forceinline__ V3T<T> rot(const T R[9], V3T<T> x) {
  return v3(fma_t(R[0], x.x, fma_t(R[1], x.y, R[2] * x.z)),
            fma_t(R[3], x.x, fma_t(R[4], x.y, R[5] * x.z)),
            fma_t(R[6], x.x, fma_t(R[7], x.y, R[8] * x.z)));
}
template <class T> __device__ __forceinline__ V3T<T> rotT(const T R[9], V3T<T> x) {
  return v3(fma_t(R[0], x.x, fma_t(R[3], x.y, R[6] * x.z)),
            fma_t(R[1], x.x, fma_t(R[4], x.y, R[7] * x.z)),
            fma_t(R[2], x.x, fma_t(R[5], x.y, R[8] * x.z)));
}
template <class T> __device__ __forceinline__ V3T<T> cross3(V3T<T> a, V3T<T> b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float tan_of(float) { return 0.f; }
__device__ __forceinline__ float tan_of(Dual a) { return a.d; }


// ---------------------------------------------------------------------------
// edge: trace forward (storing the steps), contact, and optionally adjoint
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T gstep(T phi, float c) {   // sigmoid(phi/tau) phi
  return sigmoid_t(phi, c) * phi;
}
template <class T> __device__ __forceinline__ T gstep_d(T phi, float c) {  // its derivative
  const T s = sigmoid_t(phi, c);
  return fma_t(phi * (c * kLn2), s * (1.0f - s), s);
}

template <class T, bool kAdj, int kK>
__device__ void edge_t(const float4* __restrict__ pl, int nf, V3T<T> xI, V3T<T> xII, float mI0,
                       float mII0, T phI0, T phII0, V3T<T> gI0, V3T<T> gII0, const Coef<T>& k,
                       const KParams& kp, SdfT<T>& c, V3T<T>& pe, V3T<T>& xbI, V3T<T>& xbII) {
  const V3T<T> d = v3(xII.x - xI.x, xII.y - xI.y, xII.z - xI.z);
  const T L = sqrt_t(dot3(d, d));
  const T iL = rcp_t(L);
  const V3T<T> e = v3(d.x * iL, d.y * iL, d.z * iL);
  // kK > 0: exactly kK steps (compile-time, fully unrolled, registers);
  // kK == 0: trace_iters steps (up to 16) with arrays in local memory
  constexpr int kN = kK > 0 ? kK : 16;
  const int K = kK > 0 ? kK : kp.trace_iters;
  T a[kN + 1], b[kN + 1], pa[kN], pb[kN];
  V3T<T> ga[kN], gb[kN];
  a[0] = T(0.f);
  b[0] = L;
  pa[0] = phI0;
  pb[0] = phII0;
  ga[0] = gI0;
  gb[0] = gII0;
  float ma = mI0, mb = mII0;
  for (int s = 0; s < K; ++s) {
    const T sa = gstep(pa[s], kp.c_trace), sb = gstep(pb[s], kp.c_trace);
    a[s + 1] = a[s] + sa;
    b[s + 1] = b[s] - sb;
    if (s + 1 == K) break;
    const V3T<T> qa = v3(fma_t(a[s + 1], e.x, xI.x), fma_t(a[s + 1], e.y, xI.y),
                         fma_t(a[s + 1], e.z, xI.z));
    const V3T<T> qb = v3(fma_t(b[s + 1], e.x, xI.x), fma_t(b[s + 1], e.y, xI.y),
                         fma_t(b[s + 1], e.z, xI.z));
    SdfT<T> ra, rb;
    sdf_t2<T, kAdj ? 1 : 0>(pl, nf, qa, ma - fabsf(val(sa)), qb, mb - fabsf(val(sb)), kp, ra, rb);
    pa[s + 1] = ra.phi;
    pb[s + 1] = rb.phi;
    if (kAdj) { ga[s + 1] = ra.g; gb[s + 1] = rb.g; }
    // exact max-plane values are not tracked here; a looser lower bound only
    // risks the (exact) repeat pass inside sdf_t
    ma = val(ra.phi) - kp.tau_sdf * logf((float)nf) - 1e-6f;
    mb = val(rb.phi) - kp.tau_sdf * logf((float)nf) - 1e-6f;
  }
  const T aK = a[K], bK = b[K];
  const T cI = softclip0_t(aK, L, kp.tau_clip, kp.c_clip);
  const T cII = softclip0_t(bK, L, kp.tau_clip, kp.c_clip);
  const T am = 0.5f * (cI + cII);
  pe = v3(fma_t(am, e.x, xI.x), fma_t(am, e.y, xI.y), fma_t(am, e.z, xI.z));
  const float lb = fmaxf(mI0 - val(am), mII0 - (val(L) - val(am)));
  c = sdf_t<T, kAdj ? 2 : 1>(pl, nf, pe, lb, k.nb, kp);
  if (!kAdj) return;
  // ---- reverse sweep ----
  const V3T<T> xb = contact_adjoint(c, pe, k, kp);
  V3T<T> xi = xb;                                   // d pe / d xI = I (with e fixed)
  V3T<T> eb = v3(am * xb.x, am * xb.y, am * xb.z);  // d pe / d e = am I
  const T amb = dot3(xb, e);
  // soft clip: d sc/d alpha = sig(alpha/tc) - sig((alpha - L)/tc), d sc/dL = sig((alpha - L)/tc)
  const T sIa = sigmoid_t(aK, kp.c_clip), sIb = sigmoid_t(aK - L, kp.c_clip);
  const T sJa = sigmoid_t(bK, kp.c_clip), sJb = sigmoid_t(bK - L, kp.c_clip);
  T abar = 0.5f * amb * (sIa - sIb);
  T bbar = 0.5f * amb * (sJa - sJb);
  T Lb = 0.5f * amb * (sIb + sJb);
  for (int s = K - 1; s >= 0; --s) {
    // chain I: a[s+1] = a[s] + g(phi(xI + a[s] e))
    const T pbarI = abar * gstep_d(pa[s], kp.c_trace);
    xi = v3(fma_t(pbarI, ga[s].x, xi.x), fma_t(pbarI, ga[s].y, xi.y), fma_t(pbarI, ga[s].z, xi.z));
    if (s > 0) {
      const T t = pbarI * a[s];
      eb = v3(fma_t(t, ga[s].x, eb.x), fma_t(t, ga[s].y, eb.y), fma_t(t, ga[s].z, eb.z));
      abar = fma_t(pbarI, dot3(ga[s], e), abar);
    }
    // chain II: b[s+1] = b[s] - g(phi(xI + b[s] e)), b[0] = L
    const T pbarII = -(bbar * gstep_d(pb[s], kp.c_trace));
    xi = v3(fma_t(pbarII, gb[s].x, xi.x), fma_t(pbarII, gb[s].y, xi.y), fma_t(pbarII, gb[s].z, xi.z));
    const T t2 = pbarII * b[s];
    eb = v3(fma_t(t2, gb[s].x, eb.x), fma_t(t2, gb[s].y, eb.y), fma_t(t2, gb[s].z, eb.z));
    bbar = fma_t(pbarII, dot3(gb[s], e), bbar);
  }
  Lb += bbar;   // b[0] = L
  // e = d / L, L = |d|, d = xII - xI
  const T ee = dot3(e, eb);
  const V3T<T> db = v3(fma_t(Lb, e.x, (eb.x - e.x * ee) * iL), fma_t(Lb, e.y, (eb.y - e.y * ee) * iL),
                       fma_t(Lb, e.z, (eb.z - e.z * ee) * iL));
  xbII = db;
  xbI = v3(xi.x - db.x, xi.y - db.y, xi.z - db.z);
}


// The 12 gradient components (w_A, v_A, w_B, v_B) of one pair's (or one
// work item's) forces, plus the output-transform terms (w, v) of each body,
// into g[12]; with h != NULL the tangents (H u) into h[12], each body's
// twist gradient corrected by -1/2 u_w x grad_w (the chart's second-order
// term).  uA / uB: the direction's twists of A and B (NULL for float).
template <class T>
__device__ void write_twists(V3T<T> F, V3T<T> M, V3T<T> oAw, V3T<T> oAv, V3T<T> oBw,
                             V3T<T> oBv, V3T<T> tba, const float* uA, const float* uB, float* g,
                             float* h) {
  const V3T<T> c = cross3(tba, F);
  const T gA[6] = {M.x + oAw.x, M.y + oAw.y, M.z + oAw.z, F.x + oAv.x, F.y + oAv.y, F.z + oAv.z};
  const T gB[6] = {c.x - M.x + oBw.x, c.y - M.y + oBw.y, c.z - M.z + oBw.z,
                   oBv.x - F.x, oBv.y - F.y, oBv.z - F.z};
  for (int q = 0; q < 6; ++q) {
    g[q] = val(gA[q]);
    g[6 + q] = val(gB[q]);
  }
  if (h) {
    float hA[6], hB[6];
    for (int q = 0; q < 6; ++q) { hA[q] = tan_of(gA[q]); hB[q] = tan_of(gB[q]); }
    const float wA[3] = {val(gA[0]), val(gA[1]), val(gA[2])};
    const float wB[3] = {val(gB[0]), val(gB[1]), val(gB[2])};
    hA[0] -= 0.5f * (uA[1] * wA[2] - uA[2] * wA[1]);
    hA[1] -= 0.5f * (uA[2] * wA[0] - uA[0] * wA[2]);
    hA[2] -= 0.5f * (uA[0] * wA[1] - uA[1] * wA[0]);
    hB[0] -= 0.5f * (uB[1] * wB[2] - uB[2] * wB[1]);
    hB[1] -= 0.5f * (uB[2] * wB[0] - uB[0] * wB[2]);
    hB[2] -= 0.5f * (uB[0] * wB[1] - uB[1] * wB[0]);
    for (int q = 0; q < 6; ++q) {
      h[q] = hA[q];
      h[6 + q] = hB[q];
    }
  }
}


// cotangent row yb, with PS the pose of its SDF body; with jrow the output
// tangents (J u) of the group; ow, ov: the output-transform terms of the SDF
// body's twist, d<ybar, y>/d(w_S, v_S) through p_w = R_S q + t_S and
// n_w = R_S nu / |nu| (zero for a group without a contact).
template <class T>
__device__ void form_coef(const PartT<T>& A, const float* yb, const PoseT<T>& PS, float* jrow,
                          Coef<T>& cf, V3T<T>& ow, V3T<T>& ov) {
  cf.db = yb[0];
  cf.ab = yb[1];
  cf.live = val(A.U) > 0.f;
  const V3T<T> pbw = v3(T(yb[2]), T(yb[3]), T(yb[4]));
  const V3T<T> nbw = v3(T(yb[5]), T(yb[6]), T(yb[7]));
  ow = ov = zero3t<T>();
  if (cf.live) {
    const T iU = rcp_t(A.U);
    const T d = fma_t(A.Dd, iU, A.rd), a = fma_t(A.Da, iU, A.rf);
    const V3T<T> q = axpy3(iU, A.Dp, A.rp);
    const V3T<T> nu = axpy3(iU, A.Dn, A.rn);
    const V3T<T> nuw = rot(PS.R, nu);
    const T nn = sqrt_t(dot3(nuw, nuw));
    const T inn = val(nn) > 0.f ? rcp_t(nn) : T(0.f);
    const V3T<T> nw = v3(nuw.x * inn, nuw.y * inn, nuw.z * inn);
    const V3T<T> qw = rot(PS.R, q);
    if (jrow) {
      jrow[0] = tan_of(d);
      jrow[1] = tan_of(a);
      jrow[2] = tan_of(qw.x) + tan_of(PS.t[0]);
      jrow[3] = tan_of(qw.y) + tan_of(PS.t[1]);
      jrow[4] = tan_of(qw.z) + tan_of(PS.t[2]);
      jrow[5] = tan_of(nw.x);
      jrow[6] = tan_of(nw.y);
      jrow[7] = tan_of(nw.z);
    }
    cf.M = A.M;
    cf.invU = iU;
    cf.qb = rotT(PS.R, pbw);
    const V3T<T> nbs = rotT(PS.R, nbw);
    const V3T<T> ns = rotT(PS.R, nw);
    const T nsn = dot3(ns, nbs);
    cf.nb = v3((nbs.x - ns.x * nsn) * inn, (nbs.y - ns.y * nsn) * inn, (nbs.z - ns.z * nsn) * inn);
    cf.rd = A.rd; cf.rf = A.rf; cf.rp = A.rp; cf.rn = A.rn;
    cf.gdel = (cf.db * A.Dd + cf.ab * A.Da + dot3(cf.qb, A.Dp) + dot3(cf.nb, A.Dn)) * iU;
    const V3T<T> c1 = cross3(qw, pbw), c2 = cross3(nw, nbw);
    ow = v3(c1.x + c2.x, c1.y + c2.y, c1.z + c2.z);
    ov = pbw;
  } else {
    cf.M = cf.invU = cf.gdel = cf.rd = cf.rf = T(0.f);
    cf.qb = cf.nb = cf.rp = cf.rn = zero3t<T>();
    if (jrow)
      for (int q = 0; q < 8; ++q) jrow[q] = 0.f;
  }
}

}  // namespace ccm
