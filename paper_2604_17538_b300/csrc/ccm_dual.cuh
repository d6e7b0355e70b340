// Scalar types of the derivative kernels: plain float, and a forward-mode
// dual number (value + one tangent) so that running the hand-written adjoint
// on duals gives forward-over-reverse second derivatives (H u) and, on the
// forward recomputation, the output tangents (J u).
#pragma once
#include "ccm_device.cuh"

namespace ccm {

struct Dual {
  float v, d;
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(float a) : v(a), d(0.f) {}
  __device__ __forceinline__ Dual(float a, float b) : v(a), d(b) {}
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) {
  return Dual(a.v * b.v, fmaf(a.v, b.d, a.d * b.v));
}
__device__ __forceinline__ Dual operator*(Dual a, float b) { return Dual(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator*(float a, Dual b) { return Dual(a * b.v, a * b.d); }
__device__ __forceinline__ Dual operator+(Dual a, float b) { return Dual(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(float a, Dual b) { return Dual(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(Dual a, float b) { return Dual(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(float a, Dual b) { return Dual(a - b.v, -b.d); }
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a.v += b.v; a.d += b.d; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { a.v -= b.v; a.d -= b.d; return a; }

// value of a scalar (for decisions that never carry derivatives)
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ float val(Dual a) { return a.v; }

// fused a * b + c
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ Dual fma_t(Dual a, Dual b, Dual c) {
  return Dual(fmaf(a.v, b.v, c.v), fmaf(a.v, b.d, fmaf(a.d, b.v, c.d)));
}
__device__ __forceinline__ Dual fma_t(float a, Dual b, Dual c) {
  return Dual(fmaf(a, b.v, c.v), fmaf(a, b.d, c.d));
}
__device__ __forceinline__ Dual fma_t(Dual a, float b, Dual c) {
  return Dual(fmaf(a.v, b, c.v), fmaf(a.d, b, c.d));
}

// 2^x on the SFU
__device__ __forceinline__ float ex2_t(float x) { return ex2(x); }
__device__ __forceinline__ Dual ex2_t(Dual x) {
  const float e = ex2(x.v);
  return Dual(e, e * kLn2 * x.d);
}
__device__ __forceinline__ float log2_t(float x) { return __log2f(x); }
__device__ __forceinline__ Dual log2_t(Dual x) {
  return Dual(__log2f(x.v), x.d / (x.v * kLn2));
}
__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ Dual rcp_t(Dual x) {
  const float r = __frcp_rn(x.v);
  return Dual(r, -x.d * r * r);
}
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ Dual sqrt_t(Dual x) {
  const float s = sqrtf(x.v);
  return Dual(s, s > 0.f ? 0.5f * x.d / s : 0.f);
}
__device__ __forceinline__ float log1p_t(float x) { return log1pf(x); }
__device__ __forceinline__ Dual log1p_t(Dual x) { return Dual(log1pf(x.v), x.d / (1.0f + x.v)); }
__device__ __forceinline__ float max_t(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ Dual max_t(Dual a, Dual b) { return a.v >= b.v ? a : b; }
__device__ __forceinline__ float abs_t(float a) { return fabsf(a); }
__device__ __forceinline__ Dual abs_t(Dual a) { return a.v >= 0.f ? a : -a; }

template <class T> struct V3T { T x, y, z; };
template <class T> __device__ __forceinline__ V3T<T> v3(T x, T y, T z) { return {x, y, z}; }
template <class T> __device__ __forceinline__ T dot3(V3T<T> a, V3T<T> b) {
  return fma_t(a.x, b.x, fma_t(a.y, b.y, a.z * b.z));
}

}  // namespace ccm
