// Sec. 4.4 blend partials shared by the forward and reverse kernels, on a
// scalar type T (float, or Dual for the forward-over-reverse pass).
#pragma once
#include "ccm_dual.cuh"

namespace ccm {

// ---------------------------------------------------------------------------
// Sec. 4.4 blend partials on T (online softmax).  Besides the normaliser U a
// partial keeps a reference contact r -- the one with the largest logit -- and
// the weighted differences sum_j u_j (x_j - x_r) of every blended quantity
// x = (d_c, f, p, grad phi), rather than the plain sums.  The adjoint needs
// g_c - gbar for g = ybar . (contact values); formed from differences to r it
// carries no cancellation, and it is exactly 0 for a group whose only active
// contact is r (there 1/U = 1/f can be huge near the gate edge).
// ---------------------------------------------------------------------------
template <class T> struct PartT {
  T M, U;
  T rd, rf;          // reference contact: mollified depth, transition weight
  V3T<T> rp, rn;     // reference point, gradient
  T Dd, Da;          // sum u (d_c - rd), sum u (f - rf)
  V3T<T> Dp, Dn;     // sum u (p - rp), sum u (grad phi - rn)
};

template <class T> __device__ __forceinline__ V3T<T> zero3t() { return v3(T(0.f), T(0.f), T(0.f)); }

template <class T> __device__ __forceinline__ void part_zero(PartT<T>& c) {
  c.M = T(-INFINITY);
  c.U = c.rd = c.rf = c.Dd = c.Da = T(0.f);
  c.rp = c.rn = c.Dp = c.Dn = zero3t<T>();
}

template <class T>
__device__ __forceinline__ void part_from_contact(PartT<T>& c, T f, T dc, V3T<T> p, V3T<T> g,
                                                  float c_blend) {
  if (val(f) > 0.f) {
    c.M = dc * (-c_blend);
    c.U = f;
    c.rd = dc;
    c.rf = f;
    c.rp = p;
    c.rn = g;
    c.Dd = c.Da = T(0.f);
    c.Dp = c.Dn = zero3t<T>();
  } else {
    part_zero(c);
  }
}

template <class T> __device__ __forceinline__ V3T<T> axpy3(T a, V3T<T> x, V3T<T> y) {
  return v3(fma_t(a, x.x, y.x), fma_t(a, x.y, y.y), fma_t(a, x.z, y.z));
}
template <class T> __device__ __forceinline__ V3T<T> sub3(V3T<T> a, V3T<T> b) {
  return v3(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <class T> __device__ __forceinline__ V3T<T> scale3(T a, V3T<T> x) {
  return v3(a * x.x, a * x.y, a * x.z);
}

// a <- a (+) b; the reference of the partial with the larger logit is kept
// (a's on ties), the other's differences are re-based onto it
template <class T> __device__ __forceinline__ void part_combine(PartT<T>& a, const PartT<T>& b) {
  if (val(b.M) == -INFINITY) return;
  if (val(a.M) == -INFINITY) { a = b; return; }
  const bool keep_a = val(a.M) >= val(b.M);
  const PartT<T>& H = keep_a ? a : b;   // keeps its reference
  const PartT<T>& O = keep_a ? b : a;   // re-based
  const T rO = ex2_t(O.M - H.M);
  const T uO = O.U * rO;
  PartT<T> r;
  r.M = H.M;
  r.rd = H.rd; r.rf = H.rf; r.rp = H.rp; r.rn = H.rn;
  r.U = H.U + uO;
  r.Dd = fma_t(rO, O.Dd, fma_t(uO, O.rd - H.rd, H.Dd));
  r.Da = fma_t(rO, O.Da, fma_t(uO, O.rf - H.rf, H.Da));
  r.Dp = axpy3(rO, O.Dp, axpy3(uO, sub3(O.rp, H.rp), H.Dp));
  r.Dn = axpy3(rO, O.Dn, axpy3(uO, sub3(O.rn, H.rn), H.Dn));
  a = r;
}

// folds the contacts k0 <= k < k1 of a value array [*, 8] (f, d_c, p, n) into
// acc in index order, one at a time; the values of kBatch contacts are loaded
// before the first of them is folded, so that a long group waits on one load
// latency per batch instead of one per contact (the order of the arithmetic,
// hence the result, is that of the plain loop)
template <class T>
__device__ __forceinline__ void fold_one(const T* c, float c_blend, PartT<T>& acc) {
  PartT<T> q;
  part_from_contact(q, c[0], c[1], v3(c[2], c[3], c[4]), v3(c[5], c[6], c[7]), c_blend);
  part_combine(acc, q);
}
template <class T>
__device__ __forceinline__ void fold_range(const T* cval, int64_t k0, int64_t k1, float c_blend,
                                           PartT<T>& acc) {
  constexpr int kBatch = sizeof(T) == 4 ? 4 : 2;
  int64_t k = k0;
  for (; k + kBatch <= k1; k += kBatch) {
    T v[kBatch][8];
#pragma unroll
    for (int b = 0; b < kBatch; ++b)
#pragma unroll
      for (int q = 0; q < 8; ++q) v[b][q] = cval[8 * (k + b) + q];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) fold_one(v[b], c_blend, acc);
  }
  for (; k < k1; ++k) fold_one(cval + 8 * k, c_blend, acc);
}

__device__ __forceinline__ float shfl_down_t(float v, int o) { return __shfl_down_sync(kFull, v, o); }
__device__ __forceinline__ Dual shfl_down_t(Dual v, int o) {
  return Dual(__shfl_down_sync(kFull, v.v, o), __shfl_down_sync(kFull, v.d, o));
}
__device__ __forceinline__ float shfl_xor_t(float v, int o) { return __shfl_xor_sync(kFull, v, o); }
__device__ __forceinline__ Dual shfl_xor_t(Dual v, int o) {
  return Dual(__shfl_xor_sync(kFull, v.v, o), __shfl_xor_sync(kFull, v.d, o));
}
template <class T> __device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor_t(v, o);
  return v;
}

template <class T> __device__ __forceinline__ V3T<T> shfl_down3(V3T<T> x, int o) {
  return v3(shfl_down_t(x.x, o), shfl_down_t(x.y, o), shfl_down_t(x.z, o));
}
template <class T> __device__ __forceinline__ PartT<T> part_shfl_down(const PartT<T>& c, int o) {
  PartT<T> r;
  r.M = shfl_down_t(c.M, o); r.U = shfl_down_t(c.U, o);
  r.rd = shfl_down_t(c.rd, o); r.rf = shfl_down_t(c.rf, o);
  r.rp = shfl_down3(c.rp, o); r.rn = shfl_down3(c.rn, o);
  r.Dd = shfl_down_t(c.Dd, o); r.Da = shfl_down_t(c.Da, o);
  r.Dp = shfl_down3(c.Dp, o); r.Dn = shfl_down3(c.Dn, o);
  return r;
}

template <class T> __device__ __forceinline__ V3T<T> shfl_xor3(V3T<T> x, int o) {
  return v3(shfl_xor_t(x.x, o), shfl_xor_t(x.y, o), shfl_xor_t(x.z, o));
}
template <class T> __device__ __forceinline__ PartT<T> part_shfl_xor(const PartT<T>& c, int o) {
  PartT<T> r;
  r.M = shfl_xor_t(c.M, o); r.U = shfl_xor_t(c.U, o);
  r.rd = shfl_xor_t(c.rd, o); r.rf = shfl_xor_t(c.rf, o);
  r.rp = shfl_xor3(c.rp, o); r.rn = shfl_xor3(c.rn, o);
  r.Dd = shfl_xor_t(c.Dd, o); r.Da = shfl_xor_t(c.Da, o);
  r.Dp = shfl_xor3(c.Dp, o); r.Dn = shfl_xor3(c.Dn, o);
  return r;
}

// Folds one group's vertex contacts [v0, v1) and then its edge contacts
// [e0, e1) over kSplit consecutive lanes (an aligned lane group): lane `sub`
// folds every kSplit-th contact of that sequence, in order, with kBatch
// contacts' values loaded at a time; the lanes' partials are then combined
// pairwise in lane order ((0 with 1), (2 with 3), then the pairs), the same
// operations on every lane of the group, so all of them end with the same
// partial.  The chain of dependent blends of a long group is kSplit times
// shorter than one lane's fold.  Every lane of the warp calls it (an empty
// range gives an empty partial).
template <class T, int kSplit>
__device__ void fold_split(const T* cval, int64_t v0, int64_t v1, int64_t e0, int64_t e1,
                           float c_blend, int sub, PartT<T>& acc) {
  constexpr int kBatch = sizeof(T) == 4 ? 4 : 2;
  part_zero(acc);
  const int64_t nv = v1 - v0, n = nv + (e1 - e0);
  auto at = [&](int64_t t) { return t < nv ? v0 + t : e0 + (t - nv); };
  int64_t t = sub;
  for (; t + (kBatch - 1) * kSplit < n; t += kBatch * kSplit) {
    T v[kBatch][8];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const T* c = cval + 8 * at(t + b * kSplit);
#pragma unroll
      for (int q = 0; q < 8; ++q) v[b][q] = c[q];
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) fold_one(v[b], c_blend, acc);
  }
  for (; t < n; t += kSplit) fold_one(cval + 8 * at(t), c_blend, acc);
#pragma unroll
  for (int o = 1; o < kSplit; o <<= 1) {
    const PartT<T> other = part_shfl_xor(acc, o);
    if (sub & o) {   // the lower lanes' partial first
      PartT<T> lo = other;
      part_combine(lo, acc);
      acc = lo;
    } else {
      part_combine(acc, other);
    }
  }
}

// segmented fold of lane contacts sorted by key into the group table
template <class T>
__device__ void fold_t(PartT<T> c, int key, PartT<T>* acc, int lane) {
  const unsigned seg = __match_any_sync(kFull, key);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const PartT<T> b = part_shfl_down(c, o);
    if (lane + o < 32 && ((seg >> (lane + o)) & 1u)) part_combine(c, b);
  }
  if ((__ffs(seg) - 1) == lane && key != 0xffff && val(c.M) != -INFINITY) {
    PartT<T> g = acc[key];
    part_combine(g, c);
    acc[key] = g;
  }
}

// A direction (feature piece f of a chunk, SDF piece s < kHitS) is marked
// when it produced a contact of non-zero weight.  A direction without such a
// contact contributes nothing to a group's blend nor to its adjoint (f = 0
// there, and f' = f'' = 0 at the gate's knot), so later passes visit only the
// marked ones; directions with s >= kHitS are re-gated.
constexpr int kHitS = 256;
constexpr int kHitWords = kHitS / 32;

// The hit table in shared memory keeps hw <= kHitWords words per group (as
// many as the largest SDF body needs).  A negative sg (a caller that gates by
// hits it already has) marks nothing.
__device__ __forceinline__ void mark_hit(uint32_t* hit, int hw, int g, int sg, float w) {
  if (w > 0.f && sg >= 0 && sg < 32 * hw) atomicOr(hit + g * hw + (sg >> 5), 1u << (sg & 31));
}

// What ccm_contacts_save keeps per output group for the reverse pass: the
// group's blend partial (18 floats: M, U, rd, rf, rp, rn, Dd, Da, Dp, Dn), its
// hit words (kHitWords uint32, stored bit for bit; words past the
// shared-memory table's hw are zero), the tag of the contact list the same
// forward kept (uint32; 0: none) and one zero word.
constexpr int kSavedFloats = 18 + kHitWords + 2;
constexpr int kSavedTag = 18 + kHitWords;

__device__ __forceinline__ void save_group(float* o, const PartT<float>& a, const uint32_t* hit,
                                           int hw, uint32_t tag) {
  o[0] = a.M; o[1] = a.U; o[2] = a.rd; o[3] = a.rf;
  o[4] = a.rp.x; o[5] = a.rp.y; o[6] = a.rp.z; o[7] = a.rn.x; o[8] = a.rn.y; o[9] = a.rn.z;
  o[10] = a.Dd; o[11] = a.Da;
  o[12] = a.Dp.x; o[13] = a.Dp.y; o[14] = a.Dp.z; o[15] = a.Dn.x; o[16] = a.Dn.y; o[17] = a.Dn.z;
  uint32_t* h = reinterpret_cast<uint32_t*>(o + 18);
  for (int q = 0; q < kHitWords; ++q) h[q] = q < hw ? hit[q] : 0u;
  h[kHitWords] = tag;
  h[kHitWords + 1] = 0u;
}

}  // namespace ccm
