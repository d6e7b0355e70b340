// FP64 CPU oracle for one-shot smooth contact manifolds between convex-decomposed
// bodies (arxiv 2604.17538).  TEST INFRASTRUCTURE: only the tests, the smoke
// check and the benchmark's CPU-baseline leg load this library; the product path
// never does.  It shares no code with the CUDA path.
//
// Plain, slow and written to be checked against the paper by eye.  Every value
// is computed in double precision, step by step in the paper's order:
//   Sec. 2  smooth operators: sigmoid, softplus, softclip, LSE, softmax.
//   Sec. 3  PSQ SDF: smooth intersection (Eq. smooth-intersection) of the
//           half-space SDFs phi_k = n_k.x + h_k of one convex piece.
//   Sec. 4.2 V-SDF contacts (vertex = contact point) and E-SDF contacts found
//           by sphere tracing both edge corners towards each other, soft
//           clipping to the edge and taking the midpoint.
//   Sec. 4.3 mollification: d_c = f phi + (1 - f) d_max with a C^2 transition f.
//   Sec. 4.4 blending of the contacts of one convex piece (CP group).
//
// Readings where the paper is silent (each is a named choice):
//   * piece SDF = LSE over the face planes only (no superquadric term);
//   * sphere-trace gate [[phi > 0]] softened to sigmoid(phi / tau_trace);
//   * the soft clip acts on the edge parameter alpha in [0, L];
//   * transition f_t = quintic smoothstep of s = (d_max - d) / eps on [0, 1];
//   * blend weights w_c = f_c exp(-d_c/tau_blend) / sum(f exp(-d/tau_blend));
//     group outputs d = sum w d_c, a = sum w f_c, p = sum w p_c,
//     n = normalize(sum w grad phi); a group without active contact returns
//     (d_max, 0, 0, 0);
//   * a group is one convex piece of one body; its contacts are all its
//     vertices and edges against every convex piece of the other body;
//   * outputs are in world frame, normals point out of the SDF body;
//   * pose derivatives use the twist chart R <- Exp(w) R, t <- t + v per body.
//
// Variants selected by ccmo_params.flags (forward values only):
//   * kFlagBodyUnion: the SDF of the other body is the smooth union
//     (Sec. 3.1, Eq. soft_union) of its pieces' SDFs,
//     phi_S(x) = -tau LSE(-phi_s(x) / tau) over the pieces s, with the same
//     softness tau_sdf, and every feature of a group gives one contact
//     against the whole body instead of one per piece;
//   * kFlagProject: every contact point is moved onto the SDF's isosurface
//     (Sec. 4.1), proj(p) = p - phi(p) n(p) with n the contact normal (grad
//     phi, or the normal spline), after its depth and normal were taken at p;
//   * kFlagSpline: every SDF piece is a tricubic spline (Sec. 3.2): the SDF
//     and the three normal components are each a tensor-product cubic spline
//     on the piece's voxel grid, s(x) = sum c_{kx,ky,kz} u(.) u(.) u(.) with
//     the paper's basis u (support [-2, 2]); the contact normal is the normal
//     spline, not the SDF's gradient.  Outside the grid box the SDF continues
//     as the spline at the nearest box point plus the distance to the box.
//   * kFlagUngated: the literal reading of "softmax on {d_c}" in Sec. 4.4,
//     for comparison with the gated blend above: w_c = exp(-d_c/tau_blend) /
//     sum exp(-d/tau_blend) over EVERY contact of the group, including those
//     with f_c = 0 (whose mollified depth is exactly d_max); the outputs are
//     the same sums with these weights, so no group is ever empty.
//
// Derivatives: the same templated code runs on forward-mode dual numbers.
// Dual<double,12> gives the exact gradient with respect to the 12 twist
// coordinates of a pair; Dual<Dual<double,1>,12> gives, in one pass, the
// gradient, the Hessian-vector product H u and the output tangents J u.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace ccmo {

// --------------------------------------------------------------------------
// forward-mode dual numbers (nestable: S may itself be a Dual)
// --------------------------------------------------------------------------
template <class S, int N>
struct Dual {
  S v;
  S d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = S(0.0); }
  Dual(double c) : v(c) { for (int i = 0; i < N; ++i) d[i] = S(0.0); }
  Dual(const S& c, int) : v(c) { for (int i = 0; i < N; ++i) d[i] = S(0.0); }
};

inline double val(double x) { return x; }
template <class S, int N> inline double val(const Dual<S, N>& x) { return val(x.v); }

template <class S, int N>
inline Dual<S, N> operator+(const Dual<S, N>& a, const Dual<S, N>& b) {
  Dual<S, N> r; r.v = a.v + b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class S, int N>
inline Dual<S, N> operator-(const Dual<S, N>& a, const Dual<S, N>& b) {
  Dual<S, N> r; r.v = a.v - b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class S, int N>
inline Dual<S, N> operator-(const Dual<S, N>& a) {
  Dual<S, N> r; r.v = -a.v;
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class S, int N>
inline Dual<S, N> operator*(const Dual<S, N>& a, const Dual<S, N>& b) {
  Dual<S, N> r; r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.v * b.d[i] + a.d[i] * b.v;
  return r;
}
template <class S, int N>
inline Dual<S, N> operator/(const Dual<S, N>& a, const Dual<S, N>& b) {
  Dual<S, N> r; r.v = a.v / b.v;
  S inv2 = S(1.0) / (b.v * b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) * inv2;
  return r;
}
template <class S, int N> inline Dual<S, N> operator+(const Dual<S, N>& a, double b) { return a + Dual<S, N>(b); }
template <class S, int N> inline Dual<S, N> operator+(double a, const Dual<S, N>& b) { return Dual<S, N>(a) + b; }
template <class S, int N> inline Dual<S, N> operator-(const Dual<S, N>& a, double b) { return a - Dual<S, N>(b); }
template <class S, int N> inline Dual<S, N> operator-(double a, const Dual<S, N>& b) { return Dual<S, N>(a) - b; }
template <class S, int N> inline Dual<S, N> operator*(const Dual<S, N>& a, double b) {
  Dual<S, N> r; r.v = a.v * b;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <class S, int N> inline Dual<S, N> operator*(double a, const Dual<S, N>& b) { return b * a; }
template <class S, int N> inline Dual<S, N> operator/(const Dual<S, N>& a, double b) { return a * (1.0 / b); }
template <class S, int N> inline Dual<S, N> operator/(double a, const Dual<S, N>& b) { return Dual<S, N>(a) / b; }
template <class S, int N> inline Dual<S, N>& operator+=(Dual<S, N>& a, const Dual<S, N>& b) { a = a + b; return a; }

// f(x) for a dual x given f(x.v) and f'(x.v)
template <class S, int N>
inline Dual<S, N> chain(const Dual<S, N>& x, const S& fx, const S& dfx) {
  Dual<S, N> r; r.v = fx;
  for (int i = 0; i < N; ++i) r.d[i] = dfx * x.d[i];
  return r;
}
using std::exp; using std::log; using std::log1p; using std::sqrt; using std::sin; using std::cos;
template <class S, int N> inline Dual<S, N> exp(const Dual<S, N>& x) { S e = exp(x.v); return chain(x, e, e); }
template <class S, int N> inline Dual<S, N> log(const Dual<S, N>& x) { return chain(x, log(x.v), S(1.0) / x.v); }
template <class S, int N> inline Dual<S, N> log1p(const Dual<S, N>& x) { return chain(x, log1p(x.v), S(1.0) / (S(1.0) + x.v)); }
template <class S, int N> inline Dual<S, N> sqrt(const Dual<S, N>& x) { S s = sqrt(x.v); return chain(x, s, S(0.5) / s); }
template <class S, int N> inline Dual<S, N> sin(const Dual<S, N>& x) { return chain(x, sin(x.v), cos(x.v)); }
template <class S, int N> inline Dual<S, N> cos(const Dual<S, N>& x) { return chain(x, cos(x.v), -sin(x.v)); }

// --------------------------------------------------------------------------
// small vector algebra
// --------------------------------------------------------------------------
template <class T> struct V3 { T x, y, z; };
template <class T> inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> inline V3<T> operator*(const T& s, const V3<T>& a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> inline V3<T> scale(double s, const V3<T>& a) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> zero3() { return {T(0.0), T(0.0), T(0.0)}; }

// rigid pose x_w = R x + t, R row-major
template <class T> struct Pose { T R[9]; T t[3]; };
template <class T> inline V3<T> apply(const Pose<T>& P, const V3<T>& x) {
  return {P.R[0] * x.x + P.R[1] * x.y + P.R[2] * x.z + P.t[0],
          P.R[3] * x.x + P.R[4] * x.y + P.R[5] * x.z + P.t[1],
          P.R[6] * x.x + P.R[7] * x.y + P.R[8] * x.z + P.t[2]};
}
template <class T> inline V3<T> rotate(const Pose<T>& P, const V3<T>& x) {
  return {P.R[0] * x.x + P.R[1] * x.y + P.R[2] * x.z,
          P.R[3] * x.x + P.R[4] * x.y + P.R[5] * x.z,
          P.R[6] * x.x + P.R[7] * x.y + P.R[8] * x.z};
}
// body-frame coordinates of a world point: R^T (x_w - t)
template <class T> inline V3<T> apply_inverse(const Pose<T>& P, const V3<T>& xw) {
  V3<T> d = {xw.x - P.t[0], xw.y - P.t[1], xw.z - P.t[2]};
  return {P.R[0] * d.x + P.R[3] * d.y + P.R[6] * d.z,
          P.R[1] * d.x + P.R[4] * d.y + P.R[7] * d.z,
          P.R[2] * d.x + P.R[5] * d.y + P.R[8] * d.z};
}

// twist chart: R(xi) = Exp([w]x) R0, t(xi) = t0 + v; Exp by Rodrigues' formula,
// Exp = I + a [w]x + b [w]x^2 with a = sin(th)/th, b = (1 - cos th)/th^2
// (Taylor series in th^2 near zero so that derivatives at xi = 0 are exact).
template <class T>
Pose<T> twisted(const double* pose12, const T* w, const T* v) {
  T th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  T a, b;
  if (val(th2) < 1e-6) {
    a = 1.0 - th2 * (1.0 / 6.0) + th2 * th2 * (1.0 / 120.0);
    b = 0.5 - th2 * (1.0 / 24.0) + th2 * th2 * (1.0 / 720.0);
  } else {
    T th = sqrt(th2);
    a = sin(th) / th;
    b = (1.0 - cos(th)) / th2;
  }
  // K = [w]x
  T K[9] = {T(0.0), -w[2], w[1], w[2], T(0.0), -w[0], -w[1], w[0], T(0.0)};
  T E[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T k2 = K[3 * i + 0] * K[0 + j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
      E[3 * i + j] = (i == j ? T(1.0) : T(0.0)) + a * K[3 * i + j] + b * k2;
    }
  Pose<T> P;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      P.R[3 * i + j] = E[3 * i + 0] * pose12[0 + j] + E[3 * i + 1] * pose12[3 + j] + E[3 * i + 2] * pose12[6 + j];
  for (int i = 0; i < 3; ++i) P.t[i] = pose12[9 + i] + v[i];
  return P;
}

// --------------------------------------------------------------------------
// inputs
// --------------------------------------------------------------------------
}  // namespace ccmo

extern "C" {
struct ccmo_params {
  double tau_sdf;     // LSE softness of the piece SDF (Sec. 3)
  double tau_trace;   // softness of the sphere-trace gate [[phi > 0]] (Sec. 4.2)
  double tau_clip;    // softness of the edge soft clip (Sec. 4.2)
  double tau_blend;   // softmax temperature of the blend (Sec. 4.4)
  double d_max;       // distance threshold (Sec. 4.3)
  double gate_width;  // transition bandwidth epsilon (Sec. 4.3)
  int32_t trace_iters;  // sphere-trace iterations (three in Sec. 4.2)
  int32_t flags;      // kFlagBodyUnion | kFlagProject | kFlagSpline | kFlagUngated
};
struct ccmo_geom {
  const int64_t* body_piece_off;
  const int64_t* piece_v_off;
  const int64_t* piece_f_off;
  const int64_t* piece_e_off;
  const double* verts;   // [V,3]
  const double* planes;  // [F,4]
  const int32_t* edges;  // [E,2]
  // tricubic spline SDFs (Sec. 3.2), or NULL: per piece the grid origin and
  // voxel size (ox, oy, oz, h), the voxel counts (nx, ny, nz) and the offset
  // of its coefficients, [(nx+3)(ny+3)(nz+3), 4] rows (phi, n_x, n_y, n_z)
  // with the z index fastest
  const double* spline_grid;    // [P,4]
  const int64_t* spline_dims;   // [P,4]: nx, ny, nz, first coefficient row
  const double* spline_coef;    // [rows,4]
};
}

namespace ccmo {

// --------------------------------------------------------------------------
// Sec. 2: smooth approximations of non-smooth operators
// --------------------------------------------------------------------------
// sigmoid(x) = 1 / (1 + exp(-x)); evaluated without overflow on both sides
template <class T> T sigmoid(const T& x) {
  if (val(x) >= 0.0) return 1.0 / (1.0 + exp(-x));
  T e = exp(x);
  return e / (1.0 + e);
}
// softplus s+(x) = tau log(1 + exp(x / tau)) = max(x, 0) + tau log1p(exp(-|x| / tau))
template <class T> T softplus(const T& x, double tau) {
  if (val(x) >= 0.0) return x + tau * log1p(exp(-x / tau));
  return tau * log1p(exp(x / tau));
}
// softclip(x, lo, hi) = lo + s+(x - lo) - s+(x - hi)
template <class T> T softclip(const T& x, const T& lo, const T& hi, double tau) {
  return lo + softplus(x - lo, tau) - softplus(x - hi, tau);
}

// --------------------------------------------------------------------------
// Sec. 3: SDF of a convex piece = smooth intersection of its half-spaces,
// phi(x) = LSE_tau(phi_1, ..., phi_F),  phi_k = n_k . x + h_k.
// LSE is evaluated max-shifted: m + tau log sum exp((phi_k - m) / tau).
// The gradient is the softmax-weighted sum of the plane normals.
// --------------------------------------------------------------------------
template <class T>
T piece_sdf(const double* planes, int F, const V3<T>& x, double tau, V3<T>* grad) {
  std::vector<T> phik(F);
  int kmax = 0;
  for (int k = 0; k < F; ++k) {
    const double* P = planes + 4 * k;
    phik[k] = x.x * P[0] + x.y * P[1] + x.z * P[2] + P[3];
    if (val(phik[k]) > val(phik[kmax])) kmax = k;
  }
  T m = phik[kmax];
  T S(0.0);
  std::vector<T> e(F);
  for (int k = 0; k < F; ++k) {
    e[k] = exp((phik[k] - m) / tau);
    S = S + e[k];
  }
  T phi = m + tau * log(S);
  if (grad) {
    V3<T> g = zero3<T>();
    for (int k = 0; k < F; ++k) {
      T w = e[k] / S;  // softmax weight s_argmax(phi/.)_k
      const double* P = planes + 4 * k;
      g.x = g.x + w * P[0];
      g.y = g.y + w * P[1];
      g.z = g.z + w * P[2];
    }
    *grad = g;
  }
  return phi;
}

// the SDF of one convex piece as a callable: phi(x) and, if grad, grad phi
struct PieceSdf {
  const double* planes;
  int F;
  double tau;
  template <class T> T operator()(const V3<T>& x, V3<T>* grad) const {
    return piece_sdf(planes, F, x, tau, grad);
  }
};

// --------------------------------------------------------------------------
// Sec. 3.1 Eq. soft_union: smooth union of the pieces of one body,
// phi_S(x) = -tau log sum_s exp(-phi_s(x) / tau), evaluated min-shifted:
// m - tau log sum_s exp(-(phi_s - m) / tau), m = min_s phi_s.  Its gradient
// is the softmin-weighted sum of the pieces' gradients.
// --------------------------------------------------------------------------
constexpr int32_t kFlagBodyUnion = 2;
constexpr int32_t kFlagProject = 4;
constexpr int32_t kFlagSpline = 8;
constexpr int32_t kFlagUngated = 16;

// --------------------------------------------------------------------------
// Sec. 3.2: cubic spline basis u(t) = 4 - 6|t|^2 + 3|t|^3 on |t| <= 1,
// (2 - |t|)^3 on 1 <= |t| <= 2, 0 beyond, and the tricubic spline of one
// piece.  Coefficient k of an axis sits at grid node k - 1 (k = 0..N+2), so
// the nodes i = 0..N and one extra coefficient beyond each end carry the
// N + 3 basis functions of N voxels.
// --------------------------------------------------------------------------
template <class T> T spline_u(const T& t) {
  const T a = val(t) < 0.0 ? -t : t;
  if (val(a) <= 1.0) return 4.0 - 6.0 * a * a + 3.0 * a * a * a;
  if (val(a) <= 2.0) { const T b = 2.0 - a; return b * b * b; }
  return T(0.0);
}

struct SplineSdf {
  const double* grid;   // ox, oy, oz, h
  const int64_t* dims;  // nx, ny, nz, first row
  const double* coef;   // [rows, 4]
  // value of channel ch at t (grid units), t inside [0, N] per axis
  template <class T> T channel(const T t[3], int ch) const {
    int64_t i0[3];
    for (int a = 0; a < 3; ++a) {
      i0[a] = (int64_t)std::floor(val(t[a]));
      if (i0[a] > dims[a] - 1) i0[a] = dims[a] - 1;
      if (i0[a] < 0) i0[a] = 0;
    }
    const int64_t ny = dims[1] + 3, nz = dims[2] + 3;
    T sum(0.0);
    // the 64 coefficients whose basis functions reach t: k = i0 .. i0 + 3
    for (int a = 0; a < 4; ++a) {
      const T ua = spline_u(t[0] - (double)(i0[0] + a - 1));
      for (int b = 0; b < 4; ++b) {
        const T ub = spline_u(t[1] - (double)(i0[1] + b - 1));
        for (int c = 0; c < 4; ++c) {
          const T uc = spline_u(t[2] - (double)(i0[2] + c - 1));
          const int64_t row = dims[3] + ((i0[0] + a) * ny + (i0[1] + b)) * nz + (i0[2] + c);
          sum = sum + coef[4 * row + ch] * (ua * ub * uc);
        }
      }
    }
    return sum;
  }
  template <class T> T operator()(const V3<T>& x, V3<T>* normal) const {
    // grid units, clamped to the grid box; the distance to the box is added
    const T xs[3] = {x.x, x.y, x.z};
    T t[3], out2(0.0);
    for (int a = 0; a < 3; ++a) {
      const T u = (xs[a] - grid[a]) / grid[3];
      const double hi = (double)dims[a];
      if (val(u) < 0.0) { out2 = out2 + u * u; t[a] = T(0.0); }
      else if (val(u) > hi) { out2 = out2 + (u - hi) * (u - hi); t[a] = T(hi); }
      else t[a] = u;
    }
    T phi = channel(t, 0);
    if (val(out2) > 0.0) phi = phi + grid[3] * sqrt(out2);
    if (normal) *normal = V3<T>{channel(t, 1), channel(t, 2), channel(t, 3)};
    return phi;
  }
};

struct BodyUnionSdf {
  const ccmo_geom* G;
  int64_t body;
  double tau;
  template <class T> T operator()(const V3<T>& x, V3<T>* grad) const {
    const int64_t s0 = G->body_piece_off[body], s1 = G->body_piece_off[body + 1];
    std::vector<T> phis;
    std::vector<V3<T>> gs;
    int smin = 0;
    for (int64_t s = s0; s < s1; ++s) {
      V3<T> g;
      const double* planes = G->planes + 4 * G->piece_f_off[s];
      const int F = (int)(G->piece_f_off[s + 1] - G->piece_f_off[s]);
      phis.push_back(piece_sdf(planes, F, x, tau, grad ? &g : nullptr));
      gs.push_back(g);
      if (val(phis.back()) < val(phis[smin])) smin = (int)phis.size() - 1;
    }
    T m = phis[smin];
    T S(0.0);
    std::vector<T> e(phis.size());
    for (size_t k = 0; k < phis.size(); ++k) {
      e[k] = exp(-(phis[k] - m) / tau);
      S = S + e[k];
    }
    if (grad) {
      V3<T> g = zero3<T>();
      for (size_t k = 0; k < phis.size(); ++k) g = g + (e[k] / S) * gs[k];
      *grad = g;
    }
    return m - tau * log(S);
  }
};

// --------------------------------------------------------------------------
// Sec. 4.3: C^2 non-increasing transition, 1 for d <= d_max - eps, 0 for d >= d_max
// --------------------------------------------------------------------------
template <class T> T transition(const T& d, double d_max, double eps) {
  T s = (d_max - d) / eps;
  if (val(s) <= 0.0) return T(0.0);
  if (val(s) >= 1.0) return T(1.0);
  return s * s * s * (10.0 - 15.0 * s + 6.0 * s * s);
}

template <class T> struct Contact {
  T phi, f, dc;   // SDF value, transition weight, mollified depth
  V3<T> p;        // contact point, SDF body frame
  V3<T> n;        // grad phi at p, SDF body frame
};

template <class T>
void mollify(Contact<T>& c, const ccmo_params& prm) {
  c.f = transition(c.phi, prm.d_max, prm.gate_width);
  c.dc = c.f * c.phi + (1.0 - c.f) * prm.d_max;
}

// --------------------------------------------------------------------------
// Sec. 4.2: narrow phase
// --------------------------------------------------------------------------
// Sec. 4.1 isosurface projection of a contact point: p - phi(p) n(p)
template <class T>
void project(Contact<T>& c, const ccmo_params& prm) {
  if (prm.flags & kFlagProject) c.p = c.p - c.phi * c.n;
}

// V-SDF: the vertex itself is the contact point
template <class T, class Sdf>
Contact<T> vertex_contact(const Sdf& sdf, const V3<T>& x, const ccmo_params& prm) {
  Contact<T> c;
  c.p = x;
  c.phi = sdf(x, &c.n);
  mollify(c, prm);
  project(c, prm);
  return c;
}

// E-SDF: sphere trace corner v_I along +e_t and corner v_II along -e_t,
//   p_{k+1} = p_k +/- sigmoid(phi(p_k)/tau_trace) phi(p_k) e_t,
// soft clip both traced points to the edge, and take their midpoint p^e.
template <class T, class Sdf>
V3<T> edge_point(const Sdf& sdf, const V3<T>& vI, const V3<T>& vII,
                 const ccmo_params& prm, T* alpha_out = nullptr) {
  V3<T> dv = vII - vI;
  T L = sqrt(dot(dv, dv));
  V3<T> et = (1.0 / L) * dv;
  V3<T> pI = vI, pII = vII;
  for (int k = 0; k < prm.trace_iters; ++k) {
    T phiI = sdf(pI, (V3<T>*)nullptr);
    T phiII = sdf(pII, (V3<T>*)nullptr);
    pI = pI + (sigmoid(phiI / prm.tau_trace) * phiI) * et;
    pII = pII - (sigmoid(phiII / prm.tau_trace) * phiII) * et;
  }
  // positions along the edge, clipped softly to [0, L]
  T aI = dot(pI - vI, et);
  T aII = dot(pII - vI, et);
  T cI = softclip(aI, T(0.0), L, prm.tau_clip);
  T cII = softclip(aII, T(0.0), L, prm.tau_clip);
  if (alpha_out) { alpha_out[0] = aI; alpha_out[1] = aII; alpha_out[2] = cI; alpha_out[3] = cII; }
  // midpoint of the two clipped points
  return vI + (0.5 * (cI + cII)) * et;
}

template <class T, class Sdf>
Contact<T> edge_contact(const Sdf& sdf, const V3<T>& vI, const V3<T>& vII,
                        const ccmo_params& prm) {
  Contact<T> c;
  c.p = edge_point(sdf, vI, vII, prm);
  c.phi = sdf(c.p, &c.n);
  mollify(c, prm);
  project(c, prm);
  return c;
}

// --------------------------------------------------------------------------
// Sec. 4.4: blending of all contacts of one CP group
// --------------------------------------------------------------------------
template <class T> struct Group { T d, a; V3<T> p, n; };

template <class T>
Group<T> blend(const std::vector<Contact<T>>& cs, const std::vector<V3<T>>& pw,
               const std::vector<V3<T>>& nw, const ccmo_params& prm) {
  Group<T> g;
  // logits l_c = -d_c / tau_blend over contacts with f_c > 0 (every contact
  // for the ungated reading), max-shifted
  const bool gated = !(prm.flags & kFlagUngated);
  int cmax = -1;
  for (size_t c = 0; c < cs.size(); ++c)
    if ((!gated || val(cs[c].f) > 0.0) && (cmax < 0 || val(cs[c].dc) < val(cs[cmax].dc)))
      cmax = (int)c;
  if (cmax < 0) {  // no active contact
    g.d = T(prm.d_max); g.a = T(0.0); g.p = zero3<T>(); g.n = zero3<T>();
    return g;
  }
  T M = -cs[cmax].dc / prm.tau_blend;
  T U(0.0), D(0.0), A(0.0);
  V3<T> P = zero3<T>(), N = zero3<T>();
  for (size_t c = 0; c < cs.size(); ++c) {
    if (gated && !(val(cs[c].f) > 0.0)) continue;
    T u = exp(-cs[c].dc / prm.tau_blend - M);
    if (gated) u = cs[c].f * u;
    U = U + u;
    D = D + u * cs[c].dc;
    A = A + u * cs[c].f;
    P = P + u * pw[c];
    N = N + u * nw[c];
  }
  g.d = D / U;
  g.a = A / U;
  g.p = (1.0 / U) * P;
  V3<T> nb = (1.0 / U) * N;
  T nn = dot(nb, nb);
  if (val(nn) > 0.0) g.n = (1.0 / sqrt(nn)) * nb;
  else g.n = zero3<T>();
  return g;
}

// all contacts of the CP group "feature piece fp of body F" against every SDF
// piece of body S; contact points and normals are returned in world frame
template <class T>
void group_contacts(const ccmo_geom& G, int64_t fp, const Pose<T>& PF, int64_t bodyS,
                    const Pose<T>& PS, const ccmo_params& prm, std::vector<Contact<T>>& cs,
                    std::vector<V3<T>>& pw, std::vector<V3<T>>& nw) {
  const int64_t v0 = G.piece_v_off[fp], nv = G.piece_v_off[fp + 1] - v0;
  const int64_t e0 = G.piece_e_off[fp], ne = G.piece_e_off[fp + 1] - e0;
  // feature vertices in world frame
  std::vector<V3<T>> xw(nv);
  for (int64_t i = 0; i < nv; ++i) {
    const double* v = G.verts + 3 * (v0 + i);
    xw[i] = apply(PF, V3<T>{T(v[0]), T(v[1]), T(v[2])});
  }
  // the features in the SDF body frame
  std::vector<V3<T>> x(nv);
  for (int64_t i = 0; i < nv; ++i) x[i] = apply_inverse(PS, xw[i]);
  if (prm.flags & kFlagBodyUnion) {
    // one contact per feature against the smooth union of body S's pieces
    const BodyUnionSdf sdf{&G, bodyS, prm.tau_sdf};
    for (int64_t i = 0; i < nv; ++i) cs.push_back(vertex_contact(sdf, x[i], prm));
    for (int64_t j = 0; j < ne; ++j) {
      const int32_t* e = G.edges + 2 * (e0 + j);
      cs.push_back(edge_contact(sdf, x[e[0]], x[e[1]], prm));
    }
  } else if (prm.flags & kFlagSpline) {
    // every SDF piece as its tricubic spline (Sec. 3.2)
    for (int64_t s = G.body_piece_off[bodyS]; s < G.body_piece_off[bodyS + 1]; ++s) {
      const SplineSdf sdf{G.spline_grid + 4 * s, G.spline_dims + 4 * s, G.spline_coef};
      for (int64_t i = 0; i < nv; ++i) cs.push_back(vertex_contact(sdf, x[i], prm));
      for (int64_t j = 0; j < ne; ++j) {
        const int32_t* e = G.edges + 2 * (e0 + j);
        cs.push_back(edge_contact(sdf, x[e[0]], x[e[1]], prm));
      }
    }
  } else {
    for (int64_t s = G.body_piece_off[bodyS]; s < G.body_piece_off[bodyS + 1]; ++s) {
      const PieceSdf sdf{G.planes + 4 * G.piece_f_off[s],
                         (int)(G.piece_f_off[s + 1] - G.piece_f_off[s]), prm.tau_sdf};
      for (int64_t i = 0; i < nv; ++i) cs.push_back(vertex_contact(sdf, x[i], prm));
      for (int64_t j = 0; j < ne; ++j) {
        const int32_t* e = G.edges + 2 * (e0 + j);
        cs.push_back(edge_contact(sdf, x[e[0]], x[e[1]], prm));
      }
    }
  }
  for (auto& c : cs) {
    V3<T> q = apply(PS, c.p);
    pw.push_back(q);
    nw.push_back(rotate(PS, c.n));
  }
}

// the N_A + N_B groups of one body pair: first A's pieces (features of A
// against the SDF pieces of B), then B's pieces (features of B against A)
template <class T>
void pair_groups(const ccmo_geom& G, int64_t bA, int64_t bB, const Pose<T>& PA,
                 const Pose<T>& PB, const ccmo_params& prm, std::vector<Group<T>>& out) {
  for (int side = 0; side < 2; ++side) {
    const int64_t bF = side == 0 ? bA : bB, bS = side == 0 ? bB : bA;
    const Pose<T>& PF = side == 0 ? PA : PB;
    const Pose<T>& PS = side == 0 ? PB : PA;
    for (int64_t fp = G.body_piece_off[bF]; fp < G.body_piece_off[bF + 1]; ++fp) {
      std::vector<Contact<T>> cs;
      std::vector<V3<T>> pw, nw;
      group_contacts(G, fp, PF, bS, PS, prm, cs, pw, nw);
      out.push_back(blend(cs, pw, nw, prm));
    }
  }
}

template <class T> inline void store8(const Group<T>& g, T* y) {
  y[0] = g.d; y[1] = g.a;
  y[2] = g.p.x; y[3] = g.p.y; y[4] = g.p.z;
  y[5] = g.n.x; y[6] = g.n.y; y[7] = g.n.z;
}

template <class T> Pose<T> const_pose(const double* p12) {
  Pose<T> P;
  for (int i = 0; i < 9; ++i) P.R[i] = T(p12[i]);
  for (int i = 0; i < 3; ++i) P.t[i] = T(p12[9 + i]);
  return P;
}

inline int nthreads(int t) {
#ifdef _OPENMP
  return t > 0 ? t : omp_get_max_threads();
#else
  (void)t; return 1;
#endif
}

}  // namespace ccmo

using namespace ccmo;

extern "C" {

// y[G,8] = (d, a, p_x, p_y, p_z, n_x, n_y, n_z) for every group of every pair
int ccmo_forward(const ccmo_geom* G, int64_t n, const int64_t* pa, const int64_t* pb,
                 const double* pose_a, const double* pose_b, const ccmo_params* prm,
                 const int64_t* goff, double* y, int threads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads(threads))
  for (int64_t i = 0; i < n; ++i) {
    std::vector<Group<double>> out;
    pair_groups(*G, pa[i], pb[i], const_pose<double>(pose_a + 12 * i),
                const_pose<double>(pose_b + 12 * i), *prm, out);
    for (size_t g = 0; g < out.size(); ++g) store8(out[g], y + 8 * (goff[i] + g));
  }
  return 0;
}

// gradient of L = <ybar, y> with respect to the twists (w_A, v_A, w_B, v_B)
// of every pair, evaluated at Exp(xi) T (xi = 0 when xi == NULL)
int ccmo_gradient(const ccmo_geom* G, int64_t n, const int64_t* pa, const int64_t* pb,
                  const double* pose_a, const double* pose_b, const ccmo_params* prm,
                  const int64_t* goff, const double* ybar, const double* xi, double* grad,
                  double* y, int threads) {
  typedef Dual<double, 12> D;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads(threads))
  for (int64_t i = 0; i < n; ++i) {
    D z[12];
    for (int k = 0; k < 12; ++k) {
      z[k] = D(xi ? xi[12 * i + k] : 0.0);
      z[k].d[k] = 1.0;
    }
    Pose<D> PA = twisted<D>(pose_a + 12 * i, z + 0, z + 3);
    Pose<D> PB = twisted<D>(pose_b + 12 * i, z + 6, z + 9);
    std::vector<Group<D>> out;
    pair_groups(*G, pa[i], pb[i], PA, PB, *prm, out);
    D L(0.0);
    for (size_t g = 0; g < out.size(); ++g) {
      D yy[8];
      store8(out[g], yy);
      for (int k = 0; k < 8; ++k) {
        L = L + yy[k] * ybar[8 * (goff[i] + g) + k];
        if (y) y[8 * (goff[i] + g) + k] = yy[k].v;
      }
    }
    for (int k = 0; k < 12; ++k) grad[12 * i + k] = L.d[k];
  }
  return 0;
}

// one pass of nested duals at xi = 0: gradient g, Hessian-vector product H u of
// L = <ybar, y> in the twist chart (Hessian of L(Exp(xi) T) at xi = 0) and the
// output tangents J u; any output pointer may be NULL
int ccmo_hvp(const ccmo_geom* G, int64_t n, const int64_t* pa, const int64_t* pb,
             const double* pose_a, const double* pose_b, const ccmo_params* prm,
             const int64_t* goff, const double* ybar, const double* u, double* grad,
             double* hvp, double* jvp, double* y, int threads) {
  typedef Dual<double, 1> S;
  typedef Dual<S, 12> D;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads(threads))
  for (int64_t i = 0; i < n; ++i) {
    D z[12];
    for (int k = 0; k < 12; ++k) {
      S base(0.0);
      base.d[0] = u[12 * i + k];
      z[k] = D(base, 0);
      z[k].d[k] = S(1.0);
    }
    Pose<D> PA = twisted<D>(pose_a + 12 * i, z + 0, z + 3);
    Pose<D> PB = twisted<D>(pose_b + 12 * i, z + 6, z + 9);
    std::vector<Group<D>> out;
    pair_groups(*G, pa[i], pb[i], PA, PB, *prm, out);
    D L(0.0);
    for (size_t g = 0; g < out.size(); ++g) {
      D yy[8];
      store8(out[g], yy);
      for (int k = 0; k < 8; ++k) {
        L = L + yy[k] * ybar[8 * (goff[i] + g) + k];
        if (y) y[8 * (goff[i] + g) + k] = yy[k].v.v;
        if (jvp) jvp[8 * (goff[i] + g) + k] = yy[k].v.d[0];
      }
    }
    for (int k = 0; k < 12; ++k) {
      if (grad) grad[12 * i + k] = L.d[k].v;
      if (hvp) hvp[12 * i + k] = L.d[k].d[0];
    }
  }
  return 0;
}

// ---- single steps, exposed for the pin tests ----

double ccmo_sdf(const double* planes, int F, const double* x, double tau, double* grad) {
  V3<double> g;
  double phi = piece_sdf<double>(planes, F, V3<double>{x[0], x[1], x[2]}, tau, &g);
  if (grad) { grad[0] = g.x; grad[1] = g.y; grad[2] = g.z; }
  return phi;
}

void ccmo_edge_point(const double* planes, int F, const double* vI, const double* vII,
                     const ccmo_params* prm, double* pe, double* alpha) {
  double a[4];
  const PieceSdf sdf{planes, F, prm->tau_sdf};
  V3<double> p = edge_point<double>(sdf, V3<double>{vI[0], vI[1], vI[2]},
                                    V3<double>{vII[0], vII[1], vII[2]}, *prm, a);
  pe[0] = p.x; pe[1] = p.y; pe[2] = p.z;
  if (alpha) for (int k = 0; k < 4; ++k) alpha[k] = a[k];
}

// smooth-union SDF of body `body` at x (body frame) and its gradient
double ccmo_body_sdf(const ccmo_geom* G, int64_t body, const double* x, double tau,
                     double* grad) {
  const BodyUnionSdf sdf{G, body, tau};
  V3<double> g;
  const double phi = sdf(V3<double>{x[0], x[1], x[2]}, &g);
  if (grad) { grad[0] = g.x; grad[1] = g.y; grad[2] = g.z; }
  return phi;
}

// the paper's 1-D cubic basis u(t) (Sec. 3.2)
double ccmo_spline_u(double t) { return spline_u<double>(t); }

// tricubic spline SDF of piece `piece` at x (body frame) and its normal spline
double ccmo_spline_sdf(const ccmo_geom* G, int64_t piece, const double* x, double* normal) {
  const SplineSdf sdf{G->spline_grid + 4 * piece, G->spline_dims + 4 * piece, G->spline_coef};
  V3<double> n;
  const double phi = sdf(V3<double>{x[0], x[1], x[2]}, &n);
  if (normal) { normal[0] = n.x; normal[1] = n.y; normal[2] = n.z; }
  return phi;
}

double ccmo_transition(double d, double d_max, double eps) { return transition<double>(d, d_max, eps); }
double ccmo_softclip(double x, double lo, double hi, double tau) { return softclip<double>(x, lo, hi, tau); }
double ccmo_softplus(double x, double tau) { return softplus<double>(x, tau); }
double ccmo_sigmoid(double x) { return sigmoid<double>(x); }

// every contact of one pair, for the blend tests: rows of
// (group, phi, f, d_c, p_w(3), n_w(3)); returns the number of rows (or the
// required capacity when rows == NULL)
int64_t ccmo_pair_contacts(const ccmo_geom* G, int64_t bA, int64_t bB, const double* pose_a,
                           const double* pose_b, const ccmo_params* prm, double* rows,
                           int64_t capacity) {
  Pose<double> PA = const_pose<double>(pose_a), PB = const_pose<double>(pose_b);
  int64_t cnt = 0, group = 0;
  for (int side = 0; side < 2; ++side) {
    const int64_t bF = side == 0 ? bA : bB, bS = side == 0 ? bB : bA;
    const Pose<double>& PF = side == 0 ? PA : PB;
    const Pose<double>& PS = side == 0 ? PB : PA;
    for (int64_t fp = G->body_piece_off[bF]; fp < G->body_piece_off[bF + 1]; ++fp, ++group) {
      std::vector<Contact<double>> cs;
      std::vector<V3<double>> pw, nw;
      group_contacts(*G, fp, PF, bS, PS, *prm, cs, pw, nw);
      for (size_t c = 0; c < cs.size(); ++c, ++cnt) {
        if (!rows || cnt >= capacity) continue;
        double* r = rows + 10 * cnt;
        r[0] = (double)group; r[1] = cs[c].phi; r[2] = cs[c].f; r[3] = cs[c].dc;
        r[4] = pw[c].x; r[5] = pw[c].y; r[6] = pw[c].z;
        r[7] = nw[c].x; r[8] = nw[c].y; r[9] = nw[c].z;
      }
    }
  }
  return cnt;
}

}  // extern "C"
