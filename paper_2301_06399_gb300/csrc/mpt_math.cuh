// Device math of the MPT solver: parametric points (Eqs. 13-14), the law
// residuals (Eq. 8 divided by ||X_k - X_{k-1}||, Eq. 9), their hand-derived
// Jacobian with respect to the object parameters, and the accumulation of
// the Gauss-Newton normal equations J^T J, J^T rho of Eq. 15.
//
// Everything is templated on two scalar types: R for the geometry and the
// residual, J for the Jacobian.  (float, float) is the FP32 iteration,
// (double, float) the mixed FP64 refinement, (double, double) the plain FP64
// method.  The host instantiates the same code with a counting type to give
// the FLOP model of the kernels.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define MPT_HD __host__ __device__ __forceinline__
#else
#define MPT_HD inline
#endif

namespace mpt {

// ------------------------------------------------------------- scalars --
MPT_HD float fma_(float a, float b, float c) { return fmaf(a, b, c); }
MPT_HD double fma_(double a, double b, double c) { return fma(a, b, c); }

// 1/sqrt(x).  FP32: the hardware reciprocal square root.  FP64: an FP32 seed
// refined by two Newton-Raphson steps y <- y (3 - x y^2) / 2 (each step
// squares the relative error: ~1e-7 -> ~1e-14 -> below double rounding),
// which keeps the FP64 path off the slow double-precision divide and sqrt.
MPT_HD float rsq(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}
MPT_HD float d2f_bits(double x);
MPT_HD double f2d_bits(float f);
MPT_HD double rsq(double x) {
  double y = f2d_bits(rsq(d2f_bits(x)));
  double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

// sin and cos of an FP32 argument by Cody and Waite's method ("Software
// Manual for the Elementary Functions", 1980): x = k pi/2 + r with
// k = rint(2x/pi) and |r| <= pi/4, pi/2 split over three floats and taken off
// with fused multiply-adds; then the Taylor series of sin r to r^9 and of
// cos r to r^10 (truncation below 3e-9 on |r| <= pi/4), and the quadrant
// k mod 4.  The device uses it instead of the library's sincosf: that
// carries a long path for huge arguments, and inlined at every arc
// evaluation it kept the curved solvers waiting on instruction fetch (19% of
// the curved scene's solve).  The reduction stays accurate for |x| up to
// ~1e5 (arc parameters that large only occur on diverging iterates).
// Constants: P1 + P2 + P3 = pi/2 (each the float nearest the remainder),
// 2/pi and 1/n! rounded to float.
MPT_HD void sincos_cw(float x, float& s, float& c) {
  const float k = rintf(x * 0.636619747f);
  float r = fmaf(-k, 1.57079637f, x);
  r = fmaf(-k, -4.37113883e-8f, r);
  r = fmaf(-k, -1.71512451e-15f, r);
  const float r2 = r * r;
  float ps = fmaf(r2, 2.75573188e-6f, -1.98412701e-4f);
  ps = fmaf(r2, ps, 8.33333377e-3f);
  ps = fmaf(r2, ps, -1.66666672e-1f);
  const float sr = fmaf(r * r2, ps, r);
  float pc = fmaf(r2, -2.75573200e-7f, 2.48015876e-5f);
  pc = fmaf(r2, pc, -1.38888892e-3f);
  pc = fmaf(r2, pc, 4.16666679e-2f);
  pc = fmaf(r2, pc, -0.5f);
  const float cr = fmaf(r2, pc, 1.0f);
  // quadrant: 0 (s, c), 1 (c, -s), 2 (-s, -c), 3 (-c, s); a NaN k leaves
  // NaN in r and in both results
  const float qf = k - 4.0f * floorf(0.25f * k);
  const int q = (qf >= 0.0f && qf < 4.0f) ? (int)qf : 0;
  const float s0 = (q & 1) ? cr : sr, c0 = (q & 1) ? sr : cr;
  s = (q & 2) ? -s0 : s0;
  c = (q == 1 || q == 2) ? -c0 : c0;
}

MPT_HD void sincos_(float x, float& s, float& c) {
#if defined(__CUDA_ARCH__)
  sincos_cw(x, s, c);
#else
  s = sinf(x);
  c = cosf(x);
#endif
}
MPT_HD void sincos_(double x, double& s, double& c) {
#if defined(__CUDA_ARCH__)
  sincos(x, &s, &c);
#else
  s = ::sin(x);
  c = ::cos(x);
#endif
}

// --------------------------------------------------------------- vectors --
template <class T>
struct v3 {
  T x, y, z;
};
template <class T> MPT_HD v3<T> mk(T x, T y, T z) { v3<T> r; r.x = x; r.y = y; r.z = z; return r; }
template <class T> MPT_HD v3<T> operator+(const v3<T>& a, const v3<T>& b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> MPT_HD v3<T> operator-(const v3<T>& a, const v3<T>& b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T> MPT_HD v3<T> operator-(const v3<T>& a) { return mk(-a.x, -a.y, -a.z); }
template <class T> MPT_HD v3<T> operator*(const v3<T>& a, T s) { return mk(a.x * s, a.y * s, a.z * s); }
template <class T> MPT_HD T dot(const v3<T>& a, const v3<T>& b) { return fma_(a.x, b.x, fma_(a.y, b.y, a.z * b.z)); }
// a + s * b
template <class T> MPT_HD v3<T> axpy(T s, const v3<T>& b, const v3<T>& a) {
  return mk(fma_(s, b.x, a.x), fma_(s, b.y, a.y), fma_(s, b.z, a.z));
}
template <class T> MPT_HD v3<T> cross(const v3<T>& a, const v3<T>& b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// double -> float on the integer units (truncating the mantissa; |error| <
// 1 ulp).  The mixed-precision evaluation converts every Jacobian input;
// GB300's FP64 pipe (which executes hardware conversions) is 1/64 of FP32.
MPT_HD float d2f_bits(double x) {
#if defined(__CUDA_ARCH__)
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(u >> 63) << 31;
  const unsigned ex = (unsigned)((u >> 52) & 0x7FFu);
  const unsigned m = (unsigned)((u >> 29) & 0x7FFFFFu);
  if (ex == 0x7FFu) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  const int e = (int)ex - 1023 + 127;
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  if (e <= 0) return __uint_as_float(sign);
  return __uint_as_float(sign | ((unsigned)e << 23) | m);
#else
  return (float)x;
#endif
}
// Exact float -> double, also on the integer units.  FP32 subnormals (never
// produced by the solver's magnitudes) become +-0.
MPT_HD double f2d_bits(float f) {
#if defined(__CUDA_ARCH__)
  // 32-bit halves: the low word is the mantissa's last 3 bits shifted up;
  // the high word is sign | exponent and mantissa shifted down by 3 with the
  // exponent rebiased (127 -> 1023: + 896 << 20), or all-ones for Inf/NaN.
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7FFFFFFFu;
  const uint32_t sign = u & 0x80000000u;
  uint32_t hi = (a >> 3) + 0x38000000u;
  if (a >= 0x7F800000u) hi = (a >> 3) | 0x7FF00000u;  // Inf, NaN
  if (a < 0x00800000u) hi = 0u;                        // zero, subnormal -> 0
  const uint32_t lo = a < 0x00800000u ? 0u : u << 29;
  return __hiloint2double((int)(hi | sign), (int)lo);
#else
  return (double)f;
#endif
}
template <class D, class S>
struct Conv {
  MPT_HD static D go(S x) { return D(x); }
};
template <>
struct Conv<float, double> {
  MPT_HD static float go(double x) { return d2f_bits(x); }
};
template <class D, class S> MPT_HD D conv(S x) { return Conv<D, S>::go(x); }
template <class D, class S> MPT_HD v3<D> cvt(const v3<S>& a) { return mk(conv<D>(a.x), conv<D>(a.y), conv<D>(a.z)); }

// ------------------------------------------------------------ scene record --
// 16 values per object (same layout in FP32 and FP64 copies):
//   plane       O.xyz U | u.xyz V | v.xyz d | n.xyz 0
//   paraboloid  c0.xyz t.x | c1.xyz t.y | c2.xyz t.z | 1/(4f) rho 1/(2f) f
//                 (c_j = column j of R: local axes in world)
//   line edge   P.xyz t0 | e.xyz t1 | 0 | 0
//   arc edge    C.xyz Rc | u.xyz phi0 | v.xyz phi1 | a.xyz 0   (v = a x u)
// Occluders: rectangle O.xyz U | u.xyz V | v.xyz 0 | n.xyz 0, paraboloid as above.
enum { K_PLANE = 0, K_PARAB = 1, K_LINE = 2, K_ARC = 3 };

template <class T>
struct Rec {
  T v[16];
  MPT_HD v3<T> f3(int i) const { return mk(v[i], v[i + 1], v[i + 2]); }
};

MPT_HD bool is_edge(int kind) { return kind == K_LINE || kind == K_ARC; }

// ------------------------------------------------------ parametric points --
// Point of an object at parameters (s, t) and its tangents dX/ds, dX/dt
// (Eqs. 13, 14).  Edges use s only; their second tangent is zero.
template <class T>
struct PointT {
  v3<T> X, w0, w1;
};

// CURVED = false instantiates the planes-and-straight-edges solver only (no
// paraboloid or arc branches: less code, fewer registers).
template <class T, bool TANGENTS, bool CURVED = true>
MPT_HD PointT<T> point_at(int kind, const Rec<T>& r, T s, T t) {
  PointT<T> p;
  const T zero = T(0);
  p.w1 = mk(zero, zero, zero);
  if (kind == K_PLANE) {
    p.X = axpy(t, r.f3(8), axpy(s, r.f3(4), r.f3(0)));
    if (TANGENTS) { p.w0 = r.f3(4); p.w1 = r.f3(8); }
  } else if (CURVED && kind == K_PARAB) {
    const T q4 = r.v[12], q2 = r.v[14];
    T h = (s * s + t * t) * q4;
    v3<T> base = mk(r.v[3], r.v[7], r.v[11]);
    p.X = axpy(h, r.f3(8), axpy(t, r.f3(4), axpy(s, r.f3(0), base)));
    if (TANGENTS) {
      p.w0 = axpy(s * q2, r.f3(8), r.f3(0));
      p.w1 = axpy(t * q2, r.f3(8), r.f3(4));
    }
  } else if (!CURVED || kind == K_LINE) {
    p.X = axpy(s, r.f3(4), r.f3(0));
    if (TANGENTS) p.w0 = r.f3(4);
  } else {
    T sn, cs;
    sincos_(s, sn, cs);
    const T Rc = r.v[3];
    p.X = axpy(Rc * sn, r.f3(8), axpy(Rc * cs, r.f3(4), r.f3(0)));
    if (TANGENTS) p.w0 = axpy(Rc * cs, r.f3(8), r.f3(4) * (-Rc * sn));
  }
  return p;
}

// ---------------------------------------------------- residual + normal eqs --
// Packed lower-triangular index of (i, j), i >= j.
MPT_HD constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

template <int N>
struct NormalEq {
  static constexpr int Q = 2 * N;
  static constexpr int P = Q * (Q + 1) / 2;
};

// Adds one interaction's contribution: for the (up to) six parameter
// columns of interaction k (previous point, this point, next point), the
// column vectors col[c] (3 rows for reflection, 1 for diffraction) give
// J^T J entries <col[a], col[b]> and J^T rho entries <col[a], rho>.
template <int N, int ROWS, class J>
MPT_HD void accumulate(int k, const J (&col)[6][ROWS], const bool (&live)[6], const J (&rho)[ROWS],
                       J* jtj, J* g) {
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const int ga = 2 * (k - 1) + a;  // parameter index of column a
    if (ga < 0 || ga >= 2 * N || !live[a]) continue;
    J ga_acc = J(0);
#pragma unroll
    for (int r = 0; r < ROWS; ++r) ga_acc = fma_(col[a][r], rho[r], ga_acc);
    g[ga] = g[ga] + ga_acc;
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      const int gb = 2 * (k - 1) + b;
      if (gb < 0 || gb >= 2 * N || !live[b]) continue;
      J acc = J(0);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) acc = fma_(col[a][r], col[b][r], acc);
      jtj[tri(ga, gb)] = jtj[tri(ga, gb)] + acc;
    }
  }
}

// Evaluates the cost of Eq. 15 at parameters prm (slot 2k, 2k+1 for
// interaction k; edges use slot 2k) and, when WANT_J, accumulates the normal
// equations J^T J (packed, Q = 2N) and g = J^T rho.  A = TX, B = RX.
// Returns the cost; `ok` is false when a segment has zero length.
//
// Hand-derived Jacobian.  With unit segment directions u_j and inverse
// lengths l_j, a tangent w of point k enters through the projections
//   Pi_k(w) = (w - u_k <u_k, w>) l_k        (incoming segment of point k)
//   Pr_k(w) = (w - u_{k+1} <u_{k+1}, w>) l_{k+1}   (outgoing segment)
// Reflection rho_k = r - i + 2<i,n>n, H(v) = v - 2<n,v>n:
//   d rho_k / d(point k-1) = H(Pi_k w) = H(Pr_{k-1} w)
//   d rho_k / d(point k)   = -(Pr_k w + H(Pi_k w))  (+ normal variation)
//   d rho_k / d(point k+1) = Pr_k w = Pi_{k+1} w
// Diffraction rho_k = <i,e> - <r,e>:
//   -<e, Pr_{k-1} w>,  <e, Pi_k w> + <e, Pr_k w> (+ edge variation),  -<e, Pi_{k+1} w>
// so each projection is computed once per point and shared by neighbours.
template <int N, class R, class J, bool WANT_J, bool CURVED = true>
MPT_HD R eval_path(const int (&kind)[N], const Rec<R> (&rec)[N], const R (&prm)[2 * N], const v3<R>& A,
                   const v3<R>& B, J* jtj, J* g, bool& ok) {
  PointT<R> pt[N];
#pragma unroll
  for (int k = 0; k < N; ++k)
    pt[k] = point_at<R, WANT_J, CURVED>(kind[k], rec[k], prm[2 * k], prm[2 * k + 1]);
  // segment unit vectors u[j] = (X_{j+1} - X_j)/||.||, inverse lengths il[j]
  v3<R> u[N + 1];
  R il[N + 1];
  ok = true;
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const v3<R> a = (j == 0) ? A : pt[j - 1].X;
    const v3<R> b = (j == N) ? B : pt[j].X;
    v3<R> d = b - a;
    R l2 = dot(d, d);
    ok = ok && (l2 > R(0));
    il[j] = rsq(l2);
    u[j] = d * il[j];
  }
  v3<J> PiW[N][2], PrW[N][2];
  if (WANT_J) {
#pragma unroll
    for (int i = 0; i < NormalEq<N>::P; ++i) jtj[i] = J(0);
#pragma unroll
    for (int i = 0; i < 2 * N; ++i) g[i] = J(0);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const v3<J> ui = cvt<J>(u[k]), uo = cvt<J>(u[k + 1]);
      const J li = conv<J>(il[k]), lo = conv<J>(il[k + 1]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const v3<J> w = cvt<J>(j == 0 ? pt[k].w0 : pt[k].w1);
        if (j == 1 && is_edge(kind[k])) {
          PiW[k][j] = w;  // zero tangent
          PrW[k][j] = w;
        } else {
          PiW[k][j] = axpy(-dot(ui, w), ui, w) * li;
          PrW[k][j] = axpy(-dot(uo, w), uo, w) * lo;
        }
      }
    }
  }
  R cost = R(0);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const v3<R>& ih = u[k];      // incident direction (into X_k)
    const v3<R>& rh = u[k + 1];  // departing direction
    // columns of the neighbours: live unless the neighbour is an edge's unused slot
    bool live[6];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      live[j] = (k >= 1) && (j == 0 || !is_edge(kind[k > 0 ? k - 1 : 0]));
      live[2 + j] = (j == 0) || !is_edge(kind[k]);
      live[4 + j] = (k + 1 < N) && (j == 0 || !is_edge(kind[k + 1 < N ? k + 1 : k]));
    }
    if (!is_edge(kind[k])) {
      // ---- reflection: rho = r_hat - i_hat + 2 <i_hat, n> n  (Eq. 8 / ||i||)
      v3<R> nh;
      R inv_nn = R(0);
      if (!CURVED || kind[k] == K_PLANE) {
        nh = rec[k].f3(12);
      } else {
        // n = c2 - (s/(2f)) c0 - (t/(2f)) c1  (gradient of the implicit
        // paraboloid, Eq. 2, up to sign and scale)
        const R q2 = rec[k].v[14];
        const v3<R> nraw =
            axpy(-prm[2 * k + 1] * q2, rec[k].f3(4), axpy(-prm[2 * k] * q2, rec[k].f3(0), rec[k].f3(8)));
        inv_nn = rsq(dot(nraw, nraw));
        nh = nraw * inv_nn;
      }
      const R c = dot(ih, nh);
      v3<R> rho = axpy(R(2) * c, nh, rh - ih);
      cost = fma_(rho.x, rho.x, fma_(rho.y, rho.y, fma_(rho.z, rho.z, cost)));
      if (WANT_J) {
        const v3<J> iJ = cvt<J>(ih), nJ = cvt<J>(nh);
        auto H = [&](const v3<J>& w) { return axpy(J(-2) * dot(nJ, w), nJ, w); };
        J col[6][3];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const v3<J> vp = (k >= 1) ? H(PrW[k > 0 ? k - 1 : 0][j]) : mk(J(0), J(0), J(0));
          col[j][0] = vp.x; col[j][1] = vp.y; col[j][2] = vp.z;
          v3<J> vs = -(PrW[k][j] + H(PiW[k][j]));
          if (CURVED && kind[k] == K_PARAB) {
            // d/dT of 2 <i,n> n through n: 2 (<i, dn> n + <i, n> dn),
            // dn = (I - n n^T) dn_raw / ||n_raw||, dn_raw = -c_j / (2f)
            const J q2 = conv<J>(rec[k].v[14]);
            const v3<J> craw = cvt<J>(j == 0 ? rec[k].f3(0) : rec[k].f3(4)) * (-q2);
            const v3<J> dn = axpy(-dot(nJ, craw), nJ, craw) * conv<J>(inv_nn);
            vs = axpy(J(2) * dot(iJ, dn), nJ, vs);
            vs = axpy(J(2) * conv<J>(c), dn, vs);
          }
          col[2 + j][0] = vs.x; col[2 + j][1] = vs.y; col[2 + j][2] = vs.z;
          const v3<J> vn = (k + 1 < N) ? PiW[k + 1 < N ? k + 1 : k][j] : mk(J(0), J(0), J(0));
          col[4 + j][0] = vn.x; col[4 + j][1] = vn.y; col[4 + j][2] = vn.z;
        }
        const J rr[3] = {conv<J>(rho.x), conv<J>(rho.y), conv<J>(rho.z)};
        accumulate<N, 3, J>(k, col, live, rr, jtj, g);
      }
    } else {
      // ---- diffraction: rho = <i_hat, e> - <r_hat, e>  (Eq. 9)
      v3<R> eh;
      v3<R> de;  // d e / d phi for arcs
      if (!CURVED || kind[k] == K_LINE) {
        eh = rec[k].f3(4);
      } else {
        R sn, cs;
        sincos_(prm[2 * k], sn, cs);
        eh = axpy(cs, rec[k].f3(8), rec[k].f3(4) * (-sn));
        de = axpy(-sn, rec[k].f3(8), rec[k].f3(4) * (-cs));
      }
      const R rho = dot(ih, eh) - dot(rh, eh);
      cost = fma_(rho, rho, cost);
      if (WANT_J) {
        const v3<J> eJ = cvt<J>(eh);
        J col[6][1];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          col[j][0] = (k >= 1) ? -dot(eJ, PrW[k > 0 ? k - 1 : 0][j]) : J(0);
          col[4 + j][0] = (k + 1 < N) ? -dot(eJ, PiW[k + 1 < N ? k + 1 : k][j]) : J(0);
        }
        J v = dot(eJ, PiW[k][0]) + dot(eJ, PrW[k][0]);
        if (CURVED && kind[k] == K_ARC) v = v + dot(cvt<J>(ih - rh), cvt<J>(de));  // edge direction variation
        col[2][0] = v;
        col[3][0] = J(0);
        const J rr[1] = {conv<J>(rho)};
        accumulate<N, 1, J>(k, col, live, rr, jtj, g);
      }
    }
  }
  return cost;
}

// Cholesky factorisation of the packed Q x Q matrix in place (lower), with
// relative diagonal damping mu.  Returns false when a pivot is not positive.
// Every loop runs a fixed Q trips under a compile-time guard, so that full
// unrolling leaves only constant indices (a trip count that depends on an
// outer index was not unrolled at Q = 6, 8, and the matrix went to local
// memory).
template <int Q, class J>
MPT_HD bool cholesky(J* a, J mu) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    J d = a[tri(j, j)];
#pragma unroll
    for (int k = 0; k < Q; ++k)
      if (k < j) d = fma_(-a[tri(j, k)], a[tri(j, k)], d);
    d = d + mu * a[tri(j, j)] + J(1e-30f);
    ok = ok && (d > J(0));
    const J inv = rsq(d > J(0) ? d : J(1));
    a[tri(j, j)] = inv;  // store 1/L_jj
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (i <= j) continue;
      J s = a[tri(i, j)];
#pragma unroll
      for (int k = 0; k < Q; ++k)
        if (k < j) s = fma_(-a[tri(i, k)], a[tri(j, k)], s);
      a[tri(i, j)] = s * inv;
    }
  }
  return ok;
}

// Solves (L L^T) x = -g with the factor from cholesky() (diagonal holds 1/L_jj).
template <int Q, class J>
MPT_HD void chol_solve(const J* a, const J* g, J* x) {
  J y[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    J s = -g[i];
#pragma unroll
    for (int k = 0; k < Q; ++k)
      if (k < i) s = fma_(-a[tri(i, k)], y[k], s);
    y[i] = s * a[tri(i, i)];
  }
#pragma unroll
  for (int r = 0; r < Q; ++r) {
    const int i = Q - 1 - r;
    J s = y[i];
#pragma unroll
    for (int k = 0; k < Q; ++k)
      if (k > i) s = fma_(-a[tri(k, i)], x[k], s);
    x[i] = s * a[tri(i, i)];
  }
}

}  // namespace mpt
