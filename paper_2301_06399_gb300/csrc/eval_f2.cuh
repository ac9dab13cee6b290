// The FP32 evaluation of the solver (the same arithmetic as eval_path in
// mpt_math.cuh: cost of Eq. 15 with the residuals of Eqs. 8 and 9, and the
// normal equations J^T J, J^T rho) written on paired FP32 operations.
//
// The two parameters of a point (s, t) have tangents w0, w1 that go through
// the same projections and reflections, so every quantity derived from them
// comes in pairs and is computed with the paired instructions __ffma2_rn,
// __fmul2_rn, __fadd2_rn (two lanes of FP32 work per issued instruction at
// the full FP32 rate on this GPU).  Likewise the normal equations are
// accumulated as 2 x 2 blocks over the parameter pairs of two points.  An
// edge's second tangent is zero, so its unused column contributes exact zeros
// that the caller's pinning overrides.  The solver is issue-bound, so fewer
// instructions for the same operations is what this form buys.
#pragma once

#include "mpt_math.cuh"

namespace mpt {

// Two 3-vectors stored component-wise: x = (a.x, b.x), ...
struct vp {
  float2 x, y, z;
};

__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

__device__ __forceinline__ vp make_vp(const v3<float>& a, const v3<float>& b) {
  vp r;
  r.x = make_float2(a.x, b.x);
  r.y = make_float2(a.y, b.y);
  r.z = make_float2(a.z, b.z);
  return r;
}
// (<a, w0>, <a, w1>)
__device__ __forceinline__ float2 dot_vp(const v3<float>& a, const vp& w) {
  return f2fma(bc(a.z), w.z, f2fma(bc(a.y), w.y, f2mul(bc(a.x), w.x)));
}
// w + a * s   (a broadcast vector, s a pair of scalars)
__device__ __forceinline__ vp axpy_vp(const v3<float>& a, float2 s, const vp& w) {
  vp r;
  r.x = f2fma(bc(a.x), s, w.x);
  r.y = f2fma(bc(a.y), s, w.y);
  r.z = f2fma(bc(a.z), s, w.z);
  return r;
}
__device__ __forceinline__ vp scale_vp(const vp& w, float l) {
  vp r;
  r.x = f2mul(w.x, bc(l));
  r.y = f2mul(w.y, bc(l));
  r.z = f2mul(w.z, bc(l));
  return r;
}
__device__ __forceinline__ vp add_vp(const vp& a, const vp& b) {
  vp r;
  r.x = f2add(a.x, b.x);
  r.y = f2add(a.y, b.y);
  r.z = f2add(a.z, b.z);
  return r;
}
__device__ __forceinline__ vp neg_vp(const vp& a) {
  vp r;
  r.x = make_float2(-a.x.x, -a.x.y);
  r.y = make_float2(-a.y.x, -a.y.y);
  r.z = make_float2(-a.z.x, -a.z.y);
  return r;
}
// projection of both tangents off the unit direction u, over the length 1/l
__device__ __forceinline__ vp project_vp(const vp& w, const v3<float>& u, float l) {
  const float2 d = dot_vp(u, w);
  return scale_vp(axpy_vp(u, make_float2(-d.x, -d.y), w), l);
}
// mirror of both tangents in the plane of normal n: w - 2 <n, w> n
__device__ __forceinline__ vp mirror_vp(const vp& w, const v3<float>& n) {
  const float2 d = dot_vp(n, w);
  return axpy_vp(n, f2mul(d, bc(-2.0f)), w);
}

// Normal-equation accumulators over parameter pairs: for pairs m' <= m the
// block rows r0 = (J^T J)[2m][2m'..2m'+1], r1 = (J^T J)[2m+1][2m'..2m'+1]
// (the diagonal block keeps [2m][2m] as a scalar), and g pairs.
template <int N>
struct NormalAcc {
  float2 r0[N][N], r1[N][N];
  float d0[N];
  float2 gp[N];
};

// Adds the contribution of a residual with rows rho[0..ROWS) whose columns
// for parameter pair m are col[m] (ROWS rows of pairs; live[m] false = the
// interaction does not touch point m).
template <int N, int ROWS>
__device__ __forceinline__ void acc_rows(NormalAcc<N>& a, const float2 (&col)[N][ROWS], const bool (&live)[N],
                                         const float (&rho)[ROWS]) {
#pragma unroll
  for (int m = 0; m < N; ++m) {
    if (!live[m]) continue;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) a.gp[m] = f2fma(col[m][r], bc(rho[r]), a.gp[m]);
#pragma unroll
    for (int mp = 0; mp <= m; ++mp) {
      if (!live[mp]) continue;
      if (mp == m) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          a.d0[m] = fmaf(col[m][r].x, col[m][r].x, a.d0[m]);
          a.r1[m][m] = f2fma(bc(col[m][r].y), col[m][r], a.r1[m][m]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          a.r0[m][mp] = f2fma(bc(col[m][r].x), col[mp][r], a.r0[m][mp]);
          a.r1[m][mp] = f2fma(bc(col[m][r].y), col[mp][r], a.r1[m][mp]);
        }
      }
    }
  }
}

template <int N, bool CURVED>
__device__ __forceinline__ float eval_path_f2(const int (&kind)[N], const Rec<float> (&rec)[N],
                                              const float (&prm)[2 * N], const v3<float>& A, const v3<float>& B,
                                              float* jtj, float* g, bool& ok) {
  PointT<float> pt[N];
#pragma unroll
  for (int k = 0; k < N; ++k) pt[k] = point_at<float, true, CURVED>(kind[k], rec[k], prm[2 * k], prm[2 * k + 1]);
  v3<float> u[N + 1];
  float il[N + 1];
  ok = true;
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const v3<float> a = (j == 0) ? A : pt[j - 1].X;
    const v3<float> b = (j == N) ? B : pt[j].X;
    const v3<float> d = b - a;
    const float l2 = dot(d, d);
    ok = ok && (l2 > 0.f);
    il[j] = rsq(l2);
    u[j] = d * il[j];
  }
  // projections of the tangent pairs off the incoming / outgoing segments
  vp PiW[N], PrW[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const vp W = make_vp(pt[k].w0, pt[k].w1);
    PiW[k] = project_vp(W, u[k], il[k]);
    PrW[k] = project_vp(W, u[k + 1], il[k + 1]);
  }
  NormalAcc<N> acc;
#pragma unroll
  for (int m = 0; m < N; ++m) {
    acc.d0[m] = 0.f;
    acc.gp[m] = make_float2(0.f, 0.f);
#pragma unroll
    for (int mp = 0; mp < N; ++mp) {
      acc.r0[m][mp] = make_float2(0.f, 0.f);
      acc.r1[m][mp] = make_float2(0.f, 0.f);
    }
  }
  float cost = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const v3<float>& ih = u[k];
    const v3<float>& rh = u[k + 1];
    bool live[N];
#pragma unroll
    for (int m = 0; m < N; ++m) live[m] = (m >= k - 1 && m <= k + 1);
    if (!is_edge(kind[k])) {
      // ---- reflection: rho = r_hat - i_hat + 2 <i_hat, n> n  (Eq. 8 / ||i||)
      v3<float> nh;
      float inv_nn = 0.f;
      if (!CURVED || kind[k] == K_PLANE) {
        nh = rec[k].f3(12);
      } else {
        const float q2 = rec[k].v[14];
        const v3<float> nraw =
            axpy(-prm[2 * k + 1] * q2, rec[k].f3(4), axpy(-prm[2 * k] * q2, rec[k].f3(0), rec[k].f3(8)));
        inv_nn = rsq(dot(nraw, nraw));
        nh = nraw * inv_nn;
      }
      const float c = dot(ih, nh);
      const v3<float> rho = axpy(2.0f * c, nh, rh - ih);
      cost = fmaf(rho.x, rho.x, fmaf(rho.y, rho.y, fmaf(rho.z, rho.z, cost)));
      float2 col[N][3];
#pragma unroll
      for (int m = 0; m < N; ++m) {
        vp v;
        if (m == k - 1) {
          v = mirror_vp(PrW[m], nh);
        } else if (m == k) {
          v = neg_vp(add_vp(PrW[k], mirror_vp(PiW[k], nh)));
          if (CURVED && kind[k] == K_PARAB) {
            // normal variation: 2 (<i, dn> n + <i, n> dn), dn from the parameters
            const float q2 = rec[k].v[14];
            const vp craw = make_vp(rec[k].f3(0) * (-q2), rec[k].f3(4) * (-q2));
            const float2 nc = dot_vp(nh, craw);
            const vp dn = scale_vp(axpy_vp(nh, make_float2(-nc.x, -nc.y), craw), inv_nn);
            v = axpy_vp(nh, f2mul(dot_vp(ih, dn), bc(2.0f)), v);
            v.x = f2fma(bc(2.0f * c), dn.x, v.x);
            v.y = f2fma(bc(2.0f * c), dn.y, v.y);
            v.z = f2fma(bc(2.0f * c), dn.z, v.z);
          }
        } else if (m == k + 1) {
          v = PiW[m];
        } else {
          v.x = v.y = v.z = make_float2(0.f, 0.f);
        }
        col[m][0] = v.x;
        col[m][1] = v.y;
        col[m][2] = v.z;
      }
      const float rr[3] = {rho.x, rho.y, rho.z};
      acc_rows<N, 3>(acc, col, live, rr);
    } else {
      // ---- diffraction: rho = <i_hat, e> - <r_hat, e>  (Eq. 9)
      v3<float> eh, de;
      if (!CURVED || kind[k] == K_LINE) {
        eh = rec[k].f3(4);
        de = mk(0.f, 0.f, 0.f);
      } else {
        float sn, cs;
        sincos_(prm[2 * k], sn, cs);
        eh = axpy(cs, rec[k].f3(8), rec[k].f3(4) * (-sn));
        de = axpy(-sn, rec[k].f3(8), rec[k].f3(4) * (-cs));
      }
      const float rho = dot(ih, eh) - dot(rh, eh);
      cost = fmaf(rho, rho, cost);
      float2 col[N][1];
#pragma unroll
      for (int m = 0; m < N; ++m) {
        float2 v = make_float2(0.f, 0.f);
        if (m == k - 1) {
          const float2 d = dot_vp(eh, PrW[m]);
          v = make_float2(-d.x, -d.y);
        } else if (m == k) {
          // the edge's own second parameter is unused: only column 2k
          const float2 d = f2add(dot_vp(eh, PiW[k]), dot_vp(eh, PrW[k]));
          float vx = d.x;
          if (CURVED && kind[k] == K_ARC) vx += dot(ih - rh, de);  // edge direction variation
          v = make_float2(vx, 0.f);
        } else if (m == k + 1) {
          const float2 d = dot_vp(eh, PiW[m]);
          v = make_float2(-d.x, -d.y);
        }
        col[m][0] = v;
      }
      const float rr[1] = {rho};
      acc_rows<N, 1>(acc, col, live, rr);
    }
  }
  // unpack into the packed lower triangle and g
#pragma unroll
  for (int m = 0; m < N; ++m) {
    g[2 * m] = acc.gp[m].x;
    g[2 * m + 1] = acc.gp[m].y;
    jtj[tri(2 * m, 2 * m)] = acc.d0[m];
    jtj[tri(2 * m + 1, 2 * m)] = acc.r1[m][m].x;
    jtj[tri(2 * m + 1, 2 * m + 1)] = acc.r1[m][m].y;
#pragma unroll
    for (int mp = 0; mp < m; ++mp) {
      jtj[tri(2 * m, 2 * mp)] = acc.r0[m][mp].x;
      jtj[tri(2 * m, 2 * mp + 1)] = acc.r0[m][mp].y;
      jtj[tri(2 * m + 1, 2 * mp)] = acc.r1[m][mp].x;
      jtj[tri(2 * m + 1, 2 * mp + 1)] = acc.r1[m][mp].y;
    }
  }
  return cost;
}

}  // namespace mpt
