// Adjoint of converged paths: at a solution rho(T*, theta) = 0 of Eq. 15 the
// implicit-function theorem gives dT/dtheta = -(J^T J)^{-1} J^T drho/dtheta.
// For upstream weights gL (path length) and gX (points), with
//   v = gL dL/dT + gX dX/dT,   lambda = (J^T J)^{-1} v,   z = J lambda,
// the vector-Jacobian product is
//   dtheta += gL dL/dtheta|explicit + gX dX/dtheta|explicit - z^T drho/dtheta.
// Without point weights (gX = 0) v vanishes at a solution and only the
// explicit term is left, which needs no linear solve.
// theta: TX (a fixed point before interaction 1), RX (after interaction n)
// and the offset d of each plane <n, X> = d (its points move along n).
// One thread per valid path, in float-float (about 48 significand bits).
#include "mpt_internal.cuh"

namespace mpt {

constexpr int GRAD_BLOCK = 128;

// Working precision of the adjoint: float-float (see ff.cuh).
using S = ff;

// Law residual of one interaction and the linear maps that give its rows
// for a displacement w of the previous point, this point and the next point.
struct Inter {
  bool refl;
  v3<S> ih, rh, nh, eh;
  S ia, ib;
  // reflection: H P_i w / a (prev), -(P_r w / b + H P_i w / a) (this), P_r w / b (next)
  // diffraction: -<e, P_i w>/a (prev), <e,P_i w>/a + <e,P_r w>/b (this), -<e, P_r w>/b (next)
  __device__ v3<S> Pi(const v3<S>& w) const { return axpy(-dot(ih, w), ih, w) * ia; }
  __device__ v3<S> Pr(const v3<S>& w) const { return axpy(-dot(rh, w), rh, w) * ib; }
  __device__ v3<S> H(const v3<S>& w) const { return axpy(S(-2) * dot(nh, w), nh, w); }
  // rows (3 for reflection; component x only for diffraction)
  __device__ v3<S> prev(const v3<S>& w) const {
    if (refl) return H(Pi(w));
    return mk(-dot(eh, Pi(w)), S(0), S(0));
  }
  __device__ v3<S> self(const v3<S>& w) const {
    if (refl) return -(Pr(w) + H(Pi(w)));
    return mk(dot(eh, Pi(w)) + dot(eh, Pr(w)), S(0), S(0));
  }
  __device__ v3<S> next(const v3<S>& w) const {
    if (refl) return Pr(w);
    return mk(-dot(eh, Pr(w)), S(0), S(0));
  }
};

// Contributions of one path, added to the outputs by the caller.
template <int N>
struct GradOut {
  int it, ir;
  double tx[3], rx[3];
  double obj[N];  // d/d offset of plane ids[m]; 0 for other kinds
};

// CURVED = false: scenes of planes and straight edges only (no paraboloid or
// arc branches: shorter code).
template <int N, bool CURVED>
__device__ bool grad_one(const DevScene& sc, const DevEnds& ep, const Cand& cd, const double* Tc, double gL,
                         const double* gX, bool want_tx, bool want_rx, bool want_obj, GradOut<N>& o) {
  constexpr int Q = 2 * N;
  int it_, ir_;
  pair_ends(ep, cd.pair, it_, ir_);
  const v3<S> A = load_end_ff(ep.tx, it_);
  const v3<S> B = load_end_ff(ep.rx, ir_);
  const S gLs = ff_from_double(gL);
  int kind[N];
  Rec<S> rec[N];
  S prm[Q];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    kind[k] = sc.kind[cd.ids[k]];
    rec[k] = load_obj_ff(sc, cd.ids[k]);
    prm[2 * k] = ff_from_double(Tc[2 * k]);
    prm[2 * k + 1] = ff_from_double(Tc[2 * k + 1]);
  }
  // geometry
  PointT<S> pt[N];
#pragma unroll
  for (int k = 0; k < N; ++k) pt[k] = point_at<S, true, CURVED>(kind[k], rec[k], prm[2 * k], prm[2 * k + 1]);
  v3<S> u[N + 1];
  S il[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const v3<S> a = j == 0 ? A : pt[j - 1].X;
    const v3<S> b = j == N ? B : pt[j].X;
    const v3<S> d = b - a;
    il[j] = rsq(dot(d, d));
    u[j] = d * il[j];
  }
  o.it = it_;
  o.ir = ir_;
  if (gX == nullptr) {
    // Length weights only.  A path obeys the laws of Eqs. 8-9 exactly when
    // its length is stationary in the parameters (Fermat), so dL/dT = 0,
    // v = 0, lambda = 0 and the gradient is the explicit one (envelope
    // theorem): dL/dTX = -u_0, dL/dRX = u_n, dL/dd = <u_m - u_m+1, n> for a
    // reflection on the plane <n, X> = d.  No normal matrix is needed.
    if (want_tx) {
      o.tx[0] = to_double(-gLs * u[0].x);
      o.tx[1] = to_double(-gLs * u[0].y);
      o.tx[2] = to_double(-gLs * u[0].z);
    }
    if (want_rx) {
      o.rx[0] = to_double(gLs * u[N].x);
      o.rx[1] = to_double(gLs * u[N].y);
      o.rx[2] = to_double(gLs * u[N].z);
    }
    if (want_obj) {
#pragma unroll
      for (int m = 0; m < N; ++m)
        o.obj[m] = kind[m] == K_PLANE ? to_double(gLs * dot(u[m] - u[m + 1], rec[m].f3(12))) : 0.0;
    }
    return true;
  }
  // normal matrix at the solution
  S jtj[Q * (Q + 1) / 2], g[Q];
  bool ok;
  eval_path<N, S, S, true, CURVED>(kind, rec, prm, A, B, jtj, g, ok);
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (is_edge(kind[k])) jtj[tri(2 * k + 1, 2 * k + 1)] = S(1);
  if (!cholesky<Q, S>(jtj, S(0))) return false;
  Inter in[N];
  S curv_c[N];
  S inv_nn[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    in[k].refl = !is_edge(kind[k]);
    in[k].ih = u[k];
    in[k].rh = u[k + 1];
    in[k].ia = il[k];
    in[k].ib = il[k + 1];
    inv_nn[k] = S(0);
    if (kind[k] == K_PLANE) {
      in[k].nh = rec[k].f3(12);
    } else if (CURVED && kind[k] == K_PARAB) {
      const S q2 = rec[k].v[14];
      const v3<S> nraw = axpy(-prm[2 * k + 1] * q2, rec[k].f3(4), axpy(-prm[2 * k] * q2, rec[k].f3(0), rec[k].f3(8)));
      inv_nn[k] = rsq(dot(nraw, nraw));
      in[k].nh = nraw * inv_nn[k];
    } else if (!CURVED || kind[k] == K_LINE) {
      in[k].eh = rec[k].f3(4);
    } else {
      S sn, cs;
      sincos_(prm[2 * k], sn, cs);
      in[k].eh = axpy(cs, rec[k].f3(8), rec[k].f3(4) * (-sn));
    }
    curv_c[k] = in[k].refl ? dot(in[k].ih, in[k].nh) : S(0);
  }
  // v = gL dL/dT + gX dX/dT ; dL/dX_k = u[k] - u[k+1]
  S v[Q];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    v3<S> gx = (u[k] - u[k + 1]) * gLs;
    if (gX) gx = gx + mk(ff_from_double(gX[3 * k]), ff_from_double(gX[3 * k + 1]), ff_from_double(gX[3 * k + 2]));
    v[2 * k] = -dot(gx, pt[k].w0);
    v[2 * k + 1] = is_edge(kind[k]) ? S(0) : -dot(gx, pt[k].w1);
  }
  S lam[Q];
  chol_solve<Q, S>(jtj, v, lam);  // solves (J^T J) lam = -v' = gL dL/dT + gX dX/dT
  // z_k = J_k lambda: point displacements D_k = lam_2k w0 + lam_2k+1 w1
  v3<S> D[N];
#pragma unroll
  for (int k = 0; k < N; ++k) D[k] = axpy(lam[2 * k + 1], pt[k].w1, pt[k].w0 * lam[2 * k]);
  v3<S> z[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    v3<S> r = in[k].self(D[k]);
    if (k >= 1) r = r + in[k].prev(D[k - 1]);
    if (k + 1 < N) r = r + in[k].next(D[k + 1]);
    if (CURVED && kind[k] == K_PARAB) {
      // normal variation: 2 (<i, dn> n + <i, n> dn), dn from the parameters
      const S q2 = rec[k].v[14];
      const v3<S> craw = axpy(lam[2 * k + 1], rec[k].f3(4), rec[k].f3(0) * lam[2 * k]) * (-q2);
      const v3<S> dn = axpy(-dot(in[k].nh, craw), in[k].nh, craw) * inv_nn[k];
      r = axpy(S(2) * dot(in[k].ih, dn), in[k].nh, r);
      r = axpy(S(2) * curv_c[k], dn, r);
    } else if (CURVED && kind[k] == K_ARC) {
      S sn, cs;
      sincos_(prm[2 * k], sn, cs);
      const v3<S> de = axpy(-sn, rec[k].f3(8), rec[k].f3(4) * (-cs));
      r.x = r.x + dot(in[k].ih - in[k].rh, de) * lam[2 * k];
    }
    z[k] = r;
  }
  // TX: a displacement of X_0 enters interaction 0 as "previous point"
  if (want_tx) {
    const v3<S> ex = mk(S(1), S(0), S(0)), ey = mk(S(0), S(1), S(0)), ez = mk(S(0), S(0), S(1));
    o.tx[0] = to_double(-gLs * u[0].x - dot(z[0], in[0].prev(ex)));
    o.tx[1] = to_double(-gLs * u[0].y - dot(z[0], in[0].prev(ey)));
    o.tx[2] = to_double(-gLs * u[0].z - dot(z[0], in[0].prev(ez)));
  }
  if (want_rx) {
    const v3<S> ex = mk(S(1), S(0), S(0)), ey = mk(S(0), S(1), S(0)), ez = mk(S(0), S(0), S(1));
    o.rx[0] = to_double(gLs * u[N].x - dot(z[N - 1], in[N - 1].next(ex)));
    o.rx[1] = to_double(gLs * u[N].y - dot(z[N - 1], in[N - 1].next(ey)));
    o.rx[2] = to_double(gLs * u[N].z - dot(z[N - 1], in[N - 1].next(ez)));
  }
  if (want_obj) {
#pragma unroll
    for (int m = 0; m < N; ++m) {
      o.obj[m] = 0.0;
      if (kind[m] != K_PLANE) continue;
      const v3<S> n = rec[m].f3(12);
      S gd = gLs * dot(u[m] - u[m + 1], n);
      if (gX) gd = gd + dot(mk(ff_from_double(gX[3 * m]), ff_from_double(gX[3 * m + 1]), ff_from_double(gX[3 * m + 2])), n);
      gd = gd - dot(z[m], in[m].self(n));
      if (m >= 1) gd = gd - dot(z[m - 1], in[m - 1].next(n));
      if (m + 1 < N) gd = gd - dot(z[m + 1], in[m + 1].prev(n));
      o.obj[m] = to_double(gd);
    }
  }
  return true;
}

// Adds v (W values) at dst + W * key for the lanes with `have`.  When every
// such lane of the warp has the same key (one TX; the objects of one
// sequence), the warp sums first and one lane adds; otherwise each lane adds.
template <int W>
__device__ __forceinline__ void warp_add(double* dst, bool have, int key, const double (&v)[W]) {
  const unsigned act = __ballot_sync(0xffffffffu, have);
  if (act == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(act) - 1;
  const int k0 = __shfl_sync(0xffffffffu, key, leader);
  if (__all_sync(0xffffffffu, !have || key == k0)) {
#pragma unroll
    for (int j = 0; j < W; ++j) {
      double a = have ? v[j] : 0.0;
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
      if (lane == leader) atomicAdd(dst + (int64_t)W * k0 + j, a);
    }
  } else if (have) {
#pragma unroll
    for (int j = 0; j < W; ++j) atomicAdd(dst + (int64_t)W * key + j, v[j]);
  }
}

struct GradView {
  const uint4* rec;
  int64_t rec_cap;
  const int64_t* pcand;
  const double* pT;
  int64_t pcap;
  const int64_t* count;
  const double* g_len;
  const double* g_pts;
};

// One launch per path order: every launch scans all paths and takes those of
// its order (valid paths come sorted by candidate, hence by order, so the
// lanes of a warp agree), and each order gets registers of its own.  The
// loop bounds are uniform over the block so that whole warps reach the
// aggregated atomics together.
// PTS: point weights given (the normal-matrix solve; few registers spare)
// or not (explicit gradient only: a short kernel at full occupancy).
template <int N, bool PTS, bool CURVED>
__global__ void __launch_bounds__(GRAD_BLOCK, (PTS ? (N <= 2 ? 3 : 1) : 4)) k_grad(DevScene sc, DevEnds ep,
                                                                                  GradView gv, double* g_tx,
                                                                                  double* g_rx, double* g_obj) {
  int64_t n = *gv.count;
  if (n > gv.pcap) n = gv.pcap;
  for (int64_t i0 = (int64_t)blockIdx.x * GRAD_BLOCK; i0 < n; i0 += (int64_t)gridDim.x * GRAD_BLOCK) {
    const int64_t i = i0 + threadIdx.x;
    bool have = false;
    GradOut<N> o;
    Cand cd;
    cd.order = 0;
    if (i < n) {
      const int64_t c = gv.pcand[i];
      if (c >= 0 && c < gv.rec_cap) {
        cd = decode(gv.rec[c]);
        if (cd.order == N && cand_in_range(sc, ep, cd)) {
          double Tc[2 * N];
#pragma unroll
          for (int j = 0; j < 2 * N; ++j) Tc[j] = gv.pT[(int64_t)j * gv.pcap + i];
          double gX[3 * N];
          const double* gxp = nullptr;
          if (PTS && gv.g_pts) {
#pragma unroll
            for (int j = 0; j < 3 * N; ++j) gX[j] = gv.g_pts[(int64_t)j * gv.pcap + i];
            gxp = gX;
          }
          have = grad_one<N, CURVED>(sc, ep, cd, Tc, gv.g_len[i], gxp, g_tx != nullptr, g_rx != nullptr,
                             g_obj != nullptr, o);
        }
      }
    }
    if (__ballot_sync(0xffffffffu, have) == 0) continue;
    if (g_tx) warp_add<3>(g_tx, have, o.it, o.tx);
    if (g_rx) warp_add<3>(g_rx, have, o.ir, o.rx);
    if (g_obj) {
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const double v[1] = {o.obj[m]};
        warp_add<1>(g_obj, have && o.obj[m] != 0.0, have ? cd.ids[m] : 0, v);
      }
    }
  }
}

int launch_grad(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                const mpt_paths* paths, const int64_t* d_valid_count, const double* g_len, const double* g_pts,
                double* g_tx, double* g_rx, double* g_obj, cudaStream_t st) {
  if (paths->capacity <= 0) return MPT_OK;
  GradView gv{reinterpret_cast<const uint4*>(cand->rec), cand->capacity, paths->cand, paths->T, paths->capacity, d_valid_count,
              g_len, g_pts};
  int64_t blocks = (paths->capacity + GRAD_BLOCK - 1) / GRAD_BLOCK;
  const int64_t lim = (int64_t)ctx->sms * 8;
  if (blocks > lim) blocks = lim;
  const DevEnds ep = dev_ends(ends);
  // the orders are independent (their sums meet only in atomics): order 2
  // on the caller's stream, orders 1, 3, 4 on the context's auxiliary streams
  MPT_CUDA_TRY(fork_streams(ctx, st));
  const bool curved = scene_curved(scene);
#define MPT_GRAD_K(N, P, CV, S) k_grad<N, P, CV><<<(unsigned)blocks, GRAD_BLOCK, 0, (S)>>>(scene->d, ep, gv, g_tx, g_rx, g_obj)
#define MPT_GRAD(N, S)                                         \
  {                                                            \
    if (g_pts && curved)                                       \
      MPT_GRAD_K(N, true, true, S);                            \
    else if (g_pts)                                            \
      MPT_GRAD_K(N, true, false, S);                           \
    else if (curved)                                           \
      MPT_GRAD_K(N, false, true, S);                           \
    else                                                       \
      MPT_GRAD_K(N, false, false, S);                          \
    MPT_LAUNCH_CHECK();                                        \
  }
  MPT_GRAD(2, st)
  MPT_GRAD(1, ctx->aux[0])
  MPT_GRAD(3, ctx->aux[1])
  MPT_GRAD(4, ctx->aux[2])
#undef MPT_GRAD
#undef MPT_GRAD_K
  MPT_CUDA_TRY(join_streams(ctx, st));
  return MPT_OK;
}

}  // namespace mpt
