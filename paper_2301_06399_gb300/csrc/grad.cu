// Adjoint of converged paths: at a solution rho(T*, theta) = 0 of Eq. 15 the
// implicit-function theorem gives dT/dtheta = -(J^T J)^{-1} J^T drho/dtheta.
// For upstream weights gL (path length) and gX (points), with
//   v = gL dL/dT + gX dX/dT,   lambda = (J^T J)^{-1} v,   z = J lambda,
// the vector-Jacobian product is
//   dtheta += gL dL/dtheta|explicit + gX dX/dtheta|explicit - z^T drho/dtheta.
// theta: TX (a fixed point before interaction 1), RX (after interaction n)
// and the offset d of each plane <n, X> = d (its points move along n).
// One thread per valid path, FP64 throughout (a few thousand paths).
#include "mpt_internal.cuh"

namespace mpt {

constexpr int GRAD_BLOCK = 128;

// Law residual of one interaction and the linear maps that give its rows
// for a displacement w of the previous point, this point and the next point.
struct Inter {
  bool refl;
  v3<double> ih, rh, nh, eh;
  double ia, ib;
  // reflection: H P_i w / a (prev), -(P_r w / b + H P_i w / a) (this), P_r w / b (next)
  // diffraction: -<e, P_i w>/a (prev), <e,P_i w>/a + <e,P_r w>/b (this), -<e, P_r w>/b (next)
  __device__ v3<double> Pi(const v3<double>& w) const { return axpy(-dot(ih, w), ih, w) * ia; }
  __device__ v3<double> Pr(const v3<double>& w) const { return axpy(-dot(rh, w), rh, w) * ib; }
  __device__ v3<double> H(const v3<double>& w) const { return axpy(-2.0 * dot(nh, w), nh, w); }
  // rows (3 for reflection; component x only for diffraction)
  __device__ v3<double> prev(const v3<double>& w) const {
    if (refl) return H(Pi(w));
    return mk(-dot(eh, Pi(w)), 0.0, 0.0);
  }
  __device__ v3<double> self(const v3<double>& w) const {
    if (refl) return -(Pr(w) + H(Pi(w)));
    return mk(dot(eh, Pi(w)) + dot(eh, Pr(w)), 0.0, 0.0);
  }
  __device__ v3<double> next(const v3<double>& w) const {
    if (refl) return Pr(w);
    return mk(-dot(eh, Pr(w)), 0.0, 0.0);
  }
};

template <int N>
__device__ void grad_one(const DevScene& sc, const DevEnds& ep, const Cand& cd, const double* Tc, double gL,
                         const double* gX, double* g_tx, double* g_rx, double* g_obj) {
  constexpr int Q = 2 * N;
  int it_, ir_;
  pair_ends(ep, cd.pair, it_, ir_);
  const v3<double> A = mk(ep.tx[3 * it_], ep.tx[3 * it_ + 1], ep.tx[3 * it_ + 2]);
  const v3<double> B = mk(ep.rx[3 * ir_], ep.rx[3 * ir_ + 1], ep.rx[3 * ir_ + 2]);
  int kind[N];
  Rec<double> rec[N];
  double prm[Q];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    kind[k] = sc.kind[cd.ids[k]];
    rec[k] = load_obj64(sc, cd.ids[k]);
    prm[2 * k] = Tc[2 * k];
    prm[2 * k + 1] = Tc[2 * k + 1];
  }
  // normal matrix at the solution
  double jtj[Q * (Q + 1) / 2], g[Q];
  bool ok;
  eval_path<N, double, double, true>(kind, rec, prm, A, B, jtj, g, ok);
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (is_edge(kind[k])) jtj[tri(2 * k + 1, 2 * k + 1)] = 1.0;
  if (!cholesky<Q, double>(jtj, 0.0)) return;
  // geometry
  PointT<double> pt[N];
#pragma unroll
  for (int k = 0; k < N; ++k) pt[k] = point_at<double, true>(kind[k], rec[k], prm[2 * k], prm[2 * k + 1]);
  v3<double> u[N + 1];
  double il[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const v3<double> a = j == 0 ? A : pt[j - 1].X;
    const v3<double> b = j == N ? B : pt[j].X;
    const v3<double> d = b - a;
    il[j] = rsq(dot(d, d));
    u[j] = d * il[j];
  }
  Inter in[N];
  double curv_c[N];
  double inv_nn[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    in[k].refl = !is_edge(kind[k]);
    in[k].ih = u[k];
    in[k].rh = u[k + 1];
    in[k].ia = il[k];
    in[k].ib = il[k + 1];
    inv_nn[k] = 0.0;
    if (kind[k] == K_PLANE) {
      in[k].nh = rec[k].f3(12);
    } else if (kind[k] == K_PARAB) {
      const double q2 = rec[k].v[14];
      const v3<double> nraw = axpy(-prm[2 * k + 1] * q2, rec[k].f3(4), axpy(-prm[2 * k] * q2, rec[k].f3(0), rec[k].f3(8)));
      inv_nn[k] = rsq(dot(nraw, nraw));
      in[k].nh = nraw * inv_nn[k];
    } else if (kind[k] == K_LINE) {
      in[k].eh = rec[k].f3(4);
    } else {
      double sn, cs;
      sincos_(prm[2 * k], sn, cs);
      in[k].eh = axpy(cs, rec[k].f3(8), rec[k].f3(4) * (-sn));
    }
    curv_c[k] = in[k].refl ? dot(in[k].ih, in[k].nh) : 0.0;
  }
  // v = gL dL/dT + gX dX/dT ; dL/dX_k = u[k] - u[k+1]
  double v[Q];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    v3<double> gx = (u[k] - u[k + 1]) * gL;
    if (gX) gx = gx + mk(gX[3 * k], gX[3 * k + 1], gX[3 * k + 2]);
    v[2 * k] = -dot(gx, pt[k].w0);
    v[2 * k + 1] = is_edge(kind[k]) ? 0.0 : -dot(gx, pt[k].w1);
  }
  double lam[Q];
  chol_solve<Q, double>(jtj, v, lam);  // solves (J^T J) lam = -v' = gL dL/dT + gX dX/dT
  // z_k = J_k lambda: point displacements D_k = lam_2k w0 + lam_2k+1 w1
  v3<double> D[N];
#pragma unroll
  for (int k = 0; k < N; ++k) D[k] = axpy(lam[2 * k + 1], pt[k].w1, pt[k].w0 * lam[2 * k]);
  v3<double> z[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    v3<double> r = in[k].self(D[k]);
    if (k >= 1) r = r + in[k].prev(D[k - 1]);
    if (k + 1 < N) r = r + in[k].next(D[k + 1]);
    if (kind[k] == K_PARAB) {
      // normal variation: 2 (<i, dn> n + <i, n> dn), dn from the parameters
      const double q2 = rec[k].v[14];
      const v3<double> craw = axpy(lam[2 * k + 1], rec[k].f3(4), rec[k].f3(0) * lam[2 * k]) * (-q2);
      const v3<double> dn = axpy(-dot(in[k].nh, craw), in[k].nh, craw) * inv_nn[k];
      r = axpy(2.0 * dot(in[k].ih, dn), in[k].nh, r);
      r = axpy(2.0 * curv_c[k], dn, r);
    } else if (kind[k] == K_ARC) {
      double sn, cs;
      sincos_(prm[2 * k], sn, cs);
      const v3<double> de = axpy(-sn, rec[k].f3(8), rec[k].f3(4) * (-cs));
      r.x += dot(in[k].ih - in[k].rh, de) * lam[2 * k];
    }
    z[k] = r;
  }
  // TX: a displacement of X_0 enters interaction 0 as "previous point"
  if (g_tx) {
    const v3<double> ex = mk(1.0, 0.0, 0.0), ey = mk(0.0, 1.0, 0.0), ez = mk(0.0, 0.0, 1.0);
    const double gx = -gL * u[0].x - dot(z[0], in[0].prev(ex));
    const double gy = -gL * u[0].y - dot(z[0], in[0].prev(ey));
    const double gz = -gL * u[0].z - dot(z[0], in[0].prev(ez));
    atomicAdd(g_tx + 3 * it_, gx);
    atomicAdd(g_tx + 3 * it_ + 1, gy);
    atomicAdd(g_tx + 3 * it_ + 2, gz);
  }
  if (g_rx) {
    const v3<double> ex = mk(1.0, 0.0, 0.0), ey = mk(0.0, 1.0, 0.0), ez = mk(0.0, 0.0, 1.0);
    const double gx = gL * u[N].x - dot(z[N - 1], in[N - 1].next(ex));
    const double gy = gL * u[N].y - dot(z[N - 1], in[N - 1].next(ey));
    const double gz = gL * u[N].z - dot(z[N - 1], in[N - 1].next(ez));
    atomicAdd(g_rx + 3 * ir_, gx);
    atomicAdd(g_rx + 3 * ir_ + 1, gy);
    atomicAdd(g_rx + 3 * ir_ + 2, gz);
  }
  if (g_obj) {
#pragma unroll
    for (int m = 0; m < N; ++m) {
      if (kind[m] != K_PLANE) continue;
      const v3<double> n = rec[m].f3(12);
      double gd = gL * dot(u[m] - u[m + 1], n);
      if (gX) gd += dot(mk(gX[3 * m], gX[3 * m + 1], gX[3 * m + 2]), n);
      gd -= dot(z[m], in[m].self(n));
      if (m >= 1) gd -= dot(z[m - 1], in[m - 1].next(n));
      if (m + 1 < N) gd -= dot(z[m + 1], in[m + 1].prev(n));
      atomicAdd(g_obj + cd.ids[m], gd);
    }
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

__global__ void __launch_bounds__(GRAD_BLOCK) k_grad(DevScene sc, DevEnds ep, GradView gv, double* g_tx,
                                                     double* g_rx, double* g_obj) {
  int64_t n = *gv.count;
  if (n > gv.pcap) n = gv.pcap;
  for (int64_t i = (int64_t)blockIdx.x * GRAD_BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * GRAD_BLOCK) {
    const int64_t c = gv.pcand[i];
    if (c < 0 || c >= gv.rec_cap) continue;
    const Cand cd = decode(gv.rec[c]);
    if (!cand_in_range(sc, ep, cd)) continue;
    double Tc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) Tc[j] = gv.pT[(int64_t)j * gv.pcap + i];
    double gX[12];
    const double* gxp = nullptr;
    if (gv.g_pts) {
#pragma unroll
      for (int j = 0; j < 12; ++j) gX[j] = gv.g_pts[(int64_t)j * gv.pcap + i];
      gxp = gX;
    }
    const double gL = gv.g_len[i];
    switch (cd.order) {
      case 1: grad_one<1>(sc, ep, cd, Tc, gL, gxp, g_tx, g_rx, g_obj); break;
      case 2: grad_one<2>(sc, ep, cd, Tc, gL, gxp, g_tx, g_rx, g_obj); break;
      case 3: grad_one<3>(sc, ep, cd, Tc, gL, gxp, g_tx, g_rx, g_obj); break;
      case 4: grad_one<4>(sc, ep, cd, Tc, gL, gxp, g_tx, g_rx, g_obj); break;
      default: break;
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
  k_grad<<<(unsigned)blocks, GRAD_BLOCK, 0, st>>>(scene->d, dev_ends(ends), gv, g_tx, g_rx, g_obj);
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

}  // namespace mpt
