// find_minimum_path of Algorithm 1 for every candidate: Gauss-Newton on the
// cost of Eq. 15 with a backtracking line search, one thread per candidate.
//
// Precision modes:
//   MPT_FP32             FP32 iterations only
//   MPT_FP32_FP64REFINE  FP32 iterations; candidates whose FP32 cost is below
//                        1e-8 and whose parameters lie inside their bounds up
//                        to 1e-2 m then take 1-2 Gauss-Newton steps with the
//                        residual in FP64 (Jacobian and solve in FP32) and an
//                        FP64 cost.  Every other candidate is certainly
//                        rejected by validation, so it keeps its FP32 result.
//   MPT_FP64_PLAIN       the same algorithm in FP64 throughout
//
// Scheduling: a persistent grid (blocks_per_sm x SMs) per path order; blocks
// claim tiles of consecutive candidates from a global counter (work
// stealing), so uneven convergence does not leave SMs idle.  The candidate
// layout puts pairs fastest, so a warp shares one object sequence and all
// scene loads are broadcasts.
#include <type_traits>

#include "mpt_internal.cuh"

namespace mpt {

struct SolveCfg {
  int max_iters;
  int refine_steps;
  float c_tol32, step_tol32;
  double c_tol64, step_tol64;
  double diverge;
  float prescreen_cost, prescreen_margin;
  float mu32;
  double mu64;
};

struct CandView {
  const uint4* rec;
  int64_t cap;
  const int64_t* order_begin;
  uint64_t init_seed;
};

struct SolView {
  double* T;
  double* cost;
  uint8_t* status;
  uint8_t* iters;
  uint8_t* evals;
  float* T32;
  int64_t cap;
};

template <class R>
__device__ __forceinline__ Rec<R> load_obj(const DevScene& s, int o);
template <>
__device__ __forceinline__ Rec<float> load_obj<float>(const DevScene& s, int o) { return load_obj32(s, o); }
template <>
__device__ __forceinline__ Rec<double> load_obj<double>(const DevScene& s, int o) { return load_obj64(s, o); }

// Uniform draw in [0,1) from three chained SplitMix64 rounds over (pair),
// (packed ids), (start*16 + k*2 + comp); the top 24 bits of the last output.
__device__ __forceinline__ float unit_draw(uint64_t seed, uint32_t pair, uint64_t packed, int start, int k,
                                           int comp) {
  uint64_t h = splitmix64(seed ^ (uint64_t)pair);
  h = splitmix64(h ^ packed);
  h = splitmix64(h ^ (uint64_t)(start * 16 + k * 2 + comp));
  return (float)(h >> 40) * (1.0f / 16777216.0f);
}

// Initial parameters (Algorithm 1, random_guess): start 0 projects TX (first
// half of the sequence, 2k < n) or RX (second half) onto the object; starts
// > 0 draw curved objects uniformly over their disc / angle range.
template <class R>
__device__ __forceinline__ void init_params(int kind, const Rec<R>& r, const v3<R>& Y, uint64_t seed,
                                            uint32_t pair, uint64_t packed, int start, int k, R& s, R& t) {
  t = R(0);
  if (kind == K_PLANE) {
    v3<R> w = Y - r.f3(0);
    s = dot(w, r.f3(4));
    t = dot(w, r.f3(8));
  } else if (kind == K_LINE) {
    s = dot(Y - r.f3(0), r.f3(4));
  } else if (kind == K_PARAB) {
    if (start == 0) {
      v3<R> w = Y - mk(r.v[3], r.v[7], r.v[11]);
      s = dot(w, r.f3(0));
      t = dot(w, r.f3(4));
    } else {
      const R rad = r.v[13] * R(sqrtf(unit_draw(seed, pair, packed, start, k, 0)));
      const R th = R(6.283185307179586) * R(unit_draw(seed, pair, packed, start, k, 1));
      R sn, cs;
      sincos_(th, sn, cs);
      s = rad * cs;
      t = rad * sn;
    }
  } else {
    if (start == 0) {
      v3<R> w = Y - r.f3(0);
      s = atan2(dot(w, r.f3(8)), dot(w, r.f3(4)));
    } else {
      s = r.v[7] + R(unit_draw(seed, pair, packed, start, k, 0)) * (r.v[11] - r.v[7]);
    }
  }
}

// Parameters inside the object's bounds, grown by margin m (metres).
template <class R>
__device__ __forceinline__ bool in_bounds_margin(int kind, const Rec<R>& r, R s, R t, R m) {
  if (kind == K_PLANE) return s >= -m && s <= r.v[3] + m && t >= -m && t <= r.v[7] + m;
  if (kind == K_PARAB) return s * s + t * t <= (r.v[13] + m) * (r.v[13] + m);
  if (kind == K_LINE) return s >= r.v[3] - m && s <= r.v[7] + m;
  const R twopi = R(6.283185307179586);
  R d = s - r.v[7];
  d = d - twopi * floor(d / twopi);
  const R ma = m / r.v[3];
  return d <= (r.v[11] - r.v[7]) + ma || d >= twopi - ma;
}

// Edge objects use one parameter: pin the unused slot (identity row, zero rhs).
template <int N, class J>
__device__ __forceinline__ void pin_unused(const int (&kind)[N], J* jtj, J* g) {
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (is_edge(kind[k])) {
      jtj[tri(2 * k + 1, 2 * k + 1)] = J(1);
      g[2 * k + 1] = J(0);
    }
}

// Gauss-Newton with backtracking: each evaluation returns the cost and the
// normal equations at the trial point; an accepted trial's normal equations
// give the next step directly (no separate Jacobian pass).
template <int N, class R>
struct GN {
  static constexpr int Q = 2 * N;
  static constexpr int P = Q * (Q + 1) / 2;
  R prm[Q];
  R cost;
  int iters, evals, reason;
  bool finite;

  __device__ __forceinline__ void run(const int (&kind)[N], const Rec<R> (&rec)[N], const v3<R>& A,
                                      const v3<R>& B, int max_iters, R c_tol, R step_tol, R diverge, R mu) {
    R jtj[P], g[Q], dlt[Q];
    bool ok;
    cost = eval_path<N, R, R, true>(kind, rec, prm, A, B, jtj, g, ok);
    evals = 1;
    iters = 0;
    reason = MPT_PATH_MAXITER;
    finite = ok && isfinite(cost);
    if (!finite) { reason = MPT_PATH_NONFINITE; return; }
    if (cost < c_tol) { reason = MPT_PATH_CONVERGED; return; }
    pin_unused<N, R>(kind, jtj, g);
    cholesky<Q, R>(jtj, mu);
    chol_solve<Q, R>(jtj, g, dlt);
    R alpha = R(1);
    for (int it = 0; it < max_iters; ++it) {
      R trial[Q];
      R smax = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        trial[i] = fma_(alpha, dlt[i], prm[i]);
        smax = fmax(smax, fabs(alpha * dlt[i]));
      }
      R ct = eval_path<N, R, R, true>(kind, rec, trial, A, B, jtj, g, ok);
      ++evals;
      if (ok && ct < cost) {
#pragma unroll
        for (int i = 0; i < Q; ++i) prm[i] = trial[i];
        cost = ct;
        ++iters;
        R pmax = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) pmax = fmax(pmax, fabs(prm[i]));
        if (!(pmax <= diverge)) { reason = MPT_PATH_DIVERGED; return; }
        if (cost < c_tol || smax < step_tol) { reason = MPT_PATH_CONVERGED; return; }
        pin_unused<N, R>(kind, jtj, g);
        cholesky<Q, R>(jtj, mu);
        chol_solve<Q, R>(jtj, g, dlt);
        alpha = R(1);
      } else {
        alpha = alpha * R(0.5);
        if (alpha < R(1.0 / 64.0)) { reason = MPT_PATH_STALLED; return; }
      }
    }
  }
};

template <int N, int PREC>
__device__ __forceinline__ void solve_one(const DevScene& sc, const DevEnds& ep, const CandView& cv,
                                          const SolView& out, const SolveCfg& cfg, int64_t c) {
  using R = typename std::conditional<PREC == MPT_FP64_PLAIN, double, float>::type;
  constexpr int Q = 2 * N;
  const Cand cd = decode(__ldg(cv.rec + c));
  if (!cand_in_range(sc, ep, cd) || cd.order != N) {
    out.cost[c] = (double)INFINITY;
    out.status[c] = (uint8_t)MPT_PATH_NONFINITE;
    out.iters[c] = 0;
    out.evals[c] = 0;
    return;
  }
  int it_, ir_;
  pair_ends(ep, cd.pair, it_, ir_);
  const v3<double> A64 = mk(__ldg(ep.tx + 3 * it_), __ldg(ep.tx + 3 * it_ + 1), __ldg(ep.tx + 3 * it_ + 2));
  const v3<double> B64 = mk(__ldg(ep.rx + 3 * ir_), __ldg(ep.rx + 3 * ir_ + 1), __ldg(ep.rx + 3 * ir_ + 2));
  const v3<R> A = cvt<R>(A64), B = cvt<R>(B64);
  int kind[N];
  Rec<R> rec[N];
  uint64_t packed = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) packed |= (uint64_t)(uint16_t)(k < N ? cd.ids[k] : 0xFFFF) << (16 * k);
  GN<N, R> gn;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    kind[k] = __ldg(sc.kind + cd.ids[k]);
    rec[k] = load_obj<R>(sc, cd.ids[k]);
    init_params<R>(kind[k], rec[k], (2 * k < N) ? A : B, cv.init_seed, cd.pair, packed, cd.start, k,
                   gn.prm[2 * k], gn.prm[2 * k + 1]);
  }
  if (PREC == MPT_FP64_PLAIN)
    gn.run(kind, rec, A, B, cfg.max_iters, R(cfg.c_tol64), R(cfg.step_tol64), R(cfg.diverge), R(cfg.mu64));
  else
    gn.run(kind, rec, A, B, cfg.max_iters, R(cfg.c_tol32), R(cfg.step_tol32), R(cfg.diverge), R(cfg.mu32));

  int status = gn.reason;
  double cost = (double)gn.cost;
  double T64[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) T64[i] = (double)gn.prm[i];
  if (out.T32 != nullptr) {
#pragma unroll
    for (int i = 0; i < Q; ++i) out.T32[(int64_t)i * out.cap + c] = (float)gn.prm[i];
  }
  if (PREC == MPT_FP64_PLAIN) {
    status |= MPT_PATH_REFINED;
  } else if (PREC == MPT_FP32_FP64REFINE) {
    bool pass = gn.finite && gn.cost < R(cfg.prescreen_cost) && status != MPT_PATH_DIVERGED;
#pragma unroll
    for (int k = 0; k < N; ++k)
      pass = pass && in_bounds_margin<R>(kind[k], rec[k], gn.prm[2 * k], gn.prm[2 * k + 1],
                                         R(cfg.prescreen_margin));
    if (pass) {
      // FP64 refinement: residual and cost in FP64, Jacobian and solve in FP32
      Rec<double> r64[N];
#pragma unroll
      for (int k = 0; k < N; ++k) r64[k] = load_obj64(sc, cd.ids[k]);
      float jtj[Q * (Q + 1) / 2], g[Q], dlt[Q];
      bool ok;
      double c64 = eval_path<N, double, float, true>(kind, r64, T64, A64, B64, jtj, g, ok);
      int ev = 1;
      for (int s = 0; s < cfg.refine_steps && ok && c64 >= 1e-28; ++s) {
        pin_unused<N, float>(kind, jtj, g);
        cholesky<Q, float>(jtj, cfg.mu32);
        chol_solve<Q, float>(jtj, g, dlt);
#pragma unroll
        for (int i = 0; i < Q; ++i) T64[i] += (double)dlt[i];
        c64 = eval_path<N, double, float, true>(kind, r64, T64, A64, B64, jtj, g, ok);
        ++ev;
      }
      cost = ok ? c64 : (double)INFINITY;
      (void)ev;
      status |= MPT_PATH_REFINED;
    } else {
      status |= MPT_PATH_PRESCREENED;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (i < Q) out.T[(int64_t)i * out.cap + c] = T64[i];
  out.cost[c] = cost;
  out.status[c] = (uint8_t)status;
  out.iters[c] = (uint8_t)min(gn.iters, 255);
  out.evals[c] = (uint8_t)min(gn.evals, 255);
}

template <int N, int PREC>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_solve(DevScene sc, DevEnds ep, CandView cv, SolView out,
                                                       SolveCfg cfg, unsigned long long* counter) {
  int64_t end = cv.order_begin[N];
  if (end > cv.cap) end = cv.cap;
  int64_t begin = cv.order_begin[N - 1];
  if (begin > end) begin = end;
  __shared__ int64_t s_base;
  for (;;) {
    if (threadIdx.x == 0) s_base = begin + (int64_t)atomicAdd(counter, 1ull) * SOLVE_BLOCK;
    __syncthreads();
    const int64_t base = s_base;
    __syncthreads();
    if (base >= end) break;
    const int64_t c = base + threadIdx.x;
    if (c < end) solve_one<N, PREC>(sc, ep, cv, out, cfg, c);
  }
}

// One launch over every order: each thread dispatches on its candidate's
// order (warp-uniform except where a tile straddles two orders).
template <int PREC>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_solve_mixed(DevScene sc, DevEnds ep, CandView cv,
                                                             SolView out, SolveCfg cfg,
                                                             unsigned long long* counter) {
  int64_t end = cv.order_begin[4];
  if (end > cv.cap) end = cv.cap;
  __shared__ int64_t s_base;
  for (;;) {
    if (threadIdx.x == 0) s_base = (int64_t)atomicAdd(counter, 1ull) * SOLVE_BLOCK;
    __syncthreads();
    const int64_t base = s_base;
    __syncthreads();
    if (base >= end) break;
    const int64_t c = base + threadIdx.x;
    if (c < end) {
      const int order = (int)(__ldg(&cv.rec[c].w) & 0xFFu);
      switch (order) {
        case 1: solve_one<1, PREC>(sc, ep, cv, out, cfg, c); break;
        case 2: solve_one<2, PREC>(sc, ep, cv, out, cfg, c); break;
        case 3: solve_one<3, PREC>(sc, ep, cv, out, cfg, c); break;
        default: solve_one<4, PREC>(sc, ep, cv, out, cfg, c); break;
      }
    }
  }
}

template <int PREC>
static int launch_prec(mpt_ctx* ctx, DevScene sc, DevEnds ep, CandView cv, SolView sv, SolveCfg cfg,
                       const mpt_schedule* sch, cudaStream_t st) {
  MPT_CUDA_TRY(cudaMemsetAsync(ctx->counters, 0, 8 * sizeof(unsigned long long), st));
  const int bps = (sch && sch->blocks_per_sm > 0) ? sch->blocks_per_sm : 0;
  auto grid_for = [&](const void* fn) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, SOLVE_BLOCK, 0);
    if (occ < 1) occ = 1;
    int per = bps > 0 ? (bps < occ ? bps : occ) : occ;
    return ctx->sms * per;
  };
  if (sch && sch->mixed_orders) {
    const void* fn = (const void*)k_solve_mixed<PREC>;
    k_solve_mixed<PREC><<<grid_for(fn), SOLVE_BLOCK, 0, st>>>(sc, ep, cv, sv, cfg, ctx->counters + 4);
    MPT_LAUNCH_CHECK();
    return MPT_OK;
  }
  k_solve<1, PREC><<<grid_for((const void*)k_solve<1, PREC>), SOLVE_BLOCK, 0, st>>>(sc, ep, cv, sv, cfg,
                                                                                    ctx->counters + 0);
  MPT_LAUNCH_CHECK();
  k_solve<2, PREC><<<grid_for((const void*)k_solve<2, PREC>), SOLVE_BLOCK, 0, st>>>(sc, ep, cv, sv, cfg,
                                                                                    ctx->counters + 1);
  MPT_LAUNCH_CHECK();
  k_solve<3, PREC><<<grid_for((const void*)k_solve<3, PREC>), SOLVE_BLOCK, 0, st>>>(sc, ep, cv, sv, cfg,
                                                                                    ctx->counters + 2);
  MPT_LAUNCH_CHECK();
  k_solve<4, PREC><<<grid_for((const void*)k_solve<4, PREC>), SOLVE_BLOCK, 0, st>>>(sc, ep, cv, sv, cfg,
                                                                                    ctx->counters + 3);
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

int launch_solve(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                 int precision, const mpt_schedule* sch, mpt_solutions* out, cudaStream_t st) {
  SolveCfg cfg;
  cfg.max_iters = (sch && sch->max_iters > 0) ? (sch->max_iters > 255 ? 255 : sch->max_iters) : 48;
  cfg.refine_steps = (sch && sch->refine_steps > 0) ? (sch->refine_steps > 2 ? 2 : sch->refine_steps) : 2;
  const double S = scene->d.scale;
  cfg.c_tol32 = 1e-12f;
  cfg.step_tol32 = (float)(1e-6 * S);
  cfg.c_tol64 = 1e-30;
  cfg.step_tol64 = 1e-14 * S;
  cfg.diverge = 1e3 * S;
  cfg.prescreen_cost = 1e-8f;
  cfg.prescreen_margin = 1e-2f;
  cfg.mu32 = 1e-6f;
  cfg.mu64 = 1e-12;
  CandView cv{reinterpret_cast<const uint4*>(cand->rec), cand->capacity, cand->order_begin, cand->init_seed};
  SolView sv{out->T, out->cost, out->status, out->iters, out->evals, out->T32, out->capacity};
  DevEnds ep = dev_ends(ends);
  switch (precision) {
    case MPT_FP64_PLAIN: return launch_prec<MPT_FP64_PLAIN>(ctx, scene->d, ep, cv, sv, cfg, sch, st);
    case MPT_FP32: return launch_prec<MPT_FP32>(ctx, scene->d, ep, cv, sv, cfg, sch, st);
    case MPT_FP32_FP64REFINE: return launch_prec<MPT_FP32_FP64REFINE>(ctx, scene->d, ep, cv, sv, cfg, sch, st);
    default: return MPT_ERR_ARG;
  }
}

}  // namespace mpt
