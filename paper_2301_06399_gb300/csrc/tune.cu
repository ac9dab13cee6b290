// Autotuner of the solver's schedule (mpt_autotune): the batching of
// Algorithm 1's loop over candidates x starts has knobs whose best values
// depend on the workload's mix of orders, kinds and convergence, none of
// which change any solution:
//   tile           candidates a warp claims at once (work stealing granularity)
//   refill_min     idle lanes that trigger taking new candidates
//   blocks_per_sm  resident blocks of the persistent solver grids
//   mixed_orders   one persistent launch over every order, or one per order
//   prescreen      visibility prescreen before the refinement (on / off)
//   warp_orders    orders whose FP32 iterations run one candidate per warp
//                  (none, 4, 3-4, all) instead of one per lane
// (the iteration cap is part of the method's stopping rule and is not tuned).
// The search is a coordinate descent from the library defaults, two sweeps,
// each trial timed with CUDA events as the best of two solves after a
// warm-up.  The chosen schedule is cached in the context by a workload
// signature: the scene's content hash, the candidate layout (count and order
// ranges, read back from the device), the endpoints' shape and the precision.
#include <unordered_map>

#include "mpt_internal.cuh"

namespace mpt {

struct TuneEntry {
  mpt_schedule sched;
  double ms;
};
using TuneCache = std::unordered_map<uint64_t, TuneEntry>;

void tune_cache_free(mpt_ctx* ctx) {
  delete static_cast<TuneCache*>(ctx->tune_cache);
  ctx->tune_cache = nullptr;
}

static mpt_schedule default_schedule() {
  mpt_schedule s{};
  s.block = SOLVE_BLOCK;
  return s;
}

// Best of `reps` timed solves (milliseconds), or a negative status.
static double time_solve(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                         const mpt_candidates* cand, int precision, const mpt_schedule* sch, mpt_solutions* out,
                         cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps) {
  double best = 1e30;
  for (int r = 0; r < reps; ++r) {
    if (cudaEventRecord(e0, st) != cudaSuccess) return -MPT_ERR_CUDA;
    const int rc = launch_solve(ctx, scene, ends, cand, precision, sch, out, st);
    if (rc != MPT_OK) return -rc;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -MPT_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -MPT_ERR_CUDA;
    if (ms < best) best = ms;
  }
  return best;
}

int autotune(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
             int precision, mpt_solutions* out, mpt_schedule* best, double* best_ms, cudaStream_t st) {
  // workload signature
  int64_t ob[5] = {0, 0, 0, 0, 0};
  if (cudaMemcpyAsync(ob, cand->order_begin, sizeof(ob), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MPT_ERR_CUDA;
  uint64_t key = fnv1a(&scene->signature, sizeof(uint64_t));
  key = fnv1a(ob, sizeof(ob), key);
  const int64_t shape[6] = {cand->capacity, (int64_t)ends->n_tx, (int64_t)ends->n_rx, (int64_t)ends->pair_mode,
                            (int64_t)precision, (int64_t)cand->init_seed};
  key = fnv1a(shape, sizeof(shape), key);
  if (!ctx->tune_cache) ctx->tune_cache = new TuneCache();
  TuneCache& cache = *static_cast<TuneCache*>(ctx->tune_cache);
  const auto hit = cache.find(key);
  if (hit != cache.end()) {
    *best = hit->second.sched;
    if (best_ms) *best_ms = hit->second.ms;
    return MPT_OK;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MPT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MPT_ERR_CUDA;
  }
  mpt_schedule cur = default_schedule();
  int rc = MPT_OK;
  // warm-up (scratch growth, first launches), then the defaults' time
  double t = time_solve(ctx, scene, ends, cand, precision, &cur, out, st, e0, e1, 1);
  if (t >= 0) t = time_solve(ctx, scene, ends, cand, precision, &cur, out, st, e0, e1, 2);
  double t_best = t;
  if (t < 0) rc = (int)-t;
  struct Knob {
    int32_t mpt_schedule::*field;
    int values[6];
    int n;
  };
  const Knob knobs[] = {
      {&mpt_schedule::tile, {128, 96, 64, 32}, 4},
      {&mpt_schedule::refill_min, {12, 4, 6, 8, 16, 20}, 6},
      {&mpt_schedule::blocks_per_sm, {0, 4, 3, 2}, 4},
      {&mpt_schedule::mixed_orders, {0, 1}, 2},
      {&mpt_schedule::prescreen, {1, 2}, precision == MPT_FP32_FP64REFINE ? 2 : 0},
      {&mpt_schedule::warp_orders, {0, 8, 12, 15}, precision == MPT_FP64_PLAIN ? 0 : 4},
  };
  for (int sweep = 0; sweep < 2 && rc == MPT_OK; ++sweep) {
    bool moved = false;
    for (const Knob& k : knobs) {
      for (int i = 0; i < k.n && rc == MPT_OK; ++i) {
        if (cur.*(k.field) == k.values[i]) continue;
        mpt_schedule trial = cur;
        trial.*(k.field) = k.values[i];
        const double tt = time_solve(ctx, scene, ends, cand, precision, &trial, out, st, e0, e1, 2);
        if (tt < 0) {
          rc = (int)-tt;
          break;
        }
        // a move needs a 1% gain: timing noise does not wander the choice
        if (tt < 0.99 * t_best) {
          t_best = tt;
          cur = trial;
          moved = true;
        }
      }
    }
    if (!moved) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MPT_OK) return rc;
  cache[key] = TuneEntry{cur, t_best};
  *best = cur;
  if (best_ms) *best_ms = t_best;
  return MPT_OK;
}

}  // namespace mpt
