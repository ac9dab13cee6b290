// Internal declarations shared by the CUDA translation units of libmpt.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "../../include/mpt.h"
#include "ff.cuh"
#include "mpt_math.cuh"

namespace mpt {

// Device view of a scene.  Objects are stored field-major: field f (a float4
// or double2 of the 16-value record) of object o at o32[f * n_obj + o].  The
// solver reads the objects of its candidate's sequence, which every lane of
// a warp shares, so each field load is one broadcast transaction.
struct DevScene {
  int n_obj, n_occ;
  const int32_t* kind;      // [n_obj]
  const float4* o32;        // [4][n_obj]
  const float4* a32;        // [n_obj][4]: the same FP32 records, object-major
  const double2* o64;       // [8][n_obj]
  const int32_t* occ_kind;  // [n_occ]
  const float4* c32;        // [4][n_occ]
  const double2* c64;       // [8][n_occ]
  const int4* obj_occ;      // [n_obj]: up to 4 rectangles whose plane holds every point of the object, -1 padded
  const float4* cbox;       // [2][n_occ]: occluder boxes (lo, hi) grown by 1 cm; lo.w = 0 rectangle, 1 paraboloid
  int n_grp;                // ceil(n_occ / OCC_GROUP)
  const float4* gbox;       // [2][n_grp]: boxes of groups of OCC_GROUP consecutive occluders
  const float4* aff;        // [n_obj][8]: float-float records (head, tail) x 16, object-major
  const int32_t* own_occ;   // [n_obj]: the occluder rectangle that is a plane's own facet, or -1
  const int8_t* side;       // [n_obj][n_obj] or null: side[i*n_obj + j] = +1 (-1) when object j lies wholly
                            // more than 1e-6 S in front of (behind) plane i, else 0 (0 for non-planes i)
  const float4* vtx;        // [n_obj][8] or null: FP32 points whose convex hull holds the object (rectangle
                            // corners, edge ends, paraboloid box corners, arc square corners; the last repeated;
                            // w = the number of distinct points)
  double scale;
};

constexpr int OCC_GROUP = 4;  // occluders per group box

// A segment can only meet an occluder whose box its own box overlaps (the
// boxes are grown by 1 cm at upload, far above FP32 rounding of the ends).
__device__ __forceinline__ bool box_overlap(const float4& lo, const float4& hi, const v3<float>& A,
                                            const v3<float>& B) {
  return fminf(A.x, B.x) <= hi.x && fmaxf(A.x, B.x) >= lo.x && fminf(A.y, B.y) <= hi.y &&
         fmaxf(A.y, B.y) >= lo.y && fminf(A.z, B.z) <= hi.z && fmaxf(A.z, B.z) >= lo.z;
}

// Does the segment A + t d, t in [0, 1], meet the box [lo, hi]?  Slab test
// with inv = 1/d per axis (infinite for an axis the segment does not move
// along).  A NaN (an end exactly on a face plane of an axis it does not move
// along) counts as a miss; the boxes are grown by 1 cm around their
// occluders, so such a segment cannot cross one.
__device__ __forceinline__ bool seg_box(const v3<float>& A, const v3<float>& inv, const float4& lo,
                                        const float4& hi) {
  const float x1 = (lo.x - A.x) * inv.x, x2 = (hi.x - A.x) * inv.x;
  const float y1 = (lo.y - A.y) * inv.y, y2 = (hi.y - A.y) * inv.y;
  const float z1 = (lo.z - A.z) * inv.z, z2 = (hi.z - A.z) * inv.z;
  const float t0 = fmaxf(fmaxf(fminf(x1, x2), fminf(y1, y2)), fmaxf(fminf(z1, z2), 0.f));
  const float t1 = fminf(fminf(fmaxf(x1, x2), fmaxf(y1, y2)), fminf(fmaxf(z1, z2), 1.f));
  return t0 <= t1;
}

struct DevEnds {
  const double* tx;
  const double* rx;
  int n_tx, n_rx, pair_mode;
  // p / n_rx by multiplication: q = (t + ((p - t) >> s1)) >> s2 with
  // t = umulhi(m, p) (Granlund and Montgomery, "Division by invariant
  // integers using multiplication", 1994), exact for every 32-bit p.  A
  // hardware-less integer division would take float conversions, which run
  // on GB300's slow FP64 pipe.
  uint32_t rx_m;
  int rx_s1, rx_s2;
};

__device__ __forceinline__ void pair_ends(const DevEnds& e, uint32_t p, int& it, int& ir) {
  if (e.pair_mode == 0) {
    const uint32_t t = __umulhi(e.rx_m, p);
    const uint32_t q = (t + ((p - t) >> e.rx_s1)) >> e.rx_s2;
    it = (int)q;
    ir = (int)(p - q * (uint32_t)e.n_rx);
  } else {
    it = ir = (int)p;
  }
}

__device__ __forceinline__ Rec<float> load_obj32(const DevScene& s, int o) {
  Rec<float> r;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    float4 q = __ldg(&s.o32[f * s.n_obj + o]);
    r.v[4 * f] = q.x; r.v[4 * f + 1] = q.y; r.v[4 * f + 2] = q.z; r.v[4 * f + 3] = q.w;
  }
  return r;
}
__device__ __forceinline__ Rec<float> load_obj32a(const DevScene& s, int o) {
  Rec<float> r;
  const float4* p = s.a32 + 4 * o;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    float4 q = __ldg(p + f);
    r.v[4 * f] = q.x; r.v[4 * f + 1] = q.y; r.v[4 * f + 2] = q.z; r.v[4 * f + 3] = q.w;
  }
  return r;
}
__device__ __forceinline__ Rec<double> load_obj64(const DevScene& s, int o) {
  Rec<double> r;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    double2 q = __ldg(&s.o64[f * s.n_obj + o]);
    r.v[2 * f] = q.x; r.v[2 * f + 1] = q.y;
  }
  return r;
}

// Scene values in float-float (the refinement's working precision), from
// the copy split into head and tail at upload.
__device__ __forceinline__ Rec<ff> load_obj_ff(const DevScene& s, int o) {
  Rec<ff> r;
  const float4* p = s.aff + 8 * o;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    const float4 q = __ldg(p + f);
    r.v[2 * f] = ff(q.x, q.y);
    r.v[2 * f + 1] = ff(q.z, q.w);
  }
  return r;
}
__device__ __forceinline__ v3<ff> load_end_ff(const double* p, int i) {
  return mk(ff_from_double(__ldg(p + 3 * i)), ff_from_double(__ldg(p + 3 * i + 1)),
            ff_from_double(__ldg(p + 3 * i + 2)));
}

// SplitMix64 output function (Steele, Lea, Flood 2014): mixes x + gamma.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Decoded candidate record (see mpt_candidates in mpt.h).
struct Cand {
  uint32_t pair;
  int ids[4];
  int order, start;
};
__device__ __forceinline__ Cand decode(uint4 r) {
  Cand c;
  c.pair = r.x;
  c.ids[0] = (int)(r.y & 0xFFFFu);
  c.ids[1] = (int)(r.y >> 16);
  c.ids[2] = (int)(r.z & 0xFFFFu);
  c.ids[3] = (int)(r.z >> 16);
  c.order = (int)(r.w & 0xFFu);
  c.start = (int)((r.w >> 8) & 0xFFu);
  return c;
}

// Candidate indices the scene and endpoints can serve (guards against
// records that do not belong to this scene).
__device__ __forceinline__ bool cand_in_range(const DevScene& sc, const DevEnds& ep, const Cand& cd) {
  if (cd.order < 1 || cd.order > 4) return false;
  for (int k = 0; k < cd.order; ++k)
    if (cd.ids[k] >= sc.n_obj) return false;
  int it, ir;
  pair_ends(ep, cd.pair, it, ir);
  return it < ep.n_tx && ir < ep.n_rx;
}

constexpr int SOLVE_BLOCK = 128;

}  // namespace mpt

// ------------------------------------------------------------- handles --
struct mpt_ctx {
  int device;
  int sms;
  // small persistent scratch: work-stealing counters and an error flag
  unsigned long long* counters;  // [64]
  int* err_flag;                 // [1]
  // validate scratch, grown on demand
  void* vscratch;
  size_t vscratch_bytes;
  // solver refine-list scratch, grown on demand
  void* rscratch;
  size_t rscratch_bytes;
  // FP32 endpoint copies, grown on demand
  void* escratch;
  size_t escratch_bytes;
  // candidate exclusion: per-order lists of the iterated candidates and the
  // reflection beams of every endpoint through every plane, grown on demand
  void* xscratch;
  size_t xscratch_bytes;
  // auxiliary streams for independent per-order chains, and the events that
  // fork them from and join them back to the caller's stream
  cudaStream_t aux[3];
  cudaEvent_t ev_fork, ev_join[3];
  // schedules chosen by mpt_autotune, by workload signature (tune.cu)
  void* tune_cache;
  // opt-in timing of each order's solver launch (mpt_ctx_time_solver)
  bool time_solver;
  bool ev_gn_made;
  cudaEvent_t ev_gn[4][2];
};

// Makes the auxiliary streams wait for the work enqueued on st so far.
inline cudaError_t fork_streams(mpt_ctx* ctx, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(ctx->ev_fork, st);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(ctx->aux[i], ctx->ev_fork, 0);
  return e;
}
// Makes st wait for the work enqueued on the auxiliary streams.
inline cudaError_t join_streams(mpt_ctx* ctx, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = cudaEventRecord(ctx->ev_join[i], ctx->aux[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->ev_join[i], 0);
  }
  return e;
}

struct mpt_scene {
  mpt_ctx* ctx;
  mpt::DevScene d;
  void* alloc;             // one device allocation holding every array
  int32_t* host_kind;      // host copy of the kinds
  int n_obj;
  uint64_t signature;      // FNV-1a hash of the uploaded image (workload key of mpt_autotune)
  size_t alloc_bytes;      // size of `alloc`
};

// A scene holds a paraboloid or an arc edge (kernels for planes and
// straight edges alone are instantiated without the curved branches).
inline bool scene_curved(const mpt_scene* s) {
  for (int i = 0; i < s->n_obj; ++i)
    if (s->host_kind[i] == MPT_PARABOLOID || s->host_kind[i] == MPT_ARC_EDGE) return true;
  return false;
}

#define MPT_CUDA_TRY(expr)                                                 \
  do {                                                                     \
    cudaError_t e_ = (expr);                                               \
    if (e_ != cudaSuccess) {                                               \
      std::fprintf(stderr, "libmpt: %s failed: %s\n", #expr, cudaGetErrorString(e_)); \
      return MPT_ERR_CUDA;                                                 \
    }                                                                      \
  } while (0)

#define MPT_LAUNCH_CHECK()                                                  \
  do {                                                                      \
    cudaError_t e_ = cudaGetLastError();                                    \
    if (e_ != cudaSuccess) {                                                \
      std::fprintf(stderr, "libmpt: launch failed: %s\n", cudaGetErrorString(e_)); \
      return MPT_ERR_CUDA;                                                  \
    }                                                                       \
  } while (0)

namespace mpt {
inline DevEnds dev_ends(const mpt_endpoints* e) {
  DevEnds d;
  d.tx = e->tx;
  d.rx = e->rx;
  d.n_tx = e->n_tx;
  d.n_rx = e->n_rx;
  d.pair_mode = e->pair_mode;
  // multiplier for division by n_rx (>= 1): l = ceil(log2 n_rx),
  // m = floor(2^32 (2^l - n_rx) / n_rx) + 1
  const uint32_t dv = e->n_rx > 0 ? (uint32_t)e->n_rx : 1u;
  int l = 0;
  while ((1ull << l) < dv) ++l;
  d.rx_m = (uint32_t)(((1ull << 32) * ((1ull << l) - dv)) / dv + 1);
  d.rx_s1 = l < 1 ? l : 1;
  d.rx_s2 = l - 1 > 0 ? l - 1 : 0;
  return d;
}
inline int64_t n_pairs(const mpt_endpoints* e) {
  return e->pair_mode == 0 ? (int64_t)e->n_tx * e->n_rx : (int64_t)e->n_tx;
}
int check_ends(const mpt_endpoints* e);
// launchers implemented in the .cu files
int launch_solve(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                 const mpt_candidates* cand, int precision, const mpt_schedule* sch,
                 mpt_solutions* out, cudaStream_t st);
int launch_enumerate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, int max_order,
                     const uint8_t* adj, const mpt_sampling* smp, mpt_candidates* out, cudaStream_t st);
int launch_visibility(mpt_ctx* ctx, const mpt_scene* scene, uint8_t* vis, cudaStream_t st);
// Object-side table and vertex table of a scene (DevScene::side, ::vtx),
// rebuilt whenever planes move.
constexpr int SIDE_MAX_OBJ = 4096;
int launch_side_table(const DevScene& d, cudaStream_t st);
int launch_image(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                 mpt_solutions* out, cudaStream_t st);
void tune_cache_free(mpt_ctx* ctx);
int launch_shift_planes(mpt_ctx* ctx, const mpt_scene* base, mpt_scene* dst, const double* delta, cudaStream_t st);
int autotune(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
             int precision, mpt_solutions* out, mpt_schedule* best, double* best_ms, cudaStream_t st);
// FNV-1a (Fowler, Noll, Vo) over a byte range, continuing from h.
inline uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}
int launch_field(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                 const mpt_paths* paths, const int64_t* d_valid_count, const mpt_field_params* fp, double* field,
                 cudaStream_t st);
int launch_validate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                    const mpt_candidates* cand, const mpt_solutions* sol, double tau, mpt_paths* out,
                    int64_t* d_valid_count, cudaStream_t st);
int launch_grad(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                const mpt_candidates* cand, const mpt_paths* paths, const int64_t* d_valid_count,
                const double* g_len, const double* g_pts, double* g_tx, double* g_rx, double* g_obj,
                cudaStream_t st);
}  // namespace mpt
