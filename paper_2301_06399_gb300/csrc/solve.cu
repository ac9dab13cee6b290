// find_minimum_path of Algorithm 1 for every candidate: Gauss-Newton on the
// cost of Eq. 15 with a backtracking line search, one lane per candidate.
//
// Kernel A (k_gn): a persistent grid per path order.  Each lane runs a small
// state machine; every pass of the loop performs exactly one evaluation
// (cost + normal equations at the lane's trial point) and then accepts,
// backtracks or finishes.  Lanes that finish take the next candidates of
// their warp's piece of the range (consecutive candidates, so the lanes share
// one object sequence and take the same branches), so lanes stay busy
// although candidates converge after different numbers of iterations.  No
// block-level barriers.  Endpoints are read from FP32 copies and results are
// widened to FP64 on the integer units: the FP64 pipe stays idle.
//
// Kernel B (k_refine, MPT_FP32_FP64REFINE only): candidates whose FP32 cost
// is below 1e-6, whose parameters lie within 0.1 m of their bounds and that
// the visibility prescreen does not reject are refined with mixed steps
// (residual and cost in float-float, Jacobian in FP32); ill-conditioned ones
// (near object creases) go on to a full Gauss-Newton solve (k_refine_fb, in
// FP64 spread over the lanes of a warp by default; FP64 or float-float on one
// lane on request).
// Every other candidate is rejected by validation whatever its last digits,
// so it keeps its FP32 result.
//
// MPT_FP64_PLAIN runs kernel A in FP64 (the plain GPU method); MPT_FP32 runs
// kernel A only.
#include <type_traits>

#include "eval_f2.cuh"
#include "ff.cuh"
#include "mpt_internal.cuh"

namespace mpt {

struct SolveCfg {
  int max_iters, max_evals;
  int refill_min, piece;
  int refine_steps, fallback_iters;
  float min_alpha, localmin_cost, localmin_ratio, localmin_ratio_planar;
  float c_tol32, step_tol32;
  double c_tol64, step_tol64;
  double diverge;
  float prescreen_cost, prescreen_margin;
  float mu32;
  double mu64;
  int prescreen;     // 1: visibility prescreen before the refinement
  int exclude;       // 1: half-space exclusion before iterating
  int fallback;  // k_refine_fb mode: FB_FF, FB_F64 or FB_F64_WARP
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

// Per-order refine lists: positions (candidate - first candidate of the
// order) stored in idx[first of the order ...], counts in count[order - 1].
// The first list (queued by the solver) also carries, per entry, bit 31 of
// idx = "FP32 cost below the visibility-prescreen threshold", the FP32
// parameters in prm[j * stride + entry] and the object ids and endpoint
// indices in ends[entry] (ids01, ids23, TX index, RX index), so that the
// prescreen reads neither the candidate record, the cost nor the FP64
// parameters back.
struct RefineList {
  unsigned long long* count;  // [4]
  int32_t* idx;               // [cap]
  float* prm;                 // [8][stride] or null
  uint4* ends;                // [stride] or null
  int64_t stride;
};
constexpr int32_t RL_VIS = (int32_t)0x80000000;  // idx flag: prescreen the visibility
constexpr float PRESCREEN_VIS_COST = 1e-10f;

constexpr unsigned FULL = 0xffffffffu;
constexpr int CHUNK = 256;  // candidates a warp claims at once (8 per lane)

// FP32 copies of the endpoints, made once per solve call.
__global__ void k_ends_f32(const double* tx, int n_tx, const double* rx, int n_rx, float4* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_tx) out[i] = make_float4((float)tx[3 * i], (float)tx[3 * i + 1], (float)tx[3 * i + 2], 0.f);
  else if (i < n_tx + n_rx) {
    const int j = i - n_tx;
    out[i] = make_float4((float)rx[3 * j], (float)rx[3 * j + 1], (float)rx[3 * j + 2], 0.f);
  }
}

template <class R>
__device__ __forceinline__ v3<R> load_end(const double* p64, const float4* p32, int i);
template <>
__device__ __forceinline__ v3<float> load_end<float>(const double*, const float4* p32, int i) {
  const float4 q = __ldg(p32 + i);
  return mk(q.x, q.y, q.z);
}
template <>
__device__ __forceinline__ v3<double> load_end<double>(const double* p64, const float4*, int i) {
  return mk(__ldg(p64 + 3 * i), __ldg(p64 + 3 * i + 1), __ldg(p64 + 3 * i + 2));
}
__device__ __forceinline__ double to_f64(float x) { return f2d_bits(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

template <class R>
__device__ __forceinline__ Rec<R> load_obj(const DevScene& s, int o);
template <>
__device__ __forceinline__ Rec<float> load_obj<float>(const DevScene& s, int o) { return load_obj32a(s, o); }
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
template <class R, bool CURVED = true>
__device__ __forceinline__ void init_params(int kind, const Rec<R>& r, const v3<R>& Y, uint64_t seed,
                                            uint32_t pair, uint64_t packed, int start, int k, R& s, R& t) {
  t = R(0);
  if (kind == K_PLANE) {
    v3<R> w = Y - r.f3(0);
    s = dot(w, r.f3(4));
    t = dot(w, r.f3(8));
  } else if (!CURVED || kind == K_LINE) {
    // (a solver built for planes and straight edges only sees these two)
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

// ------------------------------------------- kind patterns (planar scenes) --
// A sequence of planes and straight edges has a kind pattern PAT: bit k set
// when interaction k is an edge (one parameter, slot 2k), clear for a plane
// (two parameters, slots 2k and 2k+1).  With the pattern known at compile
// time every kind test of the evaluation folds away, an edge's record is two
// float4 instead of four, and the normal equations are factored over the
// live parameters only (the pinned slot of an edge holds exact zeros off the
// diagonal, so dropping it changes no other entry of the factor or the step).
template <int N, int PAT>
struct KindPat {
  static constexpr bool edge(int k) { return ((PAT >> k) & 1) != 0; }
  static constexpr int nq() {
    int q = 0;
    for (int k = 0; k < N; ++k) q += edge(k) ? 1 : 2;
    return q;
  }
  static constexpr int Q = nq();
  // slot (in the two-per-interaction layout) of live parameter i
  static constexpr int slot(int i) {
    int q = 0;
    for (int k = 0; k < N; ++k) {
      if (q++ == i) return 2 * k;
      if (!edge(k) && q++ == i) return 2 * k + 1;
    }
    return 0;
  }
};

// Gauss-Newton step over the live parameters of pattern PAT: the normal
// equations (packed over 2N slots) are gathered, factored with relative
// damping mu and solved; dead slots get a zero step.
template <int N, int PAT, class J>
__device__ __forceinline__ void gn_step_pat(const J* jtj, const J* g, J mu, J* dlt) {
  using KP = KindPat<N, PAT>;
  constexpr int QC = KP::Q;
  J a[QC * (QC + 1) / 2], gc[QC], x[QC];
#pragma unroll
  for (int i = 0; i < QC; ++i) {
    gc[i] = g[KP::slot(i)];
#pragma unroll
    for (int j = 0; j <= i; ++j) a[tri(i, j)] = jtj[tri(KP::slot(i), KP::slot(j))];
  }
  cholesky<QC, J>(a, mu);
  chol_solve<QC, J>(a, gc, x);
#pragma unroll
  for (int k = 0; k < 2 * N; ++k) dlt[k] = J(0);
#pragma unroll
  for (int i = 0; i < QC; ++i) dlt[KP::slot(i)] = x[i];
}

// Object record of a compile-time kind from the object-major FP32 copy: a
// plane needs all four float4 (O U | u V | v d | n), an edge the first two
// (P t0 | e t1).
template <bool EDGE>
__device__ __forceinline__ Rec<float> load_obj32_kind(const DevScene& s, int o) {
  Rec<float> r;
  const float4* p = s.a32 + 4 * o;
#pragma unroll
  for (int f = 0; f < (EDGE ? 2 : 4); ++f) {
    const float4 q = __ldg(p + f);
    r.v[4 * f] = q.x; r.v[4 * f + 1] = q.y; r.v[4 * f + 2] = q.z; r.v[4 * f + 3] = q.w;
  }
  if (EDGE) {
#pragma unroll
    for (int i = 8; i < 16; ++i) r.v[i] = 0.f;
  }
  return r;
}

template <class R, bool EDGE>
__device__ __forceinline__ Rec<R> load_obj_kind(const DevScene& s, int o) {
  if constexpr (std::is_same<R, float>::value)
    return load_obj32_kind<EDGE>(s, o);
  else
    return load_obj64(s, o);
}

// ------------------------------------------------------- exclusion pass --
// Two necessary conditions of Eq. 8 for a reflection on a bounded plane,
// tested once per candidate before any iteration (k_exclude):
//  - half-space: the outgoing segment leaves on the side of the plane that
//    the incoming one came from, so the neighbouring points of a reflection
//    lie on one side of its plane;
//  - beam: the outgoing ray is the ray from the mirror image of the previous
//    point through the reflection point, so for the first reflection the
//    next point lies in the pyramid from TX's image through the rectangle
//    (likewise for the last reflection with RX's image, backwards).
// A candidate failing either, with margins, has no path whose points lie
// inside their objects' bounds (its cost there stays above ~1e-11): it is
// written as excluded, and the others go, per order, to a list that the
// solvers iterate.  Margins: an endpoint more than 1e-5 S off the plane, an
// object wholly more than 1e-6 S off it (the FP64 side table), an object (or
// RX) wholly more than 1e-5 S outside a face of the pyramid, which is only
// used when the endpoint is more than 1e-2 S off the plane.
constexpr int BEAM_F4 = 5;  // float4 per (endpoint, object): image and signed distance, four faces (n, <n, apex>)

__device__ __forceinline__ float plane_dist32(const DevScene& s, int o, const float4& X) {
  const float4 q0 = __ldg(s.a32 + 4 * o), q3 = __ldg(s.a32 + 4 * o + 3);
  return dot(mk(q3.x, q3.y, q3.z), mk(X.x - q0.x, X.y - q0.y, X.z - q0.z));
}

// Beam of every endpoint e (TX 0..n_tx-1, then RX) through every plane o:
// beams[(e * n_obj + o) * BEAM_F4 + 0] = (image of e in the plane, signed
// distance h of e from the plane), + 1 + f = face f of the pyramid from the
// image through the rectangle (unit normal pointing into it, <normal,
// image>).  FP32, with the geometry taken relative to the rectangle's origin
// (magnitudes of the scene's size: rounding ~1e-5 m, a hundredth of the
// margins).  Non-planes get h = 0.  Grid: x over objects, y over endpoints.
__global__ void k_beams(DevScene sc, const float4* ends32, int n_ends, float4* beams) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = blockIdx.y;
  if (o >= sc.n_obj || e >= n_ends) return;
  float4* out = beams + ((int64_t)e * sc.n_obj + o) * BEAM_F4;
  if (__ldg(sc.kind + o) != K_PLANE) {
    out[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const Rec<float> r = load_obj32a(sc, o);
  const v3<float> O = r.f3(0), u = r.f3(4), v = r.f3(8), nrm = r.f3(12);
  const float4 pe = __ldg(ends32 + e);
  const v3<float> p = mk(pe.x, pe.y, pe.z) - O;  // the endpoint relative to O
  const float h = dot(nrm, p);
  const v3<float> pi = axpy(-2.0f * h, nrm, p);  // its image, relative to O
  const v3<float> C[4] = {mk(0.f, 0.f, 0.f), u * r.v[3], axpy(r.v[7], v, u * r.v[3]), v * r.v[7]};
  const v3<float> cen = axpy(0.5f * r.v[7], v, u * (0.5f * r.v[3]));
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    v3<float> nn = cross(C[f] - pi, C[(f + 1) & 3] - pi);
    if (dot(nn, cen - pi) < 0.f) nn = -nn;
    nn = nn * rsqrtf(dot(nn, nn));
    // offset in absolute coordinates: <n, O> + <n, image - O>
    out[1 + f] = make_float4(nn.x, nn.y, nn.z, dot(nn, O) + dot(nn, pi));
  }
  out[0] = make_float4(pi.x + O.x, pi.y + O.y, pi.z + O.z, h);
}

// Do the points X[0..NP) all lie more than m outside one face of beam b?
template <int NP>
__device__ __forceinline__ bool outside_beam(const float4* b, const float4 (&X)[NP], float m) {
  bool out = false;
#pragma unroll
  for (int f = 1; f <= 4; ++f) {
    const float4 q = __ldg(b + f);
    bool all = true;
#pragma unroll
    for (int k = 0; k < NP; ++k) all = all && fmaf(q.x, X[k].x, fmaf(q.y, X[k].y, q.z * X[k].z)) - q.w < -m;
    out = out || all;
  }
  return out;
}

// Exclusion bits of a reflection on plane a next to endpoint e (TX before
// the first reflection, RX after the last) and a neighbouring object b:
// xbits[(e * n_obj + a) * words + b / 32] bit b % 32 set when the
// half-space or the beam condition rules b out.  A lane holds one object b
// (its distinct vertices in registers) and a warp one word of 32 objects;
// the warp walks a range of (e, a) pairs, whose beam faces are the same for
// every lane: the range's beams (contiguous) are first copied to shared
// memory by the whole warp, so that no iteration waits on an L2 read.
constexpr int XBITS_PAIRS = 16;  // (e, a) pairs a warp walks (enough warps per SM to hide the staging)

__global__ void __launch_bounds__(128) k_exclusion_bits(DevScene sc, const float4* beams, int n_ends, int words,
                                                        uint32_t* xbits, float m_end, float m_beam, float h_min) {
  const int lane = threadIdx.x & 31;
  const int no = sc.n_obj;
  const int64_t total = (int64_t)n_ends * no;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int w = (int)(gw % words);                       // the word: objects 32 w ..
  const int64_t q0 = (gw / words) * XBITS_PAIRS;         // the first (e, a) pair
  if (q0 >= total) return;                               // warp-uniform
  const int b = w * 32 + lane;
  __shared__ float4 sbeam[4][XBITS_PAIRS * BEAM_F4];
  float4* sb = sbeam[(threadIdx.x >> 5) & 3];
  const int64_t q1 = q0 + XBITS_PAIRS < total ? q0 + XBITS_PAIRS : total;
  const int nq = (int)(q1 - q0);
  for (int i = lane; i < nq * BEAM_F4; i += 32) sb[i] = __ldg(beams + q0 * BEAM_F4 + i);
  __syncwarp();
  float4 V[8];
  int nv = 0;
  if (b < no) {
#pragma unroll
    for (int k = 0; k < 8; ++k) V[k] = __ldg(sc.vtx + (int64_t)b * 8 + k);
    nv = (int)V[0].w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) V[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  int a = (int)(q0 % no);
  for (int64_t q = q0; q < q1; ++q) {
    bool ex = false;
    if (__ldg(sc.kind + a) == K_PLANE && b < no && b != a) {
      const float4* bm = sb + (q - q0) * BEAM_F4;
      const float h = bm->w;
      const int cls = __ldg(sc.side + (int64_t)a * no + b);
      ex = (h > m_end && cls < 0) || (h < -m_end && cls > 0);
      if (fabsf(h) > h_min) {
#pragma unroll
        for (int f = 1; f <= 4; ++f) {
          const float4 fq = bm[f];
          bool all = true;
#pragma unroll
          for (int k = 0; k < 8; ++k)
            all = all && (k >= nv || fmaf(fq.x, V[k].x, fmaf(fq.y, V[k].y, fq.z * V[k].z)) - fq.w < -m_beam);
          ex = ex || all;
        }
      }
    }
    const unsigned m = __ballot_sync(FULL, ex);
    if (lane == 0) xbits[q * words + w] = m;
    if (++a == no) a = 0;
  }
}

__device__ __forceinline__ bool xbit(const uint32_t* xbits, int words, int64_t e, int no, int a, int b) {
  return (__ldg(xbits + (e * no + a) * words + (b >> 5)) >> (b & 31)) & 1u;
}

// The exclusion conditions for a candidate of order n (ids, kinds, endpoint
// indices): table lookups for the first and last reflections, the endpoint
// test of a single reflection, the side table for inner reflections.
__device__ __forceinline__ bool excluded(const DevScene& sc, const DevEnds& ep, const float4* ends32,
                                         const float4* beams, const uint32_t* xbits, int words, int n,
                                         const int (&id)[4], const int (&kind)[4], int it_, int ir_) {
  const float m_end = (float)(1e-5 * sc.scale), m_beam = (float)(1e-5 * sc.scale);
  const float h_min = (float)(1e-2 * sc.scale);
  const int no = sc.n_obj;
  // the last interaction and the one before it (selects, not indexing)
  const int idl = n == 1 ? id[0] : n == 2 ? id[1] : n == 3 ? id[2] : id[3];
  const int kl = n == 1 ? kind[0] : n == 2 ? kind[1] : n == 3 ? kind[2] : kind[3];
  const int idp = n == 2 ? id[0] : n == 3 ? id[1] : id[2];
  if (kind[0] == K_PLANE) {
    if (n == 1) {
      const float4* bm = beams + ((int64_t)it_ * no + id[0]) * BEAM_F4;
      const float a = __ldg(&bm->w);
      const float4 B = __ldg(ends32 + ep.n_tx + ir_);
      const float b = plane_dist32(sc, id[0], B);
      if ((a > m_end && b < -m_end) || (a < -m_end && b > m_end)) return true;
      const float4 X[1] = {B};
      if (fabsf(a) > h_min && outside_beam<1>(bm, X, m_beam)) return true;
    } else if (xbit(xbits, words, it_, no, id[0], id[1])) {
      return true;
    }
  }
  if (n >= 2 && kl == K_PLANE && xbit(xbits, words, (int64_t)ep.n_tx + ir_, no, idl, idp)) return true;
#pragma unroll
  for (int k = 1; k < 3; ++k)
    if (k + 1 < n && kind[k] == K_PLANE) {
      const int c0 = __ldg(sc.side + (int64_t)id[k] * no + id[k - 1]);
      const int c1 = __ldg(sc.side + (int64_t)id[k] * no + id[k + 1]);
      if (c0 * c1 < 0) return true;
    }
  return false;
}

__device__ __forceinline__ void write_excluded(const SolView& out, int64_t c) {
  out.cost[c] = (double)INFINITY;
  out.status[c] = (uint8_t)MPT_PATH_EXCLUDED;
  out.iters[c] = 0;
  out.evals[c] = 0;
}

// Eight candidates per lane, a warp on 256 consecutive ones per iteration:
// excluded candidates are written; the others (and records the solvers
// reject as malformed) are appended to the list of their order range,
// list[order_begin[o-1] + i] = candidate - order_begin[o-1], counts in
// list_count[o-1], in candidate order within the warp's 256.  The appends
// of the 256 take one atomic per order present (one counter takes every
// append, so its atomics would otherwise bound the pass).
constexpr int XC_PER_LANE = 8;

__global__ void __launch_bounds__(256) k_exclude(DevScene sc, DevEnds ep, const float4* ends32, const float4* beams,
                                                 const uint32_t* xbits, int words, CandView cv, SolView out,
                                                 int32_t* list, unsigned long long* list_count) {
  int64_t ob[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) ob[k] = cv.order_begin[k] < cv.cap ? cv.order_begin[k] : cv.cap;
  const int64_t total = ob[4];
  const unsigned lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 * XC_PER_LANE < total;
       w += n_warps) {
    const int64_t c0 = w * 32 * XC_PER_LANE + lane;
    uint32_t keep_bits = 0;  // bit j: candidate c0 + 32 j is kept
    int ord_of[XC_PER_LANE];
#pragma unroll
    for (int j = 0; j < XC_PER_LANE; ++j) {
      const int64_t c = c0 + 32 * j;
      ord_of[j] = 0;
      if (c < total) {
        const int ord = 1 + (c >= ob[1]) + (c >= ob[2]) + (c >= ob[3]);
        ord_of[j] = ord;
        const uint4 rr = __ldg(cv.rec + c);
        const int n = (int)(rr.w & 0xFFu);
        int id[4], kind[4] = {K_LINE, K_LINE, K_LINE, K_LINE};
        bool valid = n == ord;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          id[k] = (int)(((k < 2 ? rr.y : rr.z) >> (16 * (k & 1))) & 0xFFFFu);
          if (k < n) valid = valid && id[k] < sc.n_obj;
        }
        int it_, ir_;
        pair_ends(ep, rr.x, it_, ir_);
        valid = valid && it_ < ep.n_tx && ir_ < ep.n_rx;
        if (valid) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (k < n) kind[k] = __ldg(sc.kind + id[k]);
        }
        if (valid && excluded(sc, ep, ends32, beams, xbits, words, n, id, kind, it_, ir_))
          write_excluded(out, c);
        else
          keep_bits |= 1u << j;
      }
    }
    // appends: per order present, one atomic for the warp's 256
#pragma unroll
    for (int o = 1; o <= 4; ++o) {
      unsigned m[XC_PER_LANE];
      int cnt = 0;
#pragma unroll
      for (int j = 0; j < XC_PER_LANE; ++j) {
        m[j] = __ballot_sync(FULL, ((keep_bits >> j) & 1u) && ord_of[j] == o);
        cnt += __popc(m[j]);
      }
      if (cnt == 0) continue;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(list_count + (o - 1), (unsigned long long)cnt);
      base = __shfl_sync(FULL, base, 0);
#pragma unroll
      for (int j = 0; j < XC_PER_LANE; ++j) {
        if ((m[j] >> lane) & 1u)
          list[ob[o - 1] + (int64_t)base + __popc(m[j] & lt_mask)] = (int32_t)(c0 + 32 * j - ob[o - 1]);
        base += __popc(m[j]);
      }
    }
  }
}

// ------------------------------------------------------------- kernel A --
// The lanes of one warp solve the candidates of order N in [begin, end).
// With a counter, the warp claims pieces of the range as it goes (work
// stealing between warps); without one it walks [begin, end) piece by
// piece.  order_base = first candidate of order N (refine-list base).
//
// Candidate records are staged in shared memory: every claimed piece is
// copied there by cp.async (16 bytes per lane per copy) one piece ahead of
// its use, so that taking a new candidate costs a shared-memory read
// instead of a DRAM round trip.  Object records and endpoints are read from
// global memory (L1-resident, the same address for the lanes of a warp) at
// every evaluation instead of being held in registers across iterations.
//
// A lane that finishes keeps its result and goes idle; idle lanes write their
// results and take new candidates together, once cfg.refill_min of them are
// idle (or nothing else is running), so the narrow write/refill code runs for
// many lanes at once instead of once per finishing lane.
//
// Pieces are cfg.piece candidates while the range is long and shrink to 32
// as it runs out (guided self-scheduling: about half of what is left, split
// over every warp), so that warps run out of work at nearly the same time.
constexpr int GN_CHUNK = 128;  // records per staged piece (the largest piece)
constexpr int GN_WARPS = SOLVE_BLOCK / 32;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// Calls f(std::integral_constant<int, PAT>) for the lane's kind pattern, so
// that each pattern runs its own compile-time specialisation (lanes of one
// warp share a pattern except where a piece straddles two sequences).
template <int N, class F>
__device__ __forceinline__ void dispatch_pat(int pat, F&& f) {
  using std::integral_constant;
  if constexpr (N == 1) {
    if (pat == 0) f(integral_constant<int, 0>{});
    else f(integral_constant<int, 1>{});
  } else if constexpr (N == 2) {
    switch (pat) {
      case 0: f(integral_constant<int, 0>{}); break;
      case 1: f(integral_constant<int, 1>{}); break;
      case 2: f(integral_constant<int, 2>{}); break;
      default: f(integral_constant<int, 3>{}); break;
    }
  } else {
    f(integral_constant<int, -1>{});
  }
}

template <int N, class R>
__device__ __forceinline__ void load_objs(const DevScene& sc, uint32_t ids01, uint32_t ids23, Rec<R> (&rec)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const uint32_t w = k < 2 ? ids01 : ids23;
    rec[k] = load_obj<R>(sc, (int)((w >> (16 * (k & 1))) & 0xFFFFu));
  }
}

template <int N, int PREC, bool CURVED>
__device__ __forceinline__ void gn_warp(const DevScene& sc, const DevEnds& ep, const float4* ends32,
                                        const CandView& cv, const SolView& out, const SolveCfg& cfg,
                                        unsigned long long* counter, const RefineList& rl, int64_t begin,
                                        int64_t end, int64_t cand_base, int64_t order_base, const int32_t* list,
                                        uint4 (*rbuf)[GN_CHUNK], int32_t (*ibuf)[GN_CHUNK]) {
  using R = typename std::conditional<PREC == MPT_FP64_PLAIN, double, float>::type;
  constexpr int Q = 2 * N, P = Q * (Q + 1) / 2;
  const unsigned lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const R c_tol = R(PREC == MPT_FP64_PLAIN ? cfg.c_tol64 : (double)cfg.c_tol32);
  const R step_tol = R(PREC == MPT_FP64_PLAIN ? cfg.step_tol64 : (double)cfg.step_tol32);
  const R diverge = R(cfg.diverge);
  const R mu = R(PREC == MPT_FP64_PLAIN ? cfg.mu64 : (double)cfg.mu32);

  // per lane: candidate c (offset from begin; -1 = idle) and its data
  int c = -1;
  int done_c = -1;  // finished candidate whose result is not written yet
  int done_status = 0;
  bool done_push = false;
  bool exhausted = false;
  uint32_t ids01 = 0, ids23 = 0;  // object ids, 16 bits each
  int kinds = 0;                  // object kinds, 8 bits each
  int pat = 0;                    // kind pattern (bit k: interaction k is an edge)
  uint32_t pair_ = 0;             // TX/RX pair and start index (curved starts)
  int start_ = 0;
  int it_ = 0, ir_ = 0;
  R prm[Q], trial[Q], dlt[Q];
  R cost = R(0), alpha = R(1);
  R lm_ratio = R(cfg.localmin_ratio_planar);  // local-minimum test of this sequence
  int iters = 0, evals = 0;
  bool fresh = false;

  // ---- warp-uniform staging of candidate records: the current piece (being
  // taken from) and the next one (in flight)
  int64_t walk = begin;  // past the last piece seen
  // guided piece size: about half of what is left, split over every warp
  const float inv_2warps = 0.5f / (float)(gridDim.x * (blockDim.x >> 5));
  auto claim = [&](int64_t& base, int& len) {
    int size = cfg.piece;
    if (counter != nullptr) {
      // guided size from the last position seen (a slight lag is harmless)
      const int64_t guided = (int64_t)((float)(int)(end - walk) * inv_2warps);
      if (guided < size) size = guided < 32 ? 32 : (int)guided;
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(counter, (unsigned long long)size);
      b = __shfl_sync(FULL, b, 0);
      base = begin + (int64_t)b;
      walk = base + size;
    } else {
      base = walk;
      walk += size;
    }
    len = base < end ? (int)(end - base < size ? end - base : size) : 0;
  };
  // positions [begin, end) are candidates cand_base + position, or with a
  // list, candidates cand_base + list[position]
  auto stage = [&](int b, int64_t base, int len) {
    for (int k = lane; k < len; k += 32) {
      if (list != nullptr) {
        const int32_t v = __ldg(list + base + k);
        ibuf[b][k] = v;
        cp_async16(&rbuf[b][k], cv.rec + cand_base + v);
      } else {
        cp_async16(&rbuf[b][k], cv.rec + base + k);
      }
    }
    cp_async_commit();
  };
  int buf = 0;
  int64_t cur_base, nxt_base;
  int cur_len, nxt_len, cur_pos = 0;
  claim(cur_base, cur_len);
  stage(0, cur_base, cur_len);
  claim(nxt_base, nxt_len);
  stage(1, nxt_base, nxt_len);
  cp_async_wait<1>();
  __syncwarp();

  for (;;) {
    const unsigned idle = __ballot_sync(FULL, c < 0);
    if (idle == FULL || __popc(idle) >= cfg.refill_min) {
      // ---- write the results waiting in idle lanes
      if (done_c >= 0) {
        const int64_t dc = cand_base + done_c;
#pragma unroll
        for (int i = 0; i < Q; ++i) out.T[(int64_t)i * out.cap + dc] = to_f64(prm[i]);
        if (out.T32 != nullptr) {
#pragma unroll
          for (int i = 0; i < Q; ++i) out.T32[(int64_t)i * out.cap + dc] = (float)prm[i];
        }
        out.cost[dc] = to_f64(cost);
        out.status[dc] = (uint8_t)done_status;
        out.iters[dc] = (uint8_t)min(iters, 255);
        out.evals[dc] = (uint8_t)min(evals, 255);
      }
      if (PREC == MPT_FP32_FP64REFINE) {
        const unsigned pm = __ballot_sync(FULL, done_push);
        if (pm) {
          const int leader = __ffs(pm) - 1;
          unsigned long long base = 0;
          if ((int)lane == leader) base = atomicAdd(rl.count + (N - 1), (unsigned long long)__popc(pm));
          base = __shfl_sync(FULL, base, leader);
          if (done_push) {
            const int64_t pos = (int64_t)base + __popc(pm & lt_mask);
            const int64_t at = order_base + pos;
            rl.idx[at] = (int32_t)(cand_base + done_c - order_base) | (cost < R(PRESCREEN_VIS_COST) ? RL_VIS : 0);
            if (rl.prm != nullptr) {
#pragma unroll
              for (int i = 0; i < Q; ++i) rl.prm[(int64_t)i * rl.stride + at] = (float)prm[i];
              rl.ends[at] = make_uint4(ids01, ids23, (uint32_t)it_, (uint32_t)ir_);
            }
          }
        }
      }
      done_c = -1;
      done_push = false;
      // ---- take the next candidates from the staged pieces
      bool need = (c < 0) && !exhausted;
      unsigned need_mask = __ballot_sync(FULL, need);
      while (need_mask) {
        if (cur_pos >= cur_len) {
          if (nxt_len == 0) break;  // the range is done
          // the next piece becomes current; stage the one after it
          buf ^= 1;
          cur_base = nxt_base;
          cur_len = nxt_len;
          cur_pos = 0;
          cp_async_wait<0>();
          __syncwarp();
          claim(nxt_base, nxt_len);
          stage(buf ^ 1, nxt_base, nxt_len);
        }
        const int avail = cur_len - cur_pos;
        const int nneed = __popc(need_mask);
        const int rank = __popc(need_mask & lt_mask);
        const bool take = need && rank < avail;
        const int slot = cur_pos + rank;
        cur_pos += nneed < avail ? nneed : avail;
        if (take) {
          need = false;
          const int64_t idx = list != nullptr ? cand_base + ibuf[buf][slot] : cur_base + slot;
          const uint4 rr = rbuf[buf][slot];
          // a record of this solver's order whose objects and endpoints exist
          bool valid = (int)(rr.w & 0xFFu) == N;
#pragma unroll
          for (int k = 0; k < N; ++k)
            valid = valid && (int)(((k < 2 ? rr.y : rr.z) >> (16 * (k & 1))) & 0xFFFFu) < sc.n_obj;
          int t_, r_;
          pair_ends(ep, rr.x, t_, r_);
          valid = valid && t_ < ep.n_tx && r_ < ep.n_rx;
          if (valid) {
            it_ = t_;
            ir_ = r_;
            // only the record is decoded here; the initial guess is made in
            // the first pass, from the records and endpoints it loads anyway
            c = (int)(idx - cand_base);
            ids01 = rr.y;
            ids23 = rr.z;
            pair_ = rr.x;
            start_ = (int)((rr.w >> 8) & 0xFFu);
            kinds = 0;
            pat = 0;
            lm_ratio = R(cfg.localmin_ratio_planar);
#pragma unroll
            for (int k = 0; k < N; ++k) {
              const int kd = __ldg(sc.kind + (int)(((k < 2 ? rr.y : rr.z) >> (16 * (k & 1))) & 0xFFFFu));
              kinds |= kd << (8 * k);
              pat |= (kd == K_LINE ? 1 : 0) << k;
              if (CURVED && (kd == K_PARAB || kd == K_ARC)) lm_ratio = R(cfg.localmin_ratio);
            }
            fresh = true;
            iters = 0;
            evals = 0;
            alpha = R(1);
          } else {
            out.cost[idx] = (double)INFINITY;
            out.status[idx] = (uint8_t)MPT_PATH_NONFINITE;
            out.iters[idx] = 0;
            out.evals[idx] = 0;
          }
        }
        need_mask = __ballot_sync(FULL, need);
      }
      if (cur_pos >= cur_len && nxt_len == 0 && c < 0) exhausted = true;
    }
    if (__ballot_sync(FULL, c >= 0) == 0) {
      if (__ballot_sync(FULL, !exhausted || done_c >= 0) == 0) break;
      continue;
    }
    // ---- one evaluation at the trial point.  PAT >= 0: the kind pattern
    // of a planar sequence, fixed at compile time; PAT < 0: kinds decoded at
    // run time (curved scenes, the FP64 method).
    auto pass = [&](auto pat_c) {
      constexpr int PAT = decltype(pat_c)::value;
      int kind[N];
      Rec<R> rec[N];
      if constexpr (PAT >= 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const uint32_t w = k < 2 ? ids01 : ids23;
          const int o = (int)((w >> (16 * (k & 1))) & 0xFFFFu);
          kind[k] = KindPat<N, PAT>::edge(k) ? K_LINE : K_PLANE;
          if (KindPat<N, PAT>::edge(k))
            rec[k] = load_obj_kind<R, true>(sc, o);
          else
            rec[k] = load_obj_kind<R, false>(sc, o);
        }
      } else {
#pragma unroll
        for (int k = 0; k < N; ++k) kind[k] = (kinds >> (8 * k)) & 0xFF;
        load_objs<N, R>(sc, ids01, ids23, rec);
      }
      const v3<R> A = load_end<R>(ep.tx, ends32, it_);
      const v3<R> B = load_end<R>(ep.rx, ends32 + ep.n_tx, ir_);
      if (fresh) {
        // initial guess (Algorithm 1, random_guess); the ids hash (unused
        // slots 0xFFFF) seeds the extra starts of curved objects only
        uint64_t packed = 0;
        if constexpr (CURVED) {
          packed = (uint64_t)ids01 | ((uint64_t)ids23 << 32);
          if constexpr (N < 4) packed |= ~0ull << (16 * (N < 4 ? N : 0));
        }
#pragma unroll
        for (int k = 0; k < N; ++k)
          init_params<R, CURVED>(kind[k], rec[k], (2 * k < N) ? A : B, cv.init_seed, pair_, packed, start_, k,
                                 trial[2 * k], trial[2 * k + 1]);
      }
      R jtj[P], g[Q];
      bool ok;
      R ct;
      if constexpr (std::is_same<R, float>::value)
        ct = eval_path_f2<N, CURVED>(kind, rec, trial, A, B, jtj, g, ok);
      else
        ct = eval_path<N, R, R, true, CURVED>(kind, rec, trial, A, B, jtj, g, ok);
      ++evals;
      int done = -1;
      bool factor = false;
      if (fresh) {
        fresh = false;
#pragma unroll
        for (int i = 0; i < Q; ++i) prm[i] = trial[i];
        cost = ct;
        if (!(ok && isfinite(ct))) done = MPT_PATH_NONFINITE;
        else if (cost < c_tol) done = MPT_PATH_CONVERGED;
        else factor = true;
      } else if (ok && ct < cost) {
        R smax = R(0), pmax = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (PAT >= 0 && KindPat<N, (PAT < 0 ? 0 : PAT)>::edge(i / 2) && (i & 1)) continue;  // dead slot
          smax = fmax(smax, fabs(trial[i] - prm[i]));
          prm[i] = trial[i];
          pmax = fmax(pmax, fabs(prm[i]));
        }
        cost = ct;
        ++iters;
        if (!(pmax <= diverge)) done = MPT_PATH_DIVERGED;
        else if (cost < c_tol || smax < step_tol) done = MPT_PATH_CONVERGED;
        else if (iters >= cfg.max_iters) done = MPT_PATH_MAXITER;
        else factor = true;
      } else {
        alpha = alpha * R(0.5);
        if (alpha < R(cfg.min_alpha)) done = MPT_PATH_STALLED;
      }
      if (done < 0 && evals >= cfg.max_evals) done = MPT_PATH_MAXITER;
      if (factor && done < 0) {
        if constexpr (PAT >= 0) {
          gn_step_pat<N, PAT, R>(jtj, g, mu, dlt);
        } else {
          pin_unused<N, R>(kind, jtj, g);
          cholesky<Q, R>(jtj, mu);
          chol_solve<Q, R>(jtj, g, dlt);
        }
        alpha = R(1);
        // The Gauss-Newton model predicts the decrease -g.dlt; when it is a
        // small fraction of a large cost the iterate sits at a local minimum
        // with non-zero residual: no path of this sequence is near.  The
        // fraction is 0.1 for planes and straight edges, 1e-4 when a
        // paraboloid or an arc bends the cost away from its model.
        R pred = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) pred = fma_(-g[i], dlt[i], pred);
        if (iters >= 2 && cost > R(cfg.localmin_cost) && pred < lm_ratio * cost) done = MPT_PATH_STALLED;
      }
      if (done < 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) trial[i] = fma_(alpha, dlt[i], prm[i]);
      } else {
        // ---- finish: keep the result for the next batched write
        int status = done;
        if (PREC == MPT_FP64_PLAIN) status |= MPT_PATH_REFINED;
        bool pass = false;
        if (PREC == MPT_FP32_FP64REFINE) {
          pass = isfinite(cost) && cost < R(cfg.prescreen_cost) && done != MPT_PATH_DIVERGED;
#pragma unroll
          for (int k = 0; k < N; ++k)
            pass = pass && in_bounds_margin<R>(kind[k], rec[k], prm[2 * k], prm[2 * k + 1], R(cfg.prescreen_margin));
          if (!pass) status |= MPT_PATH_PRESCREENED;
        }
        done_c = c;
        done_status = status;
        done_push = pass;
        c = -1;
      }
    };
    if (c >= 0) {
      if constexpr (!CURVED && PREC != MPT_FP64_PLAIN && N <= 2)
        dispatch_pat<N>(pat, pass);
      else
        pass(std::integral_constant<int, -1>{});
    }
  }
  cp_async_wait<0>();  // nothing left in flight when the warp leaves
  __syncwarp();
}

// Resident blocks per SM the register allocation is held to: orders 1-2 of
// the FP32 solvers (the bulk of the work) 5 blocks of 128 threads (96
// registers), 4 for scenes with curved objects (5 spilled: measured 3.5%
// faster on the curved scene); orders 3-4 three (168 registers, no spill;
// measured 5% faster on order 4 than two), curved order 4 two (three would
// spill); the FP64 method fewer.
template <int N, int PREC, bool CURVED>
constexpr int gn_min_blocks() {
  if (PREC == MPT_FP64_PLAIN) return N <= 2 ? 2 : 1;
  if (N <= 2) return CURVED ? 4 : 5;
  return (N == 4 && CURVED) ? 2 : 3;
}

template <int N, int PREC, bool CURVED>
__global__ void __launch_bounds__(SOLVE_BLOCK, gn_min_blocks<N, PREC, CURVED>())
    k_gn(DevScene sc, DevEnds ep, const float4* ends32, CandView cv, SolView out, SolveCfg cfg,
         unsigned long long* counter, RefineList rl, const int32_t* list, const unsigned long long* list_count) {
  __shared__ __align__(16) uint4 rbuf[GN_WARPS][2][GN_CHUNK];
  __shared__ int32_t ibuf[GN_WARPS][2][GN_CHUNK];
  int64_t end = cv.order_begin[N];
  if (end > cv.cap) end = cv.cap;
  int64_t begin = cv.order_begin[N - 1];
  if (begin > end) begin = end;
  if (list != nullptr) {
    // the candidates of this order that the exclusion pass kept
    const int64_t n = (int64_t)*list_count < end - begin ? (int64_t)*list_count : end - begin;
    gn_warp<N, PREC, CURVED>(sc, ep, ends32, cv, out, cfg, counter, rl, 0, n, begin, begin, list + begin,
                             rbuf[threadIdx.x >> 5], ibuf[threadIdx.x >> 5]);
  } else {
    gn_warp<N, PREC, CURVED>(sc, ep, ends32, cv, out, cfg, counter, rl, begin, end, begin, begin, nullptr,
                             rbuf[threadIdx.x >> 5], ibuf[threadIdx.x >> 5]);
  }
}

// One launch over every order (uneven orders and convergence in one
// persistent grid): warps claim CHUNK-sized pieces of the whole candidate
// range and solve each piece with the solver of its order (a piece that
// straddles an order boundary is split).  Registers are those of the order-4
// solver, so per-order launches are faster when the orders come in large
// uniform ranges; mpt_autotune times both for a workload.
template <int PREC>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_gn_mixed(DevScene sc, DevEnds ep, const float4* ends32,
                                                          CandView cv, SolView out, SolveCfg cfg,
                                                          unsigned long long* counter, RefineList rl) {
  __shared__ __align__(16) uint4 rbuf[GN_WARPS][2][GN_CHUNK];
  int64_t total = cv.order_begin[4];
  if (total > cv.cap) total = cv.cap;
  const unsigned lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)CHUNK);
    base = __shfl_sync(FULL, base, 0);
    int64_t s = (int64_t)base;
    if (s >= total) break;
    const int64_t e = s + CHUNK < total ? s + CHUNK : total;
    while (s < e) {
      const int o = (int)(__ldg(&cv.rec[s].w) & 0xFFu);
      int64_t oe = (o >= 1 && o <= 4) ? cv.order_begin[o] : s + 1;
      if (oe > e) oe = e;
      if (oe <= s) oe = s + 1;
      const int64_t ob = (o >= 1 && o <= 4) ? cv.order_begin[o - 1] : 0;
      switch (o) {
        case 1: gn_warp<1, PREC, true>(sc, ep, ends32, cv, out, cfg, nullptr, rl, s, oe, s, ob, nullptr, rbuf[threadIdx.x >> 5], nullptr); break;
        case 2: gn_warp<2, PREC, true>(sc, ep, ends32, cv, out, cfg, nullptr, rl, s, oe, s, ob, nullptr, rbuf[threadIdx.x >> 5], nullptr); break;
        case 3: gn_warp<3, PREC, true>(sc, ep, ends32, cv, out, cfg, nullptr, rl, s, oe, s, ob, nullptr, rbuf[threadIdx.x >> 5], nullptr); break;
        case 4: gn_warp<4, PREC, true>(sc, ep, ends32, cv, out, cfg, nullptr, rl, s, oe, s, ob, nullptr, rbuf[threadIdx.x >> 5], nullptr); break;
        default:
          if (lane == 0) {
            out.cost[s] = (double)INFINITY;
            out.status[s] = (uint8_t)MPT_PATH_NONFINITE;
            out.iters[s] = 0;
            out.evals[s] = 0;
          }
          break;
      }
      s = oe;
    }
  }
}

// ----------------------------------------------------- visibility prescreen --
// Candidates queued for refinement whose FP32 solution is well converged
// (cost < 1e-10) and has a segment that crosses an occluder rectangle with a
// clearance of CLEAR_M on every side (both ends CLEAR_M off the plane, the
// crossing CLEAR_M inside the rectangle) are certainly blocked after
// refinement too (the refinement moves a converged point by orders of
// magnitude less), so they are rejected here; the others go to the second
// list that k_refine processes.  Paraboloid occluders never reject here.
constexpr float CLEAR_M = 0.25f;

// seg_box on paired FP32 instructions, for boxes stored as (lo.x, hi.x,
// lo.y, hi.y), (lo.z, hi.z, -, -): per axis one paired add and one paired
// multiply give ((lo - A) inv, (hi - A) inv), the same roundings as seg_box,
// so the same decisions; the segment's pairs are formed once per segment.
struct SegPairs {
  float2 nax, nay, naz, ivx, ivy, ivz;
};
__device__ __forceinline__ SegPairs seg_pairs(const v3<float>& A, const v3<float>& inv) {
  SegPairs p;
  p.nax = bc(-A.x);
  p.nay = bc(-A.y);
  p.naz = bc(-A.z);
  p.ivx = bc(inv.x);
  p.ivy = bc(inv.y);
  p.ivz = bc(inv.z);
  return p;
}
__device__ __forceinline__ bool seg_box2(const SegPairs& p, const float4& b0, const float4& b1) {
  const float2 x = f2mul(f2add(make_float2(b0.x, b0.y), p.nax), p.ivx);
  const float2 y = f2mul(f2add(make_float2(b0.z, b0.w), p.nay), p.ivy);
  const float2 z = f2mul(f2add(make_float2(b1.x, b1.y), p.naz), p.ivz);
  const float t0 = fmaxf(fmaxf(fminf(x.x, x.y), fminf(y.x, y.y)), fmaxf(fminf(z.x, z.y), 0.f));
  const float t1 = fminf(fminf(fmaxf(x.x, x.y), fmaxf(y.x, y.y)), fminf(fmaxf(z.x, z.y), 1.f));
  return t0 <= t1;
}

// Occluder o (staged in shared memory: fields 0-3 of the FP32 records, then
// the boxes lo (w = kind) and hi) crosses segment AB with a clearance of
// CLEAR_M everywhere.
__device__ __forceinline__ bool clearly_crosses(const float4* sm, int n_occ, int o, const v3<float>& A,
                                                const v3<float>& B) {
  const float4 f0 = sm[o], f1 = sm[n_occ + o], f2 = sm[2 * n_occ + o], f3 = sm[3 * n_occ + o];
  const v3<float> O = mk(f0.x, f0.y, f0.z), n = mk(f3.x, f3.y, f3.z);
  const float sA = dot(A - O, n), sB = dot(B - O, n);
  if (!((sA > CLEAR_M && sB < -CLEAR_M) || (sA < -CLEAR_M && sB > CLEAR_M))) return false;
  const float t = sA / (sA - sB);
  const v3<float> P = axpy(t, B - A, A) - O;
  const float uu = dot(P, mk(f1.x, f1.y, f1.z)), vv = dot(P, mk(f2.x, f2.y, f2.z));
  return uu > CLEAR_M && uu < f0.w - CLEAR_M && vv > CLEAR_M && vv < f1.w - CLEAR_M;
}

// Warps claim the first list 32 entries at a time; the occluders (records and boxes) are
// staged in shared memory once per block.  For up to 32 groups at a time,
// every lane first finds the groups whose boxes its segments meet (a
// warp-uniform pass), then visits only those, so lanes with different
// segments do not wait on each other's groups.
template <int N>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_vis_prescreen(DevScene sc, DevEnds ep, const float4* ends32,
                                                               CandView cv, SolView out, RefineList rl1,
                                                               RefineList rl2, unsigned long long* cursor) {
  extern __shared__ float4 occ_sm[];  // [6][n_occ] records and boxes, then [2][n_grp] group boxes
  int64_t end = cv.order_begin[N];
  if (end > cv.cap) end = cv.cap;
  int64_t begin = cv.order_begin[N - 1];
  if (begin > end) begin = end;
  int64_t n = (int64_t)rl1.count[N - 1];
  if (n > end - begin) n = end - begin;
  if (n <= 0) return;  // the whole block
  const int no = sc.n_occ, ng = sc.n_grp;
  // occluder records and boxes as they are; the group boxes interleaved as
  // pairs for the paired slab test: (lo.x, hi.x, lo.y, hi.y), (lo.z, hi.z, 0, 0)
  for (int q = threadIdx.x; q < 6 * no + 2 * ng; q += blockDim.x) {
    if (q < 6 * no) {
      occ_sm[q] = q < 4 * no ? __ldg(sc.c32 + q) : __ldg(sc.cbox + (q - 4 * no));
    } else {
      const int g = (q - 6 * no) >> 1;
      const float4 lo = __ldg(sc.gbox + g), hi = __ldg(sc.gbox + ng + g);
      occ_sm[q] = ((q - 6 * no) & 1) ? make_float4(lo.z, hi.z, 0.f, 0.f) : make_float4(lo.x, hi.x, lo.y, hi.y);
    }
  }
  __syncthreads();
  const float4* grp_sm = occ_sm + 6 * no;  // [ng][2], interleaved
  const unsigned lane = threadIdx.x & 31;
  // warps claim 32 list entries at a time
  for (;;) {
    unsigned long long wb = 0;
    if (lane == 0) wb = atomicAdd(cursor, 32ull);
    wb = __shfl_sync(FULL, wb, 0);
    if ((int64_t)wb >= n) break;
    const int64_t i = (int64_t)wb + lane;
    bool keep = false, test = false;
    int64_t c = 0;
    v3<float> P[N + 2];
    if (i < n) {
      const int32_t e = rl1.idx[begin + i];
      c = begin + (e & ~RL_VIS);
      if (c >= begin && c < end) {
        keep = true;
        if (e & RL_VIS) {
          test = true;
          const uint4 q = rl1.ends[begin + i];
          P[0] = load_end<float>(ep.tx, ends32, (int)q.z);
          P[N + 1] = load_end<float>(ep.rx, ends32 + ep.n_tx, (int)q.w);
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const int id = (int)(((k < 2 ? q.x : q.y) >> (16 * (k & 1))) & 0xFFFFu);
            const int kind = __ldg(sc.kind + id);
            const Rec<float> r = load_obj32a(sc, id);
            P[k + 1] = point_at<float, false>(kind, r, rl1.prm[(int64_t)(2 * k) * rl1.stride + begin + i],
                                              rl1.prm[(int64_t)(2 * k + 1) * rl1.stride + begin + i]).X;
          }
        }
      }
    }
    bool blocked = false;
    if (__ballot_sync(FULL, test)) {
      // segment by segment: the groups whose boxes this segment meets, then
      // only their rectangles; a lane stops at its first clear crossing
#pragma unroll
      for (int j = 0; j <= N; ++j) {
        if (!test || blocked) continue;
        const v3<float> Af = P[j], Bf = P[j + 1];
        const v3<float> inv = mk(1.0f / (Bf.x - Af.x), 1.0f / (Bf.y - Af.y), 1.0f / (Bf.z - Af.z));
        const SegPairs sp = seg_pairs(Af, inv);
        for (int g0 = 0; g0 < ng && !blocked; g0 += 32) {
          const int gn = ng - g0 < 32 ? ng - g0 : 32;
          uint32_t gm = 0;
          for (int q = 0; q < gn; ++q) gm |= (uint32_t)seg_box2(sp, grp_sm[2 * (g0 + q)], grp_sm[2 * (g0 + q) + 1]) << q;
          while (gm != 0 && !blocked) {
            const int gi = g0 + __ffs(gm) - 1;
            gm &= gm - 1;
            const int o_end = (gi + 1) * OCC_GROUP < no ? (gi + 1) * OCC_GROUP : no;
            for (int o = gi * OCC_GROUP; o < o_end && !blocked; ++o) {
              const float4 bl = occ_sm[4 * no + o], bh = occ_sm[5 * no + o];
              if (bl.w != 0.f) continue;  // rectangles only
              if (box_overlap(bl, bh, Af, Bf)) blocked = clearly_crosses(occ_sm, no, o, Af, Bf);
            }
          }
        }
      }
      if (blocked) {
        out.status[c] = (uint8_t)(out.status[c] | MPT_PATH_PRESCREENED);
        keep = false;
      }
    }
    const unsigned km = __ballot_sync(FULL, keep);
    if (km) {
      const int leader = __ffs(km) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(rl2.count + (N - 1), (unsigned long long)__popc(km));
      base = __shfl_sync(FULL, base, leader);
      if (keep) rl2.idx[begin + (int64_t)base + __popc(km & ((1u << lane) - 1u))] = (int32_t)(c - begin);
    }
  }
}

// ------------------------------------------------------------- kernel B --
// Gauss-Newton with backtracking entirely in float-float (the fallback of
// the refinement for ill-conditioned paths).  Stops as soon as the cost is
// below `stop` (the refinement target): float-float rounding puts a floor of
// ~1e-26 under the cost, where further steps only chase rounding noise.  It
// also stops at a local minimum with non-zero residual, where the model's
// predicted decrease -g.dlt is below 1e-3 of the cost (a true path has the
// prediction close to the whole cost), after 4 halvings of the step, and
// after an accepted step that does not quarter the cost.
template <int N>
__device__ ff gn_ff(const int (&kind)[N], const Rec<ff> (&rec)[N], ff (&prm)[2 * N], const v3<ff>& A,
                    const v3<ff>& B, int max_iters, float mu, float stop) {
  constexpr int Q = 2 * N, P = Q * (Q + 1) / 2;
  ff jtj[P], g[Q], dlt[Q], trial[Q], jt2[P], g2[Q];
  ff cost((float)INFINITY);
  float alpha = 1.0f;
  bool need_factor = true;
  // one evaluation site (it = -1 evaluates the start): a second inlined copy
  // of the float-float evaluation costs more in instruction fetch than the
  // extra copies below
#pragma unroll 1
  for (int it = -1; it < 2 * max_iters; ++it) {
    if (it >= 0) {
      if (!(cost.hi >= stop)) break;
      if (need_factor) {
        pin_unused<N, ff>(kind, jtj, g);
        cholesky<Q, ff>(jtj, ff(mu));
        chol_solve<Q, ff>(jtj, g, dlt);
        float pred = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) pred = fmaf(-g[i].hi, dlt[i].hi, pred);
        if (pred < 1e-3f * cost.hi) break;
        alpha = 1.0f;
        need_factor = false;
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) trial[i] = fma_(ff(alpha), dlt[i], prm[i]);
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) trial[i] = prm[i];
    }
    bool ok;
    const ff ct = eval_path<N, ff, ff, true>(kind, rec, trial, A, B, jt2, g2, ok);
    if (it < 0) {
      if (!ok) return ff((float)INFINITY);
      cost = ct;
#pragma unroll
      for (int i = 0; i < P; ++i) jtj[i] = jt2[i];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = g2[i];
      continue;
    }
    if (ok && ct < cost) {
#pragma unroll
      for (int i = 0; i < Q; ++i) prm[i] = trial[i];
#pragma unroll
      for (int i = 0; i < P; ++i) jtj[i] = jt2[i];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = g2[i];
      // near a path Gauss-Newton gains orders of magnitude per step; a step
      // that does not even quarter the cost has reached the rounding floor
      const bool stagnant = ct.hi > 0.25f * cost.hi;
      cost = ct;
      if (stagnant) break;
      need_factor = true;
    } else {
      alpha *= 0.5f;
      if (alpha < 1.0f / 16.0f) break;
    }
  }
  return cost;
}

// The fallback in FP64 arithmetic on one lane (schedule fallback = 3), with
// the rules of gn_ff: the FP64 code is a fraction of the length of the
// float-float one, which matters for a lone serial chain that otherwise waits
// on instruction fetch (measured: the order-2 fallback of the urban block
// 59 us faster than float-float).  The default spreads the same iteration
// over a warp (gn_f64_lanes below).
template <int N>
__device__ double gn_f64(const int (&kind)[N], const Rec<double> (&rec)[N], double (&prm)[2 * N], const v3<double>& A,
                         const v3<double>& B, int max_iters, double mu, double stop) {
  constexpr int Q = 2 * N, P = Q * (Q + 1) / 2;
  double jtj[P], g[Q], dlt[Q], trial[Q], jt2[P], g2[Q];
  double cost = (double)INFINITY;
  double alpha = 1.0;
  bool need_factor = true;
#pragma unroll 1
  for (int it = -1; it < 2 * max_iters; ++it) {
    if (it >= 0) {
      if (!(cost >= stop)) break;
      if (need_factor) {
        pin_unused<N, double>(kind, jtj, g);
        cholesky<Q, double>(jtj, mu);
        chol_solve<Q, double>(jtj, g, dlt);
        double pred = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) pred = fma(-g[i], dlt[i], pred);
        if (pred < 1e-3 * cost) break;
        alpha = 1.0;
        need_factor = false;
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) trial[i] = fma(alpha, dlt[i], prm[i]);
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) trial[i] = prm[i];
    }
    bool ok;
    const double ct = eval_path<N, double, double, true>(kind, rec, trial, A, B, jt2, g2, ok);
    if (it < 0) {
      if (!ok) return (double)INFINITY;
      cost = ct;
#pragma unroll
      for (int i = 0; i < P; ++i) jtj[i] = jt2[i];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = g2[i];
      continue;
    }
    if (ok && ct < cost) {
#pragma unroll
      for (int i = 0; i < Q; ++i) prm[i] = trial[i];
#pragma unroll
      for (int i = 0; i < P; ++i) jtj[i] = jt2[i];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = g2[i];
      const bool stagnant = ct > 0.25 * cost;
      cost = ct;
      if (stagnant) break;
      need_factor = true;
    } else {
      alpha *= 0.5;
      if (alpha < 1.0 / 16.0) break;
    }
  }
  return cost;
}

// ------------------------------------------- FP64 fallback across a warp --
// The FP64 pipe issues about one warp instruction per 80 cycles on each SM
// sub-partition whatever the number of active lanes, so a lone candidate's
// FP64 solve takes its count of FP64 warp instructions times that interval.
// eval_lanes computes what eval_path<N, double, double, true> computes (the
// cost of Eq. 15, J^T J and J^T rho) with the work split over the lanes of
// one warp instead of repeated in each; lane L has the roles
//   m = L / 2 < N:       point m (Eq. 13/14) and its tangent L % 2: Jacobian
//                        column L (the parameter slot of that tangent) and
//                        row L of J^T J
//   L = 2m + 1, m <= N:  segment m (X_{m-1} -> X_m; X_{-1} = TX, X_N = RX):
//                        unit vector and inverse length
//   L = 2k, k < N:       interaction k: residual (Eq. 8 / ||i||, or Eq. 9)
// and shuffles carry each piece to the lanes that use it.  Every value that
// steers the iteration (cost, J^T J, J^T rho) is gathered in the same order
// in every lane, so all lanes hold identical copies and take the same
// branches.  Lanes with no role compute values nobody reads.
// Every shuffle below runs in all 32 lanes (none sits in a branch); source
// lanes outside the warp are clamped and their values discarded.
template <class R>
__device__ __forceinline__ v3<R> shfl3(const v3<R>& v, int src) {
  src = src < 0 ? 0 : (src > 31 ? 31 : src);
  return mk(__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src), __shfl_sync(FULL, v.z, src));
}
template <class R>
__device__ __forceinline__ R shfl1(R v, int src) {
  src = src < 0 ? 0 : (src > 31 ? 31 : src);
  return __shfl_sync(FULL, v, src);
}

template <int N, class R = double, bool CURVED = true>
__device__ R eval_lanes(const int (&kind)[N], const Rec<R>& rm, const R (&prm)[2 * N], const v3<R>& A,
                        const v3<R>& B, R* jtj, R* g, bool& ok, int lane) {
  constexpr int Q = 2 * N;
  const int m = lane >> 1, j = lane & 1;
  // this lane's point: object m, parameters (s, t) = prm[2m], prm[2m + 1]
  int km = K_PLANE;
  R s = R(0), t = R(0);
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (k == m) {
      km = kind[k];
      s = prm[2 * k];
      t = prm[2 * k + 1];
    }
  const PointT<R> pt = point_at<R, true, CURVED>(km, rm, s, t);
  // segment m: unit vector u and inverse length il (lanes 2m + 1)
  const v3<R> Xprev = shfl3(pt.X, 2 * m - 2);
  const v3<R> Xa = m == 0 ? A : Xprev;
  const v3<R> Xb = m == N ? B : pt.X;
  const v3<R> d = Xb - Xa;
  const R l2 = dot(d, d);
  const R il = rsq(l2);
  const v3<R> u = d * il;
  const bool seg_lane = (j == 1) && (m <= N);
  ok = __ballot_sync(FULL, seg_lane && !(l2 > R(0))) == 0u;
  // interaction m (lanes 2m): ih = u_m, rh = u_{m+1}
  const v3<R> ih = shfl3(u, 2 * m + 1), rh = shfl3(u, 2 * m + 3);
  v3<R> ax = mk(R(0), R(0), R(0)), de = ax, rho = ax;  // axis: normal or edge direction
  R c = R(0), inv_nn = R(0);
  if (!is_edge(km)) {
    if (!CURVED || km == K_PLANE) {
      ax = rm.f3(12);
    } else {
      const R q2 = rm.v[14];
      const v3<R> nraw = axpy(-t * q2, rm.f3(4), axpy(-s * q2, rm.f3(0), rm.f3(8)));
      inv_nn = rsq(dot(nraw, nraw));
      ax = nraw * inv_nn;
    }
    c = dot(ih, ax);
    rho = axpy(R(2) * c, ax, rh - ih);
  } else {
    if (!CURVED || km == K_LINE) {
      ax = rm.f3(4);
    } else {
      R sn, cs;
      sincos_(s, sn, cs);
      ax = axpy(cs, rm.f3(8), rm.f3(4) * (-sn));
      de = axpy(-sn, rm.f3(8), rm.f3(4) * (-cs));
    }
    rho.x = dot(ih, ax) - dot(rh, ax);
  }
  const R part = fma_(rho.x, rho.x, fma_(rho.y, rho.y, rho.z * rho.z));
  R cost = R(0);
#pragma unroll
  for (int k = 0; k < N; ++k) cost += __shfl_sync(FULL, part, 2 * k);
  // Jacobian column of this lane's slot (point m, tangent j); an edge's
  // second slot is unused (zero column, pinned by the caller)
  const bool live = (m < N) && !(j == 1 && is_edge(km));
  const v3<R> w = j == 0 ? pt.w0 : pt.w1;
  const v3<R> ui = ih, uo = rh;
  const R li = shfl1(il, 2 * m + 1), lo = shfl1(il, 2 * m + 3);
  const v3<R> PiW = axpy(-dot(ui, w), ui, w) * li;
  const v3<R> PrW = axpy(-dot(uo, w), uo, w) * lo;
  // own interaction m: the lane 2m values (this lane's own when j == 0)
  const v3<R> ax_o = shfl3(ax, 2 * m), de_o = shfl3(de, 2 * m), rho_o = shfl3(rho, 2 * m);
  const R c_o = shfl1(c, 2 * m), inn_o = shfl1(inv_nn, 2 * m);
  // neighbours m - 1 and m + 1
  const v3<R> ax_p = shfl3(ax, 2 * m - 2), rho_p = shfl3(rho, 2 * m - 2);
  const v3<R> ax_n = shfl3(ax, 2 * m + 2), rho_n = shfl3(rho, 2 * m + 2);
  int kp = K_PLANE, kn = K_PLANE;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k + 1 == m) kp = kind[k];
    if (k == m + 1) kn = kind[k];
  }
  const v3<R> zero = mk(R(0), R(0), R(0));
  v3<R> cp = zero, co = zero, cn = zero;  // column blocks on interactions m-1, m, m+1
  if (live) {
    // interaction m - 1 sees this point as its next one: d rho / dX = Pi_m w
    if (m >= 1) cp = is_edge(kp) ? mk(-dot(ax_p, PiW), R(0), R(0)) : PiW;
    // interaction m + 1 sees it as its previous one: H_{m+1}(Pr_m w)
    if (m + 1 < N) cn = is_edge(kn) ? mk(-dot(ax_n, PrW), R(0), R(0)) : axpy(-R(2) * dot(ax_n, PrW), ax_n, PrW);
    if (!is_edge(km)) {
      co = -(PrW + axpy(-R(2) * dot(ax_o, PiW), ax_o, PiW));
      if (CURVED && km == K_PARAB) {
        const R q2 = rm.v[14];
        const v3<R> craw = (j == 0 ? rm.f3(0) : rm.f3(4)) * (-q2);
        const v3<R> dn = axpy(-dot(ax_o, craw), ax_o, craw) * inn_o;
        co = axpy(R(2) * dot(ih, dn), ax_o, co);
        co = axpy(R(2) * c_o, dn, co);
      }
    } else {
      R v = dot(ax_o, PiW) + dot(ax_o, PrW);
      if (CURVED && km == K_ARC) v = v + dot(ih - rh, de_o);
      co = mk(v, R(0), R(0));
    }
  }
  R gp = dot(co, rho_o);
  if (m >= 1) gp += dot(cp, rho_p);
  if (m + 1 < N) gp += dot(cn, rho_n);
  // the column over every interaction (zero away from m-1 .. m+1)
  v3<R> col[N];
#pragma unroll
  for (int k = 0; k < N; ++k) col[k] = (k + 1 == m) ? cp : (k == m) ? co : (k == m + 1) ? cn : zero;
  // row of J^T J: <col_L, col_q> over the interactions where column q lives
  R row[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    R acc = R(0);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k < (q >> 1) - 1 || k > (q >> 1) + 1) continue;
      acc = fma_(col[k].x, __shfl_sync(FULL, col[k].x, q), acc);
      acc = fma_(col[k].y, __shfl_sync(FULL, col[k].y, q), acc);
      acc = fma_(col[k].z, __shfl_sync(FULL, col[k].z, q), acc);
    }
    row[q] = acc;
  }
  // every lane gathers the packed lower triangle and the gradient
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    g[a] = __shfl_sync(FULL, gp, a);
#pragma unroll
    for (int b = 0; b <= a; ++b) jtj[tri(a, b)] = __shfl_sync(FULL, row[b], a);
  }
  return cost;
}

// gn_f64 with eval_lanes: one warp per candidate, every lane holding the
// same iterate; the factorisation and the decisions run in every lane.
template <int N>
__device__ double gn_f64_lanes(const int (&kind)[N], const Rec<double>& rm, double (&prm)[2 * N],
                               const v3<double>& A, const v3<double>& B, int max_iters, double mu, double stop,
                               int lane) {
  constexpr int Q = 2 * N, P = Q * (Q + 1) / 2;
  double jtj[P], g[Q], dlt[Q], trial[Q], jt2[P], g2[Q];
  double cost = (double)INFINITY;
  double alpha = 1.0;
  bool need_factor = true;
#pragma unroll 1
  for (int it = -1; it < 2 * max_iters; ++it) {
    if (it >= 0) {
      if (!(cost >= stop)) break;
      if (need_factor) {
        pin_unused<N, double>(kind, jtj, g);
        cholesky<Q, double>(jtj, mu);
        chol_solve<Q, double>(jtj, g, dlt);
        double pred = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) pred = fma(-g[i], dlt[i], pred);
        if (pred < 1e-3 * cost) break;
        alpha = 1.0;
        need_factor = false;
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) trial[i] = fma(alpha, dlt[i], prm[i]);
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) trial[i] = prm[i];
    }
    bool ok;
    const double ct = eval_lanes<N>(kind, rm, trial, A, B, jt2, g2, ok, lane);
    if (it < 0) {
      if (!ok) return (double)INFINITY;
      cost = ct;
#pragma unroll
      for (int i = 0; i < P; ++i) jtj[i] = jt2[i];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = g2[i];
      continue;
    }
    if (ok && ct < cost) {
#pragma unroll
      for (int i = 0; i < Q; ++i) prm[i] = trial[i];
#pragma unroll
      for (int i = 0; i < P; ++i) jtj[i] = jt2[i];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = g2[i];
      const bool stagnant = ct > 0.25 * cost;
      cost = ct;
      if (stagnant) break;
      need_factor = true;
    } else {
      alpha *= 0.5;
      if (alpha < 1.0 / 16.0) break;
    }
  }
  return cost;
}

// --------------------------------------------------- warp-per-path solver --
// The minimiser of gn_warp (Gauss-Newton on Eq. 15, the same backtracking
// search, stopping rules and FP32 tolerances) with one warp per candidate:
// the evaluation is spread over the lanes as in eval_lanes (lane L: point
// L/2 and its tangent L%2, segment, interaction) and every lane holds the
// same iterate, factorisation and decisions (the values that steer the
// iteration are gathered in the same order in every lane).  A schedule
// option (mpt_schedule.warp_orders) for solves whose lanes would diverge
// most in the one-lane form; each candidate's iterations cost about four
// times the issue slots there, so the one-lane solver is the default.
// Warps claim 32 candidates at a time, one record per lane, and walk them.
template <int N, int PREC, bool CURVED>
__global__ void __launch_bounds__(SOLVE_BLOCK) k_gn_warp(DevScene sc, DevEnds ep, const float4* ends32, CandView cv,
                                                        SolView out, SolveCfg cfg, unsigned long long* counter,
                                                        RefineList rl, const int32_t* list,
                                                        const unsigned long long* list_count) {
  constexpr int Q = 2 * N, P = Q * (Q + 1) / 2;
  const int lane = (int)(threadIdx.x & 31);
  int64_t end = cv.order_begin[N];
  if (end > cv.cap) end = cv.cap;
  int64_t begin = cv.order_begin[N - 1];
  if (begin > end) begin = end;
  // positions: candidates begin + position, or begin + list[begin + position]
  int64_t n_pos = end - begin;
  if (list != nullptr && (int64_t)*list_count < n_pos) n_pos = (int64_t)*list_count;
  const float c_tol = cfg.c_tol32, step_tol = cfg.step_tol32, mu = cfg.mu32;
  const float diverge = (float)cfg.diverge;
  for (;;) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(counter, 32ull);
    b = __shfl_sync(FULL, b, 0);
    const int64_t pos = (int64_t)b;
    if (pos >= n_pos) break;
    const int len = n_pos - pos < 32 ? (int)(n_pos - pos) : 32;
    const int32_t off = lane < len ? (list != nullptr ? __ldg(list + begin + pos + lane) : (int32_t)(pos + lane)) : 0;
    const uint4 mine = lane < len ? __ldg(cv.rec + begin + off) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
    for (int i = 0; i < len; ++i) {
      const int64_t c = begin + __shfl_sync(FULL, off, i);
      uint4 rr;
      rr.x = __shfl_sync(FULL, mine.x, i);
      rr.y = __shfl_sync(FULL, mine.y, i);
      rr.z = __shfl_sync(FULL, mine.z, i);
      rr.w = __shfl_sync(FULL, mine.w, i);
      // a record of this order whose objects and endpoints exist
      bool valid = (int)(rr.w & 0xFFu) == N;
      int ids[N];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        ids[k] = (int)(((k < 2 ? rr.y : rr.z) >> (16 * (k & 1))) & 0xFFFFu);
        valid = valid && ids[k] < sc.n_obj;
      }
      int it_, ir_;
      pair_ends(ep, rr.x, it_, ir_);
      valid = valid && it_ < ep.n_tx && ir_ < ep.n_rx;
      if (!valid) {
        if (lane == 0) {
          out.cost[c] = (double)INFINITY;
          out.status[c] = (uint8_t)MPT_PATH_NONFINITE;
          out.iters[c] = 0;
          out.evals[c] = 0;
        }
        continue;
      }
      int kind[N];
      float lm_ratio = cfg.localmin_ratio_planar;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        kind[k] = __ldg(sc.kind + ids[k]);
        if (CURVED && (kind[k] == K_PARAB || kind[k] == K_ARC)) lm_ratio = cfg.localmin_ratio;
      }
      // this lane's object (point lane / 2); lanes past the sequence hold zeros
      Rec<float> rm;
#pragma unroll
      for (int f = 0; f < 16; ++f) rm.v[f] = 0.f;
      int own = -1, km = K_PLANE;
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (k == (lane >> 1)) {
          own = ids[k];
          km = kind[k];
        }
      if (own >= 0) rm = load_obj32a(sc, own);
      const v3<float> A = load_end<float>(ep.tx, ends32, it_);
      const v3<float> B = load_end<float>(ep.rx, ends32 + ep.n_tx, ir_);
      // initial guess (Algorithm 1, random_guess): lane 2k makes object k's
      uint64_t packed = 0;
      if constexpr (CURVED) {
        packed = (uint64_t)rr.y | ((uint64_t)rr.z << 32);
        if constexpr (N < 4) packed |= ~0ull << (16 * (N < 4 ? N : 0));
      }
      float s0 = 0.f, t0 = 0.f;
      if ((lane & 1) == 0 && own >= 0)
        init_params<float, CURVED>(km, rm, (lane < N) ? A : B, cv.init_seed, rr.x, packed, (int)((rr.w >> 8) & 0xFFu),
                                   lane >> 1, s0, t0);
      float trial[Q], prm[Q], dlt[Q], jtj[P], g[Q];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        trial[2 * k] = __shfl_sync(FULL, s0, 2 * k);
        trial[2 * k + 1] = __shfl_sync(FULL, t0, 2 * k);
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) prm[q] = dlt[q] = 0.f;
      float cost = 0.f, alpha = 1.f;
      int iters = 0, evals = 0, done = -1;
      bool fresh = true;
#pragma unroll 1
      for (;;) {
        bool ok;
        const float ct = eval_lanes<N, float, CURVED>(kind, rm, trial, A, B, jtj, g, ok, lane);
        ++evals;
        bool factor = false;
        if (fresh) {
          fresh = false;
#pragma unroll
          for (int q = 0; q < Q; ++q) prm[q] = trial[q];
          cost = ct;
          if (!(ok && isfinite(ct))) done = MPT_PATH_NONFINITE;
          else if (cost < c_tol) done = MPT_PATH_CONVERGED;
          else factor = true;
        } else if (ok && ct < cost) {
          float smax = 0.f, pmax = 0.f;
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            smax = fmaxf(smax, fabsf(trial[q] - prm[q]));
            prm[q] = trial[q];
            pmax = fmaxf(pmax, fabsf(prm[q]));
          }
          cost = ct;
          ++iters;
          if (!(pmax <= diverge)) done = MPT_PATH_DIVERGED;
          else if (cost < c_tol || smax < step_tol) done = MPT_PATH_CONVERGED;
          else if (iters >= cfg.max_iters) done = MPT_PATH_MAXITER;
          else factor = true;
        } else {
          alpha = alpha * 0.5f;
          if (alpha < cfg.min_alpha) done = MPT_PATH_STALLED;
        }
        if (done < 0 && evals >= cfg.max_evals) done = MPT_PATH_MAXITER;
        if (factor && done < 0) {
          pin_unused<N, float>(kind, jtj, g);
          cholesky<Q, float>(jtj, mu);
          chol_solve<Q, float>(jtj, g, dlt);
          alpha = 1.f;
          // local minimum with non-zero residual (as in gn_warp)
          float pred = 0.f;
#pragma unroll
          for (int q = 0; q < Q; ++q) pred = fmaf(-g[q], dlt[q], pred);
          if (iters >= 2 && cost > cfg.localmin_cost && pred < lm_ratio * cost) done = MPT_PATH_STALLED;
        }
        if (done >= 0) break;
#pragma unroll
        for (int q = 0; q < Q; ++q) trial[q] = fmaf(alpha, dlt[q], prm[q]);
      }
      // ---- result: lane q writes slot q, lane 0 the rest
      int status = done;
      bool pass = false;
      if (PREC == MPT_FP32_FP64REFINE) {
        float sq = 0.f, tq = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k == (lane >> 1)) {
            sq = prm[2 * k];
            tq = prm[2 * k + 1];
          }
        const bool inb = !((lane & 1) == 0 && own >= 0) ||
                         in_bounds_margin<float>(km, rm, sq, tq, cfg.prescreen_margin);
        pass = __all_sync(FULL, inb) && isfinite(cost) && cost < cfg.prescreen_cost && done != MPT_PATH_DIVERGED;
        if (!pass) status |= MPT_PATH_PRESCREENED;
      }
      float mine_q = 0.f;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q == lane) mine_q = prm[q];
      if (lane < Q) {
        out.T[(int64_t)lane * out.cap + c] = to_f64(mine_q);
        if (out.T32 != nullptr) out.T32[(int64_t)lane * out.cap + c] = mine_q;
      }
      if (lane == 0) {
        out.cost[c] = to_f64(cost);
        out.status[c] = (uint8_t)status;
        out.iters[c] = (uint8_t)min(iters, 255);
        out.evals[c] = (uint8_t)min(evals, 255);
      }
      if (PREC == MPT_FP32_FP64REFINE && pass) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(rl.count + (N - 1), 1ull);
        pos = __shfl_sync(FULL, pos, 0);
        const int64_t at = begin + (int64_t)pos;
        if (lane == 0) {
          rl.idx[at] = (int32_t)(c - begin) | (cost < PRESCREEN_VIS_COST ? RL_VIS : 0);
          if (rl.prm != nullptr) rl.ends[at] = make_uint4(rr.y, rr.z, (uint32_t)it_, (uint32_t)ir_);
        }
        if (rl.prm != nullptr && lane < Q) rl.prm[(int64_t)lane * rl.stride + at] = mine_q;
      }
    }
  }
}

// One thread per listed candidate: up to refine_steps mixed steps (residual
// and cost in float-float, Jacobian and solve in FP32) until the cost is
// below 1e-24, extended by up to 6 steps while they still halve the cost.
// A candidate still at or above 1e-22 (ill-conditioned, near an object
// crease) is queued for k_refine_fb.  Both bounds sit above the float-float
// rounding floor of the cost (1e-28 .. 1e-23, larger for short segments far
// from the origin) and far below the acceptance threshold 1e-20.
constexpr float REFINE_STOP = 1e-24f, REFINE_TARGET = 1e-22f;

// CURVED = false: scenes of planes and straight edges only (no paraboloid or
// arc branches in the evaluation: shorter code, fewer registers).
template <int N, bool CURVED>
__global__ void __launch_bounds__(SOLVE_BLOCK, (N <= 2 ? 3 : 1)) k_refine(DevScene sc, DevEnds ep, CandView cv,
                                                                        SolView out, SolveCfg cfg, RefineList rl,
                                                                        RefineList rl3, unsigned long long* cursor) {
  constexpr int Q = 2 * N;
  int64_t end = cv.order_begin[N];
  if (end > cv.cap) end = cv.cap;
  int64_t begin = cv.order_begin[N - 1];
  if (begin > end) begin = end;
  int64_t n = (int64_t)rl.count[N - 1];
  if (n > end - begin) n = end - begin;
  const ff stop(REFINE_STOP), target(REFINE_TARGET);
  const unsigned lane = threadIdx.x & 31;
  // warps claim 32 list entries at a time (refinement lengths vary)
  for (;;) {
    unsigned long long wb = 0;
    if (lane == 0) wb = atomicAdd(cursor, 32ull);
    wb = __shfl_sync(FULL, wb, 0);
    if ((int64_t)wb >= n) break;
    const int64_t i = (int64_t)wb + lane;
    bool fallback = false;
    int64_t c = 0;
    if (i < n) {
      c = begin + (rl.idx[begin + i] & ~RL_VIS);
      if (c >= begin && c < end) {
        const Cand cd = decode(__ldg(cv.rec + c));
        int it_, ir_;
        pair_ends(ep, cd.pair, it_, ir_);
        const v3<ff> A = load_end_ff(ep.tx, it_);
        const v3<ff> B = load_end_ff(ep.rx, ir_);
        int kind[N];
        Rec<ff> rec[N];
        ff T0[Q], T[Q];
#pragma unroll
        for (int k = 0; k < N; ++k) {
          kind[k] = __ldg(sc.kind + cd.ids[k]);
          rec[k] = load_obj_ff(sc, cd.ids[k]);
        }
#pragma unroll
        for (int j = 0; j < Q; ++j) T[j] = T0[j] = ff_from_double(out.T[(int64_t)j * out.cap + c]);
        float jtj[Q * (Q + 1) / 2], g[Q], dlt[Q];
        bool ok = true;
        ff cst(0.f), prev(0.f);
        // one evaluation site (s = -1 evaluates the start): the float-float
        // evaluation is long, and a second inlined copy costs more in
        // instruction fetch than the loop control saves
#pragma unroll 1
        for (int s = -1;; ++s) {
          if (s >= 0) {
            if (!ok || !(cst >= stop)) break;
            // beyond refine_steps, up to 6 more mixed steps while the target
            // is not met and each step still halves the cost (slow linear
            // convergence of ill-conditioned paths under the FP32 Jacobian)
            if (s >= cfg.refine_steps &&
                (s >= cfg.refine_steps + 6 || cst < target || !(cst.hi < 0.5f * prev.hi)))
              break;
            prev = cst;
            pin_unused<N, float>(kind, jtj, g);
            cholesky<Q, float>(jtj, cfg.mu32);
            chol_solve<Q, float>(jtj, g, dlt);
#pragma unroll
            for (int j = 0; j < Q; ++j) T[j] = T[j] + ff(dlt[j]);
          }
          cst = eval_path<N, ff, float, true, CURVED>(kind, rec, T, A, B, jtj, g, ok);
        }
        fallback = !ok || !(cst < target);
        // the fallback starts from what is written here: the mixed result,
        // or the FP32 result (with an infinite cost) when an evaluation failed
#pragma unroll
        for (int j = 0; j < Q; ++j) out.T[(int64_t)j * out.cap + c] = to_double(ok ? T[j] : T0[j]);
        out.cost[c] = ok && finite_ff(cst) ? to_double(cst) : (double)INFINITY;
        out.status[c] = (uint8_t)(out.status[c] | MPT_PATH_REFINED | (fallback ? MPT_PATH_FALLBACK : 0));
      }
    }
    const unsigned fm = __ballot_sync(FULL, fallback);
    if (fm) {
      const int leader = __ffs(fm) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(rl3.count + (N - 1), (unsigned long long)__popc(fm));
      base = __shfl_sync(FULL, base, leader);
      if (fallback) rl3.idx[begin + (int64_t)base + __popc(fm & ((1u << lane) - 1u))] = (int32_t)(c - begin);
    }
  }
}

// The fallback of the refinement: Gauss-Newton (FP64 or float-float) for the
// queued candidates, one candidate per warp so that the few long serial
// solves run side by side on as many SM sub-partitions as there are.  MODE:
// FB_F64_WARP (the default) FP64 with the evaluation spread over the warp's
// lanes (eval_lanes); FB_F64 and FB_FF FP64 or float-float on lane 0 alone.
enum { FB_FF = 0, FB_F64 = 1, FB_F64_WARP = 2 };

template <int N, int MODE>
__global__ void __launch_bounds__(32) k_refine_fb(DevScene sc, DevEnds ep, CandView cv, SolView out, SolveCfg cfg,
                                                  RefineList rl3) {
  constexpr int Q = 2 * N;
  const int lane = (int)threadIdx.x;
  if (MODE != FB_F64_WARP && lane != 0) return;
  int64_t end = cv.order_begin[N];
  if (end > cv.cap) end = cv.cap;
  int64_t begin = cv.order_begin[N - 1];
  if (begin > end) begin = end;
  int64_t n = (int64_t)rl3.count[N - 1];
  if (n > end - begin) n = end - begin;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const int64_t c = begin + rl3.idx[begin + i];
    if (c < begin || c >= end) continue;
    const Cand cd = decode(__ldg(cv.rec + c));
    int it_, ir_;
    pair_ends(ep, cd.pair, it_, ir_);
    int kind[N];
#pragma unroll
    for (int k = 0; k < N; ++k) kind[k] = __ldg(sc.kind + cd.ids[k]);
    const double c1 = out.cost[c];
    if constexpr (MODE == FB_F64_WARP) {
      const v3<double> A = mk(ep.tx[3 * it_], ep.tx[3 * it_ + 1], ep.tx[3 * it_ + 2]);
      const v3<double> B = mk(ep.rx[3 * ir_], ep.rx[3 * ir_ + 1], ep.rx[3 * ir_ + 2]);
      // this lane's object (point lane >> 1); lanes past the sequence hold zeros
      Rec<double> rm;
#pragma unroll
      for (int f = 0; f < 16; ++f) rm.v[f] = 0.0;
      int id = -1;
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (k == (lane >> 1)) id = cd.ids[k];
      if (id >= 0) rm = load_obj64(sc, id);
      double T[Q];
#pragma unroll
      for (int j = 0; j < Q; ++j) T[j] = out.T[(int64_t)j * out.cap + c];
      const double c2 =
          gn_f64_lanes<N>(kind, rm, T, A, B, cfg.fallback_iters, cfg.mu64, (double)REFINE_TARGET, lane);
      if (lane == 0 && isfinite(c2) && c2 < c1) {
#pragma unroll
        for (int j = 0; j < Q; ++j) out.T[(int64_t)j * out.cap + c] = T[j];
        out.cost[c] = c2;
      }
    } else if constexpr (MODE == FB_F64) {
      const v3<double> A = mk(ep.tx[3 * it_], ep.tx[3 * it_ + 1], ep.tx[3 * it_ + 2]);
      const v3<double> B = mk(ep.rx[3 * ir_], ep.rx[3 * ir_ + 1], ep.rx[3 * ir_ + 2]);
      Rec<double> rec[N];
      double T[Q];
#pragma unroll
      for (int k = 0; k < N; ++k) rec[k] = load_obj64(sc, cd.ids[k]);
#pragma unroll
      for (int j = 0; j < Q; ++j) T[j] = out.T[(int64_t)j * out.cap + c];
      const double c2 = gn_f64<N>(kind, rec, T, A, B, cfg.fallback_iters, cfg.mu64, (double)REFINE_TARGET);
      if (isfinite(c2) && c2 < c1) {
#pragma unroll
        for (int j = 0; j < Q; ++j) out.T[(int64_t)j * out.cap + c] = T[j];
        out.cost[c] = c2;
      }
    } else {
      const v3<ff> A = load_end_ff(ep.tx, it_);
      const v3<ff> B = load_end_ff(ep.rx, ir_);
      Rec<ff> rec[N];
      ff T[Q];
#pragma unroll
      for (int k = 0; k < N; ++k) rec[k] = load_obj_ff(sc, cd.ids[k]);
#pragma unroll
      for (int j = 0; j < Q; ++j) T[j] = ff_from_double(out.T[(int64_t)j * out.cap + c]);
      const ff c2 = gn_ff<N>(kind, rec, T, A, B, cfg.fallback_iters, (float)cfg.mu64, REFINE_TARGET);
      if (finite_ff(c2) && to_double(c2) < c1) {
#pragma unroll
        for (int j = 0; j < Q; ++j) out.T[(int64_t)j * out.cap + c] = to_double(T[j]);
        out.cost[c] = to_double(c2);
      }
    }
  }
}

// ------------------------------------------------------------ launching --
template <class K>
static int grid_for(mpt_ctx* ctx, K kernel, const mpt_schedule* sch, size_t smem = 0) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, SOLVE_BLOCK, smem);
  if (occ < 1) occ = 1;
  if (sch && sch->blocks_per_sm > 0 && sch->blocks_per_sm < occ) occ = sch->blocks_per_sm;
  return ctx->sms * occ;
}

template <int N, int PREC>
static void launch_gn_kernel(mpt_ctx* ctx, const DevScene& sc, const DevEnds& ep, const float4* ends32,
                             const CandView& cv, const SolView& sv, const SolveCfg& cfg, const mpt_schedule* sch,
                             RefineList rl, bool curved, const int32_t* list, const unsigned long long* list_count,
                             unsigned long long* counter, cudaStream_t s);

// The solver of order N: one candidate per lane (k_gn), or one per warp
// (k_gn_warp) for the orders the schedule's warp_orders names (FP32
// precisions only).
template <int N, int PREC>
static void launch_gn(mpt_ctx* ctx, const DevScene& sc, const DevEnds& ep, const float4* ends32, const CandView& cv,
                      const SolView& sv, const SolveCfg& cfg, const mpt_schedule* sch, RefineList rl, bool curved,
                      const int32_t* list, cudaStream_t s) {
  unsigned long long* counter = ctx->counters + (N - 1);
  const unsigned long long* list_count = ctx->counters + 28 + (N - 1);
  if (ctx->time_solver) cudaEventRecord(ctx->ev_gn[N - 1][0], s);
  launch_gn_kernel<N, PREC>(ctx, sc, ep, ends32, cv, sv, cfg, sch, rl, curved, list, list_count, counter, s);
  if (ctx->time_solver) cudaEventRecord(ctx->ev_gn[N - 1][1], s);
}

template <int N, int PREC>
static void launch_gn_kernel(mpt_ctx* ctx, const DevScene& sc, const DevEnds& ep, const float4* ends32,
                             const CandView& cv, const SolView& sv, const SolveCfg& cfg, const mpt_schedule* sch,
                             RefineList rl, bool curved, const int32_t* list, const unsigned long long* list_count,
                             unsigned long long* counter, cudaStream_t s) {
  if constexpr (PREC != MPT_FP64_PLAIN) {
    if (sch != nullptr && ((sch->warp_orders >> (N - 1)) & 1) != 0) {
      if (curved)
        k_gn_warp<N, PREC, true><<<grid_for(ctx, k_gn_warp<N, PREC, true>, sch), SOLVE_BLOCK, 0, s>>>(
            sc, ep, ends32, cv, sv, cfg, counter, rl, list, list_count);
      else
        k_gn_warp<N, PREC, false><<<grid_for(ctx, k_gn_warp<N, PREC, false>, sch), SOLVE_BLOCK, 0, s>>>(
            sc, ep, ends32, cv, sv, cfg, counter, rl, list, list_count);
      return;
    }
  }
  if (curved)
    k_gn<N, PREC, true><<<grid_for(ctx, k_gn<N, PREC, true>, sch), SOLVE_BLOCK, 0, s>>>(sc, ep, ends32, cv, sv, cfg,
                                                                                       counter, rl, list, list_count);
  else
    k_gn<N, PREC, false><<<grid_for(ctx, k_gn<N, PREC, false>, sch), SOLVE_BLOCK, 0, s>>>(
        sc, ep, ends32, cv, sv, cfg, counter, rl, list, list_count);
}

template <int PREC>
static int launch_prec(mpt_ctx* ctx, const DevScene& sc, const DevEnds& ep, const float4* ends32, const CandView& cv,
                       const SolView& sv, const SolveCfg& cfg, const mpt_schedule* sch, RefineList rl,
                       RefineList rl2, bool curved, int32_t* xlist, float4* beams, uint32_t* xbits,
                       cudaStream_t st) {
  // counters[0..3]: per-order candidate cursors; [4]: mixed-order cursor;
  // [8..11]: refine list sizes; [12..15]: sizes after the visibility
  // prescreen; [16..19]: fallback queue sizes; [20..23]: refinement
  // cursors; [24..27]: prescreen cursors; [28..31]: sizes of the lists of
  // candidates the exclusion pass keeps
  MPT_CUDA_TRY(cudaMemsetAsync(ctx->counters, 0, 32 * sizeof(unsigned long long), st));
  // the exclusion pass (per-order launches only): beams of every endpoint
  // through every plane, then one pass over the candidates
  const int32_t* list = nullptr;
  if (xlist != nullptr) {
    const int n_ends = ep.n_tx + ep.n_rx;
    const int words = (sc.n_obj + 31) / 32;
    k_beams<<<dim3((sc.n_obj + 127) / 128, n_ends), 128, 0, st>>>(sc, ends32, n_ends, beams);
    MPT_LAUNCH_CHECK();
    const int64_t xwarps = ((int64_t)n_ends * sc.n_obj + XBITS_PAIRS - 1) / XBITS_PAIRS * words;
    k_exclusion_bits<<<(unsigned)((xwarps + 3) / 4), 128, 0, st>>>(sc, beams, n_ends, words, xbits,
                                                                 (float)(1e-5 * sc.scale), (float)(1e-5 * sc.scale),
                                                                 (float)(1e-2 * sc.scale));
    MPT_LAUNCH_CHECK();
    int64_t blocks = (cv.cap + 255) / 256;
    const int64_t cap_blocks = (int64_t)ctx->sms * 8;
    if (blocks > cap_blocks) blocks = cap_blocks;
    if (blocks < 1) blocks = 1;
    k_exclude<<<(unsigned)blocks, 256, 0, st>>>(sc, ep, ends32, beams, xbits, words, cv, sv, xlist,
                                                 ctx->counters + 28);
    MPT_LAUNCH_CHECK();
    list = xlist;
  }
  const size_t vsmem = (size_t)sc.n_occ * 96 + (size_t)sc.n_grp * 32;
  // the fallback queue reuses the storage of a list read by then: the first
  // list after the prescreen, else the (unused) second one
  const RefineList rl3{ctx->counters + 16, cfg.prescreen ? rl.idx : rl2.idx};
  if (sch && sch->mixed_orders) {
    k_gn_mixed<PREC><<<grid_for(ctx, k_gn_mixed<PREC>, sch), SOLVE_BLOCK, 0, st>>>(sc, ep, ends32, cv, sv, cfg,
                                                                                  ctx->counters + 4, rl);
    MPT_LAUNCH_CHECK();
  }
  // The orders are independent chains (solver, visibility prescreen,
  // refinement, fallback); order 2 stays on the caller's stream and orders
  // 1, 3, 4 run on the context's auxiliary streams, joined at the end, so
  // that the small chains and the tails of each kernel overlap.
  const bool per_order = !(sch && sch->mixed_orders);
  MPT_CUDA_TRY(fork_streams(ctx, st));
#define MPT_CHAIN(N, S)                                                                                        \
  {                                                                                                            \
    cudaStream_t s_ = (S);                                                                                     \
    if (per_order) {                                                                                           \
      launch_gn<N, PREC>(ctx, sc, ep, ends32, cv, sv, cfg, sch, rl, curved, list, s_);                          \
      MPT_LAUNCH_CHECK();                                                                                      \
    }                                                                                                          \
    if (PREC == MPT_FP32_FP64REFINE) {                                                                         \
      if (vsmem > 48 * 1024)                                                                                   \
        cudaFuncSetAttribute(k_vis_prescreen<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsmem);     \
      if (cfg.prescreen) {                                                                                     \
        k_vis_prescreen<N><<<grid_for(ctx, k_vis_prescreen<N>, nullptr, vsmem), SOLVE_BLOCK, vsmem, s_>>>(     \
            sc, ep, ends32, cv, sv, rl, rl2, ctx->counters + 24 + (N - 1));                                    \
        MPT_LAUNCH_CHECK();                                                                                    \
      }                                                                                                        \
      if (curved)                                                                                              \
        k_refine<N, true><<<grid_for(ctx, k_refine<N, true>, nullptr), SOLVE_BLOCK, 0, s_>>>(                  \
            sc, ep, cv, sv, cfg, cfg.prescreen ? rl2 : rl, rl3, ctx->counters + 20 + (N - 1));                 \
      else                                                                                                     \
        k_refine<N, false><<<grid_for(ctx, k_refine<N, false>, nullptr), SOLVE_BLOCK, 0, s_>>>(                \
            sc, ep, cv, sv, cfg, cfg.prescreen ? rl2 : rl, rl3, ctx->counters + 20 + (N - 1));                 \
      MPT_LAUNCH_CHECK();                                                                                      \
      if (cfg.fallback == FB_F64_WARP)                                                                         \
        k_refine_fb<N, FB_F64_WARP><<<ctx->sms * 4, 32, 0, s_>>>(sc, ep, cv, sv, cfg, rl3);                    \
      else if (cfg.fallback == FB_F64)                                                                         \
        k_refine_fb<N, FB_F64><<<ctx->sms * 4, 32, 0, s_>>>(sc, ep, cv, sv, cfg, rl3);                         \
      else                                                                                                     \
        k_refine_fb<N, FB_FF><<<ctx->sms * 4, 32, 0, s_>>>(sc, ep, cv, sv, cfg, rl3);                          \
      MPT_LAUNCH_CHECK();                                                                                      \
    }                                                                                                          \
  }
  MPT_CHAIN(2, st)
  MPT_CHAIN(1, ctx->aux[0])
  MPT_CHAIN(3, ctx->aux[1])
  MPT_CHAIN(4, ctx->aux[2])
#undef MPT_CHAIN
  MPT_CUDA_TRY(join_streams(ctx, st));
  return MPT_OK;
}

int launch_solve(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                 int precision, const mpt_schedule* sch, mpt_solutions* out, cudaStream_t st) {
  SolveCfg cfg;
  // Valid paths of the benchmark workloads converge within 12 accepted steps
  // and 25 evaluations; the caps leave a factor of 2 / 1.6.
  cfg.max_iters = (sch && sch->max_iters > 0) ? (sch->max_iters > 160 ? 160 : sch->max_iters) : 24;
  cfg.max_evals = cfg.max_iters * 5 / 3;
  cfg.min_alpha = 1.0f / 16.0f;
  cfg.localmin_cost = 1e-3f;
  cfg.localmin_ratio = 1e-4f;         // sequences with a paraboloid or an arc edge
  cfg.localmin_ratio_planar = 0.1f;   // planes and straight edges only
  cfg.refine_steps = (sch && sch->refine_steps > 0) ? (sch->refine_steps > 4 ? 4 : sch->refine_steps) : 2;
  cfg.refill_min = (sch && sch->refill_min > 0) ? (sch->refill_min > 32 ? 32 : sch->refill_min) : 12;
  cfg.piece = (sch && sch->tile > 0) ? (sch->tile < 32 ? 32 : (sch->tile > GN_CHUNK ? GN_CHUNK : sch->tile)) : GN_CHUNK;
  cfg.fallback_iters = 2;  // at most 5 evaluations
  cfg.prescreen = (sch && sch->prescreen == 2) ? 0 : 1;
  cfg.exclude = (sch && sch->exclude == 2) ? 0 : 1;
  cfg.fallback = !sch ? FB_F64_WARP : sch->fallback == 1 ? FB_FF : sch->fallback == 3 ? FB_F64 : FB_F64_WARP;
  const double S = scene->d.scale;
  cfg.c_tol32 = 1e-12f;
  cfg.step_tol32 = (float)(1e-6 * S);
  cfg.c_tol64 = 1e-30;
  cfg.step_tol64 = 1e-14 * S;
  cfg.diverge = 1e3 * S;
  cfg.prescreen_cost = 1e-6f;
  cfg.prescreen_margin = 0.1f;
  cfg.mu32 = 1e-6f;
  cfg.mu64 = 1e-12;
  CandView cv{reinterpret_cast<const uint4*>(cand->rec), cand->capacity, cand->order_begin, cand->init_seed};
  SolView sv{out->T, out->cost, out->status, out->iters, out->evals, out->T32, out->capacity};
  DevEnds ep = dev_ends(ends);
  RefineList rl{ctx->counters + 8, nullptr};
  RefineList rl2{ctx->counters + 12, nullptr};
  if (precision == MPT_FP32_FP64REFINE) {
    // two lists of one 4-byte position per candidate (queued, then kept),
    // the queued entries' FP32 parameters and their ids and endpoints
    const size_t need = 2 * (size_t)cand->capacity * sizeof(int32_t) + 8 * (size_t)cand->capacity * sizeof(float) +
                        (size_t)cand->capacity * sizeof(uint4) + 1024;
    if (ctx->rscratch_bytes < need) {
      if (ctx->rscratch) MPT_CUDA_TRY(cudaFreeAsync(ctx->rscratch, st));
      ctx->rscratch = nullptr;
      ctx->rscratch_bytes = 0;
      MPT_CUDA_TRY(cudaMallocAsync(&ctx->rscratch, need, st));
      ctx->rscratch_bytes = need;
    }
    rl.idx = reinterpret_cast<int32_t*>(ctx->rscratch);
    rl2.idx = rl.idx + cand->capacity;
    const size_t prm_off = ((2 * (size_t)cand->capacity * sizeof(int32_t)) + 255) & ~size_t(255);
    rl.prm = reinterpret_cast<float*>(static_cast<unsigned char*>(ctx->rscratch) + prm_off);
    const size_t ends_off = (prm_off + 8 * (size_t)cand->capacity * sizeof(float) + 255) & ~size_t(255);
    rl.ends = reinterpret_cast<uint4*>(static_cast<unsigned char*>(ctx->rscratch) + ends_off);
    rl.stride = cand->capacity;
  }
  // FP32 copies of the endpoints for the FP32 iterations
  const int n_ends = ends->n_tx + ends->n_rx;
  const size_t ebytes = (size_t)n_ends * sizeof(float4) + 256;
  if (ctx->escratch_bytes < ebytes) {
    if (ctx->escratch) MPT_CUDA_TRY(cudaFreeAsync(ctx->escratch, st));
    ctx->escratch = nullptr;
    ctx->escratch_bytes = 0;
    MPT_CUDA_TRY(cudaMallocAsync(&ctx->escratch, ebytes, st));
    ctx->escratch_bytes = ebytes;
  }
  float4* ends32 = reinterpret_cast<float4*>(ctx->escratch);
  // exclusion pass scratch: the per-order lists (4 bytes per candidate),
  // the beams of every endpoint through every object (80 bytes each) and the
  // exclusion bits of every (endpoint, plane, object)
  const size_t n_eo = (size_t)n_ends * scene->d.n_obj;
  const size_t bits_bytes = ((n_eo * ((scene->d.n_obj + 31) / 32) * sizeof(uint32_t)) + 255) & ~size_t(255);
  const bool exclude = cfg.exclude && scene->d.side != nullptr && !(sch && sch->mixed_orders) && n_ends > 0 &&
                       n_ends <= 65535 && bits_bytes <= ((size_t)1 << 28);
  int32_t* xlist = nullptr;
  float4* beams = nullptr;
  uint32_t* xbits = nullptr;
  if (exclude) {
    const size_t list_bytes = ((size_t)cand->capacity * sizeof(int32_t) + 255) & ~size_t(255);
    const size_t beam_bytes = (n_eo * BEAM_F4 * sizeof(float4) + 255) & ~size_t(255);
    const size_t need = list_bytes + beam_bytes + bits_bytes + 256;
    if (ctx->xscratch_bytes < need) {
      if (ctx->xscratch) MPT_CUDA_TRY(cudaFreeAsync(ctx->xscratch, st));
      ctx->xscratch = nullptr;
      ctx->xscratch_bytes = 0;
      MPT_CUDA_TRY(cudaMallocAsync(&ctx->xscratch, need, st));
      ctx->xscratch_bytes = need;
    }
    xlist = reinterpret_cast<int32_t*>(ctx->xscratch);
    beams = reinterpret_cast<float4*>(static_cast<unsigned char*>(ctx->xscratch) + list_bytes);
    xbits = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(ctx->xscratch) + list_bytes + beam_bytes);
  }
  if (precision != MPT_FP64_PLAIN || exclude) {
    k_ends_f32<<<(n_ends + 255) / 256, 256, 0, st>>>(ends->tx, ends->n_tx, ends->rx, ends->n_rx, ends32);
    MPT_LAUNCH_CHECK();
  }
  const bool curved = scene_curved(scene);
  switch (precision) {
    case MPT_FP64_PLAIN:
      return launch_prec<MPT_FP64_PLAIN>(ctx, scene->d, ep, ends32, cv, sv, cfg, sch, rl, rl2, curved, xlist, beams, xbits,
                                    st);
    case MPT_FP32:
      return launch_prec<MPT_FP32>(ctx, scene->d, ep, ends32, cv, sv, cfg, sch, rl, rl2, curved, xlist, beams, xbits,
                                    st);
    case MPT_FP32_FP64REFINE:
      return launch_prec<MPT_FP32_FP64REFINE>(ctx, scene->d, ep, ends32, cv, sv, cfg, sch, rl, rl2, curved, xlist, beams, xbits,
                                    st);
    default: return MPT_ERR_ARG;
  }
}

}  // namespace mpt
