// Image method (Sec. III-A, Eqs. 5-6) for the candidates whose objects are
// all planes: the paper's own baseline and, for reflection-only sequences, a
// direct alternative to the minimisation.
//
// Forward pass (Eq. 5): the images of the transmitter, I_0 = TX and
//   I_k = I_{k-1} - 2 (<I_{k-1}, n_k> - d_k) n_k        (plane <n_k, X> = d_k).
// Backward pass (Eq. 6): from X_{n+1} = RX,
//   lambda_k = (d_k - <X_{k+1}, n_k>) / <X_{k+1} - I_k, n_k>,
//   X_k = X_{k+1} + lambda_k (X_{k+1} - I_k).
// The path exists on the (unbounded) planes when every lambda_k lies strictly
// in (-1, 0): X_k is then strictly between X_{k+1} and the image I_k, i.e.
// the straight line to the image crosses the mirror.  Bounds and visibility
// are left to mpt_validate, exactly as for the minimiser's solutions.
//
// Arithmetic is float-float (pairs of FP32, 48-bit significand): images of a
// 100 m scene lie up to a few km away, beyond FP32's reach for 1e-6 m
// points, and GB300's FP64 pipe is a small fraction of its FP32 rate.  One
// thread per candidate; the objects of a candidate's sequence are shared by
// the threads of a warp (pairs are the fastest candidate index).
#include "ff.cuh"
#include "mpt_internal.cuh"

namespace mpt {

constexpr int IMG_BLOCK = 128;

// a / b in float-float: Dekker's long division (1971), a first quotient from
// the FP32 heads, then one correction from the float-float remainder.
__device__ __forceinline__ ff ff_div(const ff& a, const ff& b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = a - ff(q1) * b;
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return quick_two_sum(q1, q2);
}

struct ImgOut {
  double* T;
  double* cost;
  uint8_t* status;
  uint8_t* iters;
  uint8_t* evals;
  int64_t cap;
};

template <int N>
__device__ __forceinline__ void image_one(const DevScene& sc, const DevEnds& ep, const Cand& cd, int64_t c,
                                          const ImgOut& out) {
  int it_, ir_;
  pair_ends(ep, cd.pair, it_, ir_);
  v3<ff> n[N], O[N], U[N], V[N];
  ff d[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const Rec<ff> r = load_obj_ff(sc, cd.ids[k]);  // O U | u V | v d | n
    O[k] = r.f3(0);
    U[k] = r.f3(4);
    V[k] = r.f3(8);
    d[k] = r.v[11];
    n[k] = r.f3(12);
  }
  // Eq. 5: images of the transmitter through planes 1..N
  v3<ff> I[N + 1];
  I[0] = load_end_ff(ep.tx, it_);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const ff h = dot(I[k], n[k]) - d[k];
    I[k + 1] = axpy(ff(-2.0f) * h, n[k], I[k]);
  }
  // Eq. 6: points from the receiver back towards the transmitter
  v3<ff> X = load_end_ff(ep.rx, ir_);
  bool exists = true;
  double T[2 * N];
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const v3<ff> w = X - I[k + 1];
    const ff lam = ff_div(d[k] - dot(X, n[k]), dot(w, n[k]));
    exists = exists && lam.hi > -1.0f && lam.hi < 0.0f && isfinite(lam.hi);
    X = axpy(lam, w, X);
    const v3<ff> q = X - O[k];
    T[2 * k] = to_double(dot(q, U[k]));
    T[2 * k + 1] = to_double(dot(q, V[k]));
  }
#pragma unroll
  for (int j = 0; j < 2 * N; ++j) out.T[(int64_t)j * out.cap + c] = T[j];
  out.cost[c] = exists ? 0.0 : (double)INFINITY;
  out.status[c] = (uint8_t)((exists ? MPT_PATH_CONVERGED : MPT_PATH_STALLED) | MPT_PATH_REFINED);
  out.iters[c] = 0;
  out.evals[c] = 0;
}

// One launch per order over its candidate range (read on the device), so
// each kernel holds only its own order's registers.
template <int N>
__global__ void __launch_bounds__(IMG_BLOCK) k_image(DevScene sc, DevEnds ep, const uint4* rec,
                                                     const int64_t* order_begin, int64_t cap, ImgOut out) {
  int64_t end = order_begin[N];
  if (end > cap) end = cap;
  int64_t begin = order_begin[N - 1];
  if (begin > end) begin = end;
  for (int64_t c = begin + (int64_t)blockIdx.x * IMG_BLOCK + threadIdx.x; c < end;
       c += (int64_t)gridDim.x * IMG_BLOCK) {
    const Cand cd = decode(__ldg(rec + c));
    bool planar = cd.order == N && cand_in_range(sc, ep, cd);
#pragma unroll
    for (int k = 0; k < N; ++k) planar = planar && __ldg(sc.kind + cd.ids[k]) == K_PLANE;
    if (planar) {
      image_one<N>(sc, ep, cd, c, out);
    } else {
      out.cost[c] = (double)INFINITY;
      out.status[c] = (uint8_t)MPT_PATH_NONFINITE;
      out.iters[c] = 0;
      out.evals[c] = 0;
    }
  }
}

template <int N>
static int launch_image_order(mpt_ctx* ctx, const mpt_scene* scene, const DevEnds& ep, const mpt_candidates* cand,
                              const ImgOut& o, cudaStream_t st) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_image<N>, IMG_BLOCK, 0);
  if (occ < 1) occ = 1;
  int64_t grid = (cand->capacity + IMG_BLOCK - 1) / IMG_BLOCK;
  if (grid > (int64_t)ctx->sms * occ) grid = (int64_t)ctx->sms * occ;
  k_image<N><<<(unsigned)grid, IMG_BLOCK, 0, st>>>(scene->d, ep, reinterpret_cast<const uint4*>(cand->rec),
                                                   cand->order_begin, cand->capacity, o);
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

int launch_image(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                 mpt_solutions* out, cudaStream_t st) {
  if (cand->capacity <= 0) return MPT_OK;
  const DevEnds ep = dev_ends(ends);
  const ImgOut o{out->T, out->cost, out->status, out->iters, out->evals, out->capacity};
  int rc = launch_image_order<1>(ctx, scene, ep, cand, o, st);
  if (rc == MPT_OK) rc = launch_image_order<2>(ctx, scene, ep, cand, o, st);
  if (rc == MPT_OK) rc = launch_image_order<3>(ctx, scene, ep, cand, o, st);
  if (rc == MPT_OK) rc = launch_image_order<4>(ctx, scene, ep, cand, o, st);
  return rc;
}

}  // namespace mpt
