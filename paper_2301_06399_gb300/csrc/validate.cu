// Acceptance of Algorithm 1 ("C < threshold and X is valid") and the union
// of the valid paths into S, as a compacted list in candidate order.
//
//   k_accept   one thread per candidate: FP64 cost test, minimum segment
//              length, bounds (Sec. II: bounds are applied a posteriori),
//              then segment visibility against every occluder.  Occluder
//              records are staged into shared memory by one bulk
//              asynchronous copy per field array (cp.async.bulk completing
//              on an mbarrier).  The test runs in FP32 with a 1 mm margin;
//              decisions inside the margin are re-taken in FP64 with the
//              exact rule.  Writes one ballot word per warp and one count
//              per block.
//   k_scan     one CTA: exclusive scan of the block counts, total count.
//   k_scatter  writes each valid path at (block offset + rank in block).
#include <mutex>

#include "mpt_internal.cuh"

namespace mpt {

constexpr int ACC_BLOCK = 256;
constexpr int ACC_WARPS = ACC_BLOCK / 32;
constexpr float VIS_MARGIN = 1e-3f;     // FP32 decisions need this clearance (m)
constexpr double EPS_VIS = 1e-6;        // a crossing needs both ends > 1e-6 m off the surface
constexpr double MIN_SEG_REL = 1e-5;    // shortest accepted segment, relative to S
constexpr unsigned MBAR_SPIN_LIMIT = 1u << 22;

struct AccView {
  const uint4* rec;
  const int64_t* count;
  int64_t cap;
  const double* T;
  const double* cost;
  const uint8_t* status;
  int64_t sol_cap;
};

struct ScratchView {
  uint32_t* ballots;   // [n_blocks * ACC_WARPS]
  uint32_t* blk_count; // [n_blocks]
  int64_t* blk_off;    // [n_blocks]
};

// ---------------------------------------------------------------- PTX ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bulk global -> shared copy (no multicast); size and both addresses are
// multiples of 16 bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ------------------------------------------------------------ geometry --
// Exact FP64 rule (the same rule as the FP64 CPU reference): a rectangle
// blocks when both ends are strictly more than EPS_VIS on opposite sides and
// the crossing point is inside (inclusive); a paraboloid patch blocks when
// the segment meets it farther than EPS_VIS from both ends, inside the disc.
__device__ bool blocks64(const DevScene& s, int o, const v3<double>& A, const v3<double>& B) {
  Rec<double> r;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    double2 q = s.c64[f * s.n_occ + o];
    r.v[2 * f] = q.x; r.v[2 * f + 1] = q.y;
  }
  if (s.occ_kind[o] == 0) {
    const v3<double> O = r.f3(0), n = r.f3(12);
    const double sA = dot(A - O, n), sB = dot(B - O, n);
    if (!((sA < 0 && sB > 0) || (sA > 0 && sB < 0))) return false;
    if (!(fabs(sA) > EPS_VIS && fabs(sB) > EPS_VIS)) return false;
    const double t = sA / (sA - sB);
    const v3<double> P = axpy(t, B - A, A);
    const double uu = dot(P - O, r.f3(4)), vv = dot(P - O, r.f3(8));
    return uu >= 0 && uu <= r.v[3] && vv >= 0 && vv <= r.v[7];
  }
  // paraboloid patch in its local frame: al t^2 + be t + ga = 0
  const v3<double> t0 = mk(r.v[3], r.v[7], r.v[11]);
  const v3<double> wa = A - t0, wb = B - t0;
  const v3<double> a = mk(dot(wa, r.f3(0)), dot(wa, r.f3(4)), dot(wa, r.f3(8)));
  const v3<double> bl = mk(dot(wb, r.f3(0)), dot(wb, r.f3(4)), dot(wb, r.f3(8)));
  const v3<double> d = bl - a;
  const double q4 = r.v[12], rho = r.v[13];
  const double L = sqrt(dot(B - A, B - A));
  const double al = (d.x * d.x + d.y * d.y) * q4;
  const double be = (2.0 * a.x * d.x + 2.0 * a.y * d.y) * q4 - d.z;
  const double ga = (a.x * a.x + a.y * a.y) * q4 - a.z;
  double roots[2];
  int nr = 0;
  if (fabs(al) < 1e-300) {
    if (fabs(be) > 0) roots[nr++] = -ga / be;
  } else {
    const double disc = be * be - 4.0 * al * ga;
    if (disc >= 0) {
      const double q = -0.5 * (be + (be >= 0 ? 1.0 : -1.0) * sqrt(disc));
      roots[nr++] = q / al;
      if (q != 0) roots[nr++] = ga / q;
    }
  }
  for (int i = 0; i < nr; ++i) {
    const double t = roots[i];
    const v3<double> P = axpy(t, d, a);
    if (t * L > EPS_VIS && (1.0 - t) * L > EPS_VIS && P.x * P.x + P.y * P.y <= rho * rho) return true;
  }
  return false;
}

// FP32 rectangle test: 1 = blocked, 0 = clear, -1 = inside the margin
// (decide in FP64).
__device__ __forceinline__ int rect32(const float4* sm, int n_occ, int o, const v3<float>& A,
                                      const v3<float>& B) {
  const float4 f0 = sm[o], f1 = sm[n_occ + o], f2 = sm[2 * n_occ + o], f3 = sm[3 * n_occ + o];
  const v3<float> O = mk(f0.x, f0.y, f0.z), u = mk(f1.x, f1.y, f1.z), v = mk(f2.x, f2.y, f2.z),
                  n = mk(f3.x, f3.y, f3.z);
  const float sA = dot(A - O, n), sB = dot(B - O, n);
  const float M = VIS_MARGIN;
  if ((sA > M && sB > M) || (sA < -M && sB < -M)) return 0;
  if (!((sA > M && sB < -M) || (sA < -M && sB > M))) return -1;
  const float t = sA / (sA - sB);
  const v3<float> P = axpy(t, B - A, A) - O;
  const float uu = dot(P, u), vv = dot(P, v);
  if (uu < -M || uu > f0.w + M || vv < -M || vv > f1.w + M) return 0;
  if (uu > M && uu < f0.w - M && vv > M && vv < f1.w - M) return 1;
  return -1;
}

// Bounds of object parameters, inclusive (FP64).
__device__ __forceinline__ bool in_bounds64(int kind, const Rec<double>& r, double s, double t) {
  if (kind == K_PLANE) return s >= 0 && s <= r.v[3] && t >= 0 && t <= r.v[7];
  if (kind == K_PARAB) return sqrt(s * s + t * t) <= r.v[13];
  if (kind == K_LINE) return s >= r.v[3] && s <= r.v[7];
  const double twopi = 6.283185307179586;
  double phi = r.v[7] + fmod(s - r.v[7], twopi);
  if (phi < r.v[7]) phi += twopi;
  return phi <= r.v[11];
}

template <int N>
__device__ bool accept_one(const DevScene& sc, const DevEnds& ep, const Cand& cd, const double* Tc,
                           const float4* occ_sm, double S) {
  int it_, ir_;
  pair_ends(ep, cd.pair, it_, ir_);
  v3<double> P[N + 2];
  P[0] = mk(ep.tx[3 * it_], ep.tx[3 * it_ + 1], ep.tx[3 * it_ + 2]);
  P[N + 1] = mk(ep.rx[3 * ir_], ep.rx[3 * ir_ + 1], ep.rx[3 * ir_ + 2]);
  bool ok = true;
  int kind[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    kind[k] = sc.kind[cd.ids[k]];
    const Rec<double> r = load_obj64(sc, cd.ids[k]);
    P[k + 1] = point_at<double, false>(kind[k], r, Tc[2 * k], Tc[2 * k + 1]).X;
    ok = ok && in_bounds64(kind[k], r, Tc[2 * k], Tc[2 * k + 1]);
  }
  const double lmin = MIN_SEG_REL * S;
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const v3<double> d = P[j + 1] - P[j];
    ok = ok && (sqrt(dot(d, d)) >= lmin);
  }
  if (!ok) return false;
  // visibility of every segment against every occluder
  for (int j = 0; j <= N && ok; ++j) {
    const v3<float> Af = cvt<float>(P[j]), Bf = cvt<float>(P[j + 1]);
    // rectangles that hold an end of this segment cannot be crossed strictly
    const int own0 = j >= 1 ? sc.obj_occ[cd.ids[j - 1]] : -1;
    const int own1 = j < N ? sc.obj_occ[cd.ids[j]] : -1;
    for (int o = 0; o < sc.n_occ; ++o) {
      if (o == own0 || o == own1) continue;
      if (!box_overlap(occ_sm[4 * sc.n_occ + o], occ_sm[5 * sc.n_occ + o], Af, Bf)) continue;
      int b;
      if (sc.occ_kind[o] == 0) {
        b = rect32(occ_sm, sc.n_occ, o, Af, Bf);
        if (b < 0) b = blocks64(sc, o, P[j], P[j + 1]) ? 1 : 0;
      } else {
        b = blocks64(sc, o, P[j], P[j + 1]) ? 1 : 0;
      }
      if (b) { ok = false; break; }
    }
  }
  return ok;
}

__global__ void __launch_bounds__(ACC_BLOCK) k_accept(DevScene sc, DevEnds ep, AccView av, double tau,
                                                      ScratchView sv, int* err_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t warp_cnt[ACC_WARPS];
  float4* occ_sm = reinterpret_cast<float4*>(smem_raw);
  const uint32_t field_bytes = (uint32_t)sc.n_occ * 16u;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && sc.n_occ > 0) {
    // fields 0-3: FP32 occluder records; 4-5: their boxes (lo, hi)
    mbar_expect_tx(&bar, 6u * field_bytes);
#pragma unroll
    for (int f = 0; f < 4; ++f) bulk_g2s(occ_sm + f * sc.n_occ, sc.c32 + f * sc.n_occ, field_bytes, &bar);
#pragma unroll
    for (int f = 0; f < 2; ++f)
      bulk_g2s(occ_sm + (4 + f) * sc.n_occ, sc.cbox + f * sc.n_occ, field_bytes, &bar);
  }
  // bounded wait for the staged occluders
  bool staged = true;
  if (sc.n_occ > 0) {
    unsigned spins = 0;
    while (!mbar_try_wait(&bar, 0)) {
      if (++spins > MBAR_SPIN_LIMIT) { staged = false; break; }
    }
  }
  int64_t count = *av.count;
  if (count > av.cap) count = av.cap;
  const int64_t c = (int64_t)blockIdx.x * ACC_BLOCK + threadIdx.x;
  bool valid = false;
  if (staged && c < count) {
    const uint8_t st = av.status[c];
    const double cst = av.cost[c];
    const Cand cd = decode(av.rec[c]);
    if ((st & MPT_PATH_REFINED) && cst < tau && cand_in_range(sc, ep, cd)) {
      double Tc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) Tc[i] = i < 2 * cd.order ? av.T[(int64_t)i * av.sol_cap + c] : 0.0;
      switch (cd.order) {
        case 1: valid = accept_one<1>(sc, ep, cd, Tc, occ_sm, sc.scale); break;
        case 2: valid = accept_one<2>(sc, ep, cd, Tc, occ_sm, sc.scale); break;
        case 3: valid = accept_one<3>(sc, ep, cd, Tc, occ_sm, sc.scale); break;
        case 4: valid = accept_one<4>(sc, ep, cd, Tc, occ_sm, sc.scale); break;
        default: valid = false;
      }
    }
  }
  if (!staged && threadIdx.x == 0) {
    atomicExch(err_flag, MPT_ERR_TIMEOUT);
    // a copy that may still be in flight must land before the block exits
    unsigned spins = 0;
    while (!mbar_try_wait(&bar, 0) && ++spins < MBAR_SPIN_LIMIT) {
    }
  }
  const uint32_t ball = __ballot_sync(0xffffffffu, valid);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sv.ballots[(int64_t)blockIdx.x * ACC_WARPS + wid] = ball;
    warp_cnt[wid] = __popc(ball);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < ACC_WARPS; ++w) t += warp_cnt[w];
    sv.blk_count[blockIdx.x] = t;
  }
}

// Exclusive scan of n block counts by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan(const uint32_t* cnt, int64_t n, int64_t* off, int64_t* total) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t s_base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int64_t i0 = 0; i0 < n; i0 += 1024) {
    const int64_t i = i0 + tid;
    const int64_t v = i < n ? (int64_t)cnt[i] : 0;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int64_t w = warp_tot[lane];
      int64_t z = w;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, z, d);
        if (lane >= d) z += y;
      }
      warp_tot[lane] = z - w;
    }
    __syncthreads();
    const int64_t ex = s_base + warp_tot[wid] + (x - v);
    if (i < n) off[i] = ex;
    __syncthreads();
    if (tid == 1023) s_base = ex + v;
    __syncthreads();
  }
  if (tid == 0) *total = s_base;
}

struct PathView {
  int64_t* cand;
  double* X;
  double* T;
  double* length;
  double* cost;
  int64_t cap;
};

__global__ void __launch_bounds__(ACC_BLOCK) k_scatter(DevScene sc, DevEnds ep, AccView av, ScratchView sv,
                                                       PathView pv) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ball = sv.ballots[(int64_t)blockIdx.x * ACC_WARPS + wid];
  if (!((ball >> lane) & 1u)) return;
  int64_t pos = sv.blk_off[blockIdx.x];
  for (int w = 0; w < wid; ++w) pos += __popc(sv.ballots[(int64_t)blockIdx.x * ACC_WARPS + w]);
  pos += __popc(ball & ((1u << lane) - 1u));
  if (pos >= pv.cap) return;
  const int64_t c = (int64_t)blockIdx.x * ACC_BLOCK + threadIdx.x;
  const Cand cd = decode(av.rec[c]);
  int it_, ir_;
  pair_ends(ep, cd.pair, it_, ir_);
  v3<double> prev = mk(ep.tx[3 * it_], ep.tx[3 * it_ + 1], ep.tx[3 * it_ + 2]);
  double len = 0;
  for (int k = 0; k < 4; ++k) {
    const double s = k < cd.order ? av.T[(int64_t)(2 * k) * av.sol_cap + c] : 0.0;
    const double t = k < cd.order ? av.T[(int64_t)(2 * k + 1) * av.sol_cap + c] : 0.0;
    pv.T[(int64_t)(2 * k) * pv.cap + pos] = s;
    pv.T[(int64_t)(2 * k + 1) * pv.cap + pos] = t;
    v3<double> X = mk(0.0, 0.0, 0.0);
    if (k < cd.order) {
      const int kind = sc.kind[cd.ids[k]];
      X = point_at<double, false>(kind, load_obj64(sc, cd.ids[k]), s, t).X;
      const v3<double> d = X - prev;
      len += sqrt(dot(d, d));
      prev = X;
    }
    pv.X[(int64_t)(3 * k) * pv.cap + pos] = X.x;
    pv.X[(int64_t)(3 * k + 1) * pv.cap + pos] = X.y;
    pv.X[(int64_t)(3 * k + 2) * pv.cap + pos] = X.z;
  }
  const v3<double> B = mk(ep.rx[3 * ir_], ep.rx[3 * ir_ + 1], ep.rx[3 * ir_ + 2]);
  const v3<double> d = B - prev;
  len += sqrt(dot(d, d));
  pv.cand[pos] = c;
  pv.length[pos] = len;
  pv.cost[pos] = av.cost[c];
}

static size_t scratch_bytes(int64_t n_blocks) {
  return (size_t)n_blocks * ACC_WARPS * 4 + (size_t)n_blocks * 4 + (size_t)n_blocks * 8 + 256;
}

int launch_validate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                    const mpt_solutions* sol, double tau, mpt_paths* out, int64_t* d_valid_count, cudaStream_t st) {
  const int64_t cap = cand->capacity;
  const int64_t n_blocks = (cap + ACC_BLOCK - 1) / ACC_BLOCK;
  if (n_blocks < 1) return MPT_OK;
  const size_t need = scratch_bytes(n_blocks);
  if (ctx->vscratch_bytes < need) {
    // grows the context's scratch (stream-ordered free of the old buffer)
    if (ctx->vscratch) MPT_CUDA_TRY(cudaFreeAsync(ctx->vscratch, st));
    ctx->vscratch = nullptr;
    ctx->vscratch_bytes = 0;
    MPT_CUDA_TRY(cudaMallocAsync(&ctx->vscratch, need, st));
    ctx->vscratch_bytes = need;
  }
  unsigned char* base = reinterpret_cast<unsigned char*>(ctx->vscratch);
  ScratchView sv;
  sv.blk_off = reinterpret_cast<int64_t*>(base);
  sv.blk_count = reinterpret_cast<uint32_t*>(base + (size_t)n_blocks * 8);
  sv.ballots = reinterpret_cast<uint32_t*>(base + (size_t)n_blocks * 12);
  AccView av{reinterpret_cast<const uint4*>(cand->rec), cand->count, cap, sol->T, sol->cost, sol->status,
             sol->capacity};
  const DevEnds ep = dev_ends(ends);
  const size_t smem = (size_t)scene->d.n_occ * 96;
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(k_accept, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  k_accept<<<(unsigned)n_blocks, ACC_BLOCK, smem, st>>>(scene->d, ep, av, tau, sv, ctx->err_flag);
  MPT_LAUNCH_CHECK();
  k_scan<<<1, 1024, 0, st>>>(sv.blk_count, n_blocks, sv.blk_off, d_valid_count);
  MPT_LAUNCH_CHECK();
  PathView pv{out->cand, out->X, out->T, out->length, out->cost, out->capacity};
  k_scatter<<<(unsigned)n_blocks, ACC_BLOCK, 0, st>>>(scene->d, ep, av, sv, pv);
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

// --------------------------------------------- validation without allocation --
// Scratch of mpt_validate_noalloc: one fixed array in the library's device
// data, present on every GPU that loads the library until the process exits.
// It serves up to NOALLOC_MAX_CANDIDATES candidates (2^24): per block of 256
// candidates one 8-byte offset, one 4-byte count and eight 4-byte ballots,
// 2.9 MB in all.  Every word a call reads is written earlier in the same call
// (k_accept writes the count and ballots of every block it covers, k_scan
// every offset), so nothing needs clearing between calls; calls that overlap
// on the GPU (two streams, two host threads) race on the array.
constexpr int64_t NOALLOC_MAX_CANDIDATES = int64_t(1) << 24;
constexpr int64_t NOALLOC_MAX_BLOCKS = NOALLOC_MAX_CANDIDATES / ACC_BLOCK;
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_MAX_BLOCKS * (8 + 4 + 4 * ACC_WARPS);
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch on `device`, looked up once per device
// with that device current.  In host code the array's name only stands for
// the symbol; passing it to a kernel would not give its device address.
static int noalloc_scratch(int device, unsigned char** out) {
  static std::mutex mu;
  static void* addr[256] = {};
  if (device < 0 || device >= 256) return MPT_ERR_ARG;
  std::lock_guard<std::mutex> lock(mu);
  if (addr[device] == nullptr) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return MPT_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return MPT_ERR_CUDA;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess || p == nullptr) {
      std::fprintf(stderr, "libmpt: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return MPT_ERR_CUDA;
    }
    addr[device] = p;
  }
  *out = reinterpret_cast<unsigned char*>(addr[device]);
  return MPT_OK;
}

static int launch_validate_noalloc(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                                   const mpt_candidates* cand, const mpt_solutions* sol, double tau,
                                   mpt_paths* out, int64_t* d_valid_count, cudaStream_t st) {
  const int64_t cap = cand->capacity;
  if (cap > NOALLOC_MAX_CANDIDATES) return MPT_ERR_CAPACITY;
  const int64_t n_blocks = (cap + ACC_BLOCK - 1) / ACC_BLOCK;
  if (n_blocks < 1) return MPT_OK;
  unsigned char* base = nullptr;
  const int rc = noalloc_scratch(ctx->device, &base);
  if (rc != MPT_OK) return rc;
  ScratchView sv;
  sv.blk_off = reinterpret_cast<int64_t*>(base);
  sv.blk_count = reinterpret_cast<uint32_t*>(base + (size_t)NOALLOC_MAX_BLOCKS * 8);
  sv.ballots = reinterpret_cast<uint32_t*>(base + (size_t)NOALLOC_MAX_BLOCKS * 12);
  AccView av{reinterpret_cast<const uint4*>(cand->rec), cand->count, cap, sol->T, sol->cost, sol->status,
             sol->capacity};
  const DevEnds ep = dev_ends(ends);
  const size_t smem = (size_t)scene->d.n_occ * 96;
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(k_accept, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  k_accept<<<(unsigned)n_blocks, ACC_BLOCK, smem, st>>>(scene->d, ep, av, tau, sv, ctx->err_flag);
  MPT_LAUNCH_CHECK();
  k_scan<<<1, 1024, 0, st>>>(sv.blk_count, n_blocks, sv.blk_off, d_valid_count);
  MPT_LAUNCH_CHECK();
  PathView pv{out->cand, out->X, out->T, out->length, out->cost, out->capacity};
  k_scatter<<<(unsigned)n_blocks, ACC_BLOCK, 0, st>>>(scene->d, ep, av, sv, pv);
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

}  // namespace mpt

extern "C" int mpt_validate_noalloc(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                                    const mpt_candidates* cand, const mpt_solutions* sol, double tau,
                                    mpt_paths* out, int64_t* d_valid_count, void* stream) {
  if (!ctx || !scene || !cand || !sol || !out || !d_valid_count || !cand->rec || !cand->count || !sol->T ||
      !sol->cost || !sol->status || !out->cand || !out->X || !out->T || !out->length || !out->cost)
    return MPT_ERR_ARG;
  if (mpt::check_ends(ends) != MPT_OK) return MPT_ERR_ARG;
  if (!(tau > 0) || out->capacity < 0 || sol->capacity < cand->capacity) return MPT_ERR_ARG;
  return mpt::launch_validate_noalloc(ctx, scene, ends, cand, sol, tau, out, d_valid_count,
                                      reinterpret_cast<cudaStream_t>(stream));
}
