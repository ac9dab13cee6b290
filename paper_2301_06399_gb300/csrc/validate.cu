// Acceptance of Algorithm 1 ("C < threshold and X is valid") and the union
// of the valid paths into S, as a compacted list in candidate order.
//
// Candidates are taken in groups of GROUP (2048) consecutive indices.
//   k_flag         one block per group: lists the candidates that passed the
//                  solver's FP64 stage with cost < tau (a few percent of them)
//                  into a work list, one atomic per group.
//   k_accept_list  one thread per listed candidate: minimum segment length,
//                  bounds (Sec. II: bounds are applied a posteriori), then
//                  segment visibility against every occluder.  Occluder
//                  records and their boxes are staged into shared memory by
//                  bulk asynchronous copies (cp.async.bulk completing on an
//                  mbarrier).  The test runs in FP32 with a 1 mm margin;
//                  decisions inside the margin are re-taken in FP64 with the
//                  exact rule.  A valid candidate sets its bit in a bitmap
//                  and counts itself in its group.
//   k_accept_ovf   the same test for every candidate of a group whose
//                  entries did not fit a bounded list (fixed-size scratch).
//   k_scan         one CTA: exclusive scan of the group counts, total count.
//   k_scatter      one warp per group: writes the index of each valid
//                  candidate at (group offset + rank in group).
//   k_fill         one thread per path: parameters, points, length, cost.
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

// Parameters clearly inside the bounds in FP32: away from every bound by
// mb, which exceeds the FP32 rounding of the parameters and bounds (the
// exact FP64 test decides everything else).  Arc edges always go to FP64.
__device__ __forceinline__ bool clearly_in32(int kind, const Rec<float>& r, float s, float t, float mb) {
  if (kind == K_PLANE) return s >= mb && s <= r.v[3] - mb && t >= mb && t <= r.v[7] - mb;
  if (kind == K_PARAB) return r.v[13] > mb && s * s + t * t <= (r.v[13] - mb) * (r.v[13] - mb);
  if (kind == K_LINE) return s >= r.v[3] + mb && s <= r.v[7] - mb;
  return false;
}

// Point k (0 = TX, N + 1 = RX) of the path in FP64.
template <int N>
__device__ __forceinline__ v3<double> point64(const DevScene& sc, const DevEnds& ep, const Cand& cd, const double* Tc,
                                              int it_, int ir_, int j) {
  if (j == 0) return mk(ep.tx[3 * it_], ep.tx[3 * it_ + 1], ep.tx[3 * it_ + 2]);
  if (j == N + 1) return mk(ep.rx[3 * ir_], ep.rx[3 * ir_ + 1], ep.rx[3 * ir_ + 2]);
  const int k = j - 1;
  return point_at<double, false>(sc.kind[cd.ids[k]], load_obj64(sc, cd.ids[k]), Tc[2 * k], Tc[2 * k + 1]).X;
}

// The acceptance rule, decided in FP32 wherever the FP32 values are clear of
// the decision boundary by more than their rounding, else in FP64 with the
// exact rule (the same rule as the FP64 CPU reference):
//   bounds      clearly inside by mb = 1e-5 S + 4e-7 |bound| (FP32 parameters
//               and points are within ~1e-6 relative of the FP64 values);
//   segments    FP32 length >= 10 x the minimum length;
//   visibility  FP32 test with a 1 mm margin (rect32).
template <int N>
__device__ bool accept_one(const DevScene& sc, const DevEnds& ep, const Cand& cd, const double* Tc,
                           const float4* occ_sm, double S) {
  int it_, ir_;
  pair_ends(ep, cd.pair, it_, ir_);
  v3<float> P[N + 2];
  P[0] = mk(d2f_bits(ep.tx[3 * it_]), d2f_bits(ep.tx[3 * it_ + 1]), d2f_bits(ep.tx[3 * it_ + 2]));
  P[N + 1] = mk(d2f_bits(ep.rx[3 * ir_]), d2f_bits(ep.rx[3 * ir_ + 1]), d2f_bits(ep.rx[3 * ir_ + 2]));
  const float S32 = d2f_bits(S);
  bool exact_bounds = false;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int kind = sc.kind[cd.ids[k]];
    const Rec<float> r = load_obj32(sc, cd.ids[k]);
    const float s = d2f_bits(Tc[2 * k]), t = d2f_bits(Tc[2 * k + 1]);
    P[k + 1] = point_at<float, false>(kind, r, s, t).X;
    const float bound = kind == K_PARAB ? r.v[13] : fmaxf(fabsf(r.v[3]), fabsf(r.v[7]));
    exact_bounds = exact_bounds || !clearly_in32(kind, r, s, t, 1e-5f * S32 + 4e-7f * bound);
  }
  if (exact_bounds) {
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (!in_bounds64(sc.kind[cd.ids[k]], load_obj64(sc, cd.ids[k]), Tc[2 * k], Tc[2 * k + 1])) return false;
  }
  const double lmin = MIN_SEG_REL * S;
  const float lclear = 10.0f * d2f_bits(lmin);
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const v3<float> d = P[j + 1] - P[j];
    if (dot(d, d) >= lclear * lclear) continue;
    const v3<double> e = point64<N>(sc, ep, cd, Tc, it_, ir_, j + 1) - point64<N>(sc, ep, cd, Tc, it_, ir_, j);
    if (!(sqrt(dot(e, e)) >= lmin)) return false;
  }
  // visibility of every segment against every occluder: for up to 32 groups
  // at a time, the groups whose boxes the segment meets (a warp-uniform
  // pass), then only their occluders
  const float4* grp_sm = occ_sm + 6 * sc.n_occ;  // [2][n_grp]
  const int ng = sc.n_grp;
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const v3<float> Af = P[j], Bf = P[j + 1];
    const v3<float> inv = mk(1.0f / (Bf.x - Af.x), 1.0f / (Bf.y - Af.y), 1.0f / (Bf.z - Af.z));
    // rectangles whose plane holds an end of this segment cannot be crossed
    // strictly (both ends must be more than EPS_VIS off the plane)
    const int4 none = make_int4(-1, -1, -1, -1);
    const int4 own0 = j >= 1 ? sc.obj_occ[cd.ids[j - 1]] : none;
    const int4 own1 = j < N ? sc.obj_occ[cd.ids[j]] : none;
    for (int g0 = 0; g0 < ng; g0 += 32) {
      uint32_t gm = 0;
      const int gn = ng - g0 < 32 ? ng - g0 : 32;
      for (int q = 0; q < gn; ++q) gm |= (uint32_t)seg_box(Af, inv, grp_sm[g0 + q], grp_sm[ng + g0 + q]) << q;
      while (gm != 0) {
        const int gi = g0 + __ffs(gm) - 1;
        gm &= gm - 1;
        const int o_end = (gi + 1) * OCC_GROUP < sc.n_occ ? (gi + 1) * OCC_GROUP : sc.n_occ;
        for (int o = gi * OCC_GROUP; o < o_end; ++o) {
          if (!box_overlap(occ_sm[4 * sc.n_occ + o], occ_sm[5 * sc.n_occ + o], Af, Bf)) continue;
          if (o == own0.x || o == own0.y || o == own0.z || o == own0.w || o == own1.x || o == own1.y ||
              o == own1.z || o == own1.w)
            continue;
          int b = sc.occ_kind[o] == 0 ? rect32(occ_sm, sc.n_occ, o, Af, Bf) : -1;
          if (b < 0)
            b = blocks64(sc, o, point64<N>(sc, ep, cd, Tc, it_, ir_, j), point64<N>(sc, ep, cd, Tc, it_, ir_, j + 1))
                    ? 1
                    : 0;
          if (b) return false;
        }
      }
    }
  }
  return true;
}

// ------------------------------------------------------------ pipeline --
constexpr int GROUP = 2048;                          // candidates per group
constexpr int GROUP_WORDS = GROUP / 32;              // bitmap words per group
constexpr int FLAG_PER_THREAD = GROUP / ACC_BLOCK;   // candidates per k_flag thread
constexpr uint32_t LIST_SKIP = 0xFFFFFFFFu;          // list entry of a group that did not fit

struct ValScratch {
  unsigned long long* list_n;  // [2] list entries claimed; cursor of k_accept_list
  uint32_t* grp_count;         // [n_groups] valid paths per group
  uint32_t* words;             // [n_groups * GROUP_WORDS] one bit per valid candidate
  int64_t* grp_off;            // [n_groups] output position of the group's first path
  uint8_t* ovf;                // [n_groups] 1 = the group's entries did not fit the list
  uint32_t* list;              // [list_cap] candidates to test
  int64_t list_cap;
  int64_t n_groups;
};

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
// Scratch bytes for n_groups groups and a list of list_cap entries.  The
// first val_zero_bytes() of them (counter, counts, bitmap) are cleared by
// every call; everything after is written before it is read.
constexpr size_t val_zero_bytes(int64_t ng) {
  return al256(8) + al256((size_t)ng * 4) + al256((size_t)ng * GROUP_WORDS * 4);
}
constexpr size_t val_bytes(int64_t ng, int64_t lc) {
  return val_zero_bytes(ng) + al256((size_t)ng * 8) + al256((size_t)ng) + al256((size_t)lc * 4);
}
static ValScratch val_layout(unsigned char* base, int64_t ng, int64_t lc) {
  ValScratch v;
  size_t o = 0;
  v.list_n = reinterpret_cast<unsigned long long*>(base + o);
  o += al256(8);
  v.grp_count = reinterpret_cast<uint32_t*>(base + o);
  o += al256((size_t)ng * 4);
  v.words = reinterpret_cast<uint32_t*>(base + o);
  o += al256((size_t)ng * GROUP_WORDS * 4);
  v.grp_off = reinterpret_cast<int64_t*>(base + o);
  o += al256((size_t)ng * 8);
  v.ovf = reinterpret_cast<uint8_t*>(base + o);
  o += al256((size_t)ng);
  v.list = reinterpret_cast<uint32_t*>(base + o);
  v.list_cap = lc;
  v.n_groups = ng;
  return v;
}

__device__ __forceinline__ bool wanted(const AccView& av, int64_t c, double tau) {
  return (av.status[c] & MPT_PATH_REFINED) && av.cost[c] < tau;
}

__device__ __forceinline__ void mark_valid(const ValScratch& vs, int64_t c) {
  atomicOr(vs.words + (c >> 5), 1u << (c & 31));
  atomicAdd(vs.grp_count + c / GROUP, 1u);
}

__device__ bool accept_candidate(const DevScene& sc, const DevEnds& ep, const AccView& av, int64_t c,
                                 const float4* occ_sm) {
  const Cand cd = decode(av.rec[c]);
  if (!cand_in_range(sc, ep, cd)) return false;
  double Tc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) Tc[i] = i < 2 * cd.order ? av.T[(int64_t)i * av.sol_cap + c] : 0.0;
  switch (cd.order) {
    case 1: return accept_one<1>(sc, ep, cd, Tc, occ_sm, sc.scale);
    case 2: return accept_one<2>(sc, ep, cd, Tc, occ_sm, sc.scale);
    case 3: return accept_one<3>(sc, ep, cd, Tc, occ_sm, sc.scale);
    case 4: return accept_one<4>(sc, ep, cd, Tc, occ_sm, sc.scale);
    default: return false;
  }
}

// Stages the FP32 occluder records (fields 0-3), their boxes (fields 4-5) and
// the boxes of groups of OCC_GROUP consecutive occluders (after the fields)
// into shared memory with bulk copies; every thread waits, bounded, for them.
// On a wait that gives up, the error flag is set, thread 0 waits (again
// bounded) for the copy still in flight, and false is returned.
__device__ bool stage_occluders(const DevScene& sc, float4* occ_sm, uint64_t* bar, int* err_flag) {
  const uint32_t field_bytes = (uint32_t)sc.n_occ * 16u;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (sc.n_occ == 0) return true;
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, 6u * field_bytes + 32u * (uint32_t)sc.n_grp);
#pragma unroll
    for (int f = 0; f < 4; ++f) bulk_g2s(occ_sm + f * sc.n_occ, sc.c32 + f * sc.n_occ, field_bytes, bar);
#pragma unroll
    for (int f = 0; f < 2; ++f) bulk_g2s(occ_sm + (4 + f) * sc.n_occ, sc.cbox + f * sc.n_occ, field_bytes, bar);
    // group boxes: [2][n_grp] right after the six occluder fields
    bulk_g2s(occ_sm + 6 * sc.n_occ, sc.gbox, 32u * (uint32_t)sc.n_grp, bar);
  }
  bool staged = true;
  unsigned spins = 0;
  while (!mbar_try_wait(bar, 0)) {
    if (++spins > MBAR_SPIN_LIMIT) {
      staged = false;
      break;
    }
  }
  if (!staged) {
    atomicExch(err_flag, MPT_ERR_TIMEOUT);
    if (threadIdx.x == 0) {
      unsigned s2 = 0;
      while (!mbar_try_wait(bar, 0) && ++s2 < MBAR_SPIN_LIMIT) {
      }
    }
  }
  return staged;
}

// One block per group: the group's wanted candidates go to the list in one
// claim; a group whose entries do not all fit writes LIST_SKIP into the
// claimed positions that exist and is marked for k_accept_ovf.
__global__ void __launch_bounds__(ACC_BLOCK) k_flag(AccView av, double tau, ValScratch vs) {
  __shared__ uint32_t warp_off[ACC_WARPS];
  __shared__ unsigned long long s_base;
  __shared__ int s_fit;
  int64_t count = *av.count;
  if (count > av.cap) count = av.cap;
  const int64_t g = blockIdx.x;
  const int64_t c0 = g * GROUP;
  // thread t owns candidates c0 + FLAG_PER_THREAD t + j: their status bytes
  // come in one 8-byte load when the buffer allows it
  static_assert(FLAG_PER_THREAD == 8, "one 8-byte status load per thread");
  const int64_t ct = c0 + (int64_t)FLAG_PER_THREAD * threadIdx.x;
  uint32_t mask = 0;
  if (ct + FLAG_PER_THREAD <= count && (reinterpret_cast<uintptr_t>(av.status) & 7u) == 0) {
    const uint2 st = *reinterpret_cast<const uint2*>(av.status + ct);
#pragma unroll
    for (int j = 0; j < FLAG_PER_THREAD; ++j) {
      const uint32_t b = ((j < 4 ? st.x : st.y) >> (8 * (j & 3))) & 0xFFu;
      if ((b & MPT_PATH_REFINED) && av.cost[ct + j] < tau) mask |= 1u << j;
    }
  } else {
#pragma unroll
    for (int j = 0; j < FLAG_PER_THREAD; ++j) {
      const int64_t c = ct + j;
      if (c < count && wanted(av, c, tau)) mask |= 1u << j;
    }
  }
  const uint32_t n = __popc(mask);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = n;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_off[wid] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < ACC_WARPS; ++w) {
      const uint32_t v = warp_off[w];
      warp_off[w] = t;
      t += v;
    }
    unsigned long long base = 0;
    int fit = 1;
    if (t > 0) {
      base = atomicAdd(vs.list_n, (unsigned long long)t);
      fit = base + t <= (unsigned long long)vs.list_cap;
    }
    s_base = base;
    s_fit = fit;
    vs.ovf[g] = fit ? 0 : 1;
  }
  __syncthreads();
  if (mask) {
    unsigned long long pos = s_base + warp_off[wid] + (x - n);
#pragma unroll
    for (int j = 0; j < FLAG_PER_THREAD; ++j) {
      if (!((mask >> j) & 1u)) continue;
      if (s_fit) vs.list[pos] = (uint32_t)(ct + j);
      else if (pos < (unsigned long long)vs.list_cap) vs.list[pos] = LIST_SKIP;
      ++pos;
    }
  }
}

// Persistent grid over the list entries, one candidate per thread; warps
// claim 32 entries at a time from a cursor (vs.list_n[1]), so that blocks
// that meet cheap candidates take more of them.
constexpr int LIST_BLOCK = 128;
__global__ void __launch_bounds__(LIST_BLOCK, 3) k_accept_list(DevScene sc, DevEnds ep, AccView av, ValScratch vs,
                                                            int* err_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  float4* occ_sm = reinterpret_cast<float4*>(smem_raw);
  unsigned long long n = *vs.list_n;
  if (n > (unsigned long long)vs.list_cap) n = (unsigned long long)vs.list_cap;
  if (n == 0) return;  // the whole block
  if (!stage_occluders(sc, occ_sm, &bar, err_flag)) return;
  unsigned long long* cursor = vs.list_n + 1;
  const unsigned lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(cursor, 32ull);
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b >= n) break;
    const unsigned long long i = b + lane;
    if (i < n) {
      const uint32_t c = vs.list[i];
      if (c != LIST_SKIP && (int64_t)c < av.cap && accept_candidate(sc, ep, av, c, occ_sm)) mark_valid(vs, c);
    }
  }
}

// Groups whose entries did not fit the list: every candidate of the group.
__global__ void __launch_bounds__(ACC_BLOCK) k_accept_ovf(DevScene sc, DevEnds ep, AccView av, double tau,
                                                          ValScratch vs, int* err_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  float4* occ_sm = reinterpret_cast<float4*>(smem_raw);
  const int64_t g = blockIdx.x;
  if (!vs.ovf[g]) return;  // the whole block
  if (!stage_occluders(sc, occ_sm, &bar, err_flag)) return;
  int64_t count = *av.count;
  if (count > av.cap) count = av.cap;
  for (int j = 0; j < FLAG_PER_THREAD; ++j) {
    const int64_t c = g * GROUP + (int64_t)j * ACC_BLOCK + threadIdx.x;
    if (c < count && wanted(av, c, tau) && accept_candidate(sc, ep, av, c, occ_sm)) mark_valid(vs, c);
  }
}

// Exclusive scan of n counts by one CTA of 1024 threads; total to *total.
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

// Writes valid candidate c as path number pos: parameters, points, length.
__device__ void write_path(const DevScene& sc, const DevEnds& ep, const AccView& av, const PathView& pv, int64_t c,
                           int64_t pos) {
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
  pv.length[pos] = len;
  pv.cost[pos] = av.cost[c];
}

// One warp per group; lane l owns bitmap words 2l and 2l+1 (candidates
// 64l .. 64l+63 of the group), so a warp scan of the lanes' bit counts gives
// every valid candidate its position in candidate order.  Only the candidate
// index is written here; k_fill writes the rest, one thread per path.
__global__ void __launch_bounds__(ACC_BLOCK) k_scatter(ValScratch vs, PathView pv) {
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * ACC_WARPS + (threadIdx.x >> 5);
  if (g >= vs.n_groups) return;  // the whole warp
  const uint2 w = reinterpret_cast<const uint2*>(vs.words + g * GROUP_WORDS)[lane];
  const uint32_t n = __popc(w.x) + __popc(w.y);
  uint32_t x = n;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (n == 0) return;
  int64_t pos = vs.grp_off[g] + (int64_t)(x - n);
  const int64_t cbase = g * GROUP + (int64_t)lane * 64;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t bits = h ? w.y : w.x;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1u;
      if (pos < pv.cap) pv.cand[pos] = cbase + 32 * h + b;
      ++pos;
    }
  }
}

// Persistent grid over the written paths: parameters, points, length, cost
// of path i (consecutive threads write consecutive positions).
__global__ void __launch_bounds__(ACC_BLOCK) k_fill(DevScene sc, DevEnds ep, AccView av, const int64_t* count,
                                                    PathView pv) {
  int64_t n = *count;
  if (n > pv.cap) n = pv.cap;
  for (int64_t i = (int64_t)blockIdx.x * ACC_BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * ACC_BLOCK)
    write_path(sc, ep, av, pv, pv.cand[i], i);
}

// Enqueues the pipeline on scratch `base` (val_bytes(n_groups, list_cap)).
static int run_validate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                        const mpt_solutions* sol, double tau, mpt_paths* out, int64_t* d_valid_count,
                        unsigned char* base, int64_t n_groups, int64_t list_cap, bool may_overflow,
                        cudaStream_t st) {
  const ValScratch vs = val_layout(base, n_groups, list_cap);
  MPT_CUDA_TRY(cudaMemsetAsync(base, 0, val_zero_bytes(n_groups), st));
  AccView av{reinterpret_cast<const uint4*>(cand->rec), cand->count, cand->capacity, sol->T, sol->cost,
             sol->status, sol->capacity};
  const DevEnds ep = dev_ends(ends);
  k_flag<<<(unsigned)n_groups, ACC_BLOCK, 0, st>>>(av, tau, vs);
  MPT_LAUNCH_CHECK();
  const size_t smem = (size_t)scene->d.n_occ * 96 + (size_t)scene->d.n_grp * 32;
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(k_accept_list, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_accept_ovf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_accept_list, LIST_BLOCK, smem);
  if (occ < 1) occ = 1;
  int64_t grid = (int64_t)ctx->sms * occ;
  const int64_t need = (list_cap + LIST_BLOCK - 1) / LIST_BLOCK;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  k_accept_list<<<(unsigned)grid, LIST_BLOCK, smem, st>>>(scene->d, ep, av, vs, ctx->err_flag);
  MPT_LAUNCH_CHECK();
  if (may_overflow) {
    k_accept_ovf<<<(unsigned)n_groups, ACC_BLOCK, smem, st>>>(scene->d, ep, av, tau, vs, ctx->err_flag);
    MPT_LAUNCH_CHECK();
  }
  k_scan<<<1, 1024, 0, st>>>(vs.grp_count, n_groups, vs.grp_off, d_valid_count);
  MPT_LAUNCH_CHECK();
  PathView pv{out->cand, out->X, out->T, out->length, out->cost, out->capacity};
  k_scatter<<<(unsigned)((n_groups + ACC_WARPS - 1) / ACC_WARPS), ACC_BLOCK, 0, st>>>(vs, pv);
  MPT_LAUNCH_CHECK();
  if (out->capacity > 0) {
    int64_t fgrid = (out->capacity + ACC_BLOCK - 1) / ACC_BLOCK;
    if (fgrid > (int64_t)ctx->sms * 8) fgrid = (int64_t)ctx->sms * 8;
    k_fill<<<(unsigned)fgrid, ACC_BLOCK, 0, st>>>(scene->d, ep, av, d_valid_count, pv);
    MPT_LAUNCH_CHECK();
  }
  return MPT_OK;
}

// Candidate indices are stored in 32 bits (LIST_SKIP excluded).
constexpr int64_t MAX_CANDIDATES = (int64_t)LIST_SKIP;

int launch_validate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                    const mpt_solutions* sol, double tau, mpt_paths* out, int64_t* d_valid_count, cudaStream_t st) {
  const int64_t cap = cand->capacity;
  if (cap > MAX_CANDIDATES) return MPT_ERR_CAPACITY;
  const int64_t n_groups = (cap + GROUP - 1) / GROUP;
  if (n_groups < 1) {
    // no candidate to list: the count is still written
    MPT_CUDA_TRY(cudaMemsetAsync(d_valid_count, 0, sizeof(int64_t), st));
    return MPT_OK;
  }
  // a list as long as the candidates: it never overflows
  const size_t need = val_bytes(n_groups, cap);
  if (ctx->vscratch_bytes < need) {
    // grows the context's scratch (stream-ordered free of the old buffer)
    if (ctx->vscratch) MPT_CUDA_TRY(cudaFreeAsync(ctx->vscratch, st));
    ctx->vscratch = nullptr;
    ctx->vscratch_bytes = 0;
    MPT_CUDA_TRY(cudaMallocAsync(&ctx->vscratch, need, st));
    ctx->vscratch_bytes = need;
  }
  return run_validate(ctx, scene, ends, cand, sol, tau, out, d_valid_count,
                      reinterpret_cast<unsigned char*>(ctx->vscratch), n_groups, cap, false, st);
}

// --------------------------------------------- validation without allocation --
// Scratch of mpt_validate_noalloc: one fixed array in the library's device
// data, present on every GPU that loads the library until the process exits.
// It serves up to NOALLOC_MAX_CANDIDATES candidates (2^24) with a list of
// NOALLOC_LIST entries (2^18); groups whose entries do not fit are tested in
// full by k_accept_ovf.  3.3 MB in all.  The call clears the counter, counts
// and bitmap and writes every other word before reading it; calls that
// overlap on the GPU (two streams, two host threads) race on the array.
constexpr int64_t NOALLOC_MAX_CANDIDATES = int64_t(1) << 24;
constexpr int64_t NOALLOC_GROUPS = NOALLOC_MAX_CANDIDATES / GROUP;
constexpr int64_t NOALLOC_LIST = int64_t(1) << 18;
constexpr size_t NOALLOC_BYTES = val_bytes(NOALLOC_GROUPS, NOALLOC_LIST);
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
  const int64_t n_groups = (cap + GROUP - 1) / GROUP;
  if (n_groups < 1) {
    // no candidate to list: the count is still written
    MPT_CUDA_TRY(cudaMemsetAsync(d_valid_count, 0, sizeof(int64_t), st));
    return MPT_OK;
  }
  unsigned char* base = nullptr;
  const int rc = noalloc_scratch(ctx->device, &base);
  if (rc != MPT_OK) return rc;
  return run_validate(ctx, scene, ends, cand, sol, tau, out, d_valid_count, base, n_groups, NOALLOC_LIST, true,
                      st);
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
