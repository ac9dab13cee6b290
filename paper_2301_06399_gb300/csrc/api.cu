// C ABI entry points of libmpt: context, scene upload, argument checks and
// dispatch to the kernels, status strings and the FLOP model.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "mpt_internal.cuh"

namespace mpt {

int64_t host_candidate_count(const mpt_scene* scene, const mpt_endpoints* ends, int max_order,
                             const mpt_sampling* smp);

int check_ends(const mpt_endpoints* e) {
  if (!e || !e->tx || !e->rx || e->n_tx <= 0 || e->n_rx <= 0) return MPT_ERR_ARG;
  if (e->pair_mode != 0 && e->pair_mode != 1) return MPT_ERR_ARG;
  if (e->pair_mode == 1 && e->n_tx != e->n_rx) return MPT_ERR_ARG;
  if (n_pairs(e) > 0xFFFFFFFFll) return MPT_ERR_ARG;
  return MPT_OK;
}

// 24-value host record -> 16-value device record (see mpt_math.cuh).
static bool convert_object(int kind, const double* p, double* v) {
  for (int i = 0; i < 16; ++i) v[i] = 0.0;
  switch (kind) {
    case MPT_PLANE:
      v[0] = p[4]; v[1] = p[5]; v[2] = p[6]; v[3] = p[13];
      v[4] = p[7]; v[5] = p[8]; v[6] = p[9]; v[7] = p[14];
      v[8] = p[10]; v[9] = p[11]; v[10] = p[12]; v[11] = p[3];
      v[12] = p[0]; v[13] = p[1]; v[14] = p[2];
      return p[13] >= 0 && p[14] >= 0;
    case MPT_PARABOLOID: {
      const double f = p[12];
      if (!(f > 0) || !(p[13] > 0)) return false;
      for (int j = 0; j < 3; ++j) {
        v[4 * j + 0] = p[j];
        v[4 * j + 1] = p[3 + j];
        v[4 * j + 2] = p[6 + j];
        v[4 * j + 3] = p[9 + j];
      }
      v[12] = 1.0 / (4.0 * f); v[13] = p[13]; v[14] = 1.0 / (2.0 * f); v[15] = f;
      return true;
    }
    case MPT_LINE_EDGE:
      v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[6];
      v[4] = p[3]; v[5] = p[4]; v[6] = p[5]; v[7] = p[7];
      return p[7] >= p[6];
    case MPT_ARC_EDGE: {
      const double a[3] = {p[3], p[4], p[5]}, u[3] = {p[7], p[8], p[9]};
      v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[6];
      v[4] = u[0]; v[5] = u[1]; v[6] = u[2]; v[7] = p[10];
      v[8] = a[1] * u[2] - a[2] * u[1];
      v[9] = a[2] * u[0] - a[0] * u[2];
      v[10] = a[0] * u[1] - a[1] * u[0];
      v[11] = p[11];
      v[12] = a[0]; v[13] = a[1]; v[14] = a[2];
      return p[6] > 0 && p[11] >= p[10];
    }
    default:
      return false;
  }
}

static bool convert_occluder(int kind, const double* p, double* v) {
  for (int i = 0; i < 16; ++i) v[i] = 0.0;
  if (kind == MPT_OCC_RECT) {
    v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[9];
    v[4] = p[3]; v[5] = p[4]; v[6] = p[5]; v[7] = p[10];
    v[8] = p[6]; v[9] = p[7]; v[10] = p[8];
    v[12] = p[11]; v[13] = p[12]; v[14] = p[13];
    return true;
  }
  if (kind == MPT_OCC_PARABOLOID) return convert_object(MPT_PARABOLOID, p, v);
  return false;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace mpt

using namespace mpt;

extern "C" {

const char* mpt_status_string(int status) {
  switch (status) {
    case MPT_OK: return "MPT_OK";
    case MPT_ERR_ARG: return "MPT_ERR_ARG: invalid argument";
    case MPT_ERR_CUDA: return "MPT_ERR_CUDA: CUDA runtime error";
    case MPT_ERR_CAPACITY: return "MPT_ERR_CAPACITY: output buffer too small";
    case MPT_ERR_TIMEOUT: return "MPT_ERR_TIMEOUT: a bounded device wait gave up";
    case MPT_ERR_UNSUPPORTED: return "MPT_ERR_UNSUPPORTED: request not supported";
    default: return "unknown status";
  }
}

int mpt_ctx_create(int device, mpt_ctx** out) {
  if (!out) return MPT_ERR_ARG;
  *out = nullptr;
  int n_dev = 0;
  MPT_CUDA_TRY(cudaGetDeviceCount(&n_dev));
  if (device < 0 || device >= n_dev) return MPT_ERR_ARG;
  MPT_CUDA_TRY(cudaSetDevice(device));
  mpt_ctx* c = new mpt_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, 64 * sizeof(unsigned long long) + 256);
  if (e != cudaSuccess) {
    delete c;
    return MPT_ERR_CUDA;
  }
  cudaMemset(p, 0, 64 * sizeof(unsigned long long) + 256);
  c->counters = reinterpret_cast<unsigned long long*>(p);
  c->err_flag = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(p) + 64 * sizeof(unsigned long long));
  for (int i = 0; i < 3; ++i) {
    if (cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaFree(p);
      delete c;
      return MPT_ERR_CUDA;
    }
  }
  if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaFree(p);
    delete c;
    return MPT_ERR_CUDA;
  }
  c->vscratch = nullptr;
  c->vscratch_bytes = 0;
  c->rscratch = nullptr;
  c->rscratch_bytes = 0;
  c->escratch = nullptr;
  c->escratch_bytes = 0;
  c->xscratch = nullptr;
  c->xscratch_bytes = 0;
  c->tune_cache = nullptr;
  c->time_solver = false;
  c->ev_gn_made = false;
  *out = c;
  return MPT_OK;
}

int mpt_ctx_destroy(mpt_ctx* ctx) {
  if (!ctx) return MPT_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->vscratch) cudaFree(ctx->vscratch);
  if (ctx->rscratch) cudaFree(ctx->rscratch);
  if (ctx->escratch) cudaFree(ctx->escratch);
  if (ctx->xscratch) cudaFree(ctx->xscratch);
  cudaFree(ctx->counters);
  for (int i = 0; i < 3; ++i) {
    cudaStreamDestroy(ctx->aux[i]);
    cudaEventDestroy(ctx->ev_join[i]);
  }
  cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_gn_made)
    for (int o = 0; o < 4; ++o)
      for (int k = 0; k < 2; ++k) cudaEventDestroy(ctx->ev_gn[o][k]);
  mpt::tune_cache_free(ctx);
  delete ctx;
  return MPT_OK;
}

int mpt_ctx_sm_count(const mpt_ctx* ctx) { return ctx ? ctx->sms : 0; }

int mpt_ctx_time_solver(mpt_ctx* ctx, int on) {
  if (!ctx) return MPT_ERR_ARG;
  if (on && !ctx->ev_gn_made) {
    MPT_CUDA_TRY(cudaSetDevice(ctx->device));
    for (int o = 0; o < 4; ++o)
      for (int k = 0; k < 2; ++k)
        if (cudaEventCreate(&ctx->ev_gn[o][k]) != cudaSuccess) {
          for (int q = 0; q < 2 * o + k; ++q) cudaEventDestroy(ctx->ev_gn[q / 2][q % 2]);
          return MPT_ERR_CUDA;
        }
    ctx->ev_gn_made = true;
  }
  ctx->time_solver = on != 0;
  return MPT_OK;
}

int mpt_ctx_solver_ms(mpt_ctx* ctx, int order, float* ms) {
  if (!ctx || !ms || order < 1 || order > 4 || !ctx->ev_gn_made) return MPT_ERR_ARG;
  if (cudaEventElapsedTime(ms, ctx->ev_gn[order - 1][0], ctx->ev_gn[order - 1][1]) != cudaSuccess) {
    cudaGetLastError();
    return MPT_ERR_CUDA;
  }
  return MPT_OK;
}

int mpt_ctx_check(mpt_ctx* ctx, void* stream) {
  if (!ctx) return MPT_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int flag = 0;
  MPT_CUDA_TRY(cudaMemcpyAsync(&flag, ctx->err_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  MPT_CUDA_TRY(cudaStreamSynchronize(st));
  if (flag != 0) MPT_CUDA_TRY(cudaMemsetAsync(ctx->err_flag, 0, sizeof(int), st));
  return flag == 0 ? MPT_OK : flag;
}

namespace mpt {
// Waits on *flag (which nothing sets) for at most SELFTEST_SPINS polls
// 128 ns apart, then raises the error flag: the library's bounded-wait
// failure path, end to end.
constexpr unsigned SELFTEST_SPINS = 1u << 21;
__global__ void k_wait_selftest(const volatile int* flag, int* err_flag) {
  unsigned spins = 0;
  while (*flag == 0) {
    if (++spins > SELFTEST_SPINS) {
      atomicExch(err_flag, MPT_ERR_TIMEOUT);
      return;
    }
    __nanosleep(128);
  }
}
}  // namespace mpt

int mpt_ctx_selftest_wait(mpt_ctx* ctx, void* stream) {
  if (!ctx) return MPT_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the last counter word is zeroed at context creation and never written
  const int* flag = reinterpret_cast<const int*>(ctx->counters + 63);
  mpt::k_wait_selftest<<<1, 1, 0, st>>>(flag, ctx->err_flag);
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

int mpt_scene_upload(mpt_ctx* ctx, const mpt_scene_desc* desc, mpt_scene** out) {
  if (!ctx || !desc || !out) return MPT_ERR_ARG;
  *out = nullptr;
  const int no = desc->n_obj, nc = desc->n_occ;
  if (no < 1 || no > MPT_MAX_OBJECTS || nc < 0 || nc > MPT_MAX_OCCLUDERS) return MPT_ERR_ARG;
  if (!desc->obj_kind || !desc->obj_param || (nc > 0 && (!desc->occ_kind || !desc->occ_param)))
    return MPT_ERR_ARG;
  if (!(desc->scale > 0) || !std::isfinite(desc->scale)) return MPT_ERR_ARG;
  std::vector<double> ov((size_t)no * 16), cv((size_t)nc * 16);
  for (int o = 0; o < no; ++o)
    if (!convert_object(desc->obj_kind[o], desc->obj_param + (size_t)MPT_RECORD * o, &ov[(size_t)16 * o]))
      return MPT_ERR_ARG;
  for (int o = 0; o < nc; ++o)
    if (!convert_occluder(desc->occ_kind[o], desc->occ_param + (size_t)MPT_RECORD * o, &cv[(size_t)16 * o]))
      return MPT_ERR_ARG;
  // field-major device layout: float4 f of object o at [f * n + o]
  std::vector<float> o32((size_t)no * 16), c32((size_t)nc * 16);
  std::vector<double> o64((size_t)no * 16), c64((size_t)nc * 16);
  for (int o = 0; o < no; ++o)
    for (int i = 0; i < 16; ++i) {
      o32[((size_t)(i / 4) * no + o) * 4 + (i % 4)] = (float)ov[(size_t)16 * o + i];
      o64[((size_t)(i / 2) * no + o) * 2 + (i % 2)] = ov[(size_t)16 * o + i];
    }
  // object-major FP32 copy (the 64 bytes of object o contiguous) for the
  // solver, which reloads the records of its sequence at every evaluation:
  // one base address per object, the four float4 at constant offsets
  std::vector<float> a32((size_t)no * 16);
  for (int o = 0; o < no; ++o)
    for (int i = 0; i < 16; ++i) a32[(size_t)16 * o + i] = (float)ov[(size_t)16 * o + i];
  // object-major float-float copy (head, tail) for the refinement, the
  // adjoint and the image method: value = head + tail to about 48 bits
  std::vector<float> aff((size_t)no * 32);
  for (int o = 0; o < no; ++o)
    for (int i = 0; i < 16; ++i) {
      const double v = ov[(size_t)16 * o + i];
      const float hi = (float)v;
      aff[(size_t)32 * o + 2 * i] = hi;
      aff[(size_t)32 * o + 2 * i + 1] = (float)(v - (double)hi);
    }
  for (int o = 0; o < nc; ++o)
    for (int i = 0; i < 16; ++i) {
      c32[((size_t)(i / 4) * nc + o) * 4 + (i % 4)] = (float)cv[(size_t)16 * o + i];
      c64[((size_t)(i / 2) * nc + o) * 2 + (i % 2)] = cv[(size_t)16 * o + i];
    }
  // plane objects whose rectangle is also an occluder
  // Rectangles that hold every point an object can put on a path: for a
  // plane, rectangles in the same plane (its own rectangle first); for a
  // straight edge, rectangles whose plane contains both ends of the edge
  // (the faces that meet at it).  A segment that ends on such a plane cannot
  // cross it strictly (the visibility rule needs both ends more than 1e-6 m
  // off the plane), so validation skips them; up to 4 per object.
  std::vector<int32_t> obj_occ((size_t)no * 4, -1);
  std::vector<int32_t> own_occ((size_t)no, -1);  // the occluder that is a plane's own facet
  auto plane_dist = [&](const double* q, const double* X) {
    return (X[0] - q[0]) * q[12] + (X[1] - q[1]) * q[13] + (X[2] - q[2]) * q[14];
  };
  for (int o = 0; o < no; ++o) {
    const int kind = desc->obj_kind[o];
    if (kind != MPT_PLANE && kind != MPT_LINE_EDGE) continue;
    const double* a = &ov[(size_t)16 * o];
    int n_own = 0;
    auto add_own = [&](int q) {
      if (n_own < 4) obj_occ[(size_t)4 * o + n_own++] = q;
    };
    if (kind == MPT_PLANE) {
      for (int q = 0; q < nc; ++q) {
        if (desc->occ_kind[q] != MPT_OCC_RECT) continue;
        const double* b = &cv[(size_t)16 * q];
        // same corner, axes and extents (values 0..10 of both records)
        bool same = true;
        for (int i = 0; i < 11; ++i) same = same && a[i] == b[i];
        if (same) {
          add_own(q);
          own_occ[(size_t)o] = q;
          break;
        }
      }
    }
    for (int q = 0; q < nc; ++q) {
      if (desc->occ_kind[q] != MPT_OCC_RECT) continue;
      if (n_own > 0 && obj_occ[(size_t)4 * o] == q) continue;
      const double* b = &cv[(size_t)16 * q];
      bool on = false;
      if (kind == MPT_PLANE) {
        // coplanar: the plane's corner and both far corners lie in b's plane
        double c1[3], c2[3];
        for (int j = 0; j < 3; ++j) {
          c1[j] = a[j] + a[3] * a[4 + j];
          c2[j] = a[j] + a[7] * a[8 + j];
        }
        on = std::fabs(plane_dist(b, a)) < 1e-7 && std::fabs(plane_dist(b, c1)) < 1e-7 &&
             std::fabs(plane_dist(b, c2)) < 1e-7;
      } else {
        double e0[3], e1[3];
        for (int j = 0; j < 3; ++j) {
          e0[j] = a[j] + a[3] * a[4 + j];
          e1[j] = a[j] + a[7] * a[4 + j];
        }
        on = std::fabs(plane_dist(b, e0)) < 1e-7 && std::fabs(plane_dist(b, e1)) < 1e-7;
      }
      if (on) add_own(q);
    }
  }
  // occluder bounding boxes from FP64 corners, grown by 1 cm: rectangles from
  // their four corners, paraboloid patches from the eight corners of the
  // local box [-rho, rho]^2 x [0, rho^2 / (4f)] that holds the patch
  std::vector<float> cbox((size_t)nc * 8, 0.f);
  for (int q = 0; q < nc; ++q) {
    const double* v = &cv[(size_t)16 * q];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    auto add = [&](const double* p) {
      for (int j = 0; j < 3; ++j) {
        lo[j] = std::fmin(lo[j], p[j]);
        hi[j] = std::fmax(hi[j], p[j]);
      }
    };
    if (desc->occ_kind[q] == MPT_OCC_RECT) {
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
          double p[3];
          for (int j = 0; j < 3; ++j) p[j] = v[j] + a * v[3] * v[4 + j] + c * v[7] * v[8 + j];
          add(p);
        }
    } else {
      const double rho = v[13], zmax = rho * rho * v[12];
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c)
          for (int z = 0; z < 2; ++z) {
            const double sx = a ? rho : -rho, sy = c ? rho : -rho, sz = z ? zmax : 0.0;
            const double t0[3] = {v[3], v[7], v[11]};
            double p[3];
            for (int j = 0; j < 3; ++j) p[j] = t0[j] + sx * v[j] + sy * v[4 + j] + sz * v[8 + j];
            add(p);
          }
    }
    for (int j = 0; j < 3; ++j) {
      cbox[(size_t)4 * q + j] = (float)(lo[j] - 0.01);
      cbox[(size_t)4 * (nc + q) + j] = (float)(hi[j] + 0.01);
    }
    cbox[(size_t)4 * q + 3] = desc->occ_kind[q] == MPT_OCC_RECT ? 0.f : 1.f;  // lo.w: kind
  }
  const size_t s_kind = align256((size_t)no * 4), s_o32 = align256((size_t)no * 64),
               s_o64 = align256((size_t)no * 128), s_ck = align256((size_t)nc * 4 + 4),
               s_c32 = align256((size_t)nc * 64 + 16), s_c64 = align256((size_t)nc * 128 + 16),
               s_oo = align256((size_t)no * 16), s_cb = align256((size_t)nc * 32 + 16),
               s_a32 = align256((size_t)no * 64), s_aff = align256((size_t)no * 128),
               s_own = align256((size_t)no * 4);
  // boxes of groups of OCC_GROUP consecutive occluders (union of the members'
  // boxes): a segment that misses a group's box skips its members
  const int ng = (nc + mpt::OCC_GROUP - 1) / mpt::OCC_GROUP;
  std::vector<float> gbox((size_t)ng * 8, 0.f);
  for (int gi = 0; gi < ng; ++gi) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int q = gi * mpt::OCC_GROUP; q < nc && q < (gi + 1) * mpt::OCC_GROUP; ++q)
      for (int j = 0; j < 3; ++j) {
        lo[j] = std::fmin(lo[j], cbox[(size_t)4 * q + j]);
        hi[j] = std::fmax(hi[j], cbox[(size_t)4 * (nc + q) + j]);
      }
    for (int j = 0; j < 3; ++j) {
      gbox[(size_t)4 * gi + j] = lo[j];
      gbox[(size_t)4 * (ng + gi) + j] = hi[j];
    }
  }
  const size_t s_gb = align256((size_t)ng * 32 + 16);
  const size_t s_side = no <= mpt::SIDE_MAX_OBJ ? align256((size_t)no * no) : 0;
  const size_t s_vtx = align256((size_t)no * 128);
  const size_t total =
      s_kind + s_o32 + s_o64 + s_ck + s_c32 + s_c64 + s_oo + s_cb + s_a32 + s_gb + s_aff + s_own + s_side + s_vtx;
  MPT_CUDA_TRY(cudaSetDevice(ctx->device));
  void* mem = nullptr;
  MPT_CUDA_TRY(cudaMalloc(&mem, total));
  unsigned char* b = reinterpret_cast<unsigned char*>(mem);
  mpt_scene* s = new mpt_scene();
  s->ctx = ctx;
  s->alloc = mem;
  s->n_obj = no;
  s->host_kind = reinterpret_cast<int32_t*>(std::malloc(sizeof(int32_t) * no));
  std::memcpy(s->host_kind, desc->obj_kind, sizeof(int32_t) * no);
  // every array is laid out in one host image of the allocation and sent
  // with a single copy (one transfer instead of one per array)
  std::vector<unsigned char> image(total, 0);
  size_t off = 0;
  auto put = [&](const void* src, size_t n, size_t span) -> void* {
    void* dst = b + off;
    if (n) std::memcpy(image.data() + off, src, n);
    off += span;
    return dst;
  };
  DevScene& d = s->d;
  d.n_obj = no;
  d.n_occ = nc;
  d.kind = reinterpret_cast<const int32_t*>(put(desc->obj_kind, (size_t)no * 4, s_kind));
  d.o32 = reinterpret_cast<const float4*>(put(o32.data(), (size_t)no * 64, s_o32));
  d.o64 = reinterpret_cast<const double2*>(put(o64.data(), (size_t)no * 128, s_o64));
  d.occ_kind = reinterpret_cast<const int32_t*>(put(nc ? desc->occ_kind : nullptr, (size_t)nc * 4, s_ck));
  d.c32 = reinterpret_cast<const float4*>(put(c32.data(), (size_t)nc * 64, s_c32));
  d.c64 = reinterpret_cast<const double2*>(put(c64.data(), (size_t)nc * 128, s_c64));
  d.obj_occ = reinterpret_cast<const int4*>(put(obj_occ.data(), (size_t)no * 16, s_oo));
  d.cbox = reinterpret_cast<const float4*>(put(cbox.data(), (size_t)nc * 32, s_cb));
  d.a32 = reinterpret_cast<const float4*>(put(a32.data(), (size_t)no * 64, s_a32));
  d.n_grp = ng;
  d.gbox = reinterpret_cast<const float4*>(put(gbox.data(), (size_t)ng * 32, s_gb));
  d.aff = reinterpret_cast<const float4*>(put(aff.data(), (size_t)no * 128, s_aff));
  d.own_occ = reinterpret_cast<const int32_t*>(put(own_occ.data(), (size_t)no * 4, s_own));
  d.side = s_side ? reinterpret_cast<const int8_t*>(put(nullptr, 0, s_side)) : nullptr;  // built on the device
  d.vtx = reinterpret_cast<const float4*>(put(nullptr, 0, s_vtx));                         // likewise
  d.scale = desc->scale;
  s->signature = fnv1a(image.data(), total, fnv1a(&desc->scale, sizeof(double)));
  s->alloc_bytes = total;
  cudaError_t e = cudaMemcpy(mem, image.data(), total, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && launch_side_table(d, nullptr) != MPT_OK) e = cudaErrorLaunchFailure;
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFree(mem);
    std::free(s->host_kind);
    delete s;
    return MPT_ERR_CUDA;
  }
  *out = s;
  return MPT_OK;
}

int mpt_scene_free(mpt_scene* scene) {
  if (!scene) return MPT_ERR_ARG;
  cudaSetDevice(scene->ctx->device);
  cudaDeviceSynchronize();
  cudaFree(scene->alloc);
  std::free(scene->host_kind);
  delete scene;
  return MPT_OK;
}

int64_t mpt_candidate_count(const mpt_scene* scene, const mpt_endpoints* ends, int max_order,
                            const mpt_sampling* sampling) {
  return host_candidate_count(scene, ends, max_order, sampling);
}

int mpt_visibility(mpt_ctx* ctx, const mpt_scene* scene, uint8_t* vis, void* stream) {
  if (!ctx || !scene || !vis) return MPT_ERR_ARG;
  return launch_visibility(ctx, scene, vis, reinterpret_cast<cudaStream_t>(stream));
}

int mpt_enumerate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, int max_order,
                  const uint8_t* adj_mask, const mpt_sampling* sampling, mpt_candidates* out, void* stream) {
  if (!ctx || !scene || !out || !out->rec || !out->count || !out->order_begin || out->capacity < 0)
    return MPT_ERR_ARG;
  if (check_ends(ends) != MPT_OK) return MPT_ERR_ARG;
  return launch_enumerate(ctx, scene, ends, max_order, adj_mask, sampling, out,
                          reinterpret_cast<cudaStream_t>(stream));
}

int mpt_solve(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
              int precision, const mpt_schedule* schedule, mpt_solutions* out, void* stream) {
  if (!ctx || !scene || !cand || !out || !cand->rec || !cand->order_begin || !out->T || !out->cost ||
      !out->status || !out->iters || !out->evals)
    return MPT_ERR_ARG;
  if (check_ends(ends) != MPT_OK) return MPT_ERR_ARG;
  if (precision != MPT_FP64_PLAIN && precision != MPT_FP32 && precision != MPT_FP32_FP64REFINE) return MPT_ERR_ARG;
  if (schedule && (schedule->max_iters < 0 || schedule->refine_steps < 0 || schedule->blocks_per_sm < 0))
    return MPT_ERR_ARG;
  if (out->capacity < cand->capacity) return MPT_ERR_CAPACITY;
  if (cand->capacity > INT32_MAX) return MPT_ERR_CAPACITY;  // per-order offsets are 32-bit
  if (cand->capacity == 0) return MPT_OK;
  return launch_solve(ctx, scene, ends, cand, precision, schedule, out, reinterpret_cast<cudaStream_t>(stream));
}

int mpt_scene_shift_planes(mpt_ctx* ctx, const mpt_scene* base, mpt_scene* dst, const double* delta, void* stream) {
  if (!ctx || !base || !dst || !delta || base == dst) return MPT_ERR_ARG;
  if (base->alloc_bytes != dst->alloc_bytes || base->n_obj != dst->n_obj || base->d.n_occ != dst->d.n_occ ||
      std::memcmp(base->host_kind, dst->host_kind, sizeof(int32_t) * (size_t)base->n_obj) != 0)
    return MPT_ERR_ARG;
  return launch_shift_planes(ctx, base, dst, delta, reinterpret_cast<cudaStream_t>(stream));
}

int mpt_autotune(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                 int precision, mpt_solutions* out, mpt_schedule* best, double* best_ms, void* stream) {
  if (!ctx || !scene || !cand || !out || !best || !cand->rec || !cand->order_begin || !out->T || !out->cost ||
      !out->status || !out->iters || !out->evals)
    return MPT_ERR_ARG;
  if (check_ends(ends) != MPT_OK) return MPT_ERR_ARG;
  if (precision != MPT_FP64_PLAIN && precision != MPT_FP32 && precision != MPT_FP32_FP64REFINE) return MPT_ERR_ARG;
  if (out->capacity < cand->capacity) return MPT_ERR_CAPACITY;
  if (cand->capacity > INT32_MAX) return MPT_ERR_CAPACITY;
  if (cand->capacity == 0) {
    *best = mpt_schedule{};
    best->block = SOLVE_BLOCK;
    if (best_ms) *best_ms = 0.0;
    return MPT_OK;
  }
  return autotune(ctx, scene, ends, cand, precision, out, best, best_ms, reinterpret_cast<cudaStream_t>(stream));
}

int mpt_image_method(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                     mpt_solutions* out, void* stream) {
  if (!ctx || !scene || !cand || !out || !cand->rec || !cand->count || !cand->order_begin || !out->T ||
      !out->cost || !out->status || !out->iters || !out->evals)
    return MPT_ERR_ARG;
  if (check_ends(ends) != MPT_OK) return MPT_ERR_ARG;
  if (out->capacity < cand->capacity) return MPT_ERR_CAPACITY;
  return launch_image(ctx, scene, ends, cand, out, reinterpret_cast<cudaStream_t>(stream));
}

int mpt_validate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                 const mpt_solutions* sol, double tau, mpt_paths* out, int64_t* d_valid_count, void* stream) {
  if (!ctx || !scene || !cand || !sol || !out || !d_valid_count || !cand->rec || !cand->count || !sol->T ||
      !sol->cost || !sol->status || !out->cand || !out->X || !out->T || !out->length || !out->cost)
    return MPT_ERR_ARG;
  if (check_ends(ends) != MPT_OK) return MPT_ERR_ARG;
  if (!(tau > 0) || out->capacity < 0 || sol->capacity < cand->capacity) return MPT_ERR_ARG;
  return launch_validate(ctx, scene, ends, cand, sol, tau, out, d_valid_count,
                         reinterpret_cast<cudaStream_t>(stream));
}

int mpt_grad(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
             const mpt_paths* paths, const int64_t* d_valid_count, const double* g_len, const double* g_pts,
             double* g_tx, double* g_rx, double* g_obj, void* stream) {
  if (!ctx || !scene || !cand || !paths || !d_valid_count || !g_len || !cand->rec || !paths->cand || !paths->T)
    return MPT_ERR_ARG;
  if (check_ends(ends) != MPT_OK) return MPT_ERR_ARG;
  return launch_grad(ctx, scene, ends, cand, paths, d_valid_count, g_len, g_pts, g_tx, g_rx, g_obj,
                     reinterpret_cast<cudaStream_t>(stream));
}

int mpt_field(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
              const mpt_paths* paths, const int64_t* d_valid_count, const mpt_field_params* params, double* field,
              void* stream) {
  if (!ctx || !scene || !cand || !paths || !d_valid_count || !params || !field || !cand->rec || !paths->cand ||
      !paths->X || !(params->wavenumber > 0))
    return MPT_ERR_ARG;
  if (check_ends(ends) != MPT_OK) return MPT_ERR_ARG;
  return launch_field(ctx, scene, ends, cand, paths, d_valid_count, params, field,
                      reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
