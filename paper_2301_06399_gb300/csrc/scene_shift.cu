// Plane offsets moved on the device (mpt_scene_shift_planes): the
// differentiable configuration varies each wall's offset d in <n, X> = d, and
// the adjoint returns d(path)/d(d); evaluating the forward pass at shifted
// offsets must not need a trip through the host.  dst receives base's image
// (one device-to-device copy), then every plane object i with delta[i] != 0
// moves along its normal: corner O += delta n and d += delta in all four
// copies of its record (FP32 field-major and object-major, FP64, float-float),
// and so does the occluder rectangle that is the plane's own facet, with its
// box; the boxes of the occluder groups are then rebuilt as unions of their
// members' boxes.  Edges, other occluders and validation's lists of
// rectangles that hold an object stay base's.
#include "mpt_internal.cuh"

namespace mpt {

constexpr int SHIFT_BLOCK = 128;

__global__ void __launch_bounds__(SHIFT_BLOCK) k_shift_planes(DevScene d, const double* delta) {
  const int i = blockIdx.x * SHIFT_BLOCK + threadIdx.x;
  if (i >= d.n_obj || d.kind[i] != K_PLANE) return;
  const double dd = delta[i];
  if (dd == 0.0) return;
  // FP64 record, field-major double2: O.xyz U | u V | v d | n 0 (16 values)
  double2* o64 = const_cast<double2*>(d.o64);
  const int no = d.n_obj;
  double v[16];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    const double2 q = o64[f * no + i];
    v[2 * f] = q.x;
    v[2 * f + 1] = q.y;
  }
  const double nx = v[12], ny = v[13], nz = v[14];
  // unfused products and sums, as a host-side shift of the record would round
  v[0] = __dadd_rn(v[0], __dmul_rn(dd, nx));
  v[1] = __dadd_rn(v[1], __dmul_rn(dd, ny));
  v[2] = __dadd_rn(v[2], __dmul_rn(dd, nz));
  v[11] = __dadd_rn(v[11], dd);
#pragma unroll
  for (int f = 0; f < 8; ++f) o64[f * no + i] = make_double2(v[2 * f], v[2 * f + 1]);
  float4* o32 = const_cast<float4*>(d.o32);
  float4* a32 = const_cast<float4*>(d.a32);
  float4* aff = const_cast<float4*>(d.aff);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float4 q = make_float4(__double2float_rn(v[4 * f]), __double2float_rn(v[4 * f + 1]),
                                 __double2float_rn(v[4 * f + 2]), __double2float_rn(v[4 * f + 3]));
    o32[f * no + i] = q;
    a32[4 * i + f] = q;
  }
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    float h[2], l[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      h[j] = __double2float_rn(v[2 * f + j]);
      l[j] = __double2float_rn(__dsub_rn(v[2 * f + j], (double)h[j]));
    }
    aff[8 * i + f] = make_float4(h[0], l[0], h[1], l[1]);
  }
  // the plane's own occluder rectangle: O.xyz U | u V | v 0 | n 0
  const int q = d.own_occ[i];
  if (q < 0 || q >= d.n_occ) return;
  const int nc = d.n_occ;
  double2* c64 = const_cast<double2*>(d.c64);
  double2 c0 = c64[q], c1 = c64[nc + q];
  c0.x = __dadd_rn(c0.x, __dmul_rn(dd, nx));
  c0.y = __dadd_rn(c0.y, __dmul_rn(dd, ny));
  c1.x = __dadd_rn(c1.x, __dmul_rn(dd, nz));
  c64[q] = c0;
  c64[nc + q] = c1;
  float4* c32 = const_cast<float4*>(d.c32);
  float4 r0 = c32[q];
  r0.x = __double2float_rn(c0.x);
  r0.y = __double2float_rn(c0.y);
  r0.z = __double2float_rn(c1.x);
  c32[q] = r0;
  // its box moves with it (a translation); the 1 cm growth absorbs rounding
  float4* cbox = const_cast<float4*>(d.cbox);
  const float sx = __double2float_rn(dd * nx), sy = __double2float_rn(dd * ny), sz = __double2float_rn(dd * nz);
  float4 lo = cbox[q], hi = cbox[nc + q];
  lo.x += sx; lo.y += sy; lo.z += sz;
  hi.x += sx; hi.y += sy; hi.z += sz;
  cbox[q] = lo;
  cbox[nc + q] = hi;
}

__global__ void __launch_bounds__(SHIFT_BLOCK) k_group_boxes(DevScene d) {
  const int g = blockIdx.x * SHIFT_BLOCK + threadIdx.x;
  if (g >= d.n_grp) return;
  const int nc = d.n_occ;
  float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f), hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
  for (int q = g * OCC_GROUP; q < nc && q < (g + 1) * OCC_GROUP; ++q) {
    const float4 a = d.cbox[q], b = d.cbox[nc + q];
    lo.x = fminf(lo.x, a.x); lo.y = fminf(lo.y, a.y); lo.z = fminf(lo.z, a.z);
    hi.x = fmaxf(hi.x, b.x); hi.y = fmaxf(hi.y, b.y); hi.z = fmaxf(hi.z, b.z);
  }
  float4* gbox = const_cast<float4*>(d.gbox);
  gbox[g] = lo;
  gbox[d.n_grp + g] = hi;
}

int launch_shift_planes(mpt_ctx* ctx, const mpt_scene* base, mpt_scene* dst, const double* delta, cudaStream_t st) {
  (void)ctx;
  MPT_CUDA_TRY(cudaMemcpyAsync(dst->alloc, base->alloc, base->alloc_bytes, cudaMemcpyDeviceToDevice, st));
  const int no = dst->d.n_obj;
  k_shift_planes<<<(no + SHIFT_BLOCK - 1) / SHIFT_BLOCK, SHIFT_BLOCK, 0, st>>>(dst->d, delta);
  MPT_LAUNCH_CHECK();
  if (dst->d.n_grp > 0) {
    k_group_boxes<<<(dst->d.n_grp + SHIFT_BLOCK - 1) / SHIFT_BLOCK, SHIFT_BLOCK, 0, st>>>(dst->d);
    MPT_LAUNCH_CHECK();
  }
  return launch_side_table(dst->d, st);  // the planes moved
}

}  // namespace mpt
