// Received field of the valid paths (Sec. V, Eqs. 16-19), scalar form: the
// field of an isotropic source E0 e^{-jkr} / r (Eq. 16) carried along each
// path, where every interaction multiplies it by its coefficient, a spreading
// factor and the phase of the next segment (Eqs. 17, 18), and the paths of
// one TX/RX pair add up (Eq. 19).  With d_0 .. d_n the segment lengths and
// r_k = d_0 + ... + d_{k-1} the distance travelled to interaction k:
//   reflection   coef_R * r_k / (r_k + d_k)
//   diffraction  coef_D * sqrt(r_k / (d_k (r_k + d_k)))
// so a path contributes E0 e^{-jkL} / d_0 * prod(...), L = sum d_i (for
// reflections alone the product telescopes to the image source's E0 coef^n
// e^{-jkL} / L).  The dyadic coefficients of the paper are not given there;
// here the caller passes one complex coefficient per interaction kind.
// One thread per path, FP64; pairs accumulate with atomics.
#include "mpt_internal.cuh"

namespace mpt {

constexpr int FIELD_BLOCK = 128;

struct FieldView {
  const uint4* rec;
  int64_t rec_cap;
  const int64_t* pcand;
  const double* pX;
  int64_t pcap;
  const int64_t* count;
};

__global__ void __launch_bounds__(FIELD_BLOCK) k_field(DevScene sc, DevEnds ep, FieldView fv, mpt_field_params fp,
                                                       double* field) {
  int64_t n = *fv.count;
  if (n > fv.pcap) n = fv.pcap;
  for (int64_t i = (int64_t)blockIdx.x * FIELD_BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * FIELD_BLOCK) {
    const int64_t c = fv.pcand[i];
    if (c < 0 || c >= fv.rec_cap) continue;
    const Cand cd = decode(fv.rec[c]);
    if (!cand_in_range(sc, ep, cd)) continue;
    int it_, ir_;
    pair_ends(ep, cd.pair, it_, ir_);
    v3<double> prev = mk(ep.tx[3 * it_], ep.tx[3 * it_ + 1], ep.tx[3 * it_ + 2]);
    double d[5];
    for (int k = 0; k <= cd.order; ++k) {
      v3<double> X;
      if (k < cd.order)
        X = mk(fv.pX[(int64_t)(3 * k) * fv.pcap + i], fv.pX[(int64_t)(3 * k + 1) * fv.pcap + i],
               fv.pX[(int64_t)(3 * k + 2) * fv.pcap + i]);
      else
        X = mk(ep.rx[3 * ir_], ep.rx[3 * ir_ + 1], ep.rx[3 * ir_ + 2]);
      const v3<double> e = X - prev;
      d[k] = sqrt(dot(e, e));
      prev = X;
    }
    // amplitude (complex) and total length
    double are = fp.e0 / d[0], aim = 0.0, r = d[0], L = d[0];
    for (int k = 0; k < cd.order; ++k) {
      const bool edge = is_edge(sc.kind[cd.ids[k]]);
      const double s = d[k + 1];
      const double spread = edge ? sqrt(r / (s * (r + s))) : r / (r + s);
      const double cre = edge ? fp.diff[0] : fp.refl[0], cim = edge ? fp.diff[1] : fp.refl[1];
      const double tre = (are * cre - aim * cim) * spread, tim = (are * cim + aim * cre) * spread;
      are = tre;
      aim = tim;
      r += s;
      L += s;
    }
    double sn, cs;
    sincos(-fp.wavenumber * L, &sn, &cs);
    atomicAdd(field + 2 * (int64_t)cd.pair, are * cs - aim * sn);
    atomicAdd(field + 2 * (int64_t)cd.pair + 1, are * sn + aim * cs);
  }
}

int launch_field(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, const mpt_candidates* cand,
                 const mpt_paths* paths, const int64_t* d_valid_count, const mpt_field_params* fp, double* field,
                 cudaStream_t st) {
  if (paths->capacity <= 0) return MPT_OK;
  FieldView fv{reinterpret_cast<const uint4*>(cand->rec), cand->capacity, paths->cand, paths->X, paths->capacity,
               d_valid_count};
  int64_t blocks = (paths->capacity + FIELD_BLOCK - 1) / FIELD_BLOCK;
  if (blocks > (int64_t)ctx->sms * 8) blocks = (int64_t)ctx->sms * 8;
  k_field<<<(unsigned)blocks, FIELD_BLOCK, 0, st>>>(scene->d, dev_ends(ends), fv, *fp, field);
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

}  // namespace mpt
