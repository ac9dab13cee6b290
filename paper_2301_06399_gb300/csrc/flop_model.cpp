// FLOP model of the minimiser (host only): the kernel's own arithmetic from
// mpt_math.cuh instantiated with a scalar that counts its operations.
#include <cmath>
#include <cstdint>

#include "../../include/mpt.h"
#include "mpt_math.cuh"

namespace mpt {

// ------------------------------------------------------ FLOP counting --
// Scalar that counts its FP32-pipe operations (add/sub/mul = 1, fma = 2)
// and its special-function operations separately.
struct Cnt {
  float v;
  Cnt() : v(0) {}
  Cnt(float x) : v(x) {}   // NOLINT
  Cnt(double x) : v((float)x) {}  // NOLINT
  Cnt(int x) : v((float)x) {}  // NOLINT
};
static thread_local double g_flops = 0, g_sfu = 0;
inline Cnt operator+(Cnt a, Cnt b) { g_flops += 1; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_flops += 1; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_flops += 1; return Cnt(a.v * b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
inline bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
inline Cnt fma_(Cnt a, Cnt b, Cnt c) { g_flops += 2; return Cnt(a.v * b.v + c.v); }
inline Cnt rsq(Cnt a) { g_sfu += 1; return Cnt(1.0f / std::sqrt(a.v)); }
inline void sincos_(Cnt x, Cnt& s, Cnt& c) { g_sfu += 2; s = Cnt(std::sin(x.v)); c = Cnt(std::cos(x.v)); }

// FLOPs of one factorisation and solve over the QC live parameters.
template <int QC>
static double count_factor() {
  Cnt a[QC * (QC + 1) / 2], g[QC], x[QC];
  for (int i = 0; i < QC * (QC + 1) / 2; ++i) a[i] = Cnt(0.5f);
  for (int i = 0; i < QC; ++i) {
    a[tri(i, i)] = Cnt(4.0f);
    g[i] = Cnt(0.1f * (i + 1));
  }
  g_flops = 0;
  cholesky<QC, Cnt>(a, Cnt(1e-6f));
  chol_solve<QC, Cnt>(a, g, x);
  return g_flops;
}

template <int N>
static void count_model(const int32_t* kinds, double* f_eval, double* f_iter, double* sfu_eval) {
  int kind[N];
  Rec<Cnt> rec[N];
  Cnt prm[2 * N];
  for (int k = 0; k < N; ++k) {
    kind[k] = kinds[k];
    for (int i = 0; i < 16; ++i) rec[k].v[i] = Cnt(0.1f * (i + 1) + k);
    rec[k].v[3] = Cnt(2.0f);
    prm[2 * k] = Cnt(0.3f + k);
    prm[2 * k + 1] = Cnt(0.7f - k);
  }
  v3<Cnt> A = mk(Cnt(-5.0f), Cnt(1.0f), Cnt(3.0f)), B = mk(Cnt(6.0f), Cnt(-2.0f), Cnt(4.0f));
  constexpr int Q = 2 * N;
  Cnt jtj[Q * (Q + 1) / 2], g[Q], x[Q];
  bool ok;
  g_flops = 0;
  g_sfu = 0;
  eval_path<N, Cnt, Cnt, true>(kind, rec, prm, A, B, jtj, g, ok);
  // trial point update alpha * dlt + prm
  *f_eval = g_flops + 2.0 * Q;
  *sfu_eval = g_sfu;
  (void)x;
  // the step is algorithmically a factorisation over the live parameters:
  // two per surface interaction, one per edge (Eqs. 13-15)
  int qc = 0;
  for (int k = 0; k < N; ++k) qc += is_edge(kind[k]) ? 1 : 2;
  switch (qc) {
    case 1: *f_iter = count_factor<1>(); break;
    case 2: *f_iter = count_factor<2>(); break;
    case 3: *f_iter = count_factor<3>(); break;
    case 4: *f_iter = count_factor<4>(); break;
    case 5: *f_iter = count_factor<5>(); break;
    case 6: *f_iter = count_factor<6>(); break;
    case 7: *f_iter = count_factor<7>(); break;
    default: *f_iter = count_factor<8>(); break;
  }
}

}  // namespace mpt

using namespace mpt;

extern "C" {

int mpt_flop_model(int order, const int32_t* kinds, double* flops_per_iter, double* flops_per_eval,
                   double* sfu_per_eval) {
  if (order < 1 || order > 4 || !kinds || !flops_per_iter || !flops_per_eval) return MPT_ERR_ARG;
  for (int k = 0; k < order; ++k)
    if (kinds[k] < 0 || kinds[k] > 3) return MPT_ERR_ARG;
  double fe = 0, fi = 0, sfu = 0;
  switch (order) {
    case 1: count_model<1>(kinds, &fe, &fi, &sfu); break;
    case 2: count_model<2>(kinds, &fe, &fi, &sfu); break;
    case 3: count_model<3>(kinds, &fe, &fi, &sfu); break;
    default: count_model<4>(kinds, &fe, &fi, &sfu); break;
  }
  *flops_per_iter = fi;
  *flops_per_eval = fe;
  if (sfu_per_eval) *sfu_per_eval = sfu;
  return MPT_OK;
}

}  // extern "C"
