// FP64 CPU oracle for Min-Path-Tracing (MPT).  TEST INFRASTRUCTURE ONLY.
//
// Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
// load this library.  The CUDA library never links it and shares no code,
// headers or tables with it.  Everything here is deliberately plain: FP64
// throughout, forward-mode dual numbers for every derivative (the CUDA path
// uses hand-derived Jacobians), Gauss-Newton with a dense Gaussian
// elimination, brute-force visibility against every occluder.
//
// What each part follows in the paper (arXiv 2301.06399):
//   unknowns       the parametric form of Eqs. 13-15: every interaction
//                  point is carried on its object by its surface (s, t) or
//                  edge (t) parameters, so the constraints f_k(X_k) = 0 of
//                  Eq. 11 hold exactly and the cost is ||I(X(T))||^2 (Eq. 15)
//   residuals      Eq. 8 divided by ||X_k - X_{k-1}|| (one of the rescalings
//                  the note after Eq. 9 permits): r_hat - (i_hat - 2<i_hat,n>n)
//                  with the normal of Eq. 2; Eq. 9 as printed with the edge
//                  tangent of Eq. 4
//   minimiser      find_minimum_path of Algorithm 1 (the paper leaves the
//                  solver open; it is read as Gauss-Newton with a
//                  backtracking line search and fixed stopping rules)
//   candidates     all_simple_paths of Algorithm 1 (ordered sequences of
//                  distinct objects, up to n_t interactions), optional
//                  adjacency mask (Sec. III, Fig. 5)
//   acceptance     "C < threshold and X is valid" of Algorithm 1: bounds are
//                  applied a posteriori (Sec. II), plus segment visibility
//   gradients      implicit-function theorem at the converged path (not in the
//                  paper; built on Eq. 15)
//
// Readings where the paper is silent (the CUDA path fixes the same ones in
// its own code):
//   parametrisations  plane O + s U_ax + t V_ax; paraboloid
//                  t0 + R (s, t, (s^2 + t^2)/(4f)); line P + t e; arc
//                  C + Rc (cos t u + sin t (a x u)); the normal of Eq. 2 and
//                  the tangent of Eq. 4 follow from them (signs irrelevant)
//   threshold      tau = 1e-20 on the dimensionless cost of Eq. 15
//   degenerate     a path with a segment shorter than 1e-5 S is rejected
//                  (S = scene scale); a parameter beyond 1e3 S diverged
//   initial guess  start 0: interaction k (from 0) takes the parameters of
//                  the projection of TX if 2k < n, of RX otherwise; starts
//                  j > 0 draw curved objects uniformly over their disc area
//                  or angle range (SplitMix64 of pair, packed ids, start)
//   multi-start    sequences with a paraboloid or an arc edge are solved from
//                  the enumeration's starts_curved starts; every distinct
//                  valid root is a path (Sec. III-B)
//   bounds         inclusive parameter ranges ([0,U]x[0,V], disc, [t0,t1],
//                  arc angle modulo 2 pi)
//   visibility     a rectangle blocks a segment whose ends are both more than
//                  1e-6 m off its plane on opposite sides with the crossing
//                  inside it; a paraboloid patch blocks when the segment
//                  meets it more than 1e-6 m from both ends inside its disc;
//                  edges never block; every occluder is tested
//   ambiguity      decisions within their tolerance bands (cost within a
//                  factor 100 of tau, a segment within a factor 3 of the
//                  minimum length, 1e-6 m of a bound or of an occluder's
//                  boundary) are flagged, not compared
// Completeness of multi-root solution sets is pinned by dense scans of
// the path length's stationary points: curved sequences of every object
// kind at orders 1 and 2, and at order 3 five three-object families in all
// six orders (every kind in every position); other order-3 combinations
// run the same per-interaction code and are compared by multi-start
// agreement only.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ------------------------------------------------------------------ duals --
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0) { std::memset(d, 0, sizeof(d)); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof(d)); }  // NOLINT
};
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r;
}
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r;
}
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
template <int N> Dual<N> dsqrt(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}
template <int N> Dual<N> dsin(const Dual<N>& a) {
  Dual<N> r; r.v = std::sin(a.v); double c = std::cos(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * c;
  return r;
}
template <int N> Dual<N> dcos(const Dual<N>& a) {
  Dual<N> r; r.v = std::cos(a.v); double sn = -std::sin(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * sn;
  return r;
}
inline double dsqrt(double a) { return std::sqrt(a); }
inline double dsin(double a) { return std::sin(a); }
inline double dcos(double a) { return std::cos(a); }
template <int N> double val(const Dual<N>& a) { return a.v; }
inline double val(double a) { return a; }

template <class T>
struct V3 {
  T x, y, z;
};
template <class T> V3<T> operator+(const V3<T>& a, const V3<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> V3<T> operator-(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> V3<T> scale(const V3<T>& a, const T& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> T norm(const V3<T>& a) { return dsqrt(dot(a, a)); }
template <class T> V3<T> unit(const V3<T>& a) { T n = norm(a); return {a.x / n, a.y / n, a.z / n}; }
template <class T> V3<T> lift(const double* p) { return {T(p[0]), T(p[1]), T(p[2])}; }

using V3d = V3<double>;
inline V3d ld(const double* p) { return {p[0], p[1], p[2]}; }

// ----------------------------------------------------------------- scene --
enum { PLANE = 0, PARABOLOID = 1, LINE_EDGE = 2, ARC_EDGE = 3 };
enum { OCC_RECT = 0, OCC_PARABOLOID = 1 };
constexpr int REC = 24;

}  // namespace

extern "C" {
// Mirrors the scene arrays produced by the Python scene generators.
struct OracleScene {
  int32_t n_obj;
  const int32_t* obj_kind;
  const double* obj_param;  // [n_obj][24]
  int32_t n_occ;
  const int32_t* occ_kind;
  const double* occ_param;  // [n_occ][24]
  double scale;             // S: scene scale (divergence guard, minimum segment)
  const double* tx;         // [n_tx][3]
  int32_t n_tx;
  const double* rx;         // [n_rx][3]
  int32_t n_rx;
  int32_t pair_mode;        // 0: p = t*n_rx + r ; 1: p -> (p, p)
};
}

namespace {

inline void pair_points(const OracleScene& s, int64_t p, const double** a, const double** b) {
  if (s.pair_mode == 0) {
    *a = s.tx + 3 * (p / s.n_rx);
    *b = s.rx + 3 * (p % s.n_rx);
  } else {
    *a = s.tx + 3 * p;
    *b = s.rx + 3 * p;
  }
}

inline bool is_curved(int kind) { return kind == PARABOLOID || kind == ARC_EDGE; }
inline bool is_edge(int kind) { return kind == LINE_EDGE || kind == ARC_EDGE; }
// parameters per object: surfaces (s, t), edges (t)  (Eqs. 13, 14)
inline int dof(int kind) { return is_edge(kind) ? 1 : 2; }

// Paraboloid frame: world = t + R * local, R row-major (columns = local axes).
template <class T>
V3<T> to_local(const double* R, const double* t, const V3<T>& X) {
  V3<T> w = X - lift<T>(t);
  return {T(R[0]) * w.x + T(R[3]) * w.y + T(R[6]) * w.z,
          T(R[1]) * w.x + T(R[4]) * w.y + T(R[7]) * w.z,
          T(R[2]) * w.x + T(R[5]) * w.y + T(R[8]) * w.z};
}
template <class T>
V3<T> to_world_dir(const double* R, const V3<T>& v) {
  return {T(R[0]) * v.x + T(R[1]) * v.y + T(R[2]) * v.z,
          T(R[3]) * v.x + T(R[4]) * v.y + T(R[5]) * v.z,
          T(R[6]) * v.x + T(R[7]) * v.y + T(R[8]) * v.z};
}

// Point of object `obj` at parameters u (Eqs. 13, 14):
//   plane       X = O + s U_ax + t V_ax
//   paraboloid  X = t0 + R (s, t, (s^2 + t^2) / (4 f))
//   line edge   X = P + t e
//   arc edge    X = C + Rc (cos t u_ref + sin t (a x u_ref))
template <class T>
V3<T> point_at(const OracleScene& s, int obj, const T* u, const T* d_shift) {
  const int kind = s.obj_kind[obj];
  const double* p = s.obj_param + (size_t)REC * obj;
  if (kind == PLANE) {
    V3<T> X = lift<T>(p + 4) + scale(lift<T>(p + 7), u[0]) + scale(lift<T>(p + 10), u[1]);
    if (d_shift) X = X + scale(lift<T>(p + 0), *d_shift);  // plane moved along its normal
    return X;
  }
  if (kind == PARABOLOID) {
    V3<T> l = {u[0], u[1], (u[0] * u[0] + u[1] * u[1]) / T(4.0 * p[12])};
    return lift<T>(p + 9) + to_world_dir<T>(p, l);
  }
  if (kind == LINE_EDGE) return lift<T>(p + 0) + scale(lift<T>(p + 3), u[0]);
  V3<T> a = lift<T>(p + 3), ur = lift<T>(p + 7);
  V3<T> vr = cross(a, ur);
  T Rc(p[6]);
  return lift<T>(p + 0) + scale(ur, Rc * dcos(u[0])) + scale(vr, Rc * dsin(u[0]));
}

// Law residual of interaction k: Eq. 8 divided by ||i|| (3 rows) or Eq. 9
// (1 row), appended to out.
template <class T>
int law_residual(const OracleScene& s, int obj, const T* u, const V3<T>& Xp, const V3<T>& X,
                 const V3<T>& Xn, T* out) {
  const int kind = s.obj_kind[obj];
  const double* p = s.obj_param + (size_t)REC * obj;
  V3<T> ih = unit(X - Xp);  // incident direction
  V3<T> rh = unit(Xn - X);  // departing direction
  if (kind == PLANE || kind == PARABOLOID) {
    V3<T> nh;
    if (kind == PLANE) {
      nh = lift<T>(p + 0);
    } else {
      // gradient of f = (x^2 + y^2)/(4f) - z in the local frame (Eq. 2)
      const double f = p[12];
      V3<T> gl = {u[0] / T(2.0 * f), u[1] / T(2.0 * f), T(-1.0)};
      nh = unit(to_world_dir<T>(p, gl));
    }
    T c = T(2.0) * dot(ih, nh);
    out[0] = rh.x - (ih.x - c * nh.x);
    out[1] = rh.y - (ih.y - c * nh.y);
    out[2] = rh.z - (ih.z - c * nh.z);
    return 3;
  }
  V3<T> eh;
  if (kind == LINE_EDGE) {
    eh = lift<T>(p + 3);
  } else {
    V3<T> a = lift<T>(p + 3), ur = lift<T>(p + 7);
    V3<T> vr = cross(a, ur);
    eh = scale(ur, -dsin(u[0])) + scale(vr, dcos(u[0]));  // r'(t)/||r'(t)|| (Eq. 4)
  }
  out[0] = dot(ih, eh) - dot(rh, eh);
  return 1;
}

constexpr int MAXN = 4;
constexpr int MAXQ = 2 * MAXN;  // parameters
constexpr int MAXM = 3 * MAXN;  // residual rows

// Stacked residual (Eq. 10) of the path whose parameters are T (Eq. 15).
template <class T>
int path_residual(const OracleScene& s, int n, const int32_t* ids, const V3<T>& A, const V3<T>& B,
                  const T* Tp, const T* d_shift, T* out, V3<T>* Xout) {
  V3<T> X[MAXN];
  int off = 0;
  for (int k = 0; k < n; ++k) {
    X[k] = point_at<T>(s, ids[k], Tp + off, d_shift ? d_shift + k : nullptr);
    off += dof(s.obj_kind[ids[k]]);
  }
  int m = 0;
  off = 0;
  for (int k = 0; k < n; ++k) {
    const V3<T>& Xp = (k == 0) ? A : X[k - 1];
    const V3<T>& Xn = (k == n - 1) ? B : X[k + 1];
    m += law_residual<T>(s, ids[k], Tp + off, Xp, X[k], Xn, out + m);
    off += dof(s.obj_kind[ids[k]]);
  }
  if (Xout)
    for (int k = 0; k < n; ++k) Xout[k] = X[k];
  return m;
}

int n_params(const OracleScene& s, int n, const int32_t* ids) {
  int q = 0;
  for (int k = 0; k < n; ++k) q += dof(s.obj_kind[ids[k]]);
  return q;
}

double cost_at(const OracleScene& s, int n, const int32_t* ids, const double* a, const double* b,
               const double* Tp) {
  double r[MAXM];
  int m = path_residual<double>(s, n, ids, ld(a), ld(b), Tp, nullptr, r, nullptr);
  double c = 0;
  for (int i = 0; i < m; ++i) c += r[i] * r[i];
  return c;
}

// residual rho (m) and Jacobian J (m x q, row-major) by forward-mode duals.
int residual_jacobian(const OracleScene& s, int n, const int32_t* ids, const double* a,
                      const double* b, const double* Tp, double* rho, double* J) {
  using D = Dual<MAXQ>;
  const int q = n_params(s, n, ids);
  D u[MAXQ];
  for (int j = 0; j < q; ++j) { u[j] = D(Tp[j]); u[j].d[j] = 1.0; }
  D r[MAXM];
  int m = path_residual<D>(s, n, ids, lift<D>(a), lift<D>(b), u, nullptr, r, nullptr);
  for (int i = 0; i < m; ++i) {
    rho[i] = r[i].v;
    for (int j = 0; j < q; ++j) J[i * q + j] = r[i].d[j];
  }
  return m;
}

// Dense solve M x = rhs (Gaussian elimination, partial pivoting).  false if singular.
bool dense_solve(int u, double* M, double* rhs) {
  for (int c = 0; c < u; ++c) {
    int piv = c;
    for (int r = c + 1; r < u; ++r)
      if (std::fabs(M[r * u + c]) > std::fabs(M[piv * u + c])) piv = r;
    if (!(std::fabs(M[piv * u + c]) > 1e-300)) return false;
    if (piv != c) {
      for (int j = 0; j < u; ++j) std::swap(M[c * u + j], M[piv * u + j]);
      std::swap(rhs[c], rhs[piv]);
    }
    for (int r = c + 1; r < u; ++r) {
      double f = M[r * u + c] / M[c * u + c];
      for (int j = c; j < u; ++j) M[r * u + j] -= f * M[c * u + j];
      rhs[r] -= f * rhs[c];
    }
  }
  for (int c = u - 1; c >= 0; --c) {
    double acc = rhs[c];
    for (int j = c + 1; j < u; ++j) acc -= M[c * u + j] * rhs[j];
    rhs[c] = acc / M[c * u + c];
  }
  return true;
}

// ------------------------------------------------------- initial guesses --
uint64_t splitmix64(uint64_t x) {
  // SplitMix64 output function (Steele, Lea, Flood 2014).
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Uniform draw in [0,1) for start `start`, interaction k, component comp of a
// candidate: three chained SplitMix64 rounds over (pair), (the four object ids
// packed as 16-bit fields, -1 -> 0xFFFF), (start*16 + k*2 + comp).
double unit_draw(uint64_t seed, int64_t pair, uint64_t packed_ids, int start, int k, int comp) {
  uint64_t h = splitmix64(seed ^ (uint64_t)pair);
  h = splitmix64(h ^ packed_ids);
  h = splitmix64(h ^ (uint64_t)(start * 16 + k * 2 + comp));
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

// Initial parameters of interaction k (Algorithm 1, random_guess).  Start 0:
// the parameters of the projection onto object k of TX (first half of the
// sequence, 2k < n with k counted from 0) or of RX (second half).  Start
// j > 0: curved objects are drawn uniformly (paraboloid: over the area of its
// disc; arc: over its angle range); planes and straight edges keep the
// projection.
void initial_params(const OracleScene& s, int obj, const V3d& Y, uint64_t seed, int64_t pair,
                    uint64_t packed_ids, int start, int k, double* u) {
  const int kind = s.obj_kind[obj];
  const double* p = s.obj_param + (size_t)REC * obj;
  if (kind == PLANE) {
    V3d w = Y - ld(p + 4);
    u[0] = dot(w, ld(p + 7));
    u[1] = dot(w, ld(p + 10));
  } else if (kind == LINE_EDGE) {
    u[0] = dot(Y - ld(p), ld(p + 3));
  } else if (kind == PARABOLOID) {
    if (start == 0) {
      V3d l = to_local<double>(p, p + 9, Y);
      u[0] = l.x;
      u[1] = l.y;
    } else {
      double r = p[13] * std::sqrt(unit_draw(seed, pair, packed_ids, start, k, 0));
      double th = 2.0 * M_PI * unit_draw(seed, pair, packed_ids, start, k, 1);
      u[0] = r * std::cos(th);
      u[1] = r * std::sin(th);
    }
  } else {
    if (start == 0) {
      V3d w = Y - ld(p);
      V3d a = ld(p + 3), ur = ld(p + 7);
      u[0] = std::atan2(dot(w, cross(a, ur)), dot(w, ur));
    } else {
      u[0] = p[10] + unit_draw(seed, pair, packed_ids, start, k, 0) * (p[11] - p[10]);
    }
  }
}

// ------------------------------------------------------------ minimiser --
enum { ST_CONVERGED = 0, ST_MAXITER = 1, ST_DIVERGED = 2, ST_STALLED = 3, ST_NONFINITE = 4 };

struct SolveOut {
  double T[MAXQ];
  double cost;
  int status;
  int iters;
};

// Gauss-Newton step from the normal equations at x: (J^T J + mu diag) dx = -J^T rho,
// mu = 1e-12 relative damping.  Returns the predicted decrease -g.dx.
bool gn_step(int q, int m, const double* J, const double* rho, double* dx, double* pred) {
  double A[MAXQ * MAXQ], g[MAXQ];
  for (int i = 0; i < q; ++i) {
    g[i] = 0;
    for (int r = 0; r < m; ++r) g[i] += J[r * q + i] * rho[r];
    for (int j = 0; j < q; ++j) {
      double acc = 0;
      for (int r = 0; r < m; ++r) acc += J[r * q + i] * J[r * q + j];
      A[i * q + j] = acc;
    }
  }
  for (int i = 0; i < q; ++i) {
    A[i * q + i] += 1e-12 * A[i * q + i] + 1e-300;
    dx[i] = -g[i];
  }
  if (!dense_solve(q, A, dx)) return false;
  double p = 0;
  for (int i = 0; i < q; ++i) p -= g[i] * dx[i];
  *pred = p;
  return true;
}

// find_minimum_path (Algorithm 1) read as Gauss-Newton with a backtracking
// line search on C = ||I(X(T))||^2 (Eq. 15):
//   - each trial point T + alpha dx costs one evaluation; a trial is accepted
//     when it lowers C, then a new step is solved with alpha = 1, otherwise
//     alpha is halved; alpha < 1/16 ends the search (stalled);
//   - converged when C < 1e-30 or an accepted step moved every parameter by
//     less than 1e-14 S; at most 24 accepted steps and 40 evaluations;
//   - diverged when a parameter exceeds 1e3 S;
//   - a local minimum with non-zero residual ends the search: after two
//     accepted steps, C > 1e-3 while the Gauss-Newton model predicts a
//     decrease below r C (the model's own minimum |rho + J dx|^2 = C - pred
//     stays above (1 - r) C), with r = 0.1 when every object of the
//     sequence is a plane or a straight edge and r = 1e-4 when a paraboloid
//     or an arc edge is among them (curved objects bend the cost away from
//     its linear model, and true paths can pass through such states).
// The stopping rules above, held in one place so that a test can run the
// oracle without its early exits (oracle_set_rules) and compare the valid
// sets: the defaults are the rules the reading fixes.
struct Rules {
  int max_iters = 24;
  int max_evals = 40;
  double min_alpha = 1.0 / 16.0;
  bool localmin_exit = true;
};
Rules g_rules;

SolveOut gn_solve(const OracleScene& s, int n, const int32_t* ids, const double* a, const double* b,
                  const double* T0) {
  const Rules rules = g_rules;
  SolveOut o;
  const int q = n_params(s, n, ids);
  bool curved = false;
  for (int k = 0; k < n; ++k)
    curved = curved || s.obj_kind[ids[k]] == PARABOLOID || s.obj_kind[ids[k]] == ARC_EDGE;
  const double lm_ratio = curved ? 1e-4 : 0.1;
  double x[MAXQ], rho[MAXM], J[MAXM * MAXQ], dx[MAXQ];
  std::memcpy(x, T0, sizeof(double) * q);
  int m = residual_jacobian(s, n, ids, a, b, x, rho, J);
  double C = 0;
  for (int i = 0; i < m; ++i) C += rho[i] * rho[i];
  int evals = 1;
  o.iters = 0;
  o.status = ST_MAXITER;
  double pred = 0;
  if (!std::isfinite(C)) {
    o.status = ST_NONFINITE;
  } else if (C < 1e-30) {
    o.status = ST_CONVERGED;
  } else if (!gn_step(q, m, J, rho, dx, &pred)) {
    o.status = ST_STALLED;
  } else {
    double alpha = 1.0;
    for (;;) {
      double xt[MAXQ];
      double smax = 0;
      for (int i = 0; i < q; ++i) {
        xt[i] = x[i] + alpha * dx[i];
        smax = std::max(smax, std::fabs(alpha * dx[i]));
      }
      const double Ct = cost_at(s, n, ids, a, b, xt);
      ++evals;
      if (std::isfinite(Ct) && Ct < C) {
        std::memcpy(x, xt, sizeof(double) * q);
        C = Ct;
        ++o.iters;
        double pmax = 0;
        for (int i = 0; i < q; ++i) pmax = std::max(pmax, std::fabs(x[i]));
        if (!(pmax <= 1e3 * s.scale)) { o.status = ST_DIVERGED; break; }
        if (C < 1e-30 || smax < 1e-14 * s.scale) { o.status = ST_CONVERGED; break; }
        if (o.iters >= rules.max_iters) { o.status = ST_MAXITER; break; }
        if (evals >= rules.max_evals) { o.status = ST_MAXITER; break; }
        m = residual_jacobian(s, n, ids, a, b, x, rho, J);
        if (!gn_step(q, m, J, rho, dx, &pred)) { o.status = ST_STALLED; break; }
        alpha = 1.0;
        if (rules.localmin_exit && o.iters >= 2 && C > 1e-3 && pred < lm_ratio * C) { o.status = ST_STALLED; break; }
      } else {
        alpha *= 0.5;
        if (alpha < rules.min_alpha) { o.status = ST_STALLED; break; }
        if (evals >= rules.max_evals) { o.status = ST_MAXITER; break; }
      }
    }
  }
  std::memcpy(o.T, x, sizeof(double) * q);
  o.cost = C;
  return o;
}

// ------------------------------------------------------------ validation --
constexpr double EPS_VIS = 1e-6;   // a crossing needs both endpoints > 1e-6 m off the surface
constexpr double MIN_SEG_REL = 1e-5;  // shortest accepted segment, relative to the scene scale S
constexpr double BAND = 1e-6;      // ambiguity band half-width for geometric decisions

struct Verdict {
  bool ok;
  bool ambiguous;
};

// Interaction point inside the bounds of its object (inclusive), decided on
// its parameters: rectangle [0,U]x[0,V]; disc s^2+t^2 <= rho^2; segment
// [t0,t1]; arc angle within [phi0, phi1] modulo 2 pi.
Verdict in_bounds(const OracleScene& s, int obj, const double* u) {
  const int kind = s.obj_kind[obj];
  const double* p = s.obj_param + (size_t)REC * obj;
  Verdict v{true, false};
  if (kind == PLANE) {
    double uu = u[0], vv = u[1], U = p[13], V = p[14];
    v.ok = uu >= 0 && uu <= U && vv >= 0 && vv <= V;
    bool in_grown = uu >= -BAND && uu <= U + BAND && vv >= -BAND && vv <= V + BAND;
    bool in_shrunk = uu >= BAND && uu <= U - BAND && vv >= BAND && vv <= V - BAND;
    v.ambiguous = in_grown && !in_shrunk;
  } else if (kind == PARABOLOID) {
    double r = std::sqrt(u[0] * u[0] + u[1] * u[1]);
    v.ok = r <= p[13];
    v.ambiguous = std::fabs(r - p[13]) < BAND;
  } else if (kind == LINE_EDGE) {
    double t = u[0];
    v.ok = t >= p[6] && t <= p[7];
    v.ambiguous = std::fabs(t - p[6]) < BAND || std::fabs(t - p[7]) < BAND;
  } else {
    double phi0 = p[10], phi1 = p[11], Rc = p[6];
    double phi = phi0 + std::fmod(u[0] - phi0, 2.0 * M_PI);
    if (phi < phi0) phi += 2.0 * M_PI;
    v.ok = phi <= phi1;
    v.ambiguous = std::fabs(phi - phi0) * Rc < BAND || std::fabs(phi - phi1) * Rc < BAND ||
                  std::fabs(phi - phi0 - 2.0 * M_PI) * Rc < BAND;
  }
  return v;
}

// Does segment [A,B] cross occluder `o`?  Rules: a rectangle blocks when A
// and B lie strictly on opposite sides (both farther than EPS_VIS from the
// plane) and the crossing point is inside the rectangle (inclusive).  A
// paraboloid patch blocks when the segment meets the surface at a parameter
// whose point is farther than EPS_VIS (along the segment) from both ends and
// inside the disc (inclusive).  Edges never occlude.
Verdict blocks(const OracleScene& s, int o, const V3d& A, const V3d& B) {
  const int kind = s.occ_kind[o];
  const double* p = s.occ_param + (size_t)REC * o;
  Verdict v{false, false};
  if (kind == OCC_RECT) {
    V3d O = ld(p), u = ld(p + 3), w = ld(p + 6), n = ld(p + 11);
    double U = p[9], V = p[10];
    double sA = dot(A - O, n), sB = dot(B - O, n);
    if (!((sA < 0 && sB > 0) || (sA > 0 && sB < 0))) return v;
    double t = sA / (sA - sB);
    V3d P = A + scale(B - A, t);
    double uu = dot(P - O, u), vv = dot(P - O, w);
    bool inside = uu >= 0 && uu <= U && vv >= 0 && vv <= V;
    bool strict = std::fabs(sA) > EPS_VIS && std::fabs(sB) > EPS_VIS;
    v.ok = strict && inside;
    bool in_grown = uu >= -BAND && uu <= U + BAND && vv >= -BAND && vv <= V + BAND;
    bool in_shrunk = uu >= BAND && uu <= U - BAND && vv >= BAND && vv <= V - BAND;
    double smin = std::min(std::fabs(sA), std::fabs(sB));
    bool near_eps = smin > 0.1 * EPS_VIS && smin < 10.0 * EPS_VIS;
    v.ambiguous = (strict && in_grown && !in_shrunk) || (near_eps && in_grown);
    return v;
  }
  // paraboloid patch: local quadratic  al t^2 + be t + ga = 0
  const double* R = p;
  const double* tt = p + 9;
  const double f = p[12], rho = p[13];
  V3d a = to_local<double>(R, tt, A), bl = to_local<double>(R, tt, B);
  V3d d = bl - a;
  double L = norm(B - A);
  double al = (d.x * d.x + d.y * d.y) / (4.0 * f);
  double be = (2.0 * a.x * d.x + 2.0 * a.y * d.y) / (4.0 * f) - d.z;
  double ga = (a.x * a.x + a.y * a.y) / (4.0 * f) - a.z;
  double roots[2];
  int nr = 0;
  if (std::fabs(al) < 1e-300) {
    if (std::fabs(be) > 0) roots[nr++] = -ga / be;
  } else {
    double disc = be * be - 4.0 * al * ga;
    if (disc >= 0) {
      double q = -0.5 * (be + (be >= 0 ? 1.0 : -1.0) * std::sqrt(disc));
      roots[nr++] = q / al;
      if (q != 0) roots[nr++] = ga / q;
    }
  }
  for (int i = 0; i < nr; ++i) {
    double t = roots[i];
    V3d P = a + scale(d, t);
    double r = std::sqrt(P.x * P.x + P.y * P.y);
    double dA = t * L, dB = (1.0 - t) * L;
    bool interior = dA > EPS_VIS && dB > EPS_VIS;
    bool inside = r <= rho;
    if (interior && inside) v.ok = true;
    bool near_end = (std::fabs(dA) > 0.1 * EPS_VIS && std::fabs(dA) < 10 * EPS_VIS) ||
                    (std::fabs(dB) > 0.1 * EPS_VIS && std::fabs(dB) < 10 * EPS_VIS);
    if ((near_end && r <= rho + BAND) || (interior && std::fabs(r - rho) < BAND)) v.ambiguous = true;
  }
  return v;
}

template <class F>
void parallel_for(int64_t n, int n_threads, F&& f) {
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n_threads == 1 || n < 64) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next{0};
  const int64_t chunk = 64;
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int64_t i0 = next.fetch_add(chunk);
        if (i0 >= n) break;
        int64_t i1 = std::min(n, i0 + chunk);
        for (int64_t i = i0; i < i1; ++i) f(i);
      }
    });
  for (auto& t : th) t.join();
}

}  // namespace

extern "C" {

int oracle_abi_version() { return 2; }

int oracle_threads(int n_threads) {
  return n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
}

uint64_t oracle_splitmix64(uint64_t x) { return splitmix64(x); }

// Stopping rules of the minimiser (test hook; call before a solve, not
// during one).  Defaults: 24 accepted steps, 40 evaluations, line search
// down to alpha = 1/16, local-minimum exit on.
void oracle_set_rules(int32_t max_iters, int32_t max_evals, double min_alpha, int32_t localmin_exit) {
  g_rules.max_iters = max_iters;
  g_rules.max_evals = max_evals;
  g_rules.min_alpha = min_alpha;
  g_rules.localmin_exit = localmin_exit != 0;
}

// Candidate sequences (Algorithm 1, all_simple_paths; Sec. III).
// Orders n = 1..max_order in turn.  quota[n-1] = -1: every ordered sequence of
// n distinct objects in lexicographic order of the ids, kept only if every
// consecutive pair (a, b) has adj[a*n_obj + b] != 0 when adj is given;
// quota = q > 0: q sequences, slot sl = 0..q-1, whose draw k is
// SplitMix64(seed ^ (n << 56 | sl << 16 | k)); positions left to right take
// the (draw mod r)-th of the r objects not taken yet (in id order); every
// force_edges_every-th slot of order >= 3 first puts two consecutive edges
// (the (draw mod r)-th untaken edge, draws 0 and 1) at position
// draw_100 mod (n - 1).  Each sequence that contains a paraboloid or an arc is emitted
// `starts_curved` times (start index 0..starts_curved-1), others once.
// Returns the number of entries; writes at most `cap` of them.
int64_t oracle_enumerate(int32_t n_obj, const int32_t* obj_kind, int32_t max_order,
                         const int64_t* quota, uint64_t seed, int32_t starts_curved,
                         int32_t force_edges_every, const uint8_t* adj, int32_t* out_order,
                         int32_t* out_ids, int32_t* out_start, int64_t cap) {
  int64_t count = 0;
  std::vector<int32_t> edges;
  for (int i = 0; i < n_obj; ++i)
    if (is_edge(obj_kind[i])) edges.push_back(i);
  auto emit = [&](int n, const int32_t* ids) {
    bool curved = false;
    for (int k = 0; k < n; ++k) curved = curved || is_curved(obj_kind[ids[k]]);
    int ns = curved ? std::max(1, starts_curved) : 1;
    for (int st = 0; st < ns; ++st) {
      if (count < cap) {
        out_order[count] = n;
        for (int k = 0; k < 4; ++k) out_ids[4 * count + k] = k < n ? ids[k] : -1;
        out_start[count] = st;
      }
      ++count;
    }
  };
  for (int n = 1; n <= max_order && n <= 4; ++n) {
    int64_t q = quota[n - 1];
    if (q == 0 || n > n_obj) continue;
    if (q < 0) {
      // odometer over n-tuples, skipping tuples with repeated ids
      int32_t ids[4] = {0, 0, 0, 0};
      for (;;) {
        bool distinct = true;
        for (int i = 0; i < n && distinct; ++i)
          for (int j = i + 1; j < n; ++j)
            if (ids[i] == ids[j]) { distinct = false; break; }
        bool adjacent = true;
        if (distinct && adj)
          for (int k = 0; k + 1 < n; ++k)
            if (!adj[(size_t)ids[k] * n_obj + ids[k + 1]]) { adjacent = false; break; }
        if (distinct && adjacent) emit(n, ids);
        int pos = n - 1;
        while (pos >= 0) {
          if (++ids[pos] < n_obj) break;
          ids[pos] = 0;
          --pos;
        }
        if (pos < 0) break;
      }
      continue;
    }
    for (int64_t sl = 0; sl < q; ++sl) {
      auto draw = [&](int k) {
        uint64_t key = ((uint64_t)n << 56) | ((uint64_t)sl << 16) | (uint64_t)k;
        return splitmix64(seed ^ key);
      };
      int32_t ids[4] = {-1, -1, -1, -1};
      std::vector<char> taken(n_obj, 0);
      int k = 0;
      bool forced = n >= 3 && force_edges_every > 0 && (sl % force_edges_every) == 0 &&
                    edges.size() >= 2;
      if (forced) {
        int pfix = (int)(draw(100) % (uint64_t)(n - 1));
        for (int j = 0; j < 2; ++j) {
          int avail = (int)edges.size() - j;
          int idx = (int)(draw(k) % (uint64_t)avail);
          ++k;
          for (int e : edges) {
            if (taken[e]) continue;
            if (idx-- == 0) { ids[pfix + j] = e; taken[e] = 1; break; }
          }
        }
      }
      for (int pos = 0; pos < n; ++pos) {
        if (ids[pos] >= 0) continue;
        int avail = n_obj - k;
        int idx = (int)(draw(k) % (uint64_t)avail);
        ++k;
        for (int o = 0; o < n_obj; ++o) {
          if (taken[o]) continue;
          if (idx-- == 0) { ids[pos] = o; taken[o] = 1; break; }
        }
      }
      emit(n, ids);
    }
  }
  return count;
}

// Solve candidates [cand_begin, cand_end): entry e = c / n_pairs, pair
// p = c % n_pairs.  Outputs (indexed from cand_begin): X [.][12] interaction
// points (unused slots 0), T [.][8] parameters, cost (Eq. 15), status,
// iterations.
int oracle_solve(const OracleScene* sc, int64_t n_entries, const int32_t* ent_order,
                 const int32_t* ent_ids, const int32_t* ent_start, int64_t n_pairs,
                 int64_t cand_begin, int64_t cand_end, uint64_t init_seed, double* out_X,
                 double* out_T, double* out_cost, int32_t* out_status, int32_t* out_iters,
                 int n_threads) {
  const OracleScene& s = *sc;
  if (cand_end > n_entries * n_pairs) cand_end = n_entries * n_pairs;
  parallel_for(cand_end - cand_begin, n_threads, [&](int64_t i) {
    int64_t c = cand_begin + i;
    int64_t e = c / n_pairs, p = c % n_pairs;
    int n = ent_order[e];
    const int32_t* ids = ent_ids + 4 * e;
    const double *a, *b;
    pair_points(s, p, &a, &b);
    double T0[MAXQ];
    V3d A = ld(a), B = ld(b);
    uint64_t packed = 0;
    for (int k = 0; k < 4; ++k) packed |= (uint64_t)(uint16_t)(k < n ? ids[k] : -1) << (16 * k);
    int off = 0;
    for (int k = 0; k < n; ++k) {
      V3d Y = (2 * k < n) ? A : B;
      initial_params(s, ids[k], Y, init_seed, p, packed, ent_start[e], k, T0 + off);
      off += dof(s.obj_kind[ids[k]]);
    }
    SolveOut o = gn_solve(s, n, ids, a, b, T0);
    double r[MAXM];
    V3d X[MAXN];
    path_residual<double>(s, n, ids, A, B, o.T, nullptr, r, X);
    double* xo = out_X + 12 * i;
    for (int j = 0; j < 12; ++j) xo[j] = 0.0;
    for (int k = 0; k < n; ++k) { xo[3 * k] = X[k].x; xo[3 * k + 1] = X[k].y; xo[3 * k + 2] = X[k].z; }
    double* to = out_T + 8 * i;
    const int q = n_params(s, n, ids);
    for (int j = 0; j < 8; ++j) to[j] = j < q ? o.T[j] : 0.0;
    out_cost[i] = o.cost;
    out_status[i] = o.status;
    out_iters[i] = o.iters;
  });
  return 0;
}

// Acceptance (Algorithm 1: C < tau and X valid).  Valid needs C < tau, every
// segment at least 1e-5 S long, every point inside its object's bounds and no
// segment blocked.  ambiguous = 1 when a decision fell inside its tolerance
// band (cost in [tau/100, 100 tau], a segment within a factor 3 of the
// minimum length, a point within 1e-6 m of a bound, a crossing within the
// visibility band).  Also returns the path length.
int oracle_validate(const OracleScene* sc, int64_t n_entries, const int32_t* ent_order,
                    const int32_t* ent_ids, int64_t n_pairs, int64_t cand_begin, int64_t cand_end,
                    const double* X, const double* Tp, const double* cost, double tau,
                    int32_t* out_valid, int32_t* out_ambiguous, double* out_length, int n_threads) {
  const OracleScene& s = *sc;
  (void)n_entries;
  parallel_for(cand_end - cand_begin, n_threads, [&](int64_t i) {
    int64_t c = cand_begin + i;
    int64_t e = c / n_pairs, p = c % n_pairs;
    int n = ent_order[e];
    const int32_t* ids = ent_ids + 4 * e;
    const double *a, *b;
    pair_points(s, p, &a, &b);
    const double* x = X + 12 * i;
    const double* t = Tp + 8 * i;
    bool ok = cost[i] < tau;
    bool amb = cost[i] >= 1e-2 * tau && cost[i] <= 1e2 * tau;
    V3d P[MAXN + 2];
    P[0] = ld(a);
    for (int k = 0; k < n; ++k) P[k + 1] = ld(x + 3 * k);
    P[n + 1] = ld(b);
    double len = 0;
    const double lmin = MIN_SEG_REL * s.scale;
    for (int k = 0; k <= n; ++k) {
      double l = norm(P[k + 1] - P[k]);
      len += l;
      // consecutive points that collapse where two objects touch are not paths
      if (!(l >= lmin)) ok = false;
      if (l >= lmin / 3.0 && l <= 3.0 * lmin && cost[i] < 1e2 * tau) amb = true;
    }
    out_length[i] = len;
    bool finite = true;
    for (int j = 0; j < 3 * n; ++j) finite = finite && std::isfinite(x[j]);
    if (!finite) ok = false;
    if (finite && cost[i] < 1e2 * tau) {
      int off = 0;
      for (int k = 0; k < n; ++k) {
        Verdict v = in_bounds(s, ids[k], t + off);
        off += dof(s.obj_kind[ids[k]]);
        ok = ok && v.ok;
        amb = amb || v.ambiguous;
      }
      for (int k = 0; k <= n; ++k)
        for (int o = 0; o < s.n_occ; ++o) {
          Verdict v = blocks(s, o, P[k], P[k + 1]);
          ok = ok && !v.ok;
          amb = amb || v.ambiguous;
        }
    }
    out_valid[i] = ok ? 1 : 0;
    out_ambiguous[i] = amb ? 1 : 0;
  });
  return 0;
}

// Gradient of the path length L = sum ||X_{k+1} - X_k|| at a converged path,
// through the implicit-function theorem on rho(T, theta) = 0:
//   dT/dtheta = -(J^T J)^{-1} J^T d rho/d theta,
//   dL/dtheta = dL/dtheta|_explicit + dL/dT dT/dtheta,
//   dX/dtheta = dX/dtheta|_explicit + dX/dT dT/dtheta.
// theta = (TX[3], RX[3], d_1..d_n), d_k the offset of the plane of
// interaction k along its normal (zero column for non-planar interactions).
// Outputs: dL [6 + n], dX [3n][6 + n] row-major.
int oracle_path_grad(const OracleScene* sc, int32_t n, const int32_t* ids, const double* a,
                     const double* b, const double* Tp, double* dL, double* dX) {
  const OracleScene& s = *sc;
  constexpr int NV = MAXQ + 6 + MAXN;
  using D = Dual<NV>;
  const int q = n_params(s, n, ids), nt = 6 + n;
  D u[MAXQ];
  for (int j = 0; j < q; ++j) { u[j] = D(Tp[j]); u[j].d[j] = 1.0; }
  D A[3], B[3], dd[MAXN];
  for (int j = 0; j < 3; ++j) {
    A[j] = D(a[j]); A[j].d[q + j] = 1.0;
    B[j] = D(b[j]); B[j].d[q + 3 + j] = 1.0;
  }
  for (int k = 0; k < n; ++k) {
    dd[k] = D(0.0);
    if (s.obj_kind[ids[k]] == PLANE) dd[k].d[q + 6 + k] = 1.0;
  }
  V3<D> Av = {A[0], A[1], A[2]}, Bv = {B[0], B[1], B[2]};
  D r[MAXM];
  V3<D> X[MAXN];
  int m = path_residual<D>(s, n, ids, Av, Bv, u, dd, r, X);
  double N[MAXQ * MAXQ], dT[MAXQ * NV];
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double acc = 0;
      for (int rr = 0; rr < m; ++rr) acc += r[rr].d[i] * r[rr].d[j];
      N[i * q + j] = acc;
    }
  for (int col = 0; col < nt; ++col) {
    double M[MAXQ * MAXQ], rhs[MAXQ];
    std::memcpy(M, N, sizeof(double) * q * q);
    for (int i = 0; i < q; ++i) {
      double acc = 0;
      for (int rr = 0; rr < m; ++rr) acc += r[rr].d[i] * r[rr].d[q + col];
      rhs[i] = -acc;
    }
    if (!dense_solve(q, M, rhs)) return 1;
    for (int i = 0; i < q; ++i) dT[i * NV + col] = rhs[i];
  }
  V3<D> P[MAXN + 2];
  P[0] = Av;
  for (int k = 0; k < n; ++k) P[k + 1] = X[k];
  P[n + 1] = Bv;
  D L(0.0);
  for (int k = 0; k <= n; ++k) L = L + norm(P[k + 1] - P[k]);
  for (int col = 0; col < nt; ++col) {
    double g = L.d[q + col];
    for (int i = 0; i < q; ++i) g += L.d[i] * dT[i * NV + col];
    dL[col] = g;
  }
  for (int k = 0; k < n; ++k) {
    const D* c3[3] = {&X[k].x, &X[k].y, &X[k].z};
    for (int j = 0; j < 3; ++j)
      for (int col = 0; col < nt; ++col) {
        double g = c3[j]->d[q + col];
        for (int i = 0; i < q; ++i) g += c3[j]->d[i] * dT[i * NV + col];
        dX[(3 * k + j) * nt + col] = g;
      }
  }
  return 0;
}

// oracle_path_grad over many paths (threads over paths): path i is candidate
// cand[i] (entry cand / n_pairs, pair cand % n_pairs) with packed parameters
// T[i][8]; it writes the upstream-weighted gradient
//   w[i][j] = g_len[i] dL/dtheta_j + sum_r g_pts[i][r] dX_r/dtheta_j
// for theta = (TX[3], RX[3], d_1..d_n), j < 6 + n (the rest of the row 0).
// g_pts may be null.  Returns the number of paths whose normal matrix was
// singular (their row is left 0).
int oracle_path_grad_many(const OracleScene* sc, int64_t n_paths, const int32_t* ent_order,
                          const int32_t* ent_ids, int64_t n_pairs, const int64_t* cand, const double* Tp,
                          const double* g_len, const double* g_pts, double* w, int n_threads) {
  std::atomic<int> bad{0};
  parallel_for(n_paths, n_threads, [&](int64_t i) {
    const int64_t e = cand[i] / n_pairs, p = cand[i] % n_pairs;
    const int n = ent_order[e];
    const int32_t* ids = ent_ids + 4 * e;
    const double *a, *b;
    pair_points(*sc, p, &a, &b);
    double dL[6 + MAXN], dX[3 * MAXN * (6 + MAXN)];
    double* wi = w + (6 + MAXN) * i;
    for (int j = 0; j < 6 + MAXN; ++j) wi[j] = 0.0;
    if (oracle_path_grad(sc, n, ids, a, b, Tp + 8 * i, dL, dX) != 0) {
      ++bad;
      return;
    }
    const int nt = 6 + n;
    for (int j = 0; j < nt; ++j) {
      double acc = g_len[i] * dL[j];
      if (g_pts)
        for (int r = 0; r < 3 * n; ++r) acc += g_pts[12 * i + r] * dX[r * nt + j];
      wi[j] = acc;
    }
  });
  return bad.load();
}

// Residual and points of one path at parameters T (for tests of the oracle).
int oracle_residual(const OracleScene* sc, int32_t n, const int32_t* ids, const double* a,
                    const double* b, const double* Tp, double* rho, double* X) {
  V3d Xv[MAXN];
  int m = path_residual<double>(*sc, n, ids, ld(a), ld(b), Tp, nullptr, rho, Xv);
  for (int k = 0; k < n; ++k) { X[3 * k] = Xv[k].x; X[3 * k + 1] = Xv[k].y; X[3 * k + 2] = Xv[k].z; }
  return m;
}

// Visibility of one segment (for tests): returns 1 if blocked, sets *ambiguous.
int oracle_segment_blocked(const OracleScene* sc, const double* A, const double* B,
                           int32_t* ambiguous) {
  int blocked = 0, amb = 0;
  for (int o = 0; o < sc->n_occ; ++o) {
    Verdict v = blocks(*sc, o, ld(A), ld(B));
    blocked |= v.ok;
    amb |= v.ambiguous;
  }
  *ambiguous = amb;
  return blocked;
}

int oracle_params_in_bounds(const OracleScene* sc, int32_t obj, const double* u, int32_t* ambiguous) {
  Verdict v = in_bounds(*sc, obj, u);
  *ambiguous = v.ambiguous;
  return v.ok ? 1 : 0;
}

}  // extern "C"
