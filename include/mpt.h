/* Min-Path-Tracing (MPT) on one GPU: C ABI.
 *
 * The calls follow the problem statement of Algorithm 1 of the paper
 * (Eertmans, Oestges, Jacques, "Min-Path-Tracing: A Diffraction Aware
 * Alternative to Image Method in Ray Tracing", arXiv 2301.06399): inputs are
 * the maximum number of interactions n_t, the objects database D and the
 * BS / UE positions; the output is the set S of valid paths.
 *
 *   mpt_scene_upload  objects database D (Sec. II: implicit surfaces and
 *                     edges with their bounds; occluders)
 *   mpt_enumerate     path candidates (Algorithm 1, all_simple_paths; Sec. III)
 *   mpt_solve         find_minimum_path for every candidate (Algorithm 1;
 *                     Eqs. 8, 9, 13-15)
 *   mpt_validate      "C < threshold and X is valid" (Algorithm 1) and the
 *                     union into S, as a compacted list
 *   mpt_grad          gradients of path length / points at converged paths
 *                     (implicit-function theorem on Eq. 15; not in the paper)
 *
 * Conventions
 *   - Every call returns an int status (MPT_OK = 0); no exception crosses the
 *     ABI.  mpt_status_string() names a status.
 *   - Device buffers are allocated and owned by the caller; the library never
 *     frees them.  Opaque handles (mpt_ctx, mpt_scene) are owned by the
 *     library and released with their destroy/free call.
 *   - Work is enqueued asynchronously on the caller's CUDA stream (passed as
 *     void*, a cudaStream_t; NULL = legacy default stream).  Counts are written
 *     to device memory; no call synchronises the stream unless it says so.
 *   - Arguments are checked on the host before anything is enqueued; a bad
 *     argument returns MPT_ERR_ARG and enqueues nothing.  A CUDA launch or
 *     allocation failure returns MPT_ERR_CUDA.
 *   - One mpt_ctx per device and thread of control: calls that share a ctx
 *     must be issued from one host thread at a time, and in order on one
 *     stream (or on streams the caller orders with events).  The context's
 *     scratch (work-stealing counters, refine lists, validation scratch) is
 *     reused by every call and regrown stream-ordered on the calling stream,
 *     so two calls of one ctx that overlap on the GPU race on it.  Use one
 *     ctx per concurrent stream.
 */
#ifndef MPT_H_
#define MPT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MPT_OK = 0,
  MPT_ERR_ARG = 1,         /* invalid argument (null pointer, size, kind) */
  MPT_ERR_CUDA = 2,        /* CUDA runtime error (launch, allocation, copy) */
  MPT_ERR_CAPACITY = 3,    /* an output buffer is too small (see each call) */
  MPT_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
  MPT_ERR_UNSUPPORTED = 5  /* valid request this build does not support */
};

/* Object kinds (Sec. II).  Parameter records are double[24]:
 *   MPT_PLANE       [0:3] unit normal n, [3] d with <n,X> = d, [4:7] corner O,
 *                   [7:10] unit axis U_ax, [10:13] unit axis V_ax (n = U_ax x V_ax),
 *                   [13] U, [14] V: the facet is O + s U_ax + t V_ax, s in [0,U],
 *                   t in [0,V]
 *   MPT_PARABOLOID  [0:9] rotation R (row-major, columns = local axes in world),
 *                   [9:12] apex t0, [12] focal length f, [13] disc radius rho:
 *                   X = t0 + R (s, t, (s^2+t^2)/(4f)), s^2 + t^2 <= rho^2
 *   MPT_LINE_EDGE   [0:3] point P, [3:6] unit direction e, [6] t0, [7] t1:
 *                   X = P + t e, t in [t0, t1]
 *   MPT_ARC_EDGE    [0:3] centre C, [3:6] unit axis a, [6] radius Rc,
 *                   [7:10] unit reference u (orthogonal to a), [10] phi0,
 *                   [11] phi1: X = C + Rc (cos t u + sin t (a x u)),
 *                   t in [phi0, phi1] modulo 2 pi
 * Occluder kinds (surfaces a segment may not cross; edges never occlude):
 *   MPT_OCC_RECT       [0:3] O, [3:6] U_ax, [6:9] V_ax, [9] U, [10] V, [11:14] n
 *   MPT_OCC_PARABOLOID same record as MPT_PARABOLOID
 */
enum { MPT_PLANE = 0, MPT_PARABOLOID = 1, MPT_LINE_EDGE = 2, MPT_ARC_EDGE = 3 };
enum { MPT_OCC_RECT = 0, MPT_OCC_PARABOLOID = 1 };
#define MPT_RECORD 24
#define MPT_MAX_ORDER 4
#define MPT_MAX_OBJECTS 65535
#define MPT_MAX_OCCLUDERS 1024

/* Solver precision modes. */
enum {
  MPT_FP64_PLAIN = 0,       /* FP64 throughout (the plain GPU method) */
  MPT_FP32 = 1,             /* FP32 iterations only, no refinement */
  MPT_FP32_FP64REFINE = 2   /* FP32 iterations, then refinement of candidates
                               that pass the FP32 cost/bounds/visibility
                               prescreen in float-float arithmetic (pairs of
                               FP32, 48-bit significand; not FP64 arithmetic),
                               results stored as FP64; acceptance decisions
                               near their margins in FP64 */
};

/* Per-candidate termination status (low 4 bits) and flags. */
enum {
  MPT_PATH_CONVERGED = 0,   /* step or cost below tolerance */
  MPT_PATH_MAXITER = 1,     /* iteration cap reached */
  MPT_PATH_DIVERGED = 2,    /* a point left the cube of half-side 1e3 S */
  MPT_PATH_STALLED = 3,     /* line search could not decrease the cost */
  MPT_PATH_NONFINITE = 4,   /* NaN / Inf in the cost */
  MPT_PATH_EXCLUDED = 5,    /* no path by the half-space or beam condition of
                               Eq. 8 (see mpt_solve): not iterated, cost +inf,
                               parameters untouched, iters = evals = 0 */
  MPT_PATH_REFINED = 0x10,  /* flag: final stage ran (FP64 solve or refinement) */
  MPT_PATH_PRESCREENED = 0x20, /* flag: FP32 prescreen rejected (no refinement) */
  MPT_PATH_FALLBACK = 0x40  /* flag: refinement needed full Gauss-Newton in
                               float-float (ill-conditioned path) */
};

typedef struct mpt_ctx mpt_ctx;
typedef struct mpt_scene mpt_scene;

/* Host description of a scene (copied by mpt_scene_upload; the caller keeps
 * ownership of these arrays). */
typedef struct {
  int32_t n_obj;
  const int32_t* obj_kind;   /* host [n_obj] */
  const double* obj_param;   /* host [n_obj][MPT_RECORD] */
  int32_t n_occ;
  const int32_t* occ_kind;   /* host [n_occ] */
  const double* occ_param;   /* host [n_occ][MPT_RECORD] */
  double scale;              /* scene scale S in metres (> 0) */
} mpt_scene_desc;

/* TX / RX endpoints (device, caller-owned, read by solve/validate/grad). */
typedef struct {
  const double* tx;   /* device [n_tx][3] */
  int32_t n_tx;
  const double* rx;   /* device [n_rx][3] */
  int32_t n_rx;
  int32_t pair_mode;  /* 0: pair p = t * n_rx + r (all combinations);
                         1: pair p uses tx[p] and rx[p] (n_tx == n_rx) */
} mpt_endpoints;

/* Which sequences to enumerate.  quota[n-1] for order n: -1 = every ordered
 * sequence of n distinct objects (lexicographic order of the ids), 0 = none,
 * q > 0 = q sequences drawn with SplitMix64 (Steele, Lea, Flood 2014) from
 * `seed`, slot sl = 0..q-1 in turn.  Draw k of slot sl of order n is
 * h_k = SplitMix64(seed ^ (n << 56 | sl << 16 | k)), k counting from 0 over
 * the slot's draws.  Positions are filled left to right; each takes the
 * (h_k mod r)-th object, in id order, among the r objects not taken yet in
 * this slot.  For orders >= 3, when force_edges_every > 0, sl is a multiple of
 * it and the scene has at least two edges, the slot first places two
 * consecutive edges at position h_100 mod (n - 1): each is the (h_k mod r)-th
 * edge, in id order, of the r edges not taken yet (k = 0, 1); the remaining
 * positions then continue the draws from k = 2.  Sequences containing a
 * paraboloid or an arc are repeated `starts_curved` times with start index
 * 0..starts_curved-1.  starts_curved <= 0 means 1; the start index is held
 * in 8 bits of the candidate record, so starts_curved > 255 makes
 * mpt_enumerate return MPT_ERR_ARG and mpt_candidate_count return -1. */
typedef struct {
  int64_t quota[MPT_MAX_ORDER];
  uint64_t seed;
  int32_t starts_curved;
  int32_t force_edges_every;
} mpt_sampling;

/* Candidate list (caller-owned device buffers).  Entry e of the sequence
 * table and pair p give candidate c = e * n_pairs + p (pairs fastest, so a
 * warp shares one object sequence).  rec[c] is 16 bytes:
 *   rec[c].x = pair index p
 *   rec[c].y = id0 | id1 << 16   (0xFFFF = unused slot)
 *   rec[c].z = id2 | id3 << 16
 *   rec[c].w = order | start << 8
 * order_begin (device int64[5]) = [first candidate of order 1, of order 2,
 * of order 3, of order 4, end]; the number of candidates is order_begin[4]
 * (also written to *count). */
typedef struct {
  uint32_t* rec;         /* device [capacity][4] */
  int64_t capacity;      /* entries rec can hold */
  int64_t* count;        /* device int64[1]: number of candidates */
  int64_t* order_begin;  /* device int64[5] */
  uint64_t init_seed;    /* seed of the initial guesses of starts > 0 */
} mpt_candidates;

/* Per-candidate solver output (caller-owned device SoA, capacity >= count). */
typedef struct {
  double* T;         /* device [8][capacity]: parameters, slot j of candidate c at T[j*capacity + c] */
  double* cost;      /* device [capacity]: cost of Eq. 15 (FP64 after refinement) */
  uint8_t* status;   /* device [capacity]: MPT_PATH_* */
  uint8_t* iters;    /* device [capacity]: minimiser iterations executed */
  uint8_t* evals;    /* device [capacity]: residual evaluations executed */
  float* T32;        /* device [8][capacity] or NULL: parameters before refinement */
  int64_t capacity;
} mpt_solutions;

/* Solver schedule; NULL selects the library's defaults for the device. */
typedef struct {
  int32_t block;          /* reserved (the solver's blocks have 128 threads) */
  int32_t blocks_per_sm;  /* resident blocks per SM for the persistent grid (0: all that fit) */
  int32_t tile;           /* candidates a warp claims at once, 32..128 (0: 128); claims
                             shrink towards 32 as the range runs out */
  int32_t max_iters;      /* minimiser iteration cap (<= 160; 0: 24) */
  int32_t refine_steps;   /* mixed-precision refinement steps (1..4; 0: 2) */
  int32_t mixed_orders;   /* 1: one launch over all orders; 0: one launch per order */
  int32_t refill_min;     /* idle lanes of a warp that trigger taking new candidates
                             (1..32; 0: 12) */
  int32_t prescreen;      /* visibility prescreen before the refinement:
                             0 library default (on), 1 on, 2 off */
  int32_t fallback;       /* arithmetic of the refinement's fallback solve (the few
                             ill-conditioned candidates the mixed steps leave):
                             0 library default (2), 1 float-float on one lane,
                             2 FP64 with each candidate's evaluation spread over
                             the lanes of a warp, 3 FP64 on one lane */
  int32_t warp_orders;    /* bit n-1 set: the FP32 iterations of order n run one
                             candidate per warp, the evaluation spread over its
                             lanes (same minimiser and stopping rules); 0 (the
                             default): one candidate per lane for every order.
                             Applies to per-order launches (mixed_orders = 0) */
  int32_t exclude;        /* exclusion of candidates before iterating (see
                             mpt_solve): 0 library default (on), 1 on, 2 off
                             (every candidate iterated; the same valid paths) */
} mpt_schedule;

/* Compacted valid paths (caller-owned device buffers). */
typedef struct {
  int64_t* cand;     /* device [capacity]: candidate index */
  double* X;         /* device [12][capacity]: points, coordinate j of path i at X[j*capacity + i] */
  double* T;         /* device [8][capacity]: parameters */
  double* length;    /* device [capacity]: path length (m) */
  double* cost;      /* device [capacity] */
  int64_t capacity;
} mpt_paths;

/* ---------------------------------------------------------------- context */

/* Create a context on `device` (cudaSetDevice is called).  *out owns a few KB
 * of device scratch, grown on demand by mpt_validate. */
int mpt_ctx_create(int device, mpt_ctx** out);
int mpt_ctx_destroy(mpt_ctx* ctx);
/* Number of SMs of the context's device (host value). */
int mpt_ctx_sm_count(const mpt_ctx* ctx);
/* Opt-in timing of the solver kernel of each path order (measurement only;
 * the paper has no counterpart).  With on != 0, every later mpt_solve with
 * per-order launches records a pair of CUDA events around the launch of each
 * order's solver, on the stream that launch uses; mpt_ctx_solver_ms writes
 * the elapsed milliseconds of the last such launch of `order` (1..4) once the
 * caller has synchronised it.  Off by default; keep it off while capturing a
 * CUDA graph.  Errors: MPT_ERR_ARG (null context or output, order out of
 * range, timing never switched on), MPT_ERR_CUDA (events not created, or
 * not recorded / not complete). */
int mpt_ctx_time_solver(mpt_ctx* ctx, int on);
int mpt_ctx_solver_ms(mpt_ctx* ctx, int order, float* ms);

/* ------------------------------------------------------------------ scene */

/* Objects database D (Sec. II).  Copies the host records to the device
 * (synchronous).  Errors: MPT_ERR_ARG for unknown kinds, non-positive
 * scale, n_obj outside [1, MPT_MAX_OBJECTS], n_occ outside
 * [0, MPT_MAX_OCCLUDERS]. */
int mpt_scene_upload(mpt_ctx* ctx, const mpt_scene_desc* desc, mpt_scene** out);
int mpt_scene_free(mpt_scene* scene);

/* Plane offsets moved on the device, for gradients with respect to them
 * (the differentiable configuration varies each wall's offset d in
 * <n, X> = d; not in the paper).  dst must come from mpt_scene_upload of a
 * description of the same sizes and kinds as base (typically the same one).
 * Enqueued on `stream`: dst receives base's device image, then every plane
 * object i with delta[i] != 0 (delta: device double [n_obj]; other kinds'
 * entries ignored) moves along its normal by delta[i]: its corner and offset
 * in every copy of its record, and the occluder rectangle that is its own
 * facet, with that rectangle's bounding box; the boxes of the occluder groups
 * are rebuilt.  Edges, other occluders and validation's lists of rectangles
 * that hold an object's points stay base's.  No host round trip.  Errors:
 * MPT_ERR_ARG on null arguments, base == dst or mismatched scenes. */
int mpt_scene_shift_planes(mpt_ctx* ctx, const mpt_scene* base, mpt_scene* dst, const double* delta,
                           void* stream);

/* ---------------------------------------------------------- candidates */

/* Visibility matrix V of Algorithm 1 (its first line; Sec. III, Fig. 5),
 * written to vis (device uint8 [n_obj][n_obj], caller-owned), usable as the
 * adj_mask of mpt_enumerate.  Reading: a planar facet reflects on the side its
 * normal points to, so V[i][j] = 0 when i == j or when one of the two objects
 * is a plane and every vertex of the other (rectangle corners, edge ends, the
 * corners of a paraboloid patch's local box, the corners of the square of
 * half-side Rc around an arc's centre) lies more than 1e-6 S behind that
 * plane; otherwise 1.  Edges and paraboloids are seen from every side.  The
 * test is conservative: it removes only sequences whose planar facets would
 * have to be used from behind.  Enqueued on `stream`; MPT_ERR_ARG on null
 * arguments. */
int mpt_visibility(mpt_ctx* ctx, const mpt_scene* scene, uint8_t* vis, void* stream);

/* Candidate enumeration (Algorithm 1, all_simple_paths over the adjacency
 * matrix of Sec. III / Fig. 5; the BS row and UE column are taken as all
 * ones).  adj_mask: device uint8 [n_obj][n_obj] or NULL (complete graph);
 * applied to fully enumerated orders only.  max_order in [1, 4].  The number
 * of sequences must fit the library's table (2^24 entries); the number of
 * candidates E * n_pairs is written to *out->count and out->order_begin; when
 * it exceeds out->capacity, nothing beyond capacity is written.  When the
 * count is known on the host (no mask) and exceeds capacity, the call returns
 * MPT_ERR_CAPACITY before enqueuing anything.  With a mask the call
 * synchronises the stream once to size its sequence table. */
int mpt_enumerate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, int max_order,
                  const uint8_t* adj_mask, const mpt_sampling* sampling, mpt_candidates* out,
                  void* stream);

/* Host-side count of candidates mpt_enumerate will produce without a mask
 * (E * n_pairs); -1 on bad arguments. */
int64_t mpt_candidate_count(const mpt_scene* scene, const mpt_endpoints* ends, int max_order,
                            const mpt_sampling* sampling);

/* ---------------------------------------------------------------- solve */

/* find_minimum_path (Algorithm 1) for every candidate: Gauss-Newton with a
 * backtracking line search on the cost of Eq. 15, with residuals of Eq. 8
 * (divided by ||X_k - X_{k-1}||) and Eq. 9.  Reads min(*cand->count,
 * cand->capacity) candidates on the device.  precision: MPT_FP64_PLAIN,
 * MPT_FP32 or MPT_FP32_FP64REFINE.  out->capacity must be >= cand->capacity
 * and cand->capacity below 2^31 (MPT_ERR_CAPACITY otherwise).
 * Before iterating (per-order launches; mixed_orders = 1 iterates every
 * candidate), one pass excludes (status MPT_PATH_EXCLUDED) the candidates
 * that two consequences of Eq. 8 rule out.  The outgoing direction of a
 * reflection is the direction from the mirror image of the previous point
 * through the reflection point, so (half-space) the neighbouring points of a
 * reflection lie on one side of its plane, and (beam) after the first
 * reflection the next point lies in the pyramid from TX's mirror image
 * through the reflecting rectangle, before the last one the previous point
 * in the pyramid from RX's image.  Excluded: the first reflection with TX
 * more than 1e-5 S on one side of its plane and the next object (or RX)
 * wholly more than 1e-6 S on the other (every vertex, as for
 * mpt_visibility); the next object (or RX) wholly more than 1e-5 S outside
 * one face of the pyramid, TX being more than 1e-2 S from the plane; the
 * same for the last reflection with RX and the previous object; an inner
 * reflection with its two neighbouring objects on opposite sides.  With its
 * points inside their objects' bounds such a candidate's cost stays above
 * ~1e-11, far above any acceptance threshold: the exclusion removes no path.
 * The object-side and vertex tables are built at mpt_scene_upload (scenes of
 * at most 4096 objects); the pass uses context scratch of 4 bytes per
 * candidate and 80 + n_obj / 8 bytes per (endpoint, object), grown on
 * demand.  Scenes of more objects, more than 65535 endpoints, or exclusion
 * bits beyond 256 MB iterate every candidate. */
int mpt_solve(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
              const mpt_candidates* cand, int precision, const mpt_schedule* schedule,
              mpt_solutions* out, void* stream);

/* Image method (Sec. III-A, Eqs. 5-6), the paper's baseline, for the
 * candidates whose objects are all planes (reflection-only sequences).  For
 * each candidate of the ranges in cand->order_begin (the first
 * min(*cand->count, cand->capacity) candidates), one launch per order: forward
 * images of TX through the planes (Eq. 5), then the points back from RX
 * (Eq. 6), X_k = X_{k+1} + lambda_k (X_{k+1} - I_k), in float-float
 * arithmetic (48-bit significand), stored as FP64.  Output in `out`, the
 * layout of mpt_solve:
 *   - planar candidate whose path exists on the unbounded planes (every
 *     lambda_k strictly in (-1, 0)): T = plane parameters of its points,
 *     cost 0, status MPT_PATH_CONVERGED | MPT_PATH_REFINED;
 *   - planar candidate without such a path: cost +inf, status
 *     MPT_PATH_STALLED | MPT_PATH_REFINED (T holds the unchecked points);
 *   - any other candidate (an edge or a curved object in its sequence):
 *     cost +inf, status MPT_PATH_NONFINITE, T untouched.
 * mpt_validate then applies bounds, minimum segment length and visibility, as
 * for the minimiser's solutions.  iters and evals are written 0.  Errors:
 * MPT_ERR_ARG on null arguments, MPT_ERR_CAPACITY when out->capacity <
 * cand->capacity. */
int mpt_image_method(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                     const mpt_candidates* cand, mpt_solutions* out, void* stream);

/* Autotuner of mpt_solve's schedule for one workload (the batching of
 * Algorithm 1's loop over candidates and starts; the paper has no
 * counterpart).  Times mpt_solve on `cand` with `precision` under schedules
 * that differ only in knobs that leave the valid paths unchanged (tile,
 * refill_min, blocks_per_sm, mixed_orders and prescreen give bit-identical
 * solutions; warp_orders sums the normal equations in another order and
 * gives the same valid paths on every workload tested; the iteration cap is
 * part of the method and is not searched): a coordinate descent from the
 * defaults, two sweeps, each schedule timed with CUDA events as the best of
 * two solves.  *best receives the fastest schedule (pass it to mpt_solve),
 * *best_ms (may be NULL) its time.  The choice is cached in the context by a
 * workload signature (the scene's content hash, the candidate count and
 * per-order ranges, the endpoints' shape, the precision and the starts'
 * seed): a later call on the same workload returns it without timing.  The
 * call synchronises `stream` (it reads the order ranges back and waits for
 * its timings) and runs mpt_solve several times into `out`, which holds the
 * last trial's solutions on return (any tried schedule yields the same valid
 * paths).  Errors as mpt_solve. */
int mpt_autotune(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                 const mpt_candidates* cand, int precision, mpt_solutions* out, mpt_schedule* best,
                 double* best_ms, void* stream);

/* ------------------------------------------------------------- validate */

/* Acceptance of Algorithm 1: cost < tau (FP64), every segment longer than
 * 1e-5 S, every point inside its object's bounds, no segment blocked by an
 * occluder (Sec. II: bounds applied a posteriori).  Valid paths are written in
 * candidate order to `out`; the number of valid paths goes to *d_valid_count
 * (device int64).  If it exceeds out->capacity, only the first capacity paths
 * are written and the full count is still reported.  cand->capacity must be
 * below 2^32 - 1 (candidate indices are listed in 32 bits; MPT_ERR_CAPACITY
 * otherwise).  Occluders are staged in shared memory with bulk asynchronous
 * copies; a bounded wait on that copy that gives up sets the context's error
 * flag (see mpt_ctx_check). */
int mpt_validate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                 const mpt_candidates* cand, const mpt_solutions* sol, double tau, mpt_paths* out,
                 int64_t* d_valid_count, void* stream);

/* mpt_validate without any device allocation.  The paper has no counterpart:
 * this is a service for callers that cannot call cudaMalloc, such as
 * processes whose device memory is reserved up front by their own memory
 * manager (where one more allocation fails or breaks up the pool) and loops
 * that must not wait on the driver's allocator.  Same arguments, results and
 * errors as mpt_validate, but the call's scratch is one array in the
 * library's device data (about 3.3 MB, present on every GPU that loads the
 * library until the process exits) instead of context memory grown on demand:
 *   - cand->capacity may be at most 2^24 (16,777,216) candidates; larger
 *     requests return MPT_ERR_CAPACITY before anything is enqueued;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device made current for the lookup);
 *     make that first call before any stream capture.  The address is kept
 *     for the life of the process: after cudaDeviceReset on that device it
 *     is stale, so do not call this entry point again in that process;
 *   - the call allocates nothing (no cudaMalloc, cudaFree or allocating
 *     library routine);
 *   - every call uses the same array, which keeps the previous call's
 *     contents (the call overwrites every word it reads): calls that
 *     overlap on the GPU, from two streams or two host threads, race. */
int mpt_validate_noalloc(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
                         const mpt_candidates* cand, const mpt_solutions* sol, double tau, mpt_paths* out,
                         int64_t* d_valid_count, void* stream);

/* Reads (synchronously) and clears the context's device error flag: MPT_OK or
 * MPT_ERR_TIMEOUT when a bounded device wait gave up since the last check. */
int mpt_ctx_check(mpt_ctx* ctx, void* stream);

/* Self-test of the failure path: enqueues on `stream` one thread that waits
 * on a device flag nothing sets, with a bounded spin like the library's other
 * device waits (under a second here), gives up, raises the context's error
 * flag and returns.  The next mpt_ctx_check reports MPT_ERR_TIMEOUT and the
 * context stays usable.  Returns MPT_OK once enqueued. */
int mpt_ctx_selftest_wait(mpt_ctx* ctx, void* stream);

/* ----------------------------------------------------------------- grad */

/* Adjoint of converged paths (implicit-function theorem on rho(T, theta) = 0
 * of Eq. 15): for each of the first min(*d_valid_count, paths->capacity)
 * paths, with upstream weights g_len[i] (device double [capacity]) on the path
 * length and g_pts (device double [12][capacity] or NULL) on the points,
 * accumulates (+=, atomically) into
 *   g_tx  device double [n_tx][3]   d/d TX position
 *   g_rx  device double [n_rx][3]   d/d RX position
 *   g_obj device double [n_obj]     d/d offset d of each plane <n, X> = d
 *                                   (moved along n; other kinds get 0)
 * Any of g_tx, g_rx, g_obj may be NULL.  With g_pts NULL the length is
 * stationary at every path (Fermat: the laws of Eqs. 8-9), so its gradient
 * is the explicit one (envelope theorem: -u_0 for TX, u_n for RX,
 * <u_m - u_m+1, n> for a plane offset, u_j the unit segment directions) and
 * no linear system is solved. */
int mpt_grad(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
             const mpt_candidates* cand, const mpt_paths* paths, const int64_t* d_valid_count,
             const double* g_len, const double* g_pts, double* g_tx, double* g_rx, double* g_obj,
             void* stream);

/* ---------------------------------------------------------------- field */

/* Parameters of mpt_field: wavenumber k = 2 pi / lambda (1/m), the source's
 * field magnitude E0 at 1 m, and one complex coefficient (re, im) for every
 * reflection and one for every diffraction (the paper's dyadic coefficients
 * are not given there; a perfect conductor reflects with (-1, 0) in the
 * scalar, perpendicular-polarisation form). */
typedef struct {
  double wavenumber;
  double e0;
  double refl[2];
  double diff[2];
} mpt_field_params;

/* Received field (Sec. V, Eqs. 16-19) of the first min(*d_valid_count,
 * paths->capacity) paths, scalar form: a path with segment lengths d_0..d_n
 * (TX to the first point, ..., last point to RX) and total length L
 * contributes E0 e^{-jkL} / d_0 times, for interaction k with r_k = d_0 + ...
 * + d_{k-1}, refl * r_k / (r_k + d_k) (reflection, Eq. 17) or
 * diff * sqrt(r_k / (d_k (r_k + d_k))) (diffraction, Eq. 18); contributions
 * are added (+=, atomically) into field, device double [n_pairs][2] (re, im)
 * indexed by the candidate's TX/RX pair (Eq. 19).  MPT_ERR_ARG on null
 * arguments or a non-positive wavenumber. */
int mpt_field(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends,
              const mpt_candidates* cand, const mpt_paths* paths, const int64_t* d_valid_count,
              const mpt_field_params* params, double* field, void* stream);

/* --------------------------------------------------------------- misc */

const char* mpt_status_string(int status);
/* FLOP model of the FP32 minimiser for a sequence of `order` objects of the
 * given kinds, counted by running the kernel's own arithmetic on the host with
 * a counting scalar: flops_per_eval = FP32 add/sub/mul (1) and FMA (2) of one
 * cost + normal-equation evaluation at a trial point; flops_per_iter = those
 * of one Cholesky factorisation and solve over the live parameters (two per
 * surface interaction, one per edge); sfu_per_eval = reciprocal square
 * roots and sin/cos of one evaluation (may be NULL).  Algorithmic FLOPs of a
 * candidate = evals * flops_per_eval + iters * flops_per_iter, with evals and
 * iters as reported in mpt_solutions. */
int mpt_flop_model(int order, const int32_t* kinds, double* flops_per_iter, double* flops_per_eval,
                   double* sfu_per_eval);

#ifdef __cplusplus
}
#endif

#endif /* MPT_H_ */
