// Candidate enumeration (Algorithm 1, all_simple_paths; Sec. III).
//
// Two kernels:
//   k_sequences  one CTA builds the sequence table: for each order n, every
//                ordered sequence of n distinct objects (unranked in
//                lexicographic order, filtered by the optional adjacency
//                mask) or `quota` sequences drawn with SplitMix64; sequences
//                containing a curved object are repeated once per start.
//                A block-wide scan places each chunk's entries.
//   k_expand     writes the 16-byte candidate records c = e * n_pairs + p,
//                pairs fastest (a warp shares one sequence).
#include "mpt_internal.cuh"

namespace mpt {

constexpr int SEQ_THREADS = 1024;
constexpr int64_t MAX_ENTRIES = int64_t(1) << 24;

__host__ __device__ __forceinline__ int64_t perm_count(int64_t N, int n) {
  int64_t r = 1;
  for (int k = 0; k < n; ++k) r *= (N - k);
  return r;
}

// r-th ordered sequence of n distinct ids from [0, N), lexicographic order.
__host__ __device__ __forceinline__ void unrank(int64_t N, int n, int64_t r, int* ids) {
  int used[4];
  int nu = 0;
  for (int k = 0; k < n; ++k) {
    const int64_t rest = perm_count(N - 1 - k, n - 1 - k);
    int64_t idx = r / rest;
    r -= idx * rest;
    // idx-th id not yet used: walk the used ids in increasing order
    int o = (int)idx;
    int srt[4];
    for (int i = 0; i < nu; ++i) srt[i] = used[i];
    for (int i = 1; i < nu; ++i)
      for (int j = i; j > 0 && srt[j - 1] > srt[j]; --j) {
        int t = srt[j]; srt[j] = srt[j - 1]; srt[j - 1] = t;
      }
    for (int i = 0; i < nu; ++i)
      if (srt[i] <= o) ++o;
    ids[k] = o;
    used[nu++] = o;
  }
}

// Drawn sequence for slot `sl` of order n (quota sampling): draw k uses
// SplitMix64(seed ^ (n << 56 | sl << 16 | k)); position draws pick the
// idx-th not-yet-taken object (in id order).  Every `force_every`-th slot of
// order >= 3 first places two consecutive edges at a drawn position
// (draw 100), drawn from the edge ids.
__host__ __device__ __forceinline__ void draw_sequence(int N, const int32_t* kind, int n, int64_t sl,
                                                       uint64_t seed, int force_every, int n_edges, int* ids) {
  for (int k = 0; k < 4; ++k) ids[k] = -1;
  int taken[4];
  int nt = 0;
  int k = 0;
  auto draw = [&](int kk) {
    const uint64_t key = ((uint64_t)n << 56) | ((uint64_t)sl << 16) | (uint64_t)kk;
    return splitmix64(seed ^ key);
  };
  auto is_taken = [&](int o) {
    for (int i = 0; i < nt; ++i)
      if (taken[i] == o) return true;
    return false;
  };
  const bool forced = n >= 3 && force_every > 0 && (sl % force_every) == 0 && n_edges >= 2;
  if (forced) {
    const int pfix = (int)(draw(100) % (uint64_t)(n - 1));
    for (int j = 0; j < 2; ++j) {
      int idx = (int)(draw(k) % (uint64_t)(n_edges - j));
      ++k;
      for (int o = 0; o < N; ++o) {
        if (!is_edge(kind[o]) || is_taken(o)) continue;
        if (idx-- == 0) {
          ids[pfix + j] = o;
          taken[nt++] = o;
          break;
        }
      }
    }
  }
  for (int pos = 0; pos < n; ++pos) {
    if (ids[pos] >= 0) continue;
    int idx = (int)(draw(k) % (uint64_t)(N - k));
    ++k;
    for (int o = 0; o < N; ++o) {
      if (is_taken(o)) continue;
      if (idx-- == 0) {
        ids[pos] = o;
        taken[nt++] = o;
        break;
      }
    }
  }
  for (int pos = 0; pos < n; ++pos)
    if (ids[pos] < 0) ids[pos] = 0;  // unreachable: N - k objects are always free
}

struct SeqParams {
  int n_obj;
  int max_order;
  int64_t quota[4];
  uint64_t seed;
  int starts;
  int force_every;
  int n_edges;
};

// Sequence table entry: ids packed as in the candidate record.
struct Entry {
  uint32_t ids01, ids23, meta;
};

__global__ void __launch_bounds__(SEQ_THREADS) k_sequences(SeqParams sp, const int32_t* kind,
                                                           const uint8_t* adj, Entry* table, int64_t table_cap,
                                                           int64_t* entry_begin /* [5] */) {
  __shared__ int64_t warp_tot[SEQ_THREADS / 32];
  __shared__ int64_t s_base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int n = 1; n <= 4; ++n) {
    if (tid == 0) entry_begin[n - 1] = s_base;
    const int64_t q = (n <= sp.max_order && n <= sp.n_obj) ? sp.quota[n - 1] : 0;
    const int64_t raw = q < 0 ? perm_count(sp.n_obj, n) : q;
    for (int64_t r0 = 0; r0 < raw; r0 += SEQ_THREADS) {
      const int64_t r = r0 + tid;
      int ids[4] = {-1, -1, -1, -1};
      int cnt = 0;
      if (r < raw) {
        bool ok = true;
        if (q < 0) {
          unrank(sp.n_obj, n, r, ids);
          if (adj)
            for (int k = 0; k + 1 < n; ++k) ok = ok && adj[(int64_t)ids[k] * sp.n_obj + ids[k + 1]] != 0;
        } else {
          draw_sequence(sp.n_obj, kind, n, r, sp.seed, sp.force_every, sp.n_edges, ids);
        }
        bool curved = false;
        for (int k = 0; k < n; ++k) curved = curved || kind[ids[k]] == K_PARAB || kind[ids[k]] == K_ARC;
        cnt = ok ? (curved ? sp.starts : 1) : 0;
      }
      // block-wide exclusive scan of cnt
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
      }
      if (lane == 31) warp_tot[wid] = incl;
      __syncthreads();
      if (wid == 0) {
        int64_t v = lane < SEQ_THREADS / 32 ? warp_tot[lane] : 0;
        int64_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          int64_t y = __shfl_up_sync(0xffffffffu, x, d);
          if (lane >= d) x += y;
        }
        if (lane < SEQ_THREADS / 32) warp_tot[lane] = x - v;  // exclusive warp offsets
      }
      __syncthreads();
      const int64_t off = s_base + warp_tot[wid] + (incl - cnt);
      for (int s = 0; s < cnt; ++s) {
        const int64_t e = off + s;
        if (e < table_cap) {
          Entry en;
          en.ids01 = (uint32_t)(ids[0] & 0xFFFF) | ((uint32_t)(ids[1] & 0xFFFF) << 16);
          en.ids23 = (uint32_t)(ids[2] & 0xFFFF) | ((uint32_t)(ids[3] & 0xFFFF) << 16);
          en.meta = (uint32_t)n | ((uint32_t)s << 8);
          table[e] = en;
        }
      }
      __syncthreads();
      if (tid == SEQ_THREADS - 1) s_base = off + cnt;
      __syncthreads();
    }
  }
  if (tid == 0) entry_begin[4] = s_base;
}

// Full enumeration without a mask or curved objects: every sequence is one
// entry, so entry e of order n sits at off[n - 1] + its lexicographic rank
// and the table is written in parallel (no scan).  32-bit unranking: the
// table holds fewer than 2^24 entries.
struct FullSeq {
  int n_obj;
  int64_t off[5];  // first entry of orders 1..4, then the total
};
__global__ void k_sequences_full(FullSeq fs, Entry* table, int64_t table_cap, int64_t* entry_begin) {
  const int64_t total = fs.off[4] < table_cap ? fs.off[4] : table_cap;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g0 < 5) entry_begin[g0] = fs.off[g0];
  for (int64_t g = g0; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    int n = 1;
    while (n < 4 && g >= fs.off[n]) ++n;
    uint32_t r = (uint32_t)(g - fs.off[n - 1]);
    int ids[4] = {-1, -1, -1, -1};
    int srt[4];
    int nu = 0;
    for (int k = 0; k < n; ++k) {
      uint32_t rest = 1;
      for (int j = 0; j < n - 1 - k; ++j) rest *= (uint32_t)(fs.n_obj - 1 - k - j);
      const uint32_t idx = r / rest;
      r -= idx * rest;
      // idx-th id not yet used, walking the used ids in increasing order
      int o = (int)idx;
      for (int i = 0; i < nu; ++i)
        if (srt[i] <= o) ++o;
      ids[k] = o;
      int j = nu++;
      while (j > 0 && srt[j - 1] > o) {
        srt[j] = srt[j - 1];
        --j;
      }
      srt[j] = o;
    }
    Entry en;
    en.ids01 = (uint32_t)(ids[0] & 0xFFFF) | ((uint32_t)(ids[1] & 0xFFFF) << 16);
    en.ids23 = (uint32_t)(ids[2] & 0xFFFF) | ((uint32_t)(ids[3] & 0xFFFF) << 16);
    en.meta = (uint32_t)n;
    table[g] = en;
  }
}

__global__ void k_expand(const Entry* table, int64_t table_cap, const int64_t* entry_begin, int64_t n_pairs,
                         uint4* rec, int64_t cap, int64_t* count, int64_t* order_begin) {
  int64_t E = entry_begin[4];
  if (E > table_cap) E = table_cap;  // the table never holds more than table_cap entries
  const int64_t total = E * n_pairs;
  if (blockIdx.x == 0 && threadIdx.x < 5) order_begin[threadIdx.x] = entry_begin[threadIdx.x] * n_pairs;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = total;
  const int64_t lim = total < cap ? total : cap;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < lim; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = c / n_pairs;
    const Entry en = table[e];
    rec[c] = make_uint4((uint32_t)(c - e * n_pairs), en.ids01, en.ids23, en.meta);
  }
}

// Host mirror of the table size (no mask): exact entry count per order.
static int64_t host_entries(const int32_t* kind, const SeqParams& sp) {
  int64_t total = 0;
  int n_curved = 0;
  for (int i = 0; i < sp.n_obj; ++i) n_curved += (kind[i] == K_PARAB || kind[i] == K_ARC);
  for (int n = 1; n <= sp.max_order && n <= 4; ++n) {
    const int64_t q = n <= sp.n_obj ? sp.quota[n - 1] : 0;
    if (q == 0) continue;
    if (q < 0) {
      const int64_t all = perm_count(sp.n_obj, n);
      const int64_t flat = perm_count(sp.n_obj - n_curved, n);
      total += flat + (all - flat) * sp.starts;
    } else {
      for (int64_t sl = 0; sl < q; ++sl) {
        int ids[4];
        draw_sequence(sp.n_obj, kind, n, sl, sp.seed, sp.force_every, sp.n_edges, ids);
        bool curved = false;
        for (int k = 0; k < n; ++k) curved = curved || kind[ids[k]] == K_PARAB || kind[ids[k]] == K_ARC;
        total += curved ? sp.starts : 1;
      }
    }
  }
  return total;
}

static int seq_params(const mpt_scene* scene, int max_order, const mpt_sampling* smp, SeqParams& sp) {
  sp.n_obj = scene->n_obj;
  sp.max_order = max_order;
  for (int k = 0; k < 4; ++k) sp.quota[k] = smp ? smp->quota[k] : (k < 2 ? -1 : 0);
  sp.seed = smp ? smp->seed : 0;
  sp.starts = smp && smp->starts_curved > 0 ? smp->starts_curved : 1;
  sp.force_every = smp ? smp->force_edges_every : 0;
  sp.n_edges = 0;
  for (int i = 0; i < scene->n_obj; ++i) sp.n_edges += is_edge(scene->host_kind[i]);
  if (max_order < 1 || max_order > 4 || sp.starts > 255) return MPT_ERR_ARG;
  for (int k = 0; k < 4; ++k)
    if (sp.quota[k] < -1) return MPT_ERR_ARG;
  return MPT_OK;
}

int64_t host_candidate_count(const mpt_scene* scene, const mpt_endpoints* ends, int max_order,
                             const mpt_sampling* smp) {
  SeqParams sp;
  if (!scene || !ends || seq_params(scene, max_order, smp, sp) != MPT_OK) return -1;
  return host_entries(scene->host_kind, sp) * n_pairs(ends);
}

int launch_enumerate(mpt_ctx* ctx, const mpt_scene* scene, const mpt_endpoints* ends, int max_order,
                     const uint8_t* adj, const mpt_sampling* smp, mpt_candidates* out, cudaStream_t st) {
  SeqParams sp;
  int rc = seq_params(scene, max_order, smp, sp);
  if (rc != MPT_OK) return rc;
  const int64_t np = n_pairs(ends);
  // the unmasked entry count bounds the table (a mask only removes entries)
  const int64_t E0 = host_entries(scene->host_kind, sp);
  if (E0 > MAX_ENTRIES) return MPT_ERR_UNSUPPORTED;
  if (adj == nullptr && E0 * np > out->capacity) return MPT_ERR_CAPACITY;
  const int64_t table_cap = E0 > 0 ? E0 : 1;
  // table + entry_begin live in a temporary device buffer owned by this call
  const size_t bytes = (size_t)table_cap * sizeof(Entry) + 8 * sizeof(int64_t);
  void* buf = nullptr;
  MPT_CUDA_TRY(cudaMallocAsync(&buf, bytes, st));
  int64_t* entry_begin = reinterpret_cast<int64_t*>(buf);
  Entry* table = reinterpret_cast<Entry*>(entry_begin + 8);
  bool full = adj == nullptr;
  for (int i = 0; i < sp.n_obj && full; ++i) full = scene->host_kind[i] != K_PARAB && scene->host_kind[i] != K_ARC;
  for (int n = 1; n <= 4 && full; ++n)
    full = (n <= sp.max_order && n <= sp.n_obj) ? sp.quota[n - 1] <= 0 : true;
  if (full) {
    FullSeq fs;
    fs.n_obj = sp.n_obj;
    fs.off[0] = 0;
    for (int n = 1; n <= 4; ++n) {
      const bool on = n <= sp.max_order && n <= sp.n_obj && sp.quota[n - 1] < 0;
      fs.off[n] = fs.off[n - 1] + (on ? perm_count(sp.n_obj, n) : 0);
    }
    const int64_t blocks = (fs.off[4] + 255) / 256;
    k_sequences_full<<<(unsigned)(blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks)), 256, 0, st>>>(fs, table, table_cap,
                                                                                                 entry_begin);
  } else {
    k_sequences<<<1, SEQ_THREADS, 0, st>>>(sp, scene->d.kind, adj, table, table_cap, entry_begin);
  }
  MPT_LAUNCH_CHECK();
  bool over = false;
  if (adj != nullptr) {
    // the masked count is only known on the device: one synchronisation
    int64_t E = 0;
    MPT_CUDA_TRY(cudaMemcpyAsync(&E, entry_begin + 4, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MPT_CUDA_TRY(cudaStreamSynchronize(st));
    over = E * np > out->capacity;
  }
  const int threads = 256;
  int64_t blocks = (out->capacity + threads - 1) / threads;
  const int64_t max_blocks = (int64_t)ctx->sms * 16;
  if (blocks > max_blocks) blocks = max_blocks;
  if (blocks < 1) blocks = 1;
  k_expand<<<(unsigned)blocks, threads, 0, st>>>(table, table_cap, entry_begin, np, reinterpret_cast<uint4*>(out->rec),
                                                 out->capacity, out->count, out->order_begin);
  MPT_LAUNCH_CHECK();
  MPT_CUDA_TRY(cudaFreeAsync(buf, st));
  return over ? MPT_ERR_CAPACITY : MPT_OK;
}

// ------------------------------------------------------- visibility matrix --
// V of Algorithm 1 (its first line; Sec. III, Fig. 5) under the reading that
// a planar facet reflects on the side its normal points to: V[i][j] = 0 when
// i == j, or when one object is a plane and every vertex of the other lies
// more than delta behind that plane; otherwise 1.  Vertices bound every
// point an object can put on a path: a rectangle's corners, a line edge's
// ends, the corners of a paraboloid patch's local box, the corners of the
// square of half-side Rc around an arc's centre.  FP64; one thread per pair.
__device__ int object_vertices(const DevScene& sc, int o, v3<double> (&x)[8]) {
  const Rec<double> r = load_obj64(sc, o);
  const int kind = sc.kind[o];
  if (kind == K_PLANE) {
    const v3<double> O = r.f3(0), u = r.f3(4), v = r.f3(8);
    x[0] = O;
    x[1] = axpy(r.v[3], u, O);
    x[2] = axpy(r.v[7], v, O);
    x[3] = axpy(r.v[7], v, x[1]);
    return 4;
  }
  if (kind == K_LINE) {
    x[0] = axpy(r.v[3], r.f3(4), r.f3(0));
    x[1] = axpy(r.v[7], r.f3(4), r.f3(0));
    return 2;
  }
  if (kind == K_PARAB) {
    const v3<double> t0 = mk(r.v[3], r.v[7], r.v[11]);
    const double rho = r.v[13], h = rho * rho * r.v[12];
    int m = 0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 2; ++c)
          x[m++] = axpy(c ? h : 0.0, r.f3(8), axpy(b ? rho : -rho, r.f3(4), axpy(a ? rho : -rho, r.f3(0), t0)));
    return 8;
  }
  const double Rc = r.v[3];
  int m = 0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) x[m++] = axpy(b ? Rc : -Rc, r.f3(8), axpy(a ? Rc : -Rc, r.f3(4), r.f3(0)));
  return 4;
}

// every vertex of object j more than delta behind plane i
__device__ bool hidden_behind(const DevScene& sc, int i, int j, double delta) {
  const Rec<double> p = load_obj64(sc, i);
  const v3<double> O = p.f3(0), n = p.f3(12);
  v3<double> x[8];
  const int m = object_vertices(sc, j, x);
  for (int k = 0; k < m; ++k)
    if (!(dot(n, x[k] - O) < -delta)) return false;
  return true;
}

__global__ void k_visibility(DevScene sc, double delta, uint8_t* V) {
  const int64_t n = sc.n_obj;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * n; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / n), j = (int)(q % n);
    uint8_t v = 1;
    if (i == j) v = 0;
    else if ((sc.kind[i] == K_PLANE && hidden_behind(sc, i, j, delta)) ||
             (sc.kind[j] == K_PLANE && hidden_behind(sc, j, i, delta)))
      v = 0;
    V[q] = v;
  }
}

// side[i][j] for plane i: +1 when every vertex of object j lies more than
// delta in front of plane i (<n, X - O> > delta), -1 when every vertex lies
// more than delta behind it, else 0; 0 for non-planes i.
__global__ void k_side_table(DevScene sc, double delta, int8_t* side) {
  const int64_t n = sc.n_obj;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * n; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / n), j = (int)(q % n);
    int8_t v = 0;
    if (i != j && sc.kind[i] == K_PLANE) {
      const Rec<double> p = load_obj64(sc, i);
      const v3<double> O = p.f3(0), nrm = p.f3(12);
      v3<double> x[8];
      const int m = object_vertices(sc, j, x);
      bool front = true, behind = true;
      for (int k = 0; k < m; ++k) {
        const double h = dot(nrm, x[k] - O);
        front = front && h > delta;
        behind = behind && h < -delta;
      }
      v = front ? (int8_t)1 : behind ? (int8_t)-1 : (int8_t)0;
    }
    side[q] = v;
  }
}

// vtx[o][k]: the points of object_vertices in FP32, the last one repeated
// up to 8 (a repeated point changes no test over all of them); w holds the
// number of distinct points.
__global__ void k_vertices(DevScene sc, float4* vtx) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= sc.n_obj) return;
  v3<double> x[8];
  const int m = object_vertices(sc, o, x);
  for (int k = 0; k < 8; ++k) {
    const v3<double>& p = x[k < m ? k : m - 1];
    vtx[(int64_t)o * 8 + k] = make_float4((float)p.x, (float)p.y, (float)p.z, (float)m);
  }
}

int launch_side_table(const DevScene& d, cudaStream_t st) {
  if (d.vtx != nullptr) {
    k_vertices<<<(d.n_obj + 127) / 128, 128, 0, st>>>(d, const_cast<float4*>(d.vtx));
    MPT_LAUNCH_CHECK();
  }
  if (d.side == nullptr) return MPT_OK;
  const int64_t pairs = (int64_t)d.n_obj * d.n_obj;
  const int64_t blocks = (pairs + 255) / 256 < 1024 ? (pairs + 255) / 256 : 1024;
  k_side_table<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(d, 1e-6 * d.scale, const_cast<int8_t*>(d.side));
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

int launch_visibility(mpt_ctx* ctx, const mpt_scene* scene, uint8_t* vis, cudaStream_t st) {
  const int64_t pairs = (int64_t)scene->d.n_obj * scene->d.n_obj;
  int64_t blocks = (pairs + 255) / 256;
  if (blocks > (int64_t)ctx->sms * 16) blocks = (int64_t)ctx->sms * 16;
  if (blocks < 1) blocks = 1;
  k_visibility<<<(unsigned)blocks, 256, 0, st>>>(scene->d, 1e-6 * scene->d.scale, vis);
  MPT_LAUNCH_CHECK();
  return MPT_OK;
}

}  // namespace mpt
