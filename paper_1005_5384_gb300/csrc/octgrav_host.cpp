// octgrav_host.cpp -- host side of the GB300 tree-code library: FP64 octree
// build, cell properties and groups (Sec. 2.1), device-array layout, upload,
// launch and the C ABI declared in include/octgrav.h.
//
// Tree definition (shared with any independent implementation):
//  - root cube: centre = centre of the bounding box of the system, side =
//    longest box side * (1 + 2^-20) (1.0 when all particles coincide);
//  - quantised coordinate q = floor((x - lo) / side * 2^21) clamped to
//    [0, 2^21 - 1]; the octant of a depth-L cell's child is bit (20 - L) of q
//    on each axis (x = octant bit 0), so cells are Morton-key prefixes;
//  - a cell is a leaf when it holds <= n_leaf particles or has depth 21;
//  - groups are the cells reached first from the root that are leaves or hold
//    <= n_group particles (Sec. 2.1-2.2);
//  - per cell: tight box, boundary cube (centre = box centre, half side = half
//    the longest box side, Fig. 1), mass, centre of mass and second moments.
// The build sorts particles by Morton key (parallel LSD radix sort), splits
// key ranges level by level, and combines moments bottom-up with the
// parallel-axis theorem, all in FP64 (products accumulated with explicit fused
// multiply-adds). Compile with -ffp-contract=off: the GPU build reproduces
// these operations one for one.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/octgrav.h"
#include "octgrav_internal.h"
#include "octgrav_mlp.h"

namespace {

constexpr int kMaxDepth = OCTGRAV_MAX_DEPTH;

// Allocator whose construct() without arguments default-initialises, so that
// resize() of a vector of plain numbers leaves the new elements unwritten. The
// build's arrays are all filled completely (in parallel) right after they are
// sized; value-initialisation would first zero them on one thread (~200 MB per
// million particles).
template <class T>
struct NoInit : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInit<U>;
  };
  NoInit() = default;
  template <class U>
  NoInit(const NoInit<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using hvec = std::vector<T, NoInit<T>>;

// ---------------------------------------------------------------- errors

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(OCTGRAV_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

// ---------------------------------------------------------------- thread pool

class Pool {
 public:
  static Pool& get() {
    static Pool p;
    return p;
  }
  int size() const { return static_cast<int>(threads_.size()) + 1; }

  // Run fn(chunk) for chunk in [0, nchunks) on all workers and the caller.
  // Workers spin for a short while after a job before they sleep, so the many
  // short parallel loops of a build do not each pay a wake-up of every thread.
  void run(int nchunks, const std::function<void(int)>& fn) {
    if (nchunks <= 0) return;
    if (threads_.empty() || nchunks == 1 || in_pool_) {
      for (int c = 0; c < nchunks; ++c) fn(c);
      return;
    }
    std::lock_guard<std::mutex> one(run_mu_);  // one parallel region at a time
    job_ = &fn;
    nchunks_ = nchunks;
    next_.store(0, std::memory_order_relaxed);
    pending_.store(static_cast<int>(threads_.size()), std::memory_order_relaxed);
    gen_.fetch_add(1, std::memory_order_seq_cst);
    if (sleepers_.load(std::memory_order_seq_cst) > 0) {
      { std::lock_guard<std::mutex> g(mu_); }
      cv_.notify_all();
    }
    work();
    if (!spin_until([&] { return pending_.load(std::memory_order_acquire) == 0; })) {
      std::unique_lock<std::mutex> g(mu_);
      done_cv_.wait(g, [&] { return pending_.load(std::memory_order_acquire) == 0; });
    }
    job_ = nullptr;
  }

 private:
  Pool() {
    unsigned hc = std::thread::hardware_concurrency();
    int n = static_cast<int>(hc ? hc : 1);
    if (const char* e = getenv("OCTGRAV_THREADS")) n = std::max(1, atoi(e));
    n = std::min(n, 64);
    for (int t = 1; t < n; ++t) threads_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    stop_.store(true);
    gen_.fetch_add(1, std::memory_order_release);
    {
      std::lock_guard<std::mutex> g(mu_);
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }
  // Spin until pred() holds or ~50 us have passed; true if it holds.
  template <class P>
  static bool spin_until(P pred) {
    auto t0 = std::chrono::steady_clock::now();
    for (int k = 0;; ++k) {
      if (pred()) return true;
      if ((k & 255) == 255 && std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(50)) return pred();
    }
  }
  void work() {
    in_pool_ = true;
    for (;;) {
      int c = next_.fetch_add(1, std::memory_order_relaxed);
      if (c >= nchunks_) break;
      (*job_)(c);
    }
    in_pool_ = false;
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      if (!spin_until([&] { return gen_.load(std::memory_order_acquire) != seen; })) {
        std::unique_lock<std::mutex> g(mu_);
        sleepers_.fetch_add(1, std::memory_order_seq_cst);
        cv_.wait(g, [&] { return gen_.load(std::memory_order_seq_cst) != seen; });
        sleepers_.fetch_sub(1, std::memory_order_relaxed);
      }
      seen = gen_.load(std::memory_order_acquire);
      if (stop_.load()) return;
      work();
      if (pending_.fetch_sub(1, std::memory_order_acq_rel) == 1) {
        { std::lock_guard<std::mutex> g(mu_); }
        done_cv_.notify_all();
      }
    }
  }
  std::vector<std::thread> threads_;
  std::mutex mu_, run_mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* job_ = nullptr;
  int nchunks_ = 0;
  std::atomic<int> next_{0};
  std::atomic<int> pending_{0};
  std::atomic<int> sleepers_{0};
  std::atomic<uint64_t> gen_{0};
  std::atomic<bool> stop_{false};
  static thread_local bool in_pool_;
};
thread_local bool Pool::in_pool_ = false;

// parallel_for over [0, n) in chunks of at least `grain` elements.
void parallel_for(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& fn) {
  if (n <= 0) return;
  Pool& P = Pool::get();
  int64_t chunks = std::min<int64_t>((n + grain - 1) / grain, 8 * P.size());
  if (chunks <= 1) {
    fn(0, n);
    return;
  }
  const int64_t step = (n + chunks - 1) / chunks;
  P.run(static_cast<int>(chunks), [&](int c) {
    int64_t lo = c * step, hi = std::min(n, lo + step);
    if (lo < hi) fn(lo, hi);
  });
}

// ---------------------------------------------------------------- Morton keys

inline uint64_t spread21(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

// Stable LSD radix sort of (key, val) by key (63 significant bits, 9-bit digits).
void radix_sort(hvec<uint64_t>& key, hvec<uint32_t>& val, hvec<uint64_t>& k2, hvec<uint32_t>& v2,
                bool parallel) {
  const int64_t n = static_cast<int64_t>(key.size());
  k2.resize(n);
  v2.resize(n);
  constexpr int BITS = 9, B = 1 << BITS, PASSES = (63 + BITS - 1) / BITS;
  const int T = parallel ? std::max(1, std::min<int>(Pool::get().size(), static_cast<int>(n / 65536))) : 1;
  std::vector<int64_t> hist(static_cast<size_t>(T) * B);
  const int64_t step = (n + T - 1) / T;
  for (int pass = 0; pass < PASSES; ++pass) {
    const int sh = pass * BITS;
    auto body_hist = [&](int t) {
      int64_t* h = &hist[static_cast<size_t>(t) * B];
      std::fill(h, h + B, 0);
      const int64_t lo = t * step, hi = std::min(n, lo + step);
      for (int64_t i = lo; i < hi; ++i) ++h[(key[i] >> sh) & (B - 1)];
    };
    if (T > 1) Pool::get().run(T, body_hist); else body_hist(0);
    int64_t off = 0;
    for (int d = 0; d < B; ++d)
      for (int t = 0; t < T; ++t) {
        int64_t c = hist[static_cast<size_t>(t) * B + d];
        hist[static_cast<size_t>(t) * B + d] = off;
        off += c;
      }
    auto body_scatter = [&](int t) {
      int64_t* h = &hist[static_cast<size_t>(t) * B];
      const int64_t lo = t * step, hi = std::min(n, lo + step);
      for (int64_t i = lo; i < hi; ++i) {
        int64_t dst = h[(key[i] >> sh) & (B - 1)]++;
        k2[dst] = key[i];
        v2[dst] = val[i];
      }
    };
    if (T > 1) Pool::get().run(T, body_scatter); else body_scatter(0);
    key.swap(k2);
    val.swap(v2);
  }
}

// ---------------------------------------------------------------- one system

struct SysTree {
  int64_t n = 0;
  hvec<uint32_t> perm;  // tree position -> index within the system
  hvec<uint64_t> code;  // Morton code per tree position
  hvec<double> x;       // 3 per tree position
  hvec<double> m;
  // cells in breadth-first order (children of a node are contiguous)
  hvec<uint64_t> key;
  hvec<int32_t> depth, parent, first_child, n_child;
  hvec<int64_t> pfirst, pcount;
  hvec<double> bmin, bmax, cube, M, com, S;  // 3, 3, 4, 1, 3, 6 per cell
  hvec<int32_t> groups;                      // cell index, tree (Morton) order
  int depth_reached = 0;
  int64_t max_group = 0;
  int64_t n_leaves = 0;
  // scratch of the build (kept so that a reused SysTree allocates nothing)
  hvec<uint64_t> k2;
  hvec<uint32_t> v2;
  hvec<int64_t> splits;                      // 9 per cell of the level being split
  std::vector<int32_t> nch;                  // children per cell of that level
  std::vector<int64_t> child_base;           // first child per chunk of that level
  // empty every array but keep its memory, for a new build
  void reset() {
    n = 0;
    for (auto* v : {&perm, &v2}) v->clear();
    for (auto* v : {&code, &key, &k2}) v->clear();
    for (auto* v : {&x, &m, &bmin, &bmax, &cube, &M, &com, &S}) v->clear();
    for (auto* v : {&depth, &parent, &first_child, &n_child, &groups}) v->clear();
    for (auto* v : {&pfirst, &pcount, &splits}) v->clear();
    nch.clear();
    child_base.clear();
    depth_reached = 0;
    max_group = 0;
    n_leaves = 0;
  }
};

inline int octant_at(uint64_t code, int child_depth) {
  return static_cast<int>((code >> (3 * (kMaxDepth - child_depth))) & 7);
}

// A particle's two device records: (x_hi, y_hi, z_hi, m) and (x_lo, y_lo, z_lo, 0),
// hi = fl32(x) and lo = fl32(x - hi).
inline void particle_records(const double* x, double m, float4* rec) {
  float hi[3], lo[3];
  for (int d = 0; d < 3; ++d) {
    hi[d] = static_cast<float>(x[d]);
    lo[d] = static_cast<float>(x[d] - static_cast<double>(hi[d]));
  }
  rec[0] = make_float4(hi[0], hi[1], hi[2], static_cast<float>(m));
  rec[1] = make_float4(lo[0], lo[1], lo[2], 0.f);
}

// Where a one-system build writes its particle images during the gather (tree
// order), and what to call once they are complete (e.g. to start their upload
// while the cells are built).
struct ParticleSink {
  float4* parts = nullptr;  // 2 records per particle
  int64_t* perm = nullptr;
  int32_t* perm32 = nullptr;
  std::function<int()> ready;
  bool check_inputs = false;  // the bounding-box pass also checks the inputs (finite, masses >= 0)
};

int build_system(const double* pos, const double* mass, int64_t n, int n_leaf, int n_group,
                 bool parallel, SysTree& T, const ParticleSink* sink = nullptr) {
  T.reset();
  T.n = n;
  const int64_t grain = parallel ? 16384 : (int64_t)1 << 62;
  // ---- bounding box and root cube
  double mn[3] = {pos[0], pos[1], pos[2]}, mx[3] = {pos[0], pos[1], pos[2]};
  {
    const int64_t chunks = parallel ? std::max<int64_t>(1, std::min<int64_t>(64, n / 65536)) : 1;
    std::vector<double> part(chunks * 6);
    const int64_t step = (n + chunks - 1) / chunks;
    const bool check = sink && sink->check_inputs;
    std::vector<uint8_t> bad(chunks, 0);
    auto body = [&](int c) {
      double a[3] = {pos[0], pos[1], pos[2]}, b[3] = {pos[0], pos[1], pos[2]};
      bool ok = true;
      for (int64_t i = c * step; i < std::min(n, (c + 1) * step); ++i) {
        for (int d = 0; d < 3; ++d) {
          const double v = pos[3 * i + d];
          if (v < a[d]) a[d] = v;
          if (v > b[d]) b[d] = v;
          if (check) ok = ok && std::isfinite(v);
        }
        if (check) ok = ok && std::isfinite(mass[i]) && mass[i] >= 0;
      }
      for (int d = 0; d < 3; ++d) {
        part[6 * c + d] = a[d];
        part[6 * c + 3 + d] = b[d];
      }
      bad[c] = !ok;
    };
    if (chunks > 1) Pool::get().run(static_cast<int>(chunks), body); else body(0);
    for (int64_t c = 0; c < chunks; ++c)
      if (bad[c]) return fail(OCTGRAV_ERR_NONFINITE, "non-finite position/mass or negative mass");
    for (int64_t c = 0; c < chunks; ++c)
      for (int d = 0; d < 3; ++d) {
        mn[d] = std::min(mn[d], part[6 * c + d]);
        mx[d] = std::max(mx[d], part[6 * c + 3 + d]);
      }
  }
  double ext = mx[0] - mn[0];
  if (mx[1] - mn[1] > ext) ext = mx[1] - mn[1];
  if (mx[2] - mn[2] > ext) ext = mx[2] - mn[2];
  if (!(ext > 0)) ext = 1.0;
  const double side = ext * (1.0 + 1.0 / 1048576.0);
  double lo[3];
  for (int d = 0; d < 3; ++d) lo[d] = (mn[d] + mx[d]) * 0.5 - side * 0.5;
  const double scale = std::ldexp(1.0, kMaxDepth);
  const uint64_t qmax = (1ull << kMaxDepth) - 1;

  // ---- Morton codes and sort
  hvec<uint64_t>& code = T.code;
  hvec<uint32_t>& idx = T.perm;
  code.resize(n);
  idx.resize(n);
  parallel_for(n, grain, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      uint64_t q[3];
      for (int d = 0; d < 3; ++d) {
        const double u = (pos[3 * i + d] - lo[d]) / side;
        const double v = std::floor(u * scale);
        q[d] = v <= 0 ? 0 : (v >= static_cast<double>(qmax) ? qmax : static_cast<uint64_t>(v));
      }
      code[i] = spread21(q[0]) | (spread21(q[1]) << 1) | (spread21(q[2]) << 2);
      idx[i] = static_cast<uint32_t>(i);
    }
  });
  radix_sort(code, idx, T.k2, T.v2, parallel);
  T.x.resize(3 * n);
  T.m.resize(n);
  parallel_for(n, grain, [&](int64_t a, int64_t b) {
    constexpr int64_t ahead = 16;  // prefetch distance of the random reads
    for (int64_t t = a; t < b; ++t) {
      if (t + ahead < b) {
        const int64_t j = T.perm[t + ahead];
        __builtin_prefetch(pos + 3 * j);
        __builtin_prefetch(pos + 3 * j + 2);
        __builtin_prefetch(mass + j);
      }
      const int64_t i = T.perm[t];
      T.x[3 * t] = pos[3 * i];
      T.x[3 * t + 1] = pos[3 * i + 1];
      T.x[3 * t + 2] = pos[3 * i + 2];
      T.m[t] = mass[i];
      if (sink) {
        particle_records(&T.x[3 * t], T.m[t], sink->parts + 2 * t);
        sink->perm[t] = i;
        sink->perm32[t] = static_cast<int32_t>(i);
      }
    }
  });
  if (sink && sink->ready) {
    const int rc = sink->ready();
    if (rc) return rc;
  }

  // ---- cells, level by level
  auto push_cell = [&](uint64_t key, int depth, int32_t parent, int64_t pf, int64_t pc) {
    T.key.push_back(key);
    T.depth.push_back(depth);
    T.parent.push_back(parent);
    T.first_child.push_back(-1);
    T.n_child.push_back(0);
    T.pfirst.push_back(pf);
    T.pcount.push_back(pc);
  };
  {  // room for the usual tree size, so that the level loop rarely reallocates
    const size_t guess = static_cast<size_t>(8 * n / (n_leaf + 1) + 64);
    for (auto* v : {&T.depth, &T.parent, &T.first_child, &T.n_child}) v->reserve(guess);
    T.key.reserve(guess);
    T.pfirst.reserve(guess);
    T.pcount.reserve(guess);
  }
  push_cell(1, 0, -1, 0, n);
  std::vector<int64_t> level_begin = {0};
  hvec<int64_t>& splits = T.splits;  // read only where nch > 0
  std::vector<int32_t>& nch = T.nch;
  std::vector<int64_t>& child_base = T.child_base;
  for (int L = 0;; ++L) {
    const int64_t lb = level_begin.back(), le = static_cast<int64_t>(T.key.size());
    if (lb == le) break;
    const int64_t nl = le - lb;
    splits.resize(9 * nl);
    nch.resize(nl);
    // the level in fixed chunks: a first pass counts each chunk's children, a
    // scan over the chunk totals places them in breadth-first order, and a
    // second pass writes them
    const int64_t nchunk = parallel ? std::min<int64_t>(8 * Pool::get().size(), std::max<int64_t>(1, nl / 256)) : 1;
    const int64_t cstep = (nl + nchunk - 1) / nchunk;
    child_base.assign(nchunk + 1, 0);
    auto split_chunk = [&](int q) {
      int64_t total = 0;
      for (int64_t k = q * cstep; k < std::min(nl, (q + 1) * cstep); ++k) {
        const int64_t c = lb + k;
        const int64_t f = T.pfirst[c], cnt = T.pcount[c];
        int64_t* sp = &splits[9 * k];
        nch[k] = 0;
        if (cnt <= n_leaf || L >= kMaxDepth) continue;
        sp[0] = f;
        sp[8] = f + cnt;
        const uint64_t* base = T.code.data();
        for (int o = 1; o < 8; ++o) {
          // first position whose child octant is >= o (octants ascend inside a cell)
          const uint64_t* it = std::partition_point(base + sp[o - 1], base + f + cnt,
                                                    [&](uint64_t cd) { return octant_at(cd, L + 1) < o; });
          sp[o] = it - base;
        }
        int k8 = 0;
        for (int o = 0; o < 8; ++o) k8 += sp[o + 1] > sp[o];
        nch[k] = k8;
        total += k8;
      }
      child_base[q + 1] = total;
    };
    Pool::get().run(static_cast<int>(nchunk), split_chunk);
    for (int64_t q = 0; q < nchunk; ++q) child_base[q + 1] += child_base[q];
    const int64_t next = le + child_base[nchunk];
    if (next == le) break;
    level_begin.push_back(le);
    if (next >= (1ll << 28)) return fail(OCTGRAV_ERR_ARG, "tree too large (%lld cells)", (long long)next);
    T.key.resize(next);
    T.depth.resize(next);
    T.parent.resize(next);
    T.first_child.resize(next);
    T.n_child.resize(next);
    T.pfirst.resize(next);
    T.pcount.resize(next);
    auto emit_chunk = [&](int q) {
      int64_t w = le + child_base[q];
      for (int64_t k = q * cstep; k < std::min(nl, (q + 1) * cstep); ++k) {
        if (!nch[k]) continue;
        const int64_t c = lb + k;
        T.first_child[c] = static_cast<int32_t>(w);
        T.n_child[c] = nch[k];
        const int64_t* sp = &splits[9 * k];
        for (int o = 0; o < 8; ++o) {
          if (sp[o + 1] <= sp[o]) continue;
          T.key[w] = (T.key[c] << 3) | static_cast<uint64_t>(o);
          T.depth[w] = L + 1;
          T.parent[w] = static_cast<int32_t>(c);
          T.first_child[w] = -1;
          T.n_child[w] = 0;
          T.pfirst[w] = sp[o];
          T.pcount[w] = sp[o + 1] - sp[o];
          ++w;
        }
      }
    };
    Pool::get().run(static_cast<int>(nchunk), emit_chunk);
  }
  const int64_t nc = static_cast<int64_t>(T.key.size());
  T.depth_reached = static_cast<int>(level_begin.size()) - 1;

  // ---- cell properties, deepest level first
  T.bmin.resize(3 * nc);
  T.bmax.resize(3 * nc);
  T.cube.resize(4 * nc);
  T.M.resize(nc);
  T.com.resize(3 * nc);
  T.S.resize(6 * nc);
  level_begin.push_back(nc);
  for (int L = static_cast<int>(level_begin.size()) - 2; L >= 0; --L) {
    const int64_t lb = level_begin[L], le = level_begin[L + 1];
    parallel_for(le - lb, parallel ? 1024 : (int64_t)1 << 62, [&](int64_t a, int64_t b) {
      for (int64_t c = lb + a; c < lb + b; ++c) {
        double* bn = &T.bmin[3 * c];
        double* bx = &T.bmax[3 * c];
        double* cm = &T.com[3 * c];
        double* s6 = &T.S[6 * c];
        double Mc = 0, sx = 0, sy = 0, sz = 0;
        for (int d = 0; d < 3; ++d) {
          bn[d] = INFINITY;
          bx[d] = -INFINITY;
        }
        const int64_t f = T.pfirst[c], cnt = T.pcount[c];
        if (T.n_child[c] == 0) {
          for (int64_t t = f; t < f + cnt; ++t) {
            const double* xp = &T.x[3 * t];
            for (int d = 0; d < 3; ++d) {
              bn[d] = std::min(bn[d], xp[d]);
              bx[d] = std::max(bx[d], xp[d]);
            }
            Mc += T.m[t];
            sx = std::fma(T.m[t], xp[0], sx);
            sy = std::fma(T.m[t], xp[1], sy);
            sz = std::fma(T.m[t], xp[2], sz);
          }
        } else {
          for (int j = T.first_child[c]; j < T.first_child[c] + T.n_child[c]; ++j) {
            for (int d = 0; d < 3; ++d) {
              bn[d] = std::min(bn[d], T.bmin[3 * j + d]);
              bx[d] = std::max(bx[d], T.bmax[3 * j + d]);
            }
            Mc += T.M[j];
            sx = std::fma(T.M[j], T.com[3 * j], sx);
            sy = std::fma(T.M[j], T.com[3 * j + 1], sy);
            sz = std::fma(T.M[j], T.com[3 * j + 2], sz);
          }
        }
        double* cu = &T.cube[4 * c];
        for (int d = 0; d < 3; ++d) cu[d] = (bn[d] + bx[d]) * 0.5;
        double e = bx[0] - bn[0];
        if (bx[1] - bn[1] > e) e = bx[1] - bn[1];
        if (bx[2] - bn[2] > e) e = bx[2] - bn[2];
        cu[3] = 0.5 * e;
        T.M[c] = Mc;
        if (Mc > 0) {
          cm[0] = sx / Mc;
          cm[1] = sy / Mc;
          cm[2] = sz / Mc;
        } else {
          cm[0] = cu[0];
          cm[1] = cu[1];
          cm[2] = cu[2];
        }
        for (int q = 0; q < 6; ++q) s6[q] = 0;
        auto add_outer = [&](double w, double y0, double y1, double y2) {
          const double w0 = w * y0, w1 = w * y1, w2 = w * y2;
          s6[0] = std::fma(w0, y0, s6[0]);
          s6[1] = std::fma(w1, y1, s6[1]);
          s6[2] = std::fma(w2, y2, s6[2]);
          s6[3] = std::fma(w0, y1, s6[3]);
          s6[4] = std::fma(w0, y2, s6[4]);
          s6[5] = std::fma(w1, y2, s6[5]);
        };
        if (T.n_child[c] == 0) {
          for (int64_t t = f; t < f + cnt; ++t)
            add_outer(T.m[t], T.x[3 * t] - cm[0], T.x[3 * t + 1] - cm[1], T.x[3 * t + 2] - cm[2]);
        } else {
          for (int j = T.first_child[c]; j < T.first_child[c] + T.n_child[c]; ++j) {
            for (int q = 0; q < 6; ++q) s6[q] += T.S[6 * j + q];
            add_outer(T.M[j], T.com[3 * j] - cm[0], T.com[3 * j + 1] - cm[1], T.com[3 * j + 2] - cm[2]);
          }
        }
      }
    });
  }

  // ---- groups: first cells from the root that are leaves or hold <= n_group.
  // Such eligibility passes from a cell to its children (a child of a leaf does
  // not exist, and a child never holds more particles than its parent), so the
  // first eligible cells on the paths from the root are the eligible cells
  // whose parent is not eligible.
  auto eligible = [&](int64_t c) { return T.n_child[c] == 0 || T.pcount[c] <= n_group; };
  {
    const int64_t chunks = parallel ? std::min<int64_t>(64, std::max<int64_t>(1, nc / 8192)) : 1;
    const int64_t step = (nc + chunks - 1) / chunks;
    std::vector<std::vector<int32_t>> found(chunks);
    std::vector<int64_t> leaves(chunks, 0);
    auto body = [&](int k) {
      for (int64_t c = k * step; c < std::min(nc, (k + 1) * step); ++c) {
        leaves[k] += T.n_child[c] == 0;
        if (eligible(c) && (c == 0 || !eligible(T.parent[c]))) found[k].push_back(static_cast<int32_t>(c));
      }
    };
    if (chunks > 1) Pool::get().run(static_cast<int>(chunks), body); else body(0);
    T.n_leaves = 0;
    for (int64_t k = 0; k < chunks; ++k) {
      T.n_leaves += leaves[k];
      T.groups.insert(T.groups.end(), found[k].begin(), found[k].end());
    }
  }
  std::sort(T.groups.begin(), T.groups.end(),
            [&](int32_t a, int32_t b) { return T.pfirst[a] < T.pfirst[b]; });
  for (int32_t g : T.groups) T.max_group = std::max(T.max_group, T.pcount[g]);
  return OCTGRAV_OK;
}

// ---------------------------------------------------------------- device buffers

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  int reserve(size_t bytes) {
    if (bytes <= cap && p) return OCTGRAV_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? OCTGRAV_ERR_OOM : OCTGRAV_ERR_CUDA,
                  "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    cap = want;
    return OCTGRAV_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct Device {
  DevBuf parts, geo, link, mp, items, ibox, sysp, out, counts, ctl, dbg, mlp;
  // GPU build: tree arrays beyond the walk's, scratch, inputs and FP64 outputs
  DevBuf perm, key, props, pcount, cfirst, groups, ikey, celloff, result, scratch, in_pos, in_mass, acc64, pot64;
  DevBuf order;  // work-item processing order (octgrav_balance)
  int device = -1;
  int pageable = -1;     // kernels may read pageable host memory (-1: not asked yet)
  int64_t cell_cap = 0;  // cell capacity that last sufficed for a GPU build
  int level_hint = 0;    // depth of the last GPU build + 2 (0: none yet), caps the next level loop
  // the GPU build's kernels captured as a graph, replayed on gstream while
  // build_key (every argument, pointers included) stays the same
  cudaGraphExec_t build_exec = nullptr;
  std::vector<int64_t> build_key;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  void release_graph() {
    if (build_exec) cudaGraphExecDestroy(build_exec);
    build_exec = nullptr;
    build_key.clear();
  }
  void release() {
    release_graph();
    if (gstream) cudaStreamDestroy(gstream);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    gstream = nullptr;
    ev_in = ev_out = nullptr;
    for (DevBuf* b : {&parts, &geo, &link, &mp, &items, &ibox, &sysp, &out, &counts, &ctl, &dbg, &mlp, &perm, &key,
                      &props, &pcount, &cfirst, &groups, &ikey, &celloff, &result, &scratch, &in_pos, &in_mass,
                      &acc64, &pot64, &order})
      b->release();
    cell_cap = 0;
  }
};

}  // namespace

// ---------------------------------------------------------------- the tree object

struct octgrav_tree {
  int64_t n = 0;
  int n_leaf = 0, n_group = 0, n_sys = 0;
  int ppl = 2, ctas_per_sm = 0;
  int stage = og::STAGING_ASYNC;
  bool learned = false;             // learned opening criterion active
  float theta_lo = 0, theta_hi = 0, theta_fb = 0;
  CUtensorMap mp_map;
  std::vector<int64_t> sys_off;   // particle offsets per system (n_sys + 1)
  std::vector<int64_t> cell_off;  // cell offsets per system (n_sys + 1)
  hvec<int64_t> perm;             // tree position -> input index
  hvec<int32_t> perm32;           // the same as int32, the device image
  hvec<uint64_t> key;             // per global cell
  std::vector<int32_t> group_cell;  // per group, global cell index
  std::vector<int32_t> group_sys;
  int64_t n_cells = 0, n_leaves = 0, max_group = 0;
  int depth_reached = 0;
  // host images of the device arrays
  hvec<float4> parts, geo, mp, ibox;
  hvec<int2> link;
  hvec<int4> items;
  hvec<uint64_t> item_key;
  // host FP64 cell properties (tests / introspection)
  hvec<double> bmin, bmax, cube, M, com, S;
  hvec<int64_t> pcount;
  hvec<int32_t> cfirst;           // first particle (tree position) of every cell
  std::vector<int32_t> group_item;  // first work item of every group
  // per-system parameters (optional)
  std::vector<float4> sysp;
  bool sysp_dirty = false;
  // device state
  Device own;
  Device* dev = &own;
  bool uploaded = false;
  bool launched = false;
  // built on the GPU: the device arrays are the tree; the host images above
  // are filled on demand (host_valid)
  bool gpu = false;
  bool host_valid = true;
  bool perm_on_device = false;  // Device::perm holds the permutation (int32)
  bool parts_on_device = false;  // Device::parts already holds (or receives) the particle records
  bool pull_images = false;      // upload may pull the host images by kernel (the one-shot call, whose
                                 // images stay unchanged until it has waited for the stream)
  int64_t n_groups = 0, n_items = 0;
  bool ordered = false;  // launches take the work items in Device::order (octgrav_balance)
  hvec<int32_t> item_order;  // host image of the default order (host-built trees)
  int64_t cell_cap = 0;  // cell capacity of the device arrays of a GPU-built tree
  cudaGraphExec_t gexec = nullptr;  // captured memset + kernel (octgrav_graph_capture)
  std::vector<SysTree> sys_scratch;
};

// N-body state for the time integration, all on one device.
struct octgrav_sim {
  int64_t n = 0;
  double eps = 0, theta = 0, G = 1;
  int n_leaf = 16, n_group = 16;
  Device dev;                        // tree and build buffers, reused every step
  DevBuf x, v, m, a, phi, epart;     // FP64 state (input order) and energy partials
  int64_t steps = 0;
  int rebuild_every = 1;             // full build every k force evaluations, refit in between
  int since_build = 0;
  octgrav_tree* tree = nullptr;      // the last built tree (its buffers live in dev)
  ~octgrav_sim();
};

namespace {

// Split every group into work items of at most 32 * ppl particles.
void make_items(octgrav_tree* t) {
  const int item_max = 32 * t->ppl;
  const int64_t ng = static_cast<int64_t>(t->group_cell.size());
  t->group_item.assign(ng, 0);
  int64_t ni = 0;
  for (int64_t g = 0; g < ng; ++g) {
    t->group_item[g] = static_cast<int32_t>(ni);
    ni += (t->pcount[t->group_cell[g]] + item_max - 1) / item_max;
  }
  t->items.resize(ni);
  t->ibox.resize(4 * ni);
  t->item_key.resize(ni);
  parallel_for(ng, 1024, [&](int64_t a, int64_t b) {
    for (int64_t g = a; g < b; ++g) {
      const int64_t c = t->group_cell[g];
      const int s = t->group_sys[g];
      const int64_t root = t->cell_off[s];
      const int64_t cnt = t->pcount[c];
      const int64_t pf = t->cfirst[c];  // first particle of the group (tree position)
      float4 bx[3];
      float chi[3], clo[3];
      for (int d = 0; d < 3; ++d) {
        const double C = t->cube[4 * c + d];
        chi[d] = static_cast<float>(C);
        clo[d] = static_cast<float>(C - static_cast<double>(chi[d]));
      }
      bx[0] = make_float4(static_cast<float>(t->bmin[3 * c]), static_cast<float>(t->bmin[3 * c + 1]),
                          static_cast<float>(t->bmin[3 * c + 2]), chi[0]);
      bx[1] = make_float4(static_cast<float>(t->bmax[3 * c]), static_cast<float>(t->bmax[3 * c + 1]),
                          static_cast<float>(t->bmax[3 * c + 2]), chi[1]);
      bx[2] = make_float4(clo[0], clo[1], clo[2], chi[2]);
      float4 grange;  // (first particle, count) of the whole group, as int bits
      const int32_t gr[2] = {static_cast<int32_t>(pf), static_cast<int32_t>(cnt)};
      std::memcpy(&grange.x, &gr[0], 4);
      std::memcpy(&grange.y, &gr[1], 4);
      grange.z = grange.w = 0.f;
      int64_t k = t->group_item[g];
      for (int64_t off = 0; off < cnt; off += item_max, ++k) {
        t->items[k] = make_int4(static_cast<int>(root), static_cast<int>(pf + off),
                                static_cast<int>(std::min<int64_t>(item_max, cnt - off)), s);
        t->ibox[4 * k] = bx[0];
        t->ibox[4 * k + 1] = bx[1];
        t->ibox[4 * k + 2] = bx[2];
        t->ibox[4 * k + 3] = grange;
        t->item_key[k] = t->key[c];
      }
    }
  });
  t->n_groups = ng;
  t->n_items = ni;
  // default processing order: most particles first (a stable counting sort by count)
  std::vector<int64_t> start(item_max + 2, 0);
  for (int64_t k = 0; k < ni; ++k) ++start[item_max - t->items[k].z + 1];
  for (int b = 1; b <= item_max + 1; ++b) start[b] += start[b - 1];
  t->item_order.resize(ni);
  for (int64_t k = 0; k < ni; ++k) t->item_order[start[item_max - t->items[k].z]++] = static_cast<int32_t>(k);
  t->ordered = true;
}

// Concatenate the systems' trees into the device-array images.
// particles_done: a one-system build already wrote perm, perm32 and parts.
int assemble(octgrav_tree* t, std::vector<SysTree>& sys, bool particles_done = false) {
  const int ns = static_cast<int>(sys.size());
  t->cell_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) t->cell_off[s + 1] = t->cell_off[s] + static_cast<int64_t>(sys[s].key.size());
  const int64_t nc = t->cell_off[ns];
  if (nc >= (1ll << 28)) return fail(OCTGRAV_ERR_ARG, "too many cells (%lld)", (long long)nc);
  t->n_cells = nc;
  // one system: its FP64 cell arrays are moved, not copied, after the loop below
  const bool single = ns == 1;
  if (!particles_done) {
    t->perm.resize(t->n);
    t->perm32.resize(t->n);
    t->parts.resize(2 * t->n);
  }
  t->geo.resize(nc);
  t->link.resize(nc);
  t->mp.resize(4 * nc);
  t->cfirst.resize(nc);
  if (!single) {
    t->key.resize(nc);
    t->bmin.resize(3 * nc);
    t->bmax.resize(3 * nc);
    t->cube.resize(4 * nc);
    t->M.resize(nc);
    t->com.resize(3 * nc);
    t->S.resize(6 * nc);
    t->pcount.resize(nc);
  }
  t->group_cell.clear();
  t->group_sys.clear();
  t->n_leaves = 0;
  t->max_group = 0;
  t->depth_reached = 0;
  for (int s = 0; s < ns; ++s) {
    SysTree& T = sys[s];
    const int64_t p0 = t->sys_off[s], c0 = t->cell_off[s];
    const int64_t n = T.n, ncs = static_cast<int64_t>(T.key.size());
    if (!particles_done)
      parallel_for(n, 16384, [&](int64_t a, int64_t b) {
        for (int64_t k = a; k < b; ++k) {
          t->perm[p0 + k] = p0 + T.perm[k];
          t->perm32[p0 + k] = static_cast<int32_t>(p0 + T.perm[k]);
          particle_records(&T.x[3 * k], T.m[k], &t->parts[2 * (p0 + k)]);
        }
      });
    parallel_for(ncs, 8192, [&](int64_t a, int64_t b) {
      for (int64_t c = a; c < b; ++c) {
        const int64_t g = c0 + c;
        if (!single) t->key[g] = T.key[c];
        const double* cu = &T.cube[4 * c];
        t->geo[g] = make_float4(static_cast<float>(cu[0]), static_cast<float>(cu[1]),
                                static_cast<float>(cu[2]), static_cast<float>(cu[3]));
        if (T.n_child[c] > 0)
          t->link[g] = make_int2(static_cast<int>(c0 + T.first_child[c]), T.n_child[c]);
        else
          t->link[g] = make_int2(static_cast<int>(p0 + T.pfirst[c]), -static_cast<int>(T.pcount[c]));
        const double* cm = &T.com[3 * c];
        const double* s6 = &T.S[6 * c];
        float chi[3], clo[3];
        for (int d = 0; d < 3; ++d) {
          chi[d] = static_cast<float>(cm[d]);
          clo[d] = static_cast<float>(cm[d] - static_cast<double>(chi[d]));
        }
        const double tr = s6[0] + s6[1] + s6[2];
        t->mp[4 * g] = make_float4(chi[0], chi[1], chi[2], static_cast<float>(T.M[c]));
        t->mp[4 * g + 1] = make_float4(clo[0], clo[1], clo[2], static_cast<float>(T.pcount[c]));
        t->mp[4 * g + 2] = make_float4(static_cast<float>(3.0 * s6[0]), static_cast<float>(3.0 * s6[1]),
                                       static_cast<float>(3.0 * s6[2]), static_cast<float>(3.0 * s6[3]));
        t->mp[4 * g + 3] = make_float4(static_cast<float>(3.0 * s6[4]), static_cast<float>(3.0 * s6[5]),
                                       static_cast<float>(1.5 * tr), static_cast<float>(0.5 * tr));
        if (!single) {
          for (int d = 0; d < 3; ++d) {
            t->bmin[3 * g + d] = T.bmin[3 * c + d];
            t->bmax[3 * g + d] = T.bmax[3 * c + d];
            t->com[3 * g + d] = cm[d];
          }
          for (int d = 0; d < 4; ++d) t->cube[4 * g + d] = cu[d];
          for (int d = 0; d < 6; ++d) t->S[6 * g + d] = s6[d];
          t->M[g] = T.M[c];
          t->pcount[g] = T.pcount[c];
        }
        t->cfirst[g] = static_cast<int32_t>(p0 + T.pfirst[c]);
      }
    });
    if (single) {  // the global arrays are this system's
      t->key = std::move(T.key);
      t->bmin = std::move(T.bmin);
      t->bmax = std::move(T.bmax);
      t->cube = std::move(T.cube);
      t->M = std::move(T.M);
      t->com = std::move(T.com);
      t->S = std::move(T.S);
      t->pcount = std::move(T.pcount);
    }
    for (int32_t gc : T.groups) {
      t->group_cell.push_back(static_cast<int32_t>(c0 + gc));
      t->group_sys.push_back(s);
    }
    t->n_leaves += T.n_leaves;
    t->max_group = std::max(t->max_group, T.max_group);
    t->depth_reached = std::max(t->depth_reached, T.depth_reached);
  }
  make_items(t);
  return OCTGRAV_OK;
}

int check_inputs(const double* pos, const double* mass, int64_t n) {
  std::atomic<int> bad{0};
  parallel_for(n, 65536, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      if (!std::isfinite(pos[3 * i]) || !std::isfinite(pos[3 * i + 1]) || !std::isfinite(pos[3 * i + 2]) ||
          !std::isfinite(mass[i]) || mass[i] < 0) {
        bad.store(1);
        return;
      }
    }
  });
  return bad.load() ? fail(OCTGRAV_ERR_NONFINITE, "non-finite position/mass or negative mass") : OCTGRAV_OK;
}

// Host memory reused by a thread's one-shot calls: the per-system build
// arrays and the tree's host images keep their pages from call to call (at
// N = 1M a call otherwise touches ~200 MB of fresh memory).
struct HostCache {
  std::vector<SysTree> sys;
  octgrav_tree spare;  // holds the image vectors between calls
};

void swap_images(octgrav_tree& a, octgrav_tree& b) {
  std::swap(a.perm, b.perm);
  std::swap(a.perm32, b.perm32);
  std::swap(a.parts, b.parts);
  std::swap(a.geo, b.geo);
  std::swap(a.link, b.link);
  std::swap(a.mp, b.mp);
  std::swap(a.items, b.items);
  std::swap(a.ibox, b.ibox);
  std::swap(a.item_key, b.item_key);
  std::swap(a.key, b.key);
  std::swap(a.bmin, b.bmin);
  std::swap(a.bmax, b.bmax);
  std::swap(a.cube, b.cube);
  std::swap(a.M, b.M);
  std::swap(a.com, b.com);
  std::swap(a.S, b.S);
  std::swap(a.pcount, b.pcount);
  std::swap(a.cfirst, b.cfirst);
  std::swap(a.group_cell, b.group_cell);
  std::swap(a.group_sys, b.group_sys);
  std::swap(a.group_item, b.group_item);
  std::swap(a.item_order, b.item_order);
}

// Return a one-shot tree's memory to the cache before the tree is freed.
void give_back(octgrav_tree* t, HostCache* cache) {
  if (cache->sys.size() == 1) {  // these were moved out of the system's arrays
    SysTree& T = cache->sys[0];
    std::swap(t->key, T.key);
    std::swap(t->bmin, T.bmin);
    std::swap(t->bmax, T.bmax);
    std::swap(t->cube, T.cube);
    std::swap(t->M, T.M);
    std::swap(t->com, T.com);
    std::swap(t->S, T.S);
    std::swap(t->pcount, T.pcount);
  }
  swap_images(*t, cache->spare);
}

int check_build_args(int n_sys, const int64_t* offsets, const double* pos, const double* mass, int n_leaf,
                     int n_group, octgrav_tree** out, bool values = true) {
  if (!out) return fail(OCTGRAV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!pos || !mass || !offsets || n_sys < 1) return fail(OCTGRAV_ERR_ARG, "NULL input or n_sys < 1");
  if (n_leaf < 1 || n_group < n_leaf) return fail(OCTGRAV_ERR_ARG, "need 1 <= n_leaf <= n_group");
  if (offsets[0] != 0) return fail(OCTGRAV_ERR_ARG, "offsets[0] must be 0");
  for (int s = 0; s < n_sys; ++s)
    if (offsets[s + 1] <= offsets[s]) return fail(OCTGRAV_ERR_ARG, "empty or decreasing system %d", s);
  if (offsets[n_sys] >= (1ll << 31) - 64) return fail(OCTGRAV_ERR_ARG, "too many particles");
  return values ? check_inputs(pos, mass, offsets[n_sys]) : OCTGRAV_OK;
}

int build_common(int n_sys, const int64_t* offsets, const double* pos, const double* mass, int n_leaf,
                 int n_group, octgrav_tree** out, HostCache* cache = nullptr) {
  int rc = check_build_args(n_sys, offsets, pos, mass, n_leaf, n_group, out);
  if (rc) return rc;
  const int64_t n = offsets[n_sys];
  std::unique_ptr<octgrav_tree> t;
  try {
    t.reset(new octgrav_tree());
    t->n = n;
    t->n_leaf = n_leaf;
    t->n_group = n_group;
    t->n_sys = n_sys;
    t->sys_off.assign(offsets, offsets + n_sys + 1);
    std::vector<SysTree> local;
    std::vector<SysTree>& sys = cache ? cache->sys : local;
    sys.resize(n_sys);  // build_system empties each (reused memory stays)
    if (cache) swap_images(*t, cache->spare);
    std::vector<int> rcs(n_sys, 0);
    if (n_sys == 1) {
      rcs[0] = build_system(pos, mass, n, n_leaf, n_group, true, sys[0]);
    } else {
      Pool::get().run(n_sys, [&](int s) {
        const int64_t o = offsets[s];
        rcs[s] = build_system(pos + 3 * o, mass + o, offsets[s + 1] - o, n_leaf, n_group, false, sys[s]);
      });
    }
    for (int s = 0; s < n_sys; ++s)
      if (rcs[s]) return rcs[s];
    rc = assemble(t.get(), sys);
    if (rc) return rc;
  } catch (const std::bad_alloc&) {
    return fail(OCTGRAV_ERR_OOM, "host allocation failed");
  }
  *out = t.release();
  return OCTGRAV_OK;
}

template <class V>
int upload_vec(DevBuf& b, const V& v, cudaStream_t st) {
  const size_t bytes = v.size() * sizeof(typename V::value_type);
  int rc = b.reserve(bytes);
  if (rc) return rc;
  if (bytes) CUDA_TRY(cudaMemcpyAsync(b.p, v.data(), bytes, cudaMemcpyHostToDevice, st));
  return OCTGRAV_OK;
}

// Copy host memory to a device buffer. Where the device reads pageable host
// memory (NVLink-C2C on Grace systems) a kernel pulls it and the call returns at
// once; otherwise cudaMemcpyAsync, which returns when the source has been read.
int enqueue_h2d(Device& D, DevBuf& b, const void* src, size_t bytes, cudaStream_t st, bool* async) {
  int rc = b.reserve(bytes);
  if (rc || !bytes) return rc;
  if (D.pageable < 0) {
    int v = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, D.device));
    D.pageable = v ? 1 : 0;
  }
  const bool aligned = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(b.p) | bytes) & 15u) == 0;
  if (D.pageable == 1 && aligned) {
    cudaError_t e = og::pull_host(b.p, src, bytes, st);
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "host pull failed: %s", cudaGetErrorString(e));
    *async = true;
    return OCTGRAV_OK;
  }
  CUDA_TRY(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st));
  return OCTGRAV_OK;
}

// The one-shot call's build (one system, cached host arrays): the particle
// records and the permutation are written during the gather and start their
// way to the device (on st) while the cells are built. On return with an error
// nothing is still reading the host arrays.
int build_oneshot(const double* pos, const double* mass, int64_t n, int n_leaf, int n_group, HostCache& cache,
                  Device& D, cudaStream_t st, octgrav_tree** out) {
  const int64_t off[2] = {0, n};
  int rc = check_build_args(1, off, pos, mass, n_leaf, n_group, out, false);  // values: in the bbox pass
  if (rc) return rc;
  std::unique_ptr<octgrav_tree> t;
  bool async = false;
  try {
    t.reset(new octgrav_tree());
    t->n = n;
    t->n_leaf = n_leaf;
    t->n_group = n_group;
    t->n_sys = 1;
    t->sys_off.assign(off, off + 2);
    t->dev = &D;
    cache.sys.resize(1);
    swap_images(*t, cache.spare);
    t->perm.resize(n);
    t->perm32.resize((n + 3) & ~int64_t{3});  // whole 16-byte units for the pull
    t->parts.resize(2 * n);
    ParticleSink sink;
    sink.parts = t->parts.data();
    sink.perm = t->perm.data();
    sink.perm32 = t->perm32.data();
    sink.check_inputs = true;
    sink.ready = [&]() -> int {
      int dev = 0;
      CUDA_TRY(cudaGetDevice(&dev));
      if (D.device >= 0 && D.device != dev) D.release();
      if (D.device != dev) D.pageable = -1;
      D.device = dev;
      int r = enqueue_h2d(D, D.parts, t->parts.data(), sizeof(float4) * t->parts.size(), st, &async);
      if (!r) r = enqueue_h2d(D, D.perm, t->perm32.data(), sizeof(int32_t) * t->perm32.size(), st, &async);
      return r;
    };
    rc = build_system(pos, mass, n, n_leaf, n_group, true, cache.sys[0], &sink);
    if (!rc) rc = assemble(t.get(), cache.sys, true);
  } catch (const std::bad_alloc&) {
    rc = fail(OCTGRAV_ERR_OOM, "host allocation failed");
  }
  if (rc) {
    if (async) cudaStreamSynchronize(st);
    if (t) give_back(t.get(), &cache);
    return rc;
  }
  t->parts_on_device = true;
  t->perm_on_device = true;
  t->pull_images = true;
  *out = t.release();
  return OCTGRAV_OK;
}


int upload(octgrav_tree* t, cudaStream_t st) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  Device& D = *t->dev;
  if (D.device >= 0 && D.device != dev) {
    D.release();
  }
  D.device = dev;
  int rc;
  if (!t->gpu) {  // a GPU-built tree already lives in these arrays
    if (!t->parts_on_device &&
        ((rc = upload_vec(D.parts, t->parts, st)) || (rc = upload_vec(D.perm, t->perm32, st))))
      return rc;
    t->parts_on_device = false;  // a later re-upload copies them again
    if (t->pull_images) {
      bool async = false;
      if ((rc = enqueue_h2d(D, D.geo, t->geo.data(), sizeof(float4) * t->geo.size(), st, &async)) ||
          (rc = enqueue_h2d(D, D.link, t->link.data(), sizeof(int2) * t->link.size(), st, &async)) ||
          (rc = enqueue_h2d(D, D.mp, t->mp.data(), sizeof(float4) * t->mp.size(), st, &async)) ||
          (rc = enqueue_h2d(D, D.items, t->items.data(), sizeof(int4) * t->items.size(), st, &async)) ||
          (rc = enqueue_h2d(D, D.ibox, t->ibox.data(), sizeof(float4) * t->ibox.size(), st, &async)) ||
          (rc = enqueue_h2d(D, D.order, t->item_order.data(), sizeof(int32_t) * t->item_order.size(), st, &async)))
        return rc;
    } else if ((rc = upload_vec(D.geo, t->geo, st)) || (rc = upload_vec(D.link, t->link, st)) ||
               (rc = upload_vec(D.mp, t->mp, st)) || (rc = upload_vec(D.items, t->items, st)) ||
               (rc = upload_vec(D.ibox, t->ibox, st)) || (rc = upload_vec(D.order, t->item_order, st))) {
      return rc;
    }
    t->perm_on_device = true;
  }
  if ((rc = D.counts.reserve(t->n_items * sizeof(int2)))) return rc;
  if ((rc = D.ctl.reserve(64))) return rc;
  {
    cudaError_t e = og::encode_mp_map(&t->mp_map, D.mp.p, static_cast<int>(t->n_cells));
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "tensor map encode failed: %s", cudaGetErrorString(e));
  }
  if (!t->sysp.empty()) {
    if ((rc = upload_vec(D.sysp, t->sysp, st))) return rc;
  }
  t->sysp_dirty = false;
  t->uploaded = true;
  return OCTGRAV_OK;
}

int check_params(double eps, double theta, double G) {
  if (!(eps > 0) || !std::isfinite(eps)) return fail(OCTGRAV_ERR_ARG, "eps must be finite and > 0");
  if (!(theta >= 0) || !std::isfinite(theta)) return fail(OCTGRAV_ERR_ARG, "theta must be finite and >= 0");
  if (!std::isfinite(G)) return fail(OCTGRAV_ERR_ARG, "G must be finite");
  return OCTGRAV_OK;
}

og::KParams make_params(octgrav_tree* t, float4* out) {
  Device& D = *t->dev;
  og::KParams p{};
  p.parts = static_cast<const float4*>(D.parts.p);
  p.geo = static_cast<const float4*>(D.geo.p);
  p.link = static_cast<const int2*>(D.link.p);
  p.mp = static_cast<const float4*>(D.mp.p);
  p.items = static_cast<const int4*>(D.items.p);
  p.ibox = static_cast<const float4*>(D.ibox.p);
  p.sysp = t->sysp.empty() ? nullptr : static_cast<const float4*>(D.sysp.p);
  p.out = out;
  p.counts = static_cast<int2*>(D.counts.p);
  p.status = static_cast<int*>(D.ctl.p);
  p.work = reinterpret_cast<unsigned*>(static_cast<char*>(D.ctl.p) + 4);
  p.n_items = static_cast<int>(t->n_items);
  p.n_cells = static_cast<int>(t->n_cells);
  p.order = t->ordered ? static_cast<const int*>(D.order.p) : nullptr;
  p.stage = t->stage;
  p.mp_map = t->mp_map;
  p.n_group = t->n_group;
  if (t->learned) {
    p.mlp = static_cast<const og::MlpDevice*>(D.mlp.p);
    p.theta_lo2 = static_cast<float>(static_cast<double>(t->theta_lo) * t->theta_lo);
    p.theta_hi2 = static_cast<float>(static_cast<double>(t->theta_hi) * t->theta_hi);
    p.theta_fb2 = static_cast<float>(static_cast<double>(t->theta_fb) * t->theta_fb);
  }
  return p;
}

int launch(octgrav_tree* t, double eps, double theta, double G, float4* out, cudaStream_t st,
           bool capture, int* dbg_cell, int* dbg_leaf, int2* dbg_n, int dbg_cap) {
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  if (!t->uploaded || t->sysp_dirty) {
    if ((rc = upload(t, st))) return rc;
  }
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != t->dev->device) return fail(OCTGRAV_ERR_STATE, "tree was uploaded to device %d, current is %d",
                                         t->dev->device, dev);
  og::KParams p = make_params(t, out);
  p.sys0 = make_float4(static_cast<float>(theta * theta), static_cast<float>(eps * eps), static_cast<float>(G), 0.f);
  if (capture) {
    p.dbg_cell = dbg_cell;
    p.dbg_leaf = dbg_leaf;
    p.dbg_n = dbg_n;
    p.dbg_cap = dbg_cap;
  }
  CUDA_TRY(cudaMemsetAsync(t->dev->ctl.p, 0, 8, st));
  if (p.n_items > 0) {
    cudaError_t e = og::launch_walk_eval(p, t->ppl, t->ctas_per_sm, capture, st, nullptr);
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  }
  t->launched = true;
  return OCTGRAV_OK;
}

int read_status(octgrav_tree* t, cudaStream_t st) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, t->dev->ctl.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (h & og::ST_TIMEOUT) return fail(OCTGRAV_ERR_TIMEOUT, "device wait timed out (status %d)", h);
  if (h & og::ST_INDEX) return fail(OCTGRAV_ERR_INDEX, "walk met an out-of-range cell index");
  if (h & og::ST_STACK) return fail(OCTGRAV_ERR_STACK, "walk overflowed its node stack");
  return OCTGRAV_OK;
}

// The permutation on the device (int32); uploaded once for a host-built tree.
int device_perm(octgrav_tree* t, cudaStream_t st) {
  if (t->gpu || t->perm_on_device) return OCTGRAV_OK;
  if (static_cast<int64_t>(t->perm32.size()) != t->n) {
    t->perm32.resize(t->n);
    parallel_for(t->n, 65536, [&](int64_t a, int64_t b) {
      for (int64_t k = a; k < b; ++k) t->perm32[k] = static_cast<int32_t>(t->perm[k]);
    });
  }
  int rc = upload_vec(t->dev->perm, t->perm32, st);
  if (rc) return rc;
  t->perm_on_device = true;
  return OCTGRAV_OK;
}

// Forces into device FP64 arrays in input order (enqueued, not waited for).
int forces_dev64(octgrav_tree* t, double eps, double theta, double G, double* acc, double* pot, cudaStream_t st) {
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  if (!t->uploaded || t->sysp_dirty) {
    if ((rc = upload(t, st))) return rc;
  }
  if ((rc = t->dev->out.reserve(sizeof(float4) * t->n))) return rc;
  if ((rc = device_perm(t, st))) return rc;
  if ((rc = launch(t, eps, theta, G, static_cast<float4*>(t->dev->out.p), st, false, nullptr, nullptr, nullptr, 0)))
    return rc;
  cudaError_t e = og::gpu_unpermute(static_cast<const float4*>(t->dev->out.p), static_cast<const int*>(t->dev->perm.p),
                                    t->n, acc, pot, st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "unpermute launch failed: %s", cudaGetErrorString(e));
  return OCTGRAV_OK;
}

int forces_host(octgrav_tree* t, double eps, double theta, double G, double* acc, double* pot,
                cudaStream_t st) {
  if (!acc) return fail(OCTGRAV_ERR_ARG, "acc is NULL");
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  // unpermute on the device, copy FP64 results straight into the caller's arrays
  Device& D = *t->dev;
  if ((rc = D.acc64.reserve(24 * t->n)) || (rc = D.pot64.reserve(8 * t->n))) return rc;
  if ((rc = forces_dev64(t, eps, theta, G, static_cast<double*>(D.acc64.p), static_cast<double*>(D.pot64.p), st)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(acc, D.acc64.p, 24 * t->n, cudaMemcpyDeviceToHost, st));
  if (pot) CUDA_TRY(cudaMemcpyAsync(pot, D.pot64.p, 8 * t->n, cudaMemcpyDeviceToHost, st));
  return read_status(t, st);
}

// The one-shot calls' device buffers, one set per calling thread, released
// when the thread ends.
struct ThreadDevice {
  Device* d = nullptr;
  Device& get() {
    if (!d) d = new Device();
    return *d;
  }
  ~ThreadDevice() {
    if (d) d->release();
    delete d;
  }
};
thread_local ThreadDevice tl_device;

// ---------------------------------------------------------------- GPU build

og::GpuBuild gpu_args(octgrav_tree* t, const int64_t* offsets, const double* pos, const double* mass) {
  Device& D = *t->dev;
  const int64_t n = t->n, cap = t->cell_cap;
  og::GpuBuild a{};
  a.pos = pos;
  a.mass = mass;
  a.n = n;
  a.n_sys = t->n_sys;
  a.offsets = offsets;
  a.n_leaf = t->n_leaf;
  a.n_group = t->n_group;
  a.item_max = 32 * t->ppl;
  a.max_level = OCTGRAV_MAX_DEPTH;
  a.cap = cap;
  a.scratch = D.scratch.p;
  a.scratch_bytes = D.scratch.cap;
  a.parts = static_cast<float4*>(D.parts.p);
  a.perm = static_cast<int*>(D.perm.p);
  a.key = static_cast<uint64_t*>(D.key.p);
  a.geo = static_cast<float4*>(D.geo.p);
  a.link = static_cast<int2*>(D.link.p);
  a.mp = static_cast<float4*>(D.mp.p);
  double* pr = static_cast<double*>(D.props.p);  // bmin 3 | bmax 3 | cube 4 | M 1 | com 3 | S 6 (x cap)
  a.bmin = pr;
  a.bmax = pr + 3 * cap;
  a.cube = pr + 6 * cap;
  a.M = pr + 10 * cap;
  a.com = pr + 11 * cap;
  a.S = pr + 14 * cap;
  a.pcount = static_cast<int*>(D.pcount.p);
  a.cfirst = static_cast<int*>(D.cfirst.p);
  int* gb = static_cast<int*>(D.groups.p);  // group cell | group system | first item (x n)
  a.group_cell = gb;
  a.group_sys = gb + n;
  a.group_item = gb + 2 * n;
  a.items = static_cast<int4*>(D.items.p);
  a.ibox = static_cast<float4*>(D.ibox.p);
  a.item_key = static_cast<uint64_t*>(D.ikey.p);
  a.order = static_cast<int*>(D.order.p);
  a.cell_off = static_cast<int64_t*>(D.celloff.p);
  a.result = static_cast<int64_t*>(D.result.p);
  return a;
}

int reserve_gpu_tree(Device& D, int64_t n, int n_sys, int64_t cap) {
  int rc;
  if ((rc = D.parts.reserve(32 * n)) || (rc = D.perm.reserve(4 * n)) || (rc = D.key.reserve(8 * cap)) ||
      (rc = D.geo.reserve(16 * cap)) || (rc = D.link.reserve(8 * cap)) || (rc = D.mp.reserve(64 * cap)) ||
      (rc = D.props.reserve(160 * cap)) || (rc = D.pcount.reserve(4 * cap)) || (rc = D.cfirst.reserve(4 * cap)) ||
      (rc = D.groups.reserve(12 * n)) || (rc = D.items.reserve(16 * n)) || (rc = D.ibox.reserve(64 * n)) ||
      (rc = D.ikey.reserve(8 * n)) || (rc = D.order.reserve(4 * n)) || (rc = D.celloff.reserve(8 * (n_sys + 1))) ||
      (rc = D.result.reserve(8 * og::GB_COUNT)) || (rc = D.scratch.reserve(og::gpu_build_scratch_bytes(n, n_sys, cap))))
    return rc;
  return OCTGRAV_OK;
}

// Every argument of a GPU build (pointers included) and the system offsets:
// a captured build graph is valid while this stays the same.
std::vector<int64_t> build_key(const og::GpuBuild& a) {
  auto P = [](const void* q) { return static_cast<int64_t>(reinterpret_cast<uintptr_t>(q)); };
  std::vector<int64_t> k = {P(a.pos),     P(a.mass),     a.n,           a.n_sys,       a.n_leaf,       a.n_group,
                            a.item_max,   a.max_level,   a.cap,         P(a.scratch),  static_cast<int64_t>(a.scratch_bytes),
                            P(a.parts),   P(a.perm),     P(a.key),      P(a.geo),      P(a.link),      P(a.mp),
                            P(a.bmin),    P(a.bmax),     P(a.cube),     P(a.M),        P(a.com),       P(a.S),
                            P(a.pcount),  P(a.cfirst),   P(a.group_cell), P(a.group_sys), P(a.group_item),
                            P(a.items),   P(a.ibox),     P(a.item_key), P(a.order),    P(a.cell_off),  P(a.result)};
  k.insert(k.end(), a.offsets, a.offsets + a.n_sys + 1);
  return k;
}

// Enqueue a GPU build on st. The kernels are captured once into a graph and
// replayed on the device's own stream (ordered after and before st by
// events) while the arguments stay the same: ~125 small launches become one.
int run_build(Device& D, const og::GpuBuild& a, cudaStream_t st, bool use_graph) {
  cudaError_t e;
  if (!use_graph) {  // a one-off build: capturing would cost more than it saves
    if ((e = og::gpu_build(a, st)) != cudaSuccess)
      return fail(OCTGRAV_ERR_CUDA, "GPU build launch failed: %s", cudaGetErrorString(e));
    return OCTGRAV_OK;
  }
  if (!D.gstream) {
    CUDA_TRY(cudaStreamCreateWithFlags(&D.gstream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&D.ev_in, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&D.ev_out, cudaEventDisableTiming));
  }
  std::vector<int64_t> key = build_key(a);
  if (!D.build_exec || key != D.build_key) {
    D.release_graph();
    if ((e = og::gpu_build_tables(a, st)) != cudaSuccess)
      return fail(OCTGRAV_ERR_CUDA, "GPU build tables: %s", cudaGetErrorString(e));
    CUDA_TRY(cudaStreamBeginCapture(D.gstream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t ek = og::gpu_build_kernels(a, D.gstream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(D.gstream, &g);
    if (ek == cudaSuccess && e == cudaSuccess) e = cudaGraphInstantiate(&D.build_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ek != cudaSuccess || e != cudaSuccess) {  // not capturable here: run the kernels directly
      D.build_exec = nullptr;
      cudaGetLastError();
      if ((e = og::gpu_build_kernels(a, st)) != cudaSuccess)
        return fail(OCTGRAV_ERR_CUDA, "GPU build launch failed: %s", cudaGetErrorString(e));
      return OCTGRAV_OK;
    }
    D.build_key = std::move(key);
  }
  CUDA_TRY(cudaEventRecord(D.ev_in, st));
  CUDA_TRY(cudaStreamWaitEvent(D.gstream, D.ev_in, 0));
  CUDA_TRY(cudaGraphLaunch(D.build_exec, D.gstream));
  CUDA_TRY(cudaEventRecord(D.ev_out, D.gstream));
  CUDA_TRY(cudaStreamWaitEvent(st, D.ev_out, 0));
  return OCTGRAV_OK;
}

// Read the result block of a GPU build (waits for the stream).
int gpu_result(octgrav_tree* t, cudaStream_t st, int64_t* res) {
  CUDA_TRY(cudaMemcpyAsync(res, t->dev->result.p, 8 * og::GB_COUNT, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return OCTGRAV_OK;
}

int build_gpu_common(int n_sys, const int64_t* offsets, const double* pos, const double* mass, int n_leaf,
                     int n_group, cudaStream_t st, Device* dev, octgrav_tree** out) {
  if (!out) return fail(OCTGRAV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!pos || !mass || !offsets || n_sys < 1) return fail(OCTGRAV_ERR_ARG, "NULL input or n_sys < 1");
  if (n_leaf < 1 || n_group < n_leaf) return fail(OCTGRAV_ERR_ARG, "need 1 <= n_leaf <= n_group");
  if (offsets[0] != 0) return fail(OCTGRAV_ERR_ARG, "offsets[0] must be 0");
  for (int s = 0; s < n_sys; ++s)
    if (offsets[s + 1] <= offsets[s]) return fail(OCTGRAV_ERR_ARG, "empty or decreasing system %d", s);
  const int64_t n = offsets[n_sys];
  if (n >= (1ll << 31) - 64) return fail(OCTGRAV_ERR_ARG, "too many particles");
  std::unique_ptr<octgrav_tree> t;
  try {
    t.reset(new octgrav_tree());
    t->sys_off.assign(offsets, offsets + n_sys + 1);
  } catch (const std::bad_alloc&) {
    return fail(OCTGRAV_ERR_OOM, "host allocation failed");
  }
  t->n = n;
  t->n_leaf = n_leaf;
  t->n_group = n_group;
  t->n_sys = n_sys;
  t->gpu = true;
  t->host_valid = false;
  if (dev) t->dev = dev;
  Device& D = *t->dev;
  int cur = 0;
  CUDA_TRY(cudaGetDevice(&cur));
  if (D.device >= 0 && D.device != cur) D.release();
  D.device = cur;
  // every level holds at most n cells (they are disjoint and non-empty)
  const int64_t bound = std::min<int64_t>(22 * n + n_sys, (1ll << 28) - 1);
  int64_t cap = D.cell_cap > 0 ? D.cell_cap : 8 * n / (n_leaf + 1) + 64 * static_cast<int64_t>(n_sys) + 1024;
  if (const char* e = getenv("OCTGRAV_GPU_CELL_CAP")) {
    const long long v = atoll(e);
    if (v > 0) cap = v;
  }
  cap = std::min(std::max<int64_t>(cap, n_sys + 8), bound);  // the roots always fit
  int64_t res[og::GB_COUNT];
  int rc;
  // repeated builds on cached buffers stop the level loop two levels below the
  // previous tree's depth; a deeper tree is detected on the device and rebuilt
  int max_level = dev && D.level_hint > 0 ? std::min(D.level_hint, kMaxDepth) : kMaxDepth;
  for (;;) {
    if ((rc = reserve_gpu_tree(D, n, n_sys, cap))) return rc;
    t->cell_cap = cap;
    og::GpuBuild a = gpu_args(t.get(), offsets, pos, mass);
    a.max_level = max_level;
    if ((rc = run_build(D, a, st, dev != nullptr))) return rc;  // cached buffers: replay a graph
    if ((rc = gpu_result(t.get(), st, res))) return rc;
    if (res[og::GB_STATUS] & og::GPU_BUILD_BADINPUT)
      return fail(OCTGRAV_ERR_NONFINITE, "non-finite position/mass or negative mass");
    if ((res[og::GB_STATUS] & og::GPU_BUILD_DEEPER) && max_level < kMaxDepth) {
      max_level = kMaxDepth;
      continue;
    }
    if (!(res[og::GB_STATUS] & og::GPU_BUILD_OVERFLOW)) break;
    if (cap >= bound) return fail(OCTGRAV_ERR_ARG, "tree too large (more than %lld cells)", (long long)bound);
    cap = std::min(bound, 4 * cap);
  }
  D.cell_cap = cap;
  D.level_hint = static_cast<int>(std::min<int64_t>(kMaxDepth, res[og::GB_DEPTH] + 2));
  t->n_cells = res[og::GB_NCELLS];
  t->n_groups = res[og::GB_NGROUPS];
  t->n_items = res[og::GB_NITEMS];
  t->depth_reached = static_cast<int>(res[og::GB_DEPTH]);
  t->n_leaves = res[og::GB_NLEAVES];
  t->max_group = res[og::GB_MAXGROUP];
  t->ordered = true;  // the build wrote the default order (most particles first)
  t->cell_off.resize(n_sys + 1);
  CUDA_TRY(cudaMemcpy(t->cell_off.data(), D.celloff.p, 8 * (n_sys + 1), cudaMemcpyDeviceToHost));
  if ((rc = upload(t.get(), st))) return rc;  // counts, control word, tensor map
  *out = t.release();
  return OCTGRAV_OK;
}

// Fill the host images of a GPU-built tree (introspection and host-side paths).
int host_images(octgrav_tree* t) {
  if (!t->gpu || t->host_valid) return OCTGRAV_OK;
  Device& D = *t->dev;
  const int64_t n = t->n, nc = t->n_cells, ng = t->n_groups, ni = t->n_items, cap = t->cell_cap;
  std::vector<int32_t> p32, c32, g32;
  try {
    t->parts.resize(2 * n);
    t->geo.resize(nc);
    t->link.resize(nc);
    t->mp.resize(4 * nc);
    t->items.resize(ni);
    t->ibox.resize(4 * ni);
    t->item_key.resize(ni);
    t->key.resize(nc);
    t->perm.resize(n);
    t->bmin.resize(3 * nc);
    t->bmax.resize(3 * nc);
    t->cube.resize(4 * nc);
    t->M.resize(nc);
    t->com.resize(3 * nc);
    t->S.resize(6 * nc);
    t->pcount.resize(nc);
    t->cfirst.resize(nc);
    t->group_cell.resize(ng);
    t->group_sys.resize(ng);
    t->group_item.resize(ng);
    p32.resize(n);
    c32.resize(nc);
  } catch (const std::bad_alloc&) {
    return fail(OCTGRAV_ERR_OOM, "host allocation failed");
  }
  const double* pr = static_cast<const double*>(D.props.p);
  const int* gb = static_cast<const int*>(D.groups.p);
  const size_t zn = n, znc = nc, zni = ni, zng = ng;
  struct Copy {
    void* dst;
    const void* src;
    size_t bytes;
  } copies[] = {
      {t->parts.data(), D.parts.p, 32 * zn},         {t->geo.data(), D.geo.p, 16 * znc},
      {t->link.data(), D.link.p, 8 * znc},           {t->mp.data(), D.mp.p, 64 * znc},
      {t->items.data(), D.items.p, 16 * zni},        {t->ibox.data(), D.ibox.p, 64 * zni},
      {t->item_key.data(), D.ikey.p, 8 * zni},       {t->key.data(), D.key.p, 8 * znc},
      {p32.data(), D.perm.p, 4 * zn},                {t->bmin.data(), pr, 24 * znc},
      {t->bmax.data(), pr + 3 * cap, 24 * znc},      {t->cube.data(), pr + 6 * cap, 32 * znc},
      {t->M.data(), pr + 10 * cap, 8 * znc},         {t->com.data(), pr + 11 * cap, 24 * znc},
      {t->S.data(), pr + 14 * cap, 48 * znc},        {c32.data(), D.pcount.p, 4 * znc},
      {t->cfirst.data(), D.cfirst.p, 4 * znc},       {t->group_cell.data(), gb, 4 * zng},
      {t->group_sys.data(), gb + n, 4 * zng},        {t->group_item.data(), gb + 2 * n, 4 * zng},
  };
  for (const Copy& c : copies)
    if (c.bytes) CUDA_TRY(cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost));
  for (int64_t k = 0; k < n; ++k) t->perm[k] = p32[k];
  for (int64_t c = 0; c < nc; ++c) t->pcount[c] = c32[c];
  t->host_valid = true;
  return OCTGRAV_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

int octgrav_version(void) { return 10000; }

const char* octgrav_last_error(void) { return g_err.c_str(); }

int octgrav_build_tree(const double* pos, const double* mass, int64_t n, int n_leaf, int n_group,
                       octgrav_tree** out) {
  if (n < 1) return fail(OCTGRAV_ERR_ARG, "n must be >= 1");
  const int64_t off[2] = {0, n};
  return build_common(1, off, pos, mass, n_leaf, n_group, out);
}

int octgrav_build_batch(int n_sys, const int64_t* offsets, const double* pos, const double* mass, int n_leaf,
                        int n_group, octgrav_tree** out) {
  return build_common(n_sys, offsets, pos, mass, n_leaf, n_group, out);
}

int octgrav_tree_upload(octgrav_tree* t, void* stream) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  return upload(t, static_cast<cudaStream_t>(stream));
}

int octgrav_forces_device(octgrav_tree* t, double eps, double theta, double G, float* acc4_dev, void* stream) {
  if (!t || !acc4_dev) return fail(OCTGRAV_ERR_ARG, "NULL tree or output");
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  return launch(t, eps, theta, G, reinterpret_cast<float4*>(acc4_dev), static_cast<cudaStream_t>(stream), false,
                nullptr, nullptr, nullptr, 0);
}

int octgrav_set_system_params(octgrav_tree* t, const double* eps, const double* theta) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (!eps && !theta) {
    t->sysp.clear();
    return OCTGRAV_OK;
  }
  if (!eps || !theta) return fail(OCTGRAV_ERR_ARG, "give both eps and theta, or neither");
  std::vector<float4> sp(t->n_sys);
  for (int s = 0; s < t->n_sys; ++s) {
    int rc = check_params(eps[s], theta[s], 1.0);
    if (rc) return rc;
    sp[s] = make_float4(static_cast<float>(theta[s] * theta[s]), static_cast<float>(eps[s] * eps[s]), 1.f, 0.f);
  }
  t->sysp = std::move(sp);
  t->sysp_dirty = true;
  return OCTGRAV_OK;
}

int octgrav_forces_tree(octgrav_tree* t, double eps, double theta, double G, double* acc, double* pot,
                        void* stream) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  return forces_host(t, eps, theta, G, acc, pot, static_cast<cudaStream_t>(stream));
}

int octgrav_forces_ex(const double* pos, const double* mass, int64_t n, double eps, double theta, double G,
                      int n_leaf, int n_group, double* acc, double* pot, void* stream) {
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  if (n < 1) return fail(OCTGRAV_ERR_ARG, "n must be >= 1");
  thread_local HostCache hcache;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  octgrav_tree* t = nullptr;
  if ((rc = build_oneshot(pos, mass, n, n_leaf, n_group, hcache, tl_device.get(), st, &t))) return rc;
  rc = forces_host(t, eps, theta, G, acc, pot, st);
  if (rc) cudaStreamSynchronize(st);  // nothing may still read the cached host arrays
  give_back(t, &hcache);
  octgrav_free_tree(t);
  return rc;
}

int octgrav_forces(const double* pos, const double* mass, int64_t n, double eps, double theta, int n_leaf,
                   double* acc, double* pot) {
  return octgrav_forces_ex(pos, mass, n, eps, theta, 1.0, n_leaf, n_leaf, acc, pot, nullptr);
}

int octgrav_build_tree_gpu(const double* pos_dev, const double* mass_dev, int64_t n, int n_leaf, int n_group,
                           void* stream, octgrav_tree** out) {
  if (n < 1) return fail(OCTGRAV_ERR_ARG, "n must be >= 1");
  const int64_t off[2] = {0, n};
  return build_gpu_common(1, off, pos_dev, mass_dev, n_leaf, n_group, static_cast<cudaStream_t>(stream), nullptr, out);
}

int octgrav_build_batch_gpu(int n_sys, const int64_t* offsets, const double* pos_dev, const double* mass_dev,
                            int n_leaf, int n_group, void* stream, octgrav_tree** out) {
  return build_gpu_common(n_sys, offsets, pos_dev, mass_dev, n_leaf, n_group, static_cast<cudaStream_t>(stream),
                          nullptr, out);
}

int octgrav_forces_tree_device64(octgrav_tree* t, double eps, double theta, double G, double* acc_dev,
                                 double* pot_dev, void* stream) {
  if (!t || !acc_dev) return fail(OCTGRAV_ERR_ARG, "NULL tree or output");
  return forces_dev64(t, eps, theta, G, acc_dev, pot_dev, static_cast<cudaStream_t>(stream));
}

int octgrav_forces_gpu(const double* pos, const double* mass, int64_t n, double eps, double theta, double G,
                       int n_leaf, int n_group, double* acc, double* pot, void* stream) {
  if (!pos || !mass || !acc) return fail(OCTGRAV_ERR_ARG, "NULL input or output");
  if (n < 1) return fail(OCTGRAV_ERR_ARG, "n must be >= 1");
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Device& D = tl_device.get();
  int cur = 0;
  CUDA_TRY(cudaGetDevice(&cur));
  if (D.device >= 0 && D.device != cur) D.release();
  D.device = cur;
  if ((rc = D.in_pos.reserve(24 * n)) || (rc = D.in_mass.reserve(8 * n))) return rc;
  CUDA_TRY(cudaMemcpyAsync(D.in_pos.p, pos, 24 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(D.in_mass.p, mass, 8 * n, cudaMemcpyHostToDevice, st));
  const int64_t off[2] = {0, n};
  octgrav_tree* t = nullptr;
  if ((rc = build_gpu_common(1, off, static_cast<const double*>(D.in_pos.p), static_cast<const double*>(D.in_mass.p),
                             n_leaf, n_group, st, &D, &t)))
    return rc;
  rc = forces_host(t, eps, theta, G, acc, pot, st);
  octgrav_free_tree(t);
  return rc;
}

int octgrav_direct(const double* pos, const double* mass, int64_t n, const int64_t* targets, int64_t nt,
                   double eps, double G, double* acc, double* pot, void* stream) {
  if (!pos || !mass || !acc || !pot || n < 1 || nt < 0) return fail(OCTGRAV_ERR_ARG, "bad argument");
  if (!(eps >= 0) || !std::isfinite(eps) || !std::isfinite(G)) return fail(OCTGRAV_ERR_ARG, "need finite eps >= 0, G");
  if (!targets && nt > n) return fail(OCTGRAV_ERR_ARG, "nt > n without targets");
  if (targets)
    for (int64_t k = 0; k < nt; ++k)
      if (targets[k] < 0 || targets[k] >= n) return fail(OCTGRAV_ERR_ARG, "target %lld out of range", (long long)k);
  if (nt == 0) return OCTGRAV_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf dp, dm, dt, dpart, da, dpot;
  int rc;
  if ((rc = dp.reserve(24 * n)) || (rc = dm.reserve(8 * n)) || (rc = dt.reserve(targets ? 8 * nt : 8)) ||
      (rc = dpart.reserve(32 * og::direct_chunks(n) * nt)) || (rc = da.reserve(24 * nt)) || (rc = dpot.reserve(8 * nt)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(dp.p, pos, 24 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(dm.p, mass, 8 * n, cudaMemcpyHostToDevice, st));
  if (targets) CUDA_TRY(cudaMemcpyAsync(dt.p, targets, 8 * nt, cudaMemcpyHostToDevice, st));
  cudaError_t e = og::direct_sum(static_cast<const double*>(dp.p), static_cast<const double*>(dm.p), n,
                                 targets ? static_cast<const int64_t*>(dt.p) : nullptr, nt, eps, G,
                                 static_cast<double*>(dpart.p), static_cast<double*>(da.p),
                                 static_cast<double*>(dpot.p), st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "direct-sum launch failed: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaMemcpyAsync(acc, da.p, 24 * nt, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(pot, dpot.p, 8 * nt, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (DevBuf* b : {&dp, &dm, &dt, &dpart, &da, &dpot}) b->release();
  return OCTGRAV_OK;
}

// ---- time integration

namespace {

// Refit a GPU-built tree to new positions and masses (device arrays) on the
// scratch of its build; waits for the stream.
int refit_tree(octgrav_tree* t, const double* pos, const double* mass, cudaStream_t st) {
  const og::GpuBuild a = gpu_args(t, t->sys_off.data(), pos, mass);
  cudaError_t e = og::gpu_refit(a, st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "refit launch failed: %s", cudaGetErrorString(e));
  int64_t res[og::GB_COUNT];
  if (int rc = gpu_result(t, st, res)) return rc;
  t->host_valid = false;
  if (res[og::GB_STATUS] & og::GPU_BUILD_BADINPUT)
    return fail(OCTGRAV_ERR_NONFINITE, "non-finite position/mass or negative mass");
  return OCTGRAV_OK;
}

// Forces at the current positions: the tree built on the GPU (or refitted,
// between full builds), walk, unpermute into the state's acceleration and
// potential arrays; waits for the stream.
int sim_forces(octgrav_sim* s, cudaStream_t st) {
  const double* x = static_cast<const double*>(s->x.p);
  const double* m = static_cast<const double*>(s->m.p);
  int rc;
  if (!s->tree || s->since_build + 1 >= s->rebuild_every) {
    octgrav_free_tree(s->tree);
    s->tree = nullptr;
    const int64_t off[2] = {0, s->n};
    if ((rc = build_gpu_common(1, off, x, m, s->n_leaf, s->n_group, st, &s->dev, &s->tree))) return rc;
    s->since_build = 0;
  } else {
    if ((rc = refit_tree(s->tree, x, m, st))) return rc;
    ++s->since_build;
  }
  rc = forces_dev64(s->tree, s->eps, s->theta, s->G, static_cast<double*>(s->a.p), static_cast<double*>(s->phi.p), st);
  if (!rc) rc = read_status(s->tree, st);
  return rc;
}

}  // namespace

int octgrav_sim_create(const double* pos, const double* vel, const double* mass, int64_t n, double eps, double theta,
                       double G, int n_leaf, int n_group, void* stream, octgrav_sim** out) {
  if (!out) return fail(OCTGRAV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!pos || !vel || !mass || n < 1) return fail(OCTGRAV_ERR_ARG, "NULL input or n < 1");
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(vel[i])) return fail(OCTGRAV_ERR_NONFINITE, "non-finite velocity");
  std::unique_ptr<octgrav_sim> s(new (std::nothrow) octgrav_sim());
  if (!s) return fail(OCTGRAV_ERR_OOM, "host allocation failed");
  s->n = n;
  s->eps = eps;
  s->theta = theta;
  s->G = G;
  s->n_leaf = n_leaf;
  s->n_group = n_group;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((rc = s->x.reserve(24 * n)) || (rc = s->v.reserve(24 * n)) || (rc = s->m.reserve(8 * n)) ||
      (rc = s->a.reserve(24 * n)) || (rc = s->phi.reserve(8 * n)) || (rc = s->epart.reserve(16 * og::SIM_EBLOCKS)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(s->x.p, pos, 24 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(s->v.p, vel, 24 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(s->m.p, mass, 8 * n, cudaMemcpyHostToDevice, st));
  if ((rc = sim_forces(s.get(), st))) return rc;
  *out = s.release();
  return OCTGRAV_OK;
}

int octgrav_sim_step(octgrav_sim* s, double dt, int n_steps, void* stream) {
  if (!s) return fail(OCTGRAV_ERR_ARG, "sim is NULL");
  if (!std::isfinite(dt) || n_steps < 0) return fail(OCTGRAV_ERR_ARG, "need a finite dt and n_steps >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* x = static_cast<double*>(s->x.p);
  double* v = static_cast<double*>(s->v.p);
  const double* a = static_cast<const double*>(s->a.p);
  const double h = 0.5 * dt;
  for (int k = 0; k < n_steps; ++k) {
    cudaError_t e = og::sim_kick_drift(x, v, a, s->n, h, dt, true, st);  // v += a dt/2, x += v dt
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "kick/drift launch failed: %s", cudaGetErrorString(e));
    if (int rc = sim_forces(s, st)) return rc;
    e = og::sim_kick_drift(x, v, a, s->n, h, 0.0, false, st);  // v += a dt/2
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "kick launch failed: %s", cudaGetErrorString(e));
    ++s->steps;
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return OCTGRAV_OK;
}

int octgrav_sim_energy(octgrav_sim* s, double* kinetic, double* potential, void* stream) {
  if (!s || !kinetic || !potential) return fail(OCTGRAV_ERR_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = og::sim_energy_partials(static_cast<const double*>(s->v.p), static_cast<const double*>(s->m.p),
                                          static_cast<const double*>(s->phi.p), s->n, static_cast<double*>(s->epart.p),
                                          st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "energy launch failed: %s", cudaGetErrorString(e));
  double part[2 * og::SIM_EBLOCKS];
  CUDA_TRY(cudaMemcpyAsync(part, s->epart.p, sizeof part, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  double k = 0, w = 0;
  for (int b = 0; b < og::SIM_EBLOCKS; ++b) {
    k += part[2 * b];
    w += part[2 * b + 1];
  }
  *kinetic = k;
  *potential = w;
  return OCTGRAV_OK;
}

int octgrav_sim_state(octgrav_sim* s, double* pos, double* vel, double* acc, double* pot, void* stream) {
  if (!s) return fail(OCTGRAV_ERR_ARG, "sim is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = s->n;
  if (pos) CUDA_TRY(cudaMemcpyAsync(pos, s->x.p, 24 * n, cudaMemcpyDeviceToHost, st));
  if (vel) CUDA_TRY(cudaMemcpyAsync(vel, s->v.p, 24 * n, cudaMemcpyDeviceToHost, st));
  if (acc) CUDA_TRY(cudaMemcpyAsync(acc, s->a.p, 24 * n, cudaMemcpyDeviceToHost, st));
  if (pot) CUDA_TRY(cudaMemcpyAsync(pot, s->phi.p, 8 * n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return OCTGRAV_OK;
}

void octgrav_sim_free(octgrav_sim* s) { delete s; }

int octgrav_sim_set_rebuild(octgrav_sim* s, int every) {
  if (!s || every < 1) return fail(OCTGRAV_ERR_ARG, "NULL sim or every < 1");
  s->rebuild_every = every;
  return OCTGRAV_OK;
}

int octgrav_refit_tree_gpu(octgrav_tree* t, const double* pos_dev, const double* mass_dev, void* stream) {
  if (!t || !pos_dev || !mass_dev) return fail(OCTGRAV_ERR_ARG, "NULL argument");
  if (!t->gpu || t->dev != &t->own)
    return fail(OCTGRAV_ERR_STATE, "refit needs a tree from octgrav_build_tree_gpu / octgrav_build_batch_gpu");
  return refit_tree(t, pos_dev, mass_dev, static_cast<cudaStream_t>(stream));
}

int octgrav_status(octgrav_tree* t, void* stream) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (!t->launched) return fail(OCTGRAV_ERR_STATE, "no launch on this tree yet");
  return read_status(t, static_cast<cudaStream_t>(stream));
}

int octgrav_tree_stats(const octgrav_tree* t, int64_t* out, int n_out) {
  if (!t || !out) return fail(OCTGRAV_ERR_ARG, "NULL argument");
  const int64_t v[8] = {t->n, t->n_cells, t->n_leaves, t->n_groups, t->n_items, t->depth_reached, t->n_sys,
                        t->max_group};
  for (int k = 0; k < n_out && k < 8; ++k) out[k] = v[k];
  return OCTGRAV_OK;
}

int octgrav_tree_perm(const octgrav_tree* t, int64_t* perm) {
  if (!t || !perm) return fail(OCTGRAV_ERR_ARG, "NULL argument");
  if (int rc = host_images(const_cast<octgrav_tree*>(t))) return rc;
  std::memcpy(perm, t->perm.data(), sizeof(int64_t) * t->n);
  return OCTGRAV_OK;
}

int octgrav_tree_cell_keys(const octgrav_tree* t, uint64_t* keys) {
  if (!t || !keys) return fail(OCTGRAV_ERR_ARG, "NULL argument");
  if (int rc = host_images(const_cast<octgrav_tree*>(t))) return rc;
  std::memcpy(keys, t->key.data(), sizeof(uint64_t) * t->n_cells);
  return OCTGRAV_OK;
}

int octgrav_tree_cell_props(const octgrav_tree* t, double* bmin, double* bmax, double* cube, double* mass,
                            double* com, double* S, int64_t* count) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "NULL argument");
  if (int rc = host_images(const_cast<octgrav_tree*>(t))) return rc;
  const size_t nc = static_cast<size_t>(t->n_cells);
  if (bmin) std::memcpy(bmin, t->bmin.data(), 24 * nc);
  if (bmax) std::memcpy(bmax, t->bmax.data(), 24 * nc);
  if (cube) std::memcpy(cube, t->cube.data(), 32 * nc);
  if (mass) std::memcpy(mass, t->M.data(), 8 * nc);
  if (com) std::memcpy(com, t->com.data(), 24 * nc);
  if (S) std::memcpy(S, t->S.data(), 48 * nc);
  if (count) std::memcpy(count, t->pcount.data(), 8 * nc);
  return OCTGRAV_OK;
}

int octgrav_item_info(const octgrav_tree* t, uint64_t* group_key, int64_t* first, int32_t* count, int32_t* sys) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (int rc = host_images(const_cast<octgrav_tree*>(t))) return rc;
  for (size_t k = 0; k < t->items.size(); ++k) {
    if (group_key) group_key[k] = t->item_key[k];
    if (first) first[k] = t->items[k].y;
    if (count) count[k] = t->items[k].z;
    if (sys) sys[k] = t->items[k].w;
  }
  return OCTGRAV_OK;
}

int octgrav_interaction_counts(octgrav_tree* t, int64_t* out, void* stream) {
  if (!t || !out) return fail(OCTGRAV_ERR_ARG, "NULL argument");
  if (!t->launched) return fail(OCTGRAV_ERR_STATE, "no launch on this tree yet");
  if (int rc = host_images(t)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int2> c(t->items.size());
  if (!c.empty())
    CUDA_TRY(cudaMemcpyAsync(c.data(), t->dev->counts.p, sizeof(int2) * c.size(), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  int64_t npp = 0, npc = 0;
  for (size_t k = 0; k < c.size(); ++k) {
    const int64_t np = t->items[k].z;
    npc += np * c[k].x;
    npp += np * (c[k].y - 1);
  }
  out[0] = npp;
  out[1] = npc;
  out[2] = 38 * npp + 70 * npc;
  return OCTGRAV_OK;
}

int octgrav_debug_lists(octgrav_tree* t, double theta, int cap, uint64_t* cell_keys, int32_t* n_cell,
                        uint64_t* leaf_keys, int32_t* n_leaf, void* stream) {
  if (!t || cap < 1 || !cell_keys || !n_cell || !leaf_keys || !n_leaf) return fail(OCTGRAV_ERR_ARG, "bad argument");
  int rc = check_params(1.0, theta, 1.0);
  if (rc) return rc;
  if ((rc = host_images(t))) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t ni = t->items.size();
  if (!t->uploaded || t->sysp_dirty) {
    if ((rc = upload(t, st))) return rc;
  }
  if ((rc = t->dev->out.reserve(sizeof(float4) * t->n))) return rc;
  const size_t bytes = ni * cap * 8 + ni * sizeof(int2);
  if ((rc = t->dev->dbg.reserve(bytes))) return rc;
  int* dcell = static_cast<int*>(t->dev->dbg.p);
  int* dleaf = dcell + ni * cap;
  int2* dn = reinterpret_cast<int2*>(dleaf + ni * cap);
  if ((rc = launch(t, 1.0, theta, 1.0, static_cast<float4*>(t->dev->out.p), st, true, dcell, dleaf, dn, cap)))
    return rc;
  std::vector<int> hc(ni * cap), hl(ni * cap);
  std::vector<int2> hn(ni);
  CUDA_TRY(cudaMemcpyAsync(hc.data(), dcell, 4 * ni * cap, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hl.data(), dleaf, 4 * ni * cap, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hn.data(), dn, sizeof(int2) * ni, cudaMemcpyDeviceToHost, st));
  if ((rc = read_status(t, st))) return rc;
  bool trunc = false;
  for (size_t k = 0; k < ni; ++k) {
    n_cell[k] = hn[k].x;
    n_leaf[k] = hn[k].y;
    trunc |= hn[k].x > cap || hn[k].y > cap;
    for (int e = 0; e < std::min(cap, hn[k].x); ++e) cell_keys[k * cap + e] = t->key[hc[k * cap + e]];
    for (int e = 0; e < std::min(cap, hn[k].y); ++e) leaf_keys[k * cap + e] = t->key[hl[k * cap + e]];
  }
  if (trunc) return fail(OCTGRAV_ERR_LIST, "a list was longer than cap = %d", cap);
  return OCTGRAV_OK;
}

int octgrav_balance(octgrav_tree* t, int mode, void* stream) {
  if (!t || mode < 0 || mode > 2) return fail(OCTGRAV_ERR_ARG, "NULL tree or mode not 0/1/2");
  if (mode == 0) {
    t->ordered = false;
    return OCTGRAV_OK;
  }
  if (mode == 1 && !t->launched) return fail(OCTGRAV_ERR_STATE, "no launch on this tree yet");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t ni = t->n_items;
  std::vector<int2> c(mode == 1 ? ni : 0);
  std::vector<int4> it(ni);
  if (ni) {
    if (mode == 1)
      CUDA_TRY(cudaMemcpyAsync(c.data(), t->dev->counts.p, sizeof(int2) * ni, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(it.data(), t->dev->items.p, sizeof(int4) * ni, cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  // cost of an item: its particles times the flops of its lists (mode 1), or
  // its particles alone (mode 2, no launch needed)
  std::vector<double> cost(ni);
  for (int64_t k = 0; k < ni; ++k)
    cost[k] = static_cast<double>(it[k].z) * (mode == 1 ? 70.0 * c[k].x + 38.0 * (c[k].y - 1) : 1.0);
  std::vector<int32_t> order(ni);
  for (int64_t k = 0; k < ni; ++k) order[k] = static_cast<int32_t>(k);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  int rc = t->dev->order.reserve(4 * std::max<int64_t>(1, ni));
  if (rc) return rc;
  if (ni) CUDA_TRY(cudaMemcpyAsync(t->dev->order.p, order.data(), 4 * ni, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (!t->gpu) t->item_order.assign(order.begin(), order.end());  // a later re-upload keeps it
  t->ordered = true;
  return OCTGRAV_OK;
}

int octgrav_set_launch(octgrav_tree* t, int particles_per_lane, int ctas_per_sm) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (particles_per_lane != 1 && particles_per_lane != 2) return fail(OCTGRAV_ERR_ARG, "particles_per_lane must be 1 or 2");
  if (ctas_per_sm < 0) return fail(OCTGRAV_ERR_ARG, "ctas_per_sm must be >= 0");
  t->ctas_per_sm = ctas_per_sm;
  if (particles_per_lane != t->ppl) {
    t->ppl = particles_per_lane;
    if (t->gpu) {  // items and their default order rebuilt on the device  // rebuild the work items on the device
      const og::GpuBuild a = gpu_args(t, t->sys_off.data(), nullptr, nullptr);
      cudaError_t e = og::gpu_build_items(a, nullptr);
      if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "GPU item build failed: %s", cudaGetErrorString(e));
      int64_t res[og::GB_COUNT];
      if (int rc = gpu_result(t, nullptr, res)) return rc;
      t->n_items = res[og::GB_NITEMS];
      t->ordered = true;
      t->host_valid = false;
      if (int rc = t->dev->counts.reserve(t->n_items * sizeof(int2))) return rc;
    } else {
      make_items(t);
      t->uploaded = false;
    }
  }
  return OCTGRAV_OK;
}

int octgrav_forces_noalloc(octgrav_tree* t, void* arena, size_t* arena_bytes, double eps, double theta,
                           double G, float* acc4_dev, void* stream) {
  if (!t || !arena_bytes) return fail(OCTGRAV_ERR_ARG, "NULL tree or arena_bytes");
  if (int rc = host_images(t)) return rc;
  // arena layout: the device arrays, each starting on a 256-byte boundary
  const size_t sizes[7] = {t->parts.size() * sizeof(float4), t->geo.size() * sizeof(float4),
                           t->link.size() * sizeof(int2),    t->mp.size() * sizeof(float4),
                           t->items.size() * sizeof(int4),   t->ibox.size() * sizeof(float4),
                           t->sysp.size() * sizeof(float4)};
  size_t offs[7], total = 0;
  for (int k = 0; k < 7; ++k) {
    offs[k] = total;
    total += (sizes[k] + 255) & ~static_cast<size_t>(255);
  }
  if (!arena) {
    *arena_bytes = total;
    return OCTGRAV_OK;
  }
  if (*arena_bytes < total)
    return fail(OCTGRAV_ERR_ARG, "arena of %zu bytes is smaller than the %zu bytes needed", *arena_bytes, total);
  if (reinterpret_cast<uintptr_t>(arena) % 256) return fail(OCTGRAV_ERR_ARG, "arena must be 256-byte aligned");
  if (t->items.size() > static_cast<size_t>(OCTGRAV_NOALLOC_MAX_ITEMS))
    return fail(OCTGRAV_ERR_ARG, "tree has %zu work items; the allocation-free path takes at most %d",
                t->items.size(), OCTGRAV_NOALLOC_MAX_ITEMS);
  if (!acc4_dev) return fail(OCTGRAV_ERR_ARG, "NULL output");
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* a = static_cast<char*>(arena);
  const void* src[7] = {t->parts.data(), t->geo.data(), t->link.data(), t->mp.data(),
                        t->items.data(), t->ibox.data(), t->sysp.data()};
  for (int k = 0; k < 7; ++k)
    if (sizes[k]) CUDA_TRY(cudaMemcpyAsync(a + offs[k], src[k], sizes[k], cudaMemcpyHostToDevice, st));
  og::KParams p{};
  p.parts = reinterpret_cast<const float4*>(a + offs[0]);
  p.geo = reinterpret_cast<const float4*>(a + offs[1]);
  p.link = reinterpret_cast<const int2*>(a + offs[2]);
  p.mp = reinterpret_cast<const float4*>(a + offs[3]);
  p.items = reinterpret_cast<const int4*>(a + offs[4]);
  p.ibox = reinterpret_cast<const float4*>(a + offs[5]);
  p.sysp = t->sysp.empty() ? nullptr : reinterpret_cast<const float4*>(a + offs[6]);
  p.sys0 = make_float4(static_cast<float>(theta * theta), static_cast<float>(eps * eps), static_cast<float>(G), 0.f);
  p.out = reinterpret_cast<float4*>(acc4_dev);
  p.n_items = static_cast<int>(t->items.size());
  p.n_cells = static_cast<int>(t->n_cells);
  p.stage = t->stage;
  {
    cudaError_t e = og::encode_mp_map(&p.mp_map, a + offs[3], static_cast<int>(t->n_cells));
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "tensor map encode failed: %s", cudaGetErrorString(e));
  }
  int bits = 0;
  cudaError_t e = og::launch_walk_eval_noalloc(p, t->ppl, t->ctas_per_sm, st, &bits);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "allocation-free launch failed: %s", cudaGetErrorString(e));
  if (bits & og::ST_TIMEOUT) return fail(OCTGRAV_ERR_TIMEOUT, "device wait timed out (status %d)", bits);
  if (bits & og::ST_INDEX) return fail(OCTGRAV_ERR_INDEX, "walk met an out-of-range cell index");
  if (bits & og::ST_STACK) return fail(OCTGRAV_ERR_STACK, "walk overflowed its node stack");
  return OCTGRAV_OK;
}

int octgrav_graph_capture(octgrav_tree* t, double eps, double theta, double G, float* acc4_dev, void* stream) {
  if (!t || !acc4_dev) return fail(OCTGRAV_ERR_ARG, "NULL tree or output");
  if (!stream) return fail(OCTGRAV_ERR_ARG, "graph capture needs a non-default stream");
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!t->uploaded || t->sysp_dirty) {
    if ((rc = upload(t, st))) return rc;
  }
  CUDA_TRY(cudaStreamSynchronize(st));  // uploads from pageable memory cannot be captured
  og::LaunchInfo li;
  cudaError_t e = og::prepare_walk_eval(t->ppl, t->stage, t->ctas_per_sm, &li);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "kernel preparation failed: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  rc = launch(t, eps, theta, G, reinterpret_cast<float4*>(acc4_dev), st, false, nullptr, nullptr, nullptr, 0);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
  if (t->gexec) cudaGraphExecDestroy(t->gexec);
  t->gexec = exec;
  return OCTGRAV_OK;
}

int octgrav_graph_launch(octgrav_tree* t, void* stream) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (!t->gexec) return fail(OCTGRAV_ERR_STATE, "no captured graph on this tree");
  CUDA_TRY(cudaGraphLaunch(t->gexec, static_cast<cudaStream_t>(stream)));
  t->launched = true;
  return OCTGRAV_OK;
}

int octgrav_autotune(int n_sys, const int64_t* offsets, const double* pos, const double* mass, int n_leaf,
                     double eps, double theta, const int* n_group_cand, int n_cand, int* best, double* best_ms,
                     void* stream) {
  if (!offsets || !pos || !mass || !n_group_cand || n_cand < 1 || !best || n_sys < 1)
    return fail(OCTGRAV_ERR_ARG, "bad argument");
  int rc = check_params(eps, theta, 1.0);
  if (rc) return rc;
  // results are cached per (systems, log2 N, theta, eps, n_leaf, candidate set)
  static std::mutex mu;
  static std::vector<std::pair<std::vector<double>, std::vector<double>>> cache;
  std::vector<double> key = {static_cast<double>(n_sys), std::floor(std::log2(static_cast<double>(offsets[n_sys]))),
                             theta, eps, static_cast<double>(n_leaf)};
  for (int c = 0; c < n_cand; ++c) key.push_back(n_group_cand[c]);
  {
    std::lock_guard<std::mutex> g(mu);
    for (auto& kv : cache)
      if (kv.first == key) {
        best[0] = static_cast<int>(kv.second[0]);
        best[1] = static_cast<int>(kv.second[1]);
        best[2] = 0;
        if (best_ms) *best_ms = kv.second[2];
        return OCTGRAV_OK;
      }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf outb;
  if ((rc = outb.reserve(sizeof(float4) * offsets[n_sys]))) return rc;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  double bms = 1e300;
  int bng = -1, bppl = 2;
  for (int c = 0; c < n_cand && rc == OCTGRAV_OK; ++c) {
    if (n_group_cand[c] < n_leaf) continue;
    octgrav_tree* t = nullptr;
    if ((rc = build_common(n_sys, offsets, pos, mass, n_leaf, n_group_cand[c], &t))) break;
    for (int ppl = 1; ppl <= 2 && rc == OCTGRAV_OK; ++ppl) {
      if ((rc = octgrav_set_launch(t, ppl, 0))) break;
      float4* out = static_cast<float4*>(outb.p);
      if ((rc = launch(t, eps, theta, 1.0, out, st, false, nullptr, nullptr, nullptr, 0))) break;
      if ((rc = octgrav_balance(t, 1, st))) break;  // time the longest-first order
      std::vector<float> ms;
      for (int k = 0; k < 3 && rc == OCTGRAV_OK; ++k) {
        cudaEventRecord(e0, st);
        rc = launch(t, eps, theta, 1.0, out, st, false, nullptr, nullptr, nullptr, 0);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(OCTGRAV_ERR_CUDA, "event sync failed");
        float v = 0;
        cudaEventElapsedTime(&v, e0, e1);
        ms.push_back(v);
      }
      if (rc) break;
      if ((rc = read_status(t, st))) break;
      std::sort(ms.begin(), ms.end());
      if (ms[1] < bms) {
        bms = ms[1];
        bng = n_group_cand[c];
        bppl = ppl;
      }
    }
    octgrav_free_tree(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  outb.release();
  if (rc) return rc;
  if (bng < 0) return fail(OCTGRAV_ERR_ARG, "no candidate n_group >= n_leaf");
  best[0] = bng;
  best[1] = bppl;
  best[2] = 0;
  if (best_ms) *best_ms = bms;
  std::lock_guard<std::mutex> g(mu);
  cache.push_back({key, {static_cast<double>(bng), static_cast<double>(bppl), bms}});
  return OCTGRAV_OK;
}

// ---- learned opening criterion

static uint16_t to_bf16(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return static_cast<uint16_t>(u >> 16);
  u += 0x7fffu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}
static uint32_t pack2(float lo, float hi) { return to_bf16(lo) | (static_cast<uint32_t>(to_bf16(hi)) << 16); }

int octgrav_set_criterion(octgrav_tree* t, const float* record, double tau, double theta_lo, double theta_hi,
                          double theta_fb) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (!record) {
    t->learned = false;
    return OCTGRAV_OK;
  }
  if (!(theta_lo >= 0 && theta_hi >= theta_lo && theta_fb >= 0) || !std::isfinite(tau) || !std::isfinite(theta_hi))
    return fail(OCTGRAV_ERR_ARG, "need 0 <= theta_lo <= theta_hi, theta_fb >= 0 and a finite tau");
  const float* mu = record;
  const float* sg = record + 12;
  const float* xmin = record + 24;
  const float* xmax = record + 36;
  const float* w = record + 48;
  const float* W1 = w;
  const float* b1 = W1 + og::MLP_NH * og::MLP_NF;
  const float* W2 = b1 + og::MLP_NH;
  const float* b2 = W2 + og::MLP_NH * og::MLP_NH;
  const float* w3 = b2 + og::MLP_NH;
  og::MlpDevice D;
  std::memset(&D, 0, sizeof D);
  auto w1 = [&](int u, int k) { return k < og::MLP_NF ? W1[u * og::MLP_NF + k] : 0.f; };
  for (int j = 0; j < 8; ++j)
    for (int L = 0; L < 32; ++L) {  // B fragment of W1^T: rows k = 2(L%4)+{0,1}, +8; column u = 8j + L/4
      const int u = 8 * j + L / 4, k = 2 * (L % 4);
      D.w1f[j][L] = make_uint2(pack2(w1(u, k), w1(u, k + 1)), pack2(w1(u, k + 8), w1(u, k + 9)));
    }
  for (int kk = 0; kk < 4; ++kk)
    for (int j = 0; j < 8; ++j)
      for (int L = 0; L < 32; ++L) {
        const int u = 8 * j + L / 4, k = 16 * kk + 2 * (L % 4);
        const float* r = W2 + u * og::MLP_NH;
        D.w2f[kk][j][L] = make_uint2(pack2(r[k], r[k + 1]), pack2(r[k + 8], r[k + 9]));
      }
  for (int j = 0; j < og::MLP_NH; ++j) {
    D.b1[j] = b1[j];
    D.b2[j] = b2[j];
    D.w3[j] = w3[j];
  }
  for (int i = 0; i < 16; ++i) {
    const bool v = i < og::MLP_NF;
    D.mu[i] = v ? mu[i] : 0.f;
    D.isig[i] = v ? 1.f / sg[i] : 0.f;
    D.xmin[i] = v ? xmin[i] : 0.f;
    D.xmax[i] = v ? xmax[i] : 0.f;
  }
  D.b3 = w3[og::MLP_NH];
  D.tau = static_cast<float>(tau);
  int rc = t->dev->mlp.reserve(sizeof D);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpy(t->dev->mlp.p, &D, sizeof D, cudaMemcpyHostToDevice));
  t->learned = true;
  t->theta_lo = static_cast<float>(theta_lo);
  t->theta_hi = static_cast<float>(theta_hi);
  t->theta_fb = static_cast<float>(theta_fb);
  return OCTGRAV_OK;
}

// Host copy of the walk's FP32 opening test (same operations, no contraction).
static bool open_f32_host(const float4& g, const float4& b0, const float4& b1, float theta2, float* d2out) {
  const float h = g.w;
  const float gmin[3] = {b0.x, b0.y, b0.z}, gmax[3] = {b1.x, b1.y, b1.z}, c[3] = {g.x, g.y, g.z};
  float d[3];
  for (int k = 0; k < 3; ++k) {
    const float below = gmin[k] - (c[k] + h), above = (c[k] - h) - gmax[k];
    const float tt = below > above ? below : above;
    d[k] = tt > 0.f ? tt : 0.f;
  }
  const float d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
  if (d2out) *d2out = d2;
  return 4.0f * (h * h) >= theta2 * d2;
}

int octgrav_mlp_samples(octgrav_tree* t, const int64_t* groups, int64_t n_groups, double theta_walk, double eps,
                        float* features, float* labels, int64_t* pairs, int64_t cap, int64_t* n_out, void* stream) {
  if (!t || !groups || n_groups < 0 || !n_out) return fail(OCTGRAV_ERR_ARG, "bad argument");
  int rc = check_params(eps, theta_walk, 1.0);
  if (rc) return rc;
  if ((rc = host_images(t))) return rc;
  const int64_t ngr = static_cast<int64_t>(t->group_cell.size());
  const float th2 = static_cast<float>(theta_walk * theta_walk);
  std::vector<int32_t> s_item, s_cell;
  std::vector<int64_t> s_group;
  int max_count = 1;
  for (int64_t q = 0; q < n_groups; ++q) {
    const int64_t g = groups[q];
    if (g < 0 || g >= ngr) return fail(OCTGRAV_ERR_ARG, "group index %lld out of range", (long long)g);
    const int item = t->group_item[g];
    const int4 it = t->items[item];
    const float4 b0 = t->ibox[4 * item], b1 = t->ibox[4 * item + 1];
    max_count = std::max<int>(max_count, static_cast<int>(t->pcount[t->group_cell[g]]));
    std::vector<int32_t> stack;
    if (t->link[it.x].y > 0) stack.push_back(it.x);
    while (!stack.empty()) {
      const int node = stack.back();
      stack.pop_back();
      const int2 lk = t->link[node];
      for (int c = lk.x; c < lk.x + lk.y; ++c) {
        float d2 = 0.f;
        const bool op = open_f32_host(t->geo[c], b0, b1, th2, &d2);
        if (t->geo[c].w > 0.f && d2 > 0.f) {
          s_item.push_back(item);
          s_cell.push_back(c);
          s_group.push_back(g);
        }
        if (op && t->link[c].y > 0) stack.push_back(c);
      }
    }
  }
  const int64_t ns = static_cast<int64_t>(s_item.size());
  *n_out = ns;
  if (!features || !labels || cap <= 0 || ns == 0) return OCTGRAV_OK;
  const int64_t nw = std::min(ns, cap);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!t->uploaded || t->sysp_dirty) {
    if ((rc = upload(t, st))) return rc;
  }
  // reference accelerations: the same walk at theta = 0.3 with the plain test
  const bool learned = t->learned;
  t->learned = false;
  if ((rc = t->dev->out.reserve(sizeof(float4) * t->n))) { t->learned = learned; return rc; }
  rc = launch(t, eps, 0.3, 1.0, static_cast<float4*>(t->dev->out.p), st, false, nullptr, nullptr, nullptr, 0);
  t->learned = learned;
  if (rc) return rc;
  if ((rc = read_status(t, st))) return rc;
  // per-cell (first, count) and FP64 moments
  const int64_t nc = t->n_cells;
  std::vector<int2> fc(nc);
  for (int64_t c = 0; c < nc; ++c) fc[c] = make_int2(t->cfirst[c], static_cast<int>(t->pcount[c]));
  DevBuf b_item, b_cell, b_fc, b_com, b_M, b_S, b_feat, b_lab;
  if ((rc = b_item.reserve(4 * nw)) || (rc = b_cell.reserve(4 * nw)) || (rc = b_fc.reserve(8 * nc)) ||
      (rc = b_com.reserve(24 * nc)) || (rc = b_M.reserve(8 * nc)) || (rc = b_S.reserve(48 * nc)) ||
      (rc = b_feat.reserve(4 * og::MLP_NF * nw)) || (rc = b_lab.reserve(8 * nw)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(b_item.p, s_item.data(), 4 * nw, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_cell.p, s_cell.data(), 4 * nw, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_fc.p, fc.data(), 8 * nc, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_com.p, t->com.data(), 24 * nc, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_M.p, t->M.data(), 8 * nc, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_S.p, t->S.data(), 48 * nc, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(b_lab.p, 0, 8 * nw, st));
  og::MlpSampleArgs a{};
  a.n = static_cast<int>(nw);
  a.chunks = (max_count + 31) / 32;
  a.item = static_cast<const int*>(b_item.p);
  a.cell = static_cast<const int*>(b_cell.p);
  a.items = static_cast<const int4*>(t->dev->items.p);
  a.ibox = static_cast<const float4*>(t->dev->ibox.p);
  a.geo = static_cast<const float4*>(t->dev->geo.p);
  a.mp = static_cast<const float4*>(t->dev->mp.p);
  a.parts = static_cast<const float4*>(t->dev->parts.p);
  a.link_first_count = static_cast<const int2*>(b_fc.p);
  a.com64 = static_cast<const double*>(b_com.p);
  a.M64 = static_cast<const double*>(b_M.p);
  a.S64 = static_cast<const double*>(b_S.p);
  a.aref = static_cast<const float4*>(t->dev->out.p);
  a.eps2 = eps * eps;
  a.n_group = t->n_group;
  a.feat = static_cast<float*>(b_feat.p);
  a.label64 = static_cast<double*>(b_lab.p);
  cudaError_t e = og::mlp_sample_features(a, st);
  if (e == cudaSuccess) e = og::mlp_sample_labels(a, st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "sample kernels failed: %s", cudaGetErrorString(e));
  std::vector<double> lab(nw);
  CUDA_TRY(cudaMemcpyAsync(features, b_feat.p, 4 * og::MLP_NF * nw, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(lab.data(), b_lab.p, 8 * nw, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t k = 0; k < nw; ++k) {
    labels[k] = static_cast<float>(lab[k]);
    if (pairs) {
      pairs[2 * k] = s_group[k];
      pairs[2 * k + 1] = s_cell[k];
    }
  }
  return OCTGRAV_OK;
}

static double splitmix_uniform(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0);
}

int octgrav_mlp_grad(const float* params, const float* x, const float* target, int64_t n, float* grad, float* loss,
                     void* stream) {
  if (!params || !x || !target || n < 1 || n > (1 << 30) || !grad) return fail(OCTGRAV_ERR_ARG, "bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf bw, bx, bt, bg, bl;
  int rc;
  if ((rc = bw.reserve(4 * og::MLP_NPARAM)) || (rc = bx.reserve(4 * og::MLP_NF * n)) || (rc = bt.reserve(4 * n)) ||
      (rc = bg.reserve(4 * og::MLP_NPARAM)) || (rc = bl.reserve(4)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(bw.p, params, 4 * og::MLP_NPARAM, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(bx.p, x, 4 * og::MLP_NF * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(bt.p, target, 4 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(bg.p, 0, 4 * og::MLP_NPARAM, st));
  CUDA_TRY(cudaMemsetAsync(bl.p, 0, 4, st));
  cudaError_t e = og::mlp_grad(static_cast<float*>(bw.p), static_cast<float*>(bx.p), static_cast<float*>(bt.p),
                               static_cast<int>(n), static_cast<int>(n), 0, 0, true, static_cast<float*>(bg.p),
                               static_cast<float*>(bl.p), st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "gradient kernel failed: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaMemcpyAsync(grad, bg.p, 4 * og::MLP_NPARAM, cudaMemcpyDeviceToHost, st));
  float l = 0;
  CUDA_TRY(cudaMemcpyAsync(&l, bl.p, 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return OCTGRAV_OK;
}

int octgrav_mlp_train(const float* features, const float* labels, int64_t n, int steps, int batch, double lr,
                      uint64_t seed, float* record, float* final_loss, void* stream) {
  if (!features || !labels || !record || n < 2 || n > (1 << 30) || steps < 1 || batch < 1 || !(lr > 0))
    return fail(OCTGRAV_ERR_ARG, "bad argument");
  const int F = og::MLP_NF;
  // targets: log10 of the error label; inputs standardised per feature
  std::vector<float> y(n), X(static_cast<size_t>(n) * F);
  double mu[og::MLP_NF] = {0}, sd[og::MLP_NF] = {0};
  for (int64_t k = 0; k < n; ++k)
    for (int i = 0; i < F; ++i) mu[i] += features[k * F + i];
  for (int i = 0; i < F; ++i) mu[i] /= static_cast<double>(n);
  for (int64_t k = 0; k < n; ++k)
    for (int i = 0; i < F; ++i) sd[i] += (features[k * F + i] - mu[i]) * (features[k * F + i] - mu[i]);
  for (int i = 0; i < F; ++i) sd[i] = std::max(std::sqrt(sd[i] / static_cast<double>(n)), 1e-6);
  float xmin[og::MLP_NF], xmax[og::MLP_NF];
  for (int i = 0; i < F; ++i) { xmin[i] = INFINITY; xmax[i] = -INFINITY; }
  for (int64_t k = 0; k < n; ++k) {
    y[k] = static_cast<float>(std::log10(std::max(static_cast<double>(labels[k]), 1e-12)));
    for (int i = 0; i < F; ++i) {
      const float v = static_cast<float>((features[k * F + i] - mu[i]) / sd[i]);
      X[k * F + i] = v;
      xmin[i] = std::min(xmin[i], v);
      xmax[i] = std::max(xmax[i], v);
    }
  }
  // He-uniform initialisation from a counter-based generator
  std::vector<float> w(og::MLP_NPARAM, 0.f);
  uint64_t rs = seed;
  const int NH = og::MLP_NH;
  for (int k = 0; k < NH * F; ++k) w[k] = static_cast<float>((2 * splitmix_uniform(rs) - 1) * std::sqrt(6.0 / F));
  float* W2 = w.data() + NH * F + NH;
  for (int k = 0; k < NH * NH; ++k) W2[k] = static_cast<float>((2 * splitmix_uniform(rs) - 1) * std::sqrt(6.0 / NH));
  float* w3 = W2 + NH * NH + NH;
  for (int k = 0; k < NH; ++k) w3[k] = static_cast<float>((2 * splitmix_uniform(rs) - 1) * std::sqrt(3.0 / NH));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf bx, by, bw, bm, bv, bg, bl;
  int rc;
  if ((rc = bx.reserve(4 * X.size())) || (rc = by.reserve(4 * n)) || (rc = bw.reserve(4 * og::MLP_NPARAM)) ||
      (rc = bm.reserve(4 * og::MLP_NPARAM)) || (rc = bv.reserve(4 * og::MLP_NPARAM)) ||
      (rc = bg.reserve(4 * og::MLP_NPARAM)) || (rc = bl.reserve(4)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(bx.p, X.data(), 4 * X.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(by.p, y.data(), 4 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(bw.p, w.data(), 4 * og::MLP_NPARAM, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(bm.p, 0, 4 * og::MLP_NPARAM, st));
  CUDA_TRY(cudaMemsetAsync(bv.p, 0, 4 * og::MLP_NPARAM, st));
  const int B = static_cast<int>(std::min<int64_t>(batch, n));
  for (int k = 1; k <= steps; ++k) {
    CUDA_TRY(cudaMemsetAsync(bg.p, 0, 4 * og::MLP_NPARAM, st));
    CUDA_TRY(cudaMemsetAsync(bl.p, 0, 4, st));
    cudaError_t e = og::mlp_grad(static_cast<float*>(bw.p), static_cast<float*>(bx.p), static_cast<float*>(by.p),
                                 static_cast<int>(n), B, k, seed, false, static_cast<float*>(bg.p),
                                 static_cast<float*>(bl.p), st);
    if (e == cudaSuccess)
      e = og::mlp_adam(static_cast<float*>(bw.p), static_cast<float*>(bm.p), static_cast<float*>(bv.p),
                       static_cast<float*>(bg.p), static_cast<float>(lr), k, st);
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "training kernels failed: %s", cudaGetErrorString(e));
  }
  float l = 0;
  CUDA_TRY(cudaMemcpyAsync(w.data(), bw.p, 4 * og::MLP_NPARAM, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(&l, bl.p, 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < F; ++i) {
    record[i] = static_cast<float>(mu[i]);
    record[12 + i] = static_cast<float>(sd[i]);
    record[24 + i] = xmin[i];
    record[36 + i] = xmax[i];
  }
  std::memcpy(record + 48, w.data(), 4 * og::MLP_NPARAM);
  if (final_loss) *final_loss = l;
  return OCTGRAV_OK;
}

int octgrav_set_staging(octgrav_tree* t, int mode) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (mode < og::STAGING_BULK || mode > og::STAGING_GATHER4) return fail(OCTGRAV_ERR_ARG, "staging mode must be 0, 1 or 2");
  t->stage = mode;
  return OCTGRAV_OK;
}

void octgrav_free_tree(octgrav_tree* t) {
  if (!t) return;
  if (t->gexec) cudaGraphExecDestroy(t->gexec);
  t->own.release();
  delete t;
}

}  // extern "C"

octgrav_sim::~octgrav_sim() {
  octgrav_free_tree(tree);
  for (DevBuf* b : {&x, &v, &m, &a, &phi, &epart}) b->release();
  dev.release();
}
