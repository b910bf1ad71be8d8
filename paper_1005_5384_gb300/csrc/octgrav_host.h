// octgrav_host.h -- declarations shared by the host-side translation units of
// the library (not installed): the thread pool, the FP64 build's per-system
// arrays, the device buffers, the tree object and the helpers that the C ABI
// files call. octgrav_host_build.cpp builds trees (Sec. 2.1), octgrav_host.cpp
// uploads, launches and exports the C ABI, octgrav_host_mlp.cpp exports the
// learned criterion's calls.
#pragma once
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
#include <nvtx3/nvToolsExt.h>

#include "../../include/octgrav.h"
#include "octgrav_internal.h"

namespace ogh {

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

// Records the message for octgrav_last_error() (thread-local) and returns code.
int fail(int code, const char* fmt, ...);
extern thread_local std::string g_err;  // the calling thread's last message

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(OCTGRAV_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

// An NVTX range for profilers (no cost without one attached): "octgrav:<name>".
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

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

// parallel_for over [0, n) in chunks of at least `grain` elements.
void parallel_for(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& fn);

// Stable LSD radix sort of (key, val) by key (63 significant bits).
void radix_sort(hvec<uint64_t>& key, hvec<uint32_t>& val, hvec<uint64_t>& k2, hvec<uint32_t>& v2,
                bool parallel);

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
  double* phase_ms = nullptr;  // if set: durations of the build's phases 0..6 (octgrav_oneshot_phases)
  bool check_inputs = false;  // the bounding-box pass also checks the inputs (finite, masses >= 0)
};

// Build one system's tree from its particles (FP64): sort, cells, properties, groups.
int build_system(const double* pos, const double* mass, int64_t n, int n_leaf, int n_group,
                 bool parallel, SysTree& T, const ParticleSink* sink = nullptr);

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
  DevBuf split;  // per-part outputs of a list-split launch (octgrav_set_split)
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
                      &acc64, &pot64, &order, &split})
      b->release();
    cell_cap = 0;
  }
};

}  // namespace ogh

// ---------------------------------------------------------------- the tree object

struct octgrav_tree {
  int64_t n = 0;
  int n_leaf = 0, n_group = 0, n_sys = 0;
  int ppl = 2, ctas_per_sm = 0;
  int fault_stack_cap = 0, fault_drop_item = 0;  // failure injection (octgrav_set_fault; 0 = off)
  int nparts = 1;  // list split of every work item over this many warps (octgrav_set_split)
  int stage = og::STAGING_ASYNC;
  bool learned = false;             // learned opening criterion active
  float theta_lo = 0, theta_hi = 0, theta_fb = 0;
  int mlp_device = -1;              // device holding the criterion's network (dev->mlp)
  CUtensorMap mp_map;
  std::vector<int64_t> sys_off;   // particle offsets per system (n_sys + 1)
  std::vector<int64_t> cell_off;  // cell offsets per system (n_sys + 1)
  ogh::hvec<int64_t> perm;             // tree position -> input index
  ogh::hvec<int32_t> perm32;           // the same as int32, the device image
  ogh::hvec<uint64_t> key;             // per global cell
  std::vector<int32_t> group_cell;  // per group, global cell index
  std::vector<int32_t> group_sys;
  int64_t n_cells = 0, n_leaves = 0, max_group = 0;
  int depth_reached = 0;
  // host images of the device arrays
  ogh::hvec<float4> parts, geo, mp, ibox;
  ogh::hvec<int2> link;
  ogh::hvec<int4> items;
  ogh::hvec<uint64_t> item_key;
  // host FP64 cell properties (tests / introspection)
  ogh::hvec<double> bmin, bmax, cube, M, com, S;
  ogh::hvec<int64_t> pcount;
  ogh::hvec<int32_t> cfirst;           // first particle (tree position) of every cell
  std::vector<int32_t> group_item;  // first work item of every group
  // per-system parameters (optional)
  std::vector<float4> sysp;
  bool sysp_dirty = false;
  // device state
  ogh::Device own;
  ogh::Device* dev = &own;
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
  ogh::hvec<int32_t> item_order;  // host image of the default order (host-built trees)
  int64_t cell_cap = 0;  // cell capacity of the device arrays of a GPU-built tree
  cudaGraphExec_t gexec = nullptr;  // captured memset + kernel (octgrav_graph_capture)
};

// N-body state for the time integration, all on one device.
struct octgrav_sim {
  int64_t n = 0;
  double eps = 0, theta = 0, G = 1;
  int n_leaf = 16, n_group = 16;
  ogh::Device dev;                        // tree and build buffers, reused every step
  ogh::DevBuf x, v, m, a, phi, epart;     // FP64 state (input order) and energy partials
  int64_t steps = 0;
  int rebuild_every = 1;             // full build every k force evaluations, refit in between
  int since_build = 0;
  octgrav_tree* tree = nullptr;      // the last built tree (its buffers live in dev)
  ~octgrav_sim();
};

namespace ogh {

// Work items are cut with og::next_item_size's split except under a learned
// criterion, whose network step a split item would repeat.
inline bool item_split(const octgrav_tree* t) { return !t->learned; }
// Work items of every group, and their default processing order.
void make_items(octgrav_tree* t);
// make_items again (host-built tree) or the GPU build's item step (GPU-built
// tree), after a change of ppl or of item_split(t); drops a captured graph.
int rebuild_items(octgrav_tree* t);
// Concatenate the systems' trees into the device-array images;
// particles_done: a one-system build already wrote perm, perm32 and parts.
int assemble(octgrav_tree* t, std::vector<SysTree>& sys, bool particles_done = false);
// ERR_NONFINITE unless every position and mass is finite and every mass >= 0.
int check_inputs(const double* pos, const double* mass, int64_t n);

// octgrav_host.cpp
int upload(octgrav_tree* t, cudaStream_t st);
int check_params(double eps, double theta, double G);
// Capture buffers of a debug launch (device arrays; see og::KParams).
struct CaptureArgs {
  int* cell = nullptr;
  int* leaf = nullptr;
  int2* n = nullptr;
  int cap = 0;
  const int* slot = nullptr;
  int2* net = nullptr;
  int* net_n = nullptr;
  int net_cap = 0;
};
// One walk-and-evaluate launch of t into out (tree order); cap != nullptr runs
// the capture variant.
int launch(octgrav_tree* t, double eps, double theta, double G, float4* out, cudaStream_t st,
           const CaptureArgs* cap = nullptr);
int read_status(octgrav_tree* t, cudaStream_t st);
int host_images(octgrav_tree* t);

}  // namespace ogh
