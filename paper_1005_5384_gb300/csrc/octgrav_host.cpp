// octgrav_host.cpp -- the device side of a tree on the host: device buffers,
// upload, launch, the one-shot calls, the GPU build's host glue, the time
// integration and the C ABI declared in include/octgrav.h (the learned
// criterion's calls are in octgrav_host_mlp.cpp, the FP64 build in
// octgrav_host_build.cpp).
#include "octgrav_host.h"

namespace ogh {

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
  Range range("octgrav:host_build");
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
    if (const char* e = getenv("OCTGRAV_HOST_PULL")) v = v && atoi(e) != 0;  // 0: always cudaMemcpyAsync
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
                  Device& D, cudaStream_t st, octgrav_tree** out, double* phase_ms = nullptr) {
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
    sink.phase_ms = phase_ms;
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
    const auto ta = std::chrono::steady_clock::now();
    if (!rc) rc = assemble(t.get(), cache.sys, true);
    if (phase_ms) phase_ms[7] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ta).count();
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
  p.stack_cap = t->fault_stack_cap;
  p.drop_item = t->fault_drop_item;
  if (t->learned) {
    p.mlp = static_cast<const og::MlpDevice*>(D.mlp.p);
    p.theta_lo2 = static_cast<float>(static_cast<double>(t->theta_lo) * t->theta_lo);
    p.theta_hi2 = static_cast<float>(static_cast<double>(t->theta_hi) * t->theta_hi);
    p.theta_fb2 = static_cast<float>(static_cast<double>(t->theta_fb) * t->theta_fb);
  }
  return p;
}

// Parts of a list-split launch of t (1: no split): only plain-criterion,
// cp.async-staged launches that capture no lists split.
int split_parts(const octgrav_tree* t, bool capture) {
  return (t->nparts > 1 && !capture && !t->learned && t->stage == og::STAGING_ASYNC) ? t->nparts : 1;
}

int launch(octgrav_tree* t, double eps, double theta, double G, float4* out, cudaStream_t st,
           const CaptureArgs* cap) {
  const bool capture = cap != nullptr;
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
    p.dbg_cell = cap->cell;
    p.dbg_leaf = cap->leaf;
    p.dbg_n = cap->n;
    p.dbg_cap = cap->cap;
    p.dbg_slot = cap->slot;
    p.dbg_net = cap->net;
    p.dbg_net_n = cap->net_n;
    p.dbg_net_cap = cap->net_cap;
  }
  CUDA_TRY(cudaMemsetAsync(t->dev->ctl.p, 0, 8, st));
  const int nparts = split_parts(t, capture);
  if (nparts > 1) {  // the parts' outputs are summed into out below; counts are accumulated
    if ((rc = t->dev->split.reserve(sizeof(float4) * nparts * static_cast<size_t>(t->n)))) return rc;
    p.nparts = nparts;
    p.n = static_cast<int>(t->n);
    p.part_out = static_cast<float4*>(t->dev->split.p);
    CUDA_TRY(cudaMemsetAsync(t->dev->counts.p, 0, sizeof(int2) * t->n_items, st));
  }
  if (p.n_items > 0) {
    cudaError_t e = og::launch_walk_eval(p, t->ppl, t->ctas_per_sm, capture, st, nullptr);
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    if (nparts > 1 && (e = og::split_sum(p.part_out, nparts, p.n, out, st)) != cudaSuccess)
      return fail(OCTGRAV_ERR_CUDA, "split sum launch failed: %s", cudaGetErrorString(e));
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
// ev (optional, 3 events): recorded before the upload, before the launch and after it.
int forces_dev64(octgrav_tree* t, double eps, double theta, double G, double* acc, double* pot, cudaStream_t st,
                 cudaEvent_t* ev = nullptr) {
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  if (ev) CUDA_TRY(cudaEventRecord(ev[0], st));
  if (!t->uploaded || t->sysp_dirty) {
    if ((rc = upload(t, st))) return rc;
  }
  if ((rc = t->dev->out.reserve(sizeof(float4) * t->n))) return rc;
  if ((rc = device_perm(t, st))) return rc;
  if (ev) CUDA_TRY(cudaEventRecord(ev[1], st));
  if ((rc = launch(t, eps, theta, G, static_cast<float4*>(t->dev->out.p), st)))
    return rc;
  if (ev) CUDA_TRY(cudaEventRecord(ev[2], st));
  cudaError_t e = og::gpu_unpermute(static_cast<const float4*>(t->dev->out.p), static_cast<const int*>(t->dev->perm.p),
                                    t->n, acc, pot, st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "unpermute launch failed: %s", cudaGetErrorString(e));
  return OCTGRAV_OK;
}

// ev (optional, 4 events): those of forces_dev64, then one after the copies out.
int forces_host(octgrav_tree* t, double eps, double theta, double G, double* acc, double* pot,
                cudaStream_t st, cudaEvent_t* ev = nullptr) {
  if (!acc) return fail(OCTGRAV_ERR_ARG, "acc is NULL");
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  // unpermute on the device, copy FP64 results straight into the caller's arrays
  Device& D = *t->dev;
  if ((rc = D.acc64.reserve(24 * t->n)) || (rc = D.pot64.reserve(8 * t->n))) return rc;
  if ((rc = forces_dev64(t, eps, theta, G, static_cast<double*>(D.acc64.p), static_cast<double*>(D.pot64.p), st,
                         ev)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(acc, D.acc64.p, 24 * t->n, cudaMemcpyDeviceToHost, st));
  if (pot) CUDA_TRY(cudaMemcpyAsync(pot, D.pot64.p, 8 * t->n, cudaMemcpyDeviceToHost, st));
  if (ev) CUDA_TRY(cudaEventRecord(ev[3], st));
  return read_status(t, st);
}

// The one-shot calls' device buffers, one set per calling thread, released
// when the thread ends.
struct ThreadDevice {
  Device* d = nullptr;
  cudaEvent_t ev[4] = {};  // phase events of the last one-shot host-build call
  double phase_ms[OCTGRAV_ONESHOT_PHASES] = {};
  bool timed = false;
  Device& get() {
    if (!d) d = new Device();
    return *d;
  }
  cudaEvent_t* events() {
    for (cudaEvent_t& e : ev)
      if (!e && cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return ev;
  }
  ~ThreadDevice() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
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
  a.item_split = item_split(t) ? 1 : 0;
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
                            a.item_max,   a.item_split, a.max_level,   a.cap,         P(a.scratch),  static_cast<int64_t>(a.scratch_bytes),
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
  Range range("octgrav:gpu_build");
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

// Cut the work items again (after a change of ppl or of the item rule) with
// their default order, on the device for a GPU-built tree. A captured graph
// refers to the old items and is dropped.
int rebuild_items(octgrav_tree* t) {
  if (t->gexec) {
    cudaGraphExecDestroy(t->gexec);
    t->gexec = nullptr;
  }
  if (t->gpu) {
    const og::GpuBuild a = gpu_args(t, t->sys_off.data(), nullptr, nullptr);
    cudaError_t e = og::gpu_build_items(a, nullptr);
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "GPU item build failed: %s", cudaGetErrorString(e));
    int64_t res[og::GB_COUNT];
    if (int rc = gpu_result(t, nullptr, res)) return rc;
    t->n_items = res[og::GB_NITEMS];
    t->ordered = true;
    t->host_valid = false;
    return t->dev->counts.reserve(t->n_items * sizeof(int2));
  }
  make_items(t);
  t->uploaded = false;
  return OCTGRAV_OK;
}

}  // namespace ogh

using namespace ogh;

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
  return launch(t, eps, theta, G, reinterpret_cast<float4*>(acc4_dev), static_cast<cudaStream_t>(stream));
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
  ThreadDevice& TD = tl_device;
  double* ph = TD.phase_ms;
  TD.timed = false;
  const auto t0 = std::chrono::steady_clock::now();
  octgrav_tree* t = nullptr;
  {
    Range r("octgrav:host_build");
    if ((rc = build_oneshot(pos, mass, n, n_leaf, n_group, hcache, TD.get(), st, &t, ph))) return rc;
  }
  const auto t1 = std::chrono::steady_clock::now();
  cudaEvent_t* ev = TD.events();
  {
    Range r("octgrav:forces");
    rc = forces_host(t, eps, theta, G, acc, pot, st, ev);
  }
  if (rc) cudaStreamSynchronize(st);  // nothing may still read the cached host arrays
  give_back(t, &hcache);
  octgrav_free_tree(t);
  if (!rc) {
    const auto t2 = std::chrono::steady_clock::now();
    ph[8] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    float e01 = 0.f, e12 = 0.f, e23 = 0.f;
    if (ev && cudaEventElapsedTime(&e01, ev[0], ev[1]) == cudaSuccess &&
        cudaEventElapsedTime(&e12, ev[1], ev[2]) == cudaSuccess && cudaEventElapsedTime(&e23, ev[2], ev[3]) == cudaSuccess) {
      ph[9] = e01;
      ph[10] = e12;
      ph[11] = e23;
    } else {
      ph[9] = ph[10] = ph[11] = -1.0;
    }
    ph[12] = std::chrono::duration<double, std::milli>(t2 - t0).count();
    TD.timed = true;
  }
  return rc;
}

int octgrav_oneshot_phases(double* ms, int n_out) {
  if (!ms || n_out < 0) return fail(OCTGRAV_ERR_ARG, "NULL output or n_out < 0");
  if (!tl_device.timed) return fail(OCTGRAV_ERR_STATE, "no completed octgrav_forces_ex call on this thread");
  const int k = std::min(n_out, static_cast<int>(OCTGRAV_ONESHOT_PHASES));
  for (int i = 0; i < k; ++i) ms[i] = tl_device.phase_ms[i];
  return k;
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

int octgrav_forces_batched_ex(int n_sys, const int64_t* offsets, const double* pos, const double* mass,
                              const double* eps, const double* theta, double G, int n_leaf, int n_group,
                              double* acc, double* pot, void* stream) {
  if (n_sys < 1 || !offsets || !pos || !mass || !eps || !theta || !acc)
    return fail(OCTGRAV_ERR_ARG, "NULL input or output, or n_sys < 1");
  if (offsets[0] != 0) return fail(OCTGRAV_ERR_ARG, "offsets[0] must be 0");
  for (int s = 0; s < n_sys; ++s) {
    if (offsets[s + 1] <= offsets[s]) return fail(OCTGRAV_ERR_ARG, "empty or decreasing system %d", s);
    int rc = check_params(eps[s], theta[s], G);
    if (rc) return rc;
  }
  const int64_t n = offsets[n_sys];
  if (n >= (1ll << 31) - 64) return fail(OCTGRAV_ERR_ARG, "too many particles");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Device& D = tl_device.get();
  int cur = 0;
  CUDA_TRY(cudaGetDevice(&cur));
  if (D.device >= 0 && D.device != cur) D.release();
  D.device = cur;
  int rc;
  if ((rc = D.in_pos.reserve(24 * n)) || (rc = D.in_mass.reserve(8 * n))) return rc;
  CUDA_TRY(cudaMemcpyAsync(D.in_pos.p, pos, 24 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(D.in_mass.p, mass, 8 * n, cudaMemcpyHostToDevice, st));
  octgrav_tree* t = nullptr;
  if ((rc = build_gpu_common(n_sys, offsets, static_cast<const double*>(D.in_pos.p),
                             static_cast<const double*>(D.in_mass.p), n_leaf, n_group, st, &D, &t)))
    return rc;
  if (!(rc = octgrav_set_system_params(t, eps, theta))) rc = forces_host(t, eps[0], theta[0], G, acc, pot, st);
  octgrav_free_tree(t);
  return rc;
}

int octgrav_forces_batched(int n_sys, const int64_t* offsets, const double* pos, const double* mass,
                           const double* eps, const double* theta, double* acc, double* pot, void* stream) {
  return octgrav_forces_batched_ex(n_sys, offsets, pos, mass, eps, theta, 1.0, 16, 256, acc, pot, stream);
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
  Range range("octgrav:sim_step");
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

int octgrav_debug_walk(octgrav_tree* t, double theta, int64_t n_sel, const int64_t* items, int cap,
                       uint64_t* cell_keys, int32_t* n_cell, uint64_t* leaf_keys, int32_t* n_leaf, int net_cap,
                       uint64_t* net_keys, float* net_y, int32_t* n_net, void* stream) {
  if (!t || cap < 1 || !cell_keys || !n_cell || !leaf_keys || !n_leaf || net_cap < 0 ||
      (net_cap > 0 && (!net_keys || !net_y || !n_net)))
    return fail(OCTGRAV_ERR_ARG, "bad argument");
  int rc = check_params(1.0, theta, 1.0);
  if (rc) return rc;
  if ((rc = host_images(t))) return rc;
  const int64_t ni = static_cast<int64_t>(t->items.size());
  const int64_t ns = items ? n_sel : ni;
  if (ns < 0) return fail(OCTGRAV_ERR_ARG, "n_sel < 0");
  std::vector<int> slot;
  if (items) {
    slot.assign(static_cast<size_t>(ni), -1);
    for (int64_t r = 0; r < ns; ++r) {
      if (items[r] < 0 || items[r] >= ni) return fail(OCTGRAV_ERR_ARG, "item %lld out of range", (long long)items[r]);
      if (slot[items[r]] >= 0) return fail(OCTGRAV_ERR_ARG, "item %lld listed twice", (long long)items[r]);
      slot[items[r]] = static_cast<int>(r);
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!t->uploaded || t->sysp_dirty) {
    if ((rc = upload(t, st))) return rc;
  }
  if ((rc = t->dev->out.reserve(sizeof(float4) * t->n))) return rc;
  const size_t zs = static_cast<size_t>(ns), zc = static_cast<size_t>(cap), zn = static_cast<size_t>(net_cap);
  const size_t bytes = zs * zc * 8 + zs * sizeof(int2) + zs * zn * sizeof(int2) + zs * 4 + slot.size() * 4 + 64;
  if ((rc = t->dev->dbg.reserve(bytes))) return rc;
  CaptureArgs ca;
  ca.cell = static_cast<int*>(t->dev->dbg.p);
  ca.leaf = ca.cell + zs * zc;
  ca.n = reinterpret_cast<int2*>(ca.leaf + zs * zc);
  ca.cap = cap;
  ca.net = ca.n + zs;
  ca.net_n = reinterpret_cast<int*>(ca.net + zs * zn);
  ca.net_cap = net_cap;
  int* dslot = ca.net_n + zs;
  if (!items) {
    ca.slot = nullptr;
  } else {
    ca.slot = dslot;
    if (!slot.empty()) CUDA_TRY(cudaMemcpyAsync(dslot, slot.data(), 4 * slot.size(), cudaMemcpyHostToDevice, st));
  }
  if (zs) CUDA_TRY(cudaMemsetAsync(ca.net_n, 0, 4 * zs, st));
  if (net_cap == 0) ca.net = nullptr, ca.net_n = nullptr;
  if ((rc = launch(t, 1.0, theta, 1.0, static_cast<float4*>(t->dev->out.p), st, &ca))) return rc;
  std::vector<int> hc(zs * zc), hl(zs * zc), hnn(zs);
  std::vector<int2> hn(zs), hnet(zs * zn);
  if (zs) {
    CUDA_TRY(cudaMemcpyAsync(hc.data(), ca.cell, 4 * zs * zc, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hl.data(), ca.leaf, 4 * zs * zc, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hn.data(), ca.n, sizeof(int2) * zs, cudaMemcpyDeviceToHost, st));
    if (net_cap > 0) {
      CUDA_TRY(cudaMemcpyAsync(hnet.data(), ca.net, sizeof(int2) * zs * zn, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaMemcpyAsync(hnn.data(), ca.net_n, 4 * zs, cudaMemcpyDeviceToHost, st));
    }
  }
  if ((rc = read_status(t, st))) return rc;
  bool trunc = false;
  for (size_t k = 0; k < zs; ++k) {
    n_cell[k] = hn[k].x;
    n_leaf[k] = hn[k].y;
    trunc |= hn[k].x > cap || hn[k].y > cap;
    for (int e = 0; e < std::min(cap, hn[k].x); ++e) cell_keys[k * zc + e] = t->key[hc[k * zc + e]];
    for (int e = 0; e < std::min(cap, hn[k].y); ++e) leaf_keys[k * zc + e] = t->key[hl[k * zc + e]];
    if (net_cap > 0) {
      n_net[k] = hnn[k];
      trunc |= hnn[k] > net_cap;
      for (int e = 0; e < std::min(net_cap, hnn[k]); ++e) {
        const int2 v = hnet[k * zn + e];
        const bool in_range = v.x >= 0;
        net_keys[k * zn + e] = t->key[in_range ? v.x : ~v.x];
        float y;
        std::memcpy(&y, &v.y, 4);
        net_y[k * zn + e] = in_range ? y : NAN;
      }
    }
  }
  if (trunc) return fail(OCTGRAV_ERR_LIST, "a list was longer than its capture buffer");
  return OCTGRAV_OK;
}

int octgrav_debug_lists(octgrav_tree* t, double theta, int cap, uint64_t* cell_keys, int32_t* n_cell,
                        uint64_t* leaf_keys, int32_t* n_leaf, void* stream) {
  return octgrav_debug_walk(t, theta, 0, nullptr, cap, cell_keys, n_cell, leaf_keys, n_leaf, 0, nullptr, nullptr,
                            nullptr, stream);
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
    return rebuild_items(t);
  }
  return OCTGRAV_OK;
}

int octgrav_forces_noalloc(octgrav_tree* t, void* arena, size_t* arena_bytes, double eps, double theta,
                           double G, float* acc4_dev, void* stream) {
  if (!t || !arena_bytes) return fail(OCTGRAV_ERR_ARG, "NULL tree or arena_bytes");
  // a GPU-built tree is copied device to device from its own arrays; a
  // host-built one from its host images
  const bool from_device = t->gpu;
  const size_t n = static_cast<size_t>(t->n), nc = static_cast<size_t>(t->n_cells),
               ni = static_cast<size_t>(t->n_items);
  // arena layout: the device arrays, each starting on a 256-byte boundary
  const size_t sizes[7] = {2 * n * sizeof(float4), nc * sizeof(float4),     nc * sizeof(int2),
                           4 * nc * sizeof(float4), ni * sizeof(int4),      4 * ni * sizeof(float4),
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
  if (ni > static_cast<size_t>(OCTGRAV_NOALLOC_MAX_ITEMS))
    return fail(OCTGRAV_ERR_ARG, "tree has %zu work items; the allocation-free path takes at most %d", ni,
                OCTGRAV_NOALLOC_MAX_ITEMS);
  if (!acc4_dev) return fail(OCTGRAV_ERR_ARG, "NULL output");
  int rc = check_params(eps, theta, G);
  if (rc) return rc;
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (from_device && t->dev->device != dev)
    return fail(OCTGRAV_ERR_STATE, "tree was built on device %d, current is %d", t->dev->device, dev);
  if (t->learned && t->mlp_device != dev)
    return fail(OCTGRAV_ERR_STATE, "the learned criterion was set on device %d, current is %d", t->mlp_device, dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* a = static_cast<char*>(arena);
  if (from_device) {
    const Device& D = *t->dev;
    const void* src[6] = {D.parts.p, D.geo.p, D.link.p, D.mp.p, D.items.p, D.ibox.p};
    for (int k = 0; k < 6; ++k)
      if (sizes[k]) CUDA_TRY(cudaMemcpyAsync(a + offs[k], src[k], sizes[k], cudaMemcpyDeviceToDevice, st));
  } else {
    const void* src[6] = {t->parts.data(), t->geo.data(), t->link.data(), t->mp.data(), t->items.data(),
                          t->ibox.data()};
    for (int k = 0; k < 6; ++k)
      if (sizes[k]) CUDA_TRY(cudaMemcpyAsync(a + offs[k], src[k], sizes[k], cudaMemcpyHostToDevice, st));
  }
  if (sizes[6]) CUDA_TRY(cudaMemcpyAsync(a + offs[6], t->sysp.data(), sizes[6], cudaMemcpyHostToDevice, st));
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
  p.n_items = static_cast<int>(ni);
  p.n_cells = static_cast<int>(nc);
  p.stage = t->stage;
  p.n_group = t->n_group;
  if (t->learned) {  // the network stays in the tree's own device memory (set_criterion)
    p.mlp = static_cast<const og::MlpDevice*>(t->dev->mlp.p);
    p.theta_lo2 = static_cast<float>(static_cast<double>(t->theta_lo) * t->theta_lo);
    p.theta_hi2 = static_cast<float>(static_cast<double>(t->theta_hi) * t->theta_hi);
    p.theta_fb2 = static_cast<float>(static_cast<double>(t->theta_fb) * t->theta_fb);
  }
  {
    cudaError_t e = og::encode_mp_map(&p.mp_map, a + offs[3], static_cast<int>(nc));
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
  if (const int np = split_parts(t, false); np > 1) {  // allocate outside the capture
    if ((rc = t->dev->split.reserve(sizeof(float4) * np * static_cast<size_t>(t->n)))) return rc;
  }
  og::LaunchInfo li;
  cudaError_t e = og::prepare_walk_eval(t->ppl, t->stage, t->ctas_per_sm, &li);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "kernel preparation failed: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  rc = launch(t, eps, theta, G, reinterpret_cast<float4*>(acc4_dev), st);
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

// Coarse descriptor of how the particles are spread, for the autotuner's cache:
// quartiles of the distance of (up to 4096, evenly strided) particles from
// their system's bounding-box centre, over the box's half diagonal, as log2
// rounded to halves. A Plummer sphere, a uniform cube and a thin disc differ.
static std::vector<double> spread_descriptor(int n_sys, const int64_t* offsets, const double* pos) {
  std::vector<double> r;
  const int64_t n = offsets[n_sys];
  const int64_t stride = std::max<int64_t>(1, n / 4096);
  std::vector<double> lo(3 * n_sys, INFINITY), hi(3 * n_sys, -INFINITY);
  int s = 0;
  for (int64_t i = 0; i < n; ++i) {
    while (i >= offsets[s + 1]) ++s;
    for (int k = 0; k < 3; ++k) {
      lo[3 * s + k] = std::min(lo[3 * s + k], pos[3 * i + k]);
      hi[3 * s + k] = std::max(hi[3 * s + k], pos[3 * i + k]);
    }
  }
  s = 0;
  for (int64_t i = 0; i < n; i += stride) {
    while (i >= offsets[s + 1]) ++s;
    double d2 = 0, h2 = 0;
    for (int k = 0; k < 3; ++k) {
      const double c = 0.5 * (lo[3 * s + k] + hi[3 * s + k]), h = 0.5 * (hi[3 * s + k] - lo[3 * s + k]);
      d2 += (pos[3 * i + k] - c) * (pos[3 * i + k] - c);
      h2 += h * h;
    }
    r.push_back(h2 > 0 ? std::sqrt(d2 / h2) : 0.0);
  }
  std::sort(r.begin(), r.end());
  std::vector<double> q;
  for (double f : {0.25, 0.5, 0.75}) {
    const double v = r[static_cast<size_t>(f * (r.size() - 1))];
    q.push_back(std::round(2.0 * std::log2(std::max(v, 1e-6))) / 2.0);
  }
  return q;
}

// The autotuner behind octgrav_autotune (tune_staging = false) and
// octgrav_autotune_ex. Writes n_group, particles per lane, split, staging.
static int autotune_common(int n_sys, const int64_t* offsets, const double* pos, const double* mass, int n_leaf,
                           double eps, double theta, const int* n_group_cand, int n_cand, bool tune_staging,
                           int* best4, double* best_ms, void* stream) {
  if (!offsets || !pos || !mass || !n_group_cand || n_cand < 1 || !best4 || n_sys < 1)
    return fail(OCTGRAV_ERR_ARG, "bad argument");
  int rc = check_params(eps, theta, 1.0);
  if (rc) return rc;
  if (offsets[0] != 0) return fail(OCTGRAV_ERR_ARG, "offsets[0] must be 0");
  for (int s = 0; s < n_sys; ++s)
    if (offsets[s + 1] <= offsets[s]) return fail(OCTGRAV_ERR_ARG, "empty or decreasing system %d", s);
  // results are cached per (systems, log2 N, theta, eps, n_leaf, spread of the
  // particles, what is tuned, candidate set)
  static std::mutex mu;
  static std::vector<std::pair<std::vector<double>, std::vector<double>>> cache;
  std::vector<double> key = {static_cast<double>(n_sys), std::floor(std::log2(static_cast<double>(offsets[n_sys]))),
                             theta, eps, static_cast<double>(n_leaf), tune_staging ? 1.0 : 0.0};
  for (double q : spread_descriptor(n_sys, offsets, pos)) key.push_back(q);
  for (int c = 0; c < n_cand; ++c) key.push_back(n_group_cand[c]);
  {
    std::lock_guard<std::mutex> g(mu);
    for (auto& kv : cache)
      if (kv.first == key) {
        for (int k = 0; k < 4; ++k) best4[k] = static_cast<int>(kv.second[k]);
        if (best_ms) *best_ms = kv.second[4];
        return OCTGRAV_OK;
      }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf outb;
  if ((rc = outb.reserve(sizeof(float4) * offsets[n_sys]))) return rc;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float4* out = static_cast<float4*>(outb.p);
  // median of three timed launches, the items taken longest first
  auto time_tree = [&](octgrav_tree* t, double* ms_out) -> int {
    int r;
    if ((r = launch(t, eps, theta, 1.0, out, st))) return r;
    if ((r = octgrav_balance(t, 1, st))) return r;
    std::vector<float> ms;
    for (int k = 0; k < 3; ++k) {
      cudaEventRecord(e0, st);
      if ((r = launch(t, eps, theta, 1.0, out, st))) return r;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "event sync failed");
      float v = 0;
      cudaEventElapsedTime(&v, e0, e1);
      ms.push_back(v);
    }
    if ((r = read_status(t, st))) return r;
    std::sort(ms.begin(), ms.end());
    *ms_out = ms[1];
    return OCTGRAV_OK;
  };
  double bms = 1e300;
  int bng = -1, bppl = 2, bsplit = 1, bstage = og::STAGING_ASYNC;
  for (int c = 0; c < n_cand && rc == OCTGRAV_OK; ++c) {
    if (n_group_cand[c] < n_leaf) continue;
    octgrav_tree* t = nullptr;
    if ((rc = build_common(n_sys, offsets, pos, mass, n_leaf, n_group_cand[c], &t))) break;
    // list splits only where the work items are too few to fill the GPU
    const int max_split = t->n_items < 4 * 152 * 16 ? 8 : 1;
    for (int trial = 0; trial < 2 * 4 && rc == OCTGRAV_OK; ++trial) {
      const int ppl = 1 + trial % 2, split = 1 << (trial / 2);
      if (split > max_split) break;
      if ((rc = octgrav_set_launch(t, ppl, 0)) || (rc = octgrav_set_split(t, split))) break;
      double ms = 0;
      if ((rc = time_tree(t, &ms))) break;
      if (ms < bms) {
        bms = ms;
        bng = n_group_cand[c];
        bppl = ppl;
        bsplit = split;
      }
    }
    octgrav_free_tree(t);
  }
  // the staging of the accepted cell records, for the winner (a split runs
  // with per-lane cp.async staging only)
  if (rc == OCTGRAV_OK && tune_staging && bng >= 0 && bsplit == 1) {
    octgrav_tree* t = nullptr;
    if (!(rc = build_common(n_sys, offsets, pos, mass, n_leaf, bng, &t)) && !(rc = octgrav_set_launch(t, bppl, 0))) {
      for (int stage : {og::STAGING_BULK, og::STAGING_GATHER4}) {
        double ms = 0;
        if ((rc = octgrav_set_staging(t, stage)) || (rc = time_tree(t, &ms))) break;
        if (ms < bms) {
          bms = ms;
          bstage = stage;
        }
      }
    }
    octgrav_free_tree(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  outb.release();
  if (rc) return rc;
  if (bng < 0) return fail(OCTGRAV_ERR_ARG, "no candidate n_group >= n_leaf");
  best4[0] = bng;
  best4[1] = bppl;
  best4[2] = bsplit;
  best4[3] = bstage;
  if (best_ms) *best_ms = bms;
  std::lock_guard<std::mutex> g(mu);
  cache.push_back({key, {static_cast<double>(bng), static_cast<double>(bppl), static_cast<double>(bsplit),
                         static_cast<double>(bstage), bms}});
  return OCTGRAV_OK;
}

int octgrav_autotune(int n_sys, const int64_t* offsets, const double* pos, const double* mass, int n_leaf,
                     double eps, double theta, const int* n_group_cand, int n_cand, int* best, double* best_ms,
                     void* stream) {
  int b[4];
  int rc = autotune_common(n_sys, offsets, pos, mass, n_leaf, eps, theta, n_group_cand, n_cand, false, b, best_ms,
                           stream);
  if (rc == OCTGRAV_OK)
    for (int k = 0; k < 3; ++k) best[k] = b[k];
  return rc;
}

int octgrav_autotune_ex(int n_sys, const int64_t* offsets, const double* pos, const double* mass, int n_leaf,
                        double eps, double theta, const int* n_group_cand, int n_cand, int* best, int n_best,
                        double* best_ms, void* stream) {
  if (n_best < 1 || !best) return fail(OCTGRAV_ERR_ARG, "no room for the result");
  int b[4];
  int rc = autotune_common(n_sys, offsets, pos, mass, n_leaf, eps, theta, n_group_cand, n_cand, true, b, best_ms,
                           stream);
  if (rc == OCTGRAV_OK)
    for (int k = 0; k < std::min(n_best, 4); ++k) best[k] = b[k];
  return rc;
}

int octgrav_set_split(octgrav_tree* t, int nparts) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (nparts < 1 || nparts > 16) return fail(OCTGRAV_ERR_ARG, "nparts must be in [1, 16]");
  if (static_cast<int64_t>(nparts) * t->n_items >= (1ll << 31))
    return fail(OCTGRAV_ERR_ARG, "too many work items to split %d ways", nparts);
  t->nparts = nparts;
  return OCTGRAV_OK;
}

int octgrav_set_fault(octgrav_tree* t, int stack_cap, int64_t drop_item) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (stack_cap < 0 || drop_item < -1 || drop_item >= t->n_items)
    return fail(OCTGRAV_ERR_ARG, "stack_cap must be >= 0 and drop_item in [-1, n_items)");
  t->fault_stack_cap = stack_cap;
  t->fault_drop_item = static_cast<int>(drop_item + 1);
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
