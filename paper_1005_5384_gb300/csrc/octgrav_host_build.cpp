// octgrav_host_build.cpp -- the FP64 octree build on the host: cells, cell
// properties and groups (Sec. 2.1), the device-array images of a tree and its
// work items, and the thread pool it runs on.
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
#include "octgrav_host.h"

namespace ogh {

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

// Stable sort of (key, val) by key (63 significant bits). An LSD radix sort
// with 9-bit digits orders the top 45 bits (five passes instead of seven);
// runs of keys equal in those bits (particles sharing a cell of level 15, rare
// unless particles nearly coincide) are then sorted stably by the low 18 bits.
// The result is the order of a full stable sort: by key, equal keys in input
// order.
constexpr int kLowBits = 18;
void radix_sort(hvec<uint64_t>& key, hvec<uint32_t>& val, hvec<uint64_t>& k2, hvec<uint32_t>& v2,
                bool parallel) {
  const int64_t n = static_cast<int64_t>(key.size());
  k2.resize(n);
  v2.resize(n);
  constexpr int BITS = 9, B = 1 << BITS, PASSES = (63 - kLowBits + BITS - 1) / BITS;
  const int T = parallel ? std::max(1, std::min<int>(Pool::get().size(), static_cast<int>(n / 65536))) : 1;
  std::vector<int64_t> hist(static_cast<size_t>(T) * B);
  const int64_t step = (n + T - 1) / T;
  for (int pass = 0; pass < PASSES; ++pass) {
    const int sh = kLowBits + pass * BITS;
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
  // Runs of equal top bits, each found by the chunk holding its first key (a
  // read-only pass), then sorted by their chunk (disjoint ranges).
  const int chunks = T;
  const int64_t cstep = (n + chunks - 1) / chunks;
  std::vector<std::vector<std::pair<int64_t, int64_t>>> runs(chunks);
  auto top = [&](int64_t i) { return key[i] >> kLowBits; };
  auto body_find = [&](int t) {
    const int64_t lo = t * cstep, hi = std::min(n, lo + cstep);
    for (int64_t i = lo; i < hi; ++i) {
      if (i > 0 && top(i) == top(i - 1)) continue;  // not the first key of its run
      int64_t j = i + 1;
      while (j < n && top(j) == top(i)) ++j;
      if (j - i > 1) runs[t].emplace_back(i, j);
      i = j - 1;
    }
  };
  if (chunks > 1) Pool::get().run(chunks, body_find); else body_find(0);
  auto body_fix = [&](int t) {
    std::vector<std::pair<uint64_t, uint32_t>> r;
    for (const auto& [i, j] : runs[t]) {
      if (j - i <= 32) {  // the usual case, two or three keys: insertion sort (stable)
        for (int64_t a = i + 1; a < j; ++a) {
          const uint64_t k = key[a];
          const uint32_t v = val[a];
          int64_t b = a;
          for (; b > i && key[b - 1] > k; --b) {
            key[b] = key[b - 1];
            val[b] = val[b - 1];
          }
          key[b] = k;
          val[b] = v;
        }
        continue;
      }
      r.clear();
      for (int64_t k = i; k < j; ++k) r.emplace_back(key[k], val[k]);
      std::stable_sort(r.begin(), r.end(),
                       [](const std::pair<uint64_t, uint32_t>& x, const std::pair<uint64_t, uint32_t>& y) {
                         return x.first < y.first;
                       });
      for (int64_t k = i; k < j; ++k) {
        key[k] = r[k - i].first;
        val[k] = r[k - i].second;
      }
    }
  };
  if (chunks > 1) Pool::get().run(chunks, body_fix); else body_fix(0);
}

int build_system(const double* pos, const double* mass, int64_t n, int n_leaf, int n_group,
                 bool parallel, SysTree& T, const ParticleSink* sink) {
  T.reset();
  T.n = n;
  const int64_t grain = parallel ? 16384 : (int64_t)1 << 62;
  auto clock0 = std::chrono::steady_clock::now();
  auto mark = [&](int k) {  // phase durations for octgrav_oneshot_phases
    if (!sink || !sink->phase_ms) return;
    const auto now = std::chrono::steady_clock::now();
    sink->phase_ms[k] = std::chrono::duration<double, std::milli>(now - clock0).count();
    clock0 = now;
  };
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

  mark(0);
  // ---- Morton codes and sort
  hvec<uint64_t>& code = T.code;
  hvec<uint32_t>& idx = T.perm;
  code.resize(n);
  idx.resize(n);
  const double rscale = (1.0 / side) * scale;
  parallel_for(n, grain, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i) {
      uint64_t q[3];
      for (int d = 0; d < 3; ++d) {
        // q = floor(fl(fl(x - lo) / side) * 2^21) without the division where
        // it is safe: c = fl(x - lo) * rscale lies within 4 ulp (< 2^-29, for
        // c <= 2^21) of fl(fl(x - lo) / side) * 2^21, so the floors agree
        // unless an integer lies within 2^-28 of c; then the division decides
        // (the GPU build takes the same steps)
        const double dx = pos[3 * i + d] - lo[d];
        const double c = dx * rscale;
        double v = std::floor(c - 0x1p-28);
        if (v != std::floor(c + 0x1p-28)) v = std::floor((dx / side) * scale);
        q[d] = v <= 0 ? 0 : (v >= static_cast<double>(qmax) ? qmax : static_cast<uint64_t>(v));
      }
      code[i] = spread21(q[0]) | (spread21(q[1]) << 1) | (spread21(q[2]) << 2);
      idx[i] = static_cast<uint32_t>(i);
    }
  });
  mark(1);
  radix_sort(code, idx, T.k2, T.v2, parallel);
  mark(2);
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

  mark(3);
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

  mark(4);
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

  mark(5);
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
  // Order the groups by first particle. They were found level by level, and a
  // level's cells are in key order, i.e. in first-particle order: the list is a
  // few sorted runs (one per level), merged pairwise here (first particles are
  // distinct, so this is the order a full sort would give).
  {
    auto by_first = [&](int32_t a, int32_t b) { return T.pfirst[a] < T.pfirst[b]; };
    std::vector<size_t> bounds = {0};
    for (size_t i = 1; i < T.groups.size(); ++i)
      if (by_first(T.groups[i], T.groups[i - 1])) bounds.push_back(i);
    bounds.push_back(T.groups.size());
    while (bounds.size() > 2) {
      std::vector<size_t> next = {0};
      const size_t runs = bounds.size() - 1;
      for (size_t k = 0; k < runs; k += 2) {
        if (k + 1 < runs)
          std::inplace_merge(T.groups.begin() + bounds[k], T.groups.begin() + bounds[k + 1],
                             T.groups.begin() + bounds[k + 2], by_first);
        next.push_back(bounds[std::min(k + 2, runs)]);
      }
      bounds.swap(next);
    }
  }
  for (int32_t g : T.groups) T.max_group = std::max(T.max_group, T.pcount[g]);
  mark(6);
  return OCTGRAV_OK;
}

// Split every group into work items of at most 32 * ppl particles, cut by
// og::next_item_size (a 33..48-particle rest split in two unless the tree has
// a learned criterion, which would repeat its network for both pieces).
void make_items(octgrav_tree* t) {
  const int item_max = 32 * t->ppl;
  const bool split = item_split(t);
  const int64_t ng = static_cast<int64_t>(t->group_cell.size());
  t->group_item.assign(ng, 0);
  int64_t ni = 0;
  for (int64_t g = 0; g < ng; ++g) {
    t->group_item[g] = static_cast<int32_t>(ni);
    ni += og::item_count(t->pcount[t->group_cell[g]], item_max, split);
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
      for (int64_t off = 0, sz; off < cnt; off += sz, ++k) {
        sz = og::next_item_size(static_cast<int>(cnt - off), item_max, split);
        t->items[k] = make_int4(static_cast<int>(root), static_cast<int>(pf + off), static_cast<int>(sz), s);
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
int assemble(octgrav_tree* t, std::vector<SysTree>& sys, bool particles_done) {
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

}  // namespace ogh
