// octgrav_build.cu -- the octree build of Sec. 2.1 on the GPU: Morton keys,
// a stable LSD radix sort, the level-by-level split of key ranges, the
// bottom-up cell properties, the groups and the work items, written straight
// into the device arrays the walk kernel reads.
//
// The result equals the host build (octgrav_host.cpp) byte for byte: the same
// FP64 operations in the same order (this file is compiled with -fmad=false,
// the host with -ffp-contract=off), the same stable sort, and the same array
// layout (cells of each system in breadth-first order, systems one after the
// other). Every kernel reads its sizes from device memory, so the whole build
// is enqueued without a host round trip; the host reads one result block at
// the end (cell capacity overflow there means: enlarge and build again).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "octgrav_internal.h"

namespace og {
namespace {

constexpr int MAXD = 21;          // depth limit (Morton keys of 3 x 21 bits)
constexpr int NLEV = MAXD + 1;    // levels 0..21
constexpr int TB = 256;           // threads per block
constexpr int IPT = 16;           // elements per thread in the chunked kernels
constexpr int TILE = TB * IPT;    // particles per chunk (sort, box, keys)
constexpr int GL = 4096;          // blocks of the level kernels
constexpr int GLT = 1024;         // threads of the level scan (GL / GLT entries each)
constexpr unsigned FULL = 0xffffffffu;
constexpr int LBINS = 32;  // leaf size bins of the moment pass (32 = "32 or more")
constexpr int IBINS = 256; // work-item size bins of the default processing order (item_max <= 256)

struct SysGeo {  // root cube of a system: lower corner, side, 2^21 * fl(1 / side)
  double lo[3], side, rscale;
};

struct Chunk {  // TILE particles (or fewer) of one system
  int sys, first, count, cs;  // system, first particle, count, first chunk of the system
  int nbs, pad0, pad1, pad2;  // chunks of the system
};

// Scratch layout (byte offsets into one allocation).
struct Layout {
  size_t keyA, keyB, valA, valB, cnt, dtot, part, sg, xs, ms, chunks, offs, chunk0;
  size_t ckey, cpar, cpf, cpc, csys, cfc, cnc, spl, lpre, bsum, lvl, misc;
  size_t sstart, send, lofs, ni, lorder, lhist, ihist, gmark, gidx, gcell, nitem, ioff, sblk;
  size_t total;
};

inline size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

Layout layout(int64_t n, int n_sys, int64_t n_chunks, int64_t cap) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += al(bytes);
    return at;
  };
  L.keyA = take(8 * n);
  L.keyB = take(8 * n);
  L.valA = take(4 * n);
  L.valB = take(4 * n);
  L.cnt = take(4 * 256 * n_chunks);
  L.dtot = take(4 * 256 * static_cast<size_t>(n_sys));
  L.part = take(8 * 6 * n_chunks);
  L.sg = take(sizeof(SysGeo) * n_sys);
  L.xs = take(24 * n);
  L.ms = take(8 * n);
  L.chunks = take(sizeof(Chunk) * n_chunks);
  L.offs = take(8 * (n_sys + 1));
  L.chunk0 = take(4 * (n_sys + 1));
  L.ckey = take(8 * cap);
  L.cpar = take(4 * cap);
  L.cpf = take(4 * cap);
  L.cpc = take(4 * cap);
  L.csys = take(4 * cap);
  L.cfc = take(4 * cap);
  L.cnc = take(4 * cap);
  L.spl = take(4 * 9 * std::min<int64_t>(n, cap));
  L.lpre = take(4 * std::min<int64_t>(n, cap));
  L.bsum = take(4 * GL);
  L.lvl = take(4 * (NLEV + 2));
  L.misc = take(4 * 16);
  L.sstart = take(4 * static_cast<size_t>(n_sys) * NLEV);
  L.send = take(4 * static_cast<size_t>(n_sys) * NLEV);
  L.lofs = take(4 * static_cast<size_t>(n_sys) * NLEV);
  L.ni = take(n_sys > 1 ? 4 * cap : 0);
  L.lorder = take(4 * cap);
  L.lhist = take(4 * 2 * LBINS);
  L.ihist = take(4 * 2 * IBINS);
  L.gmark = take(4 * n);
  L.gidx = take(4 * n);
  L.gcell = take(4 * n);
  L.nitem = take(4 * n);
  L.ioff = take(4 * n);
  L.sblk = take(4 * ((n + TILE - 1) / TILE + 1));
  L.total = o;
  return L;
}

// misc[] slots (int)
enum { M_NGROUPS = 0, M_NITEMS = 1, M_NLEAVES = 2, M_MAXGROUP = 3, M_STATUS = 4 };

template <class T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

__device__ __forceinline__ uint64_t spread21(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

// Integer key with the order of `<` on non-NaN doubles (the two zeros equal),
// so that min / max run on the integer pipe (FP64 is slow on this part).
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b == (-0x7fffffffffffffffLL - 1) ? 0 : b ^ 0x7fffffffffffffffLL);
}
// min / max with the tie rule of std::min / std::max (the first argument
// wins ties, so signed zeros come out as on the host)
__device__ __forceinline__ double lesser(double a, double b) { return order_key(b) < order_key(a) ? b : a; }
__device__ __forceinline__ double greater(double a, double b) { return order_key(a) < order_key(b) ? b : a; }

__device__ __forceinline__ int octant_at(uint64_t code, int child_depth) {
  return static_cast<int>((code >> (3 * (MAXD - child_depth))) & 7);
}

// Exclusive block-wide scan of one int per thread (TB threads); returns the
// exclusive prefix and writes the block total to *total.
__device__ int block_scan_excl(int v, int* total) {
  __shared__ int warp_tot[TB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < TB / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(FULL, t, d);
      if (lane >= d) t += y;
    }
    if (lane < TB / 32) warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  const int before = w ? warp_tot[w - 1] : 0;
  *total = warp_tot[TB / 32 - 1];
  __syncthreads();  // warp_tot is reused by the next call
  return before + x - v;
}

// ---------------------------------------------------------------- keys and sort

// Bounding box per chunk; flags non-finite coordinates or masses and
// negative masses.
__global__ void __launch_bounds__(TB) k_bbox(const double* __restrict__ pos, const double* __restrict__ mass,
                                             const Chunk* __restrict__ ch, double* __restrict__ part,
                                             int* __restrict__ misc) {
  const Chunk c = ch[blockIdx.x];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (int k = threadIdx.x; k < c.count; k += TB) {
    const int64_t i = c.first + k;
    for (int d = 0; d < 3; ++d) {
      const double v = pos[3 * i + d];
      bad |= !isfinite(v);
      mn[d] = lesser(mn[d], v);
      mx[d] = greater(mx[d], v);
    }
    const double m = mass[i];
    bad |= !isfinite(m) || m < 0;
  }
  __shared__ double red[6][TB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = 0; d < 3; ++d) {
    for (int s = 16; s; s >>= 1) {
      mn[d] = lesser(mn[d], __shfl_xor_sync(FULL, mn[d], s));
      mx[d] = greater(mx[d], __shfl_xor_sync(FULL, mx[d], s));
    }
    if (lane == 0) {
      red[d][w] = mn[d];
      red[3 + d][w] = mx[d];
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&misc[M_STATUS], GPU_BUILD_BADINPUT);
  if (threadIdx.x < 6) {
    double v = red[threadIdx.x][0];
    for (int k = 1; k < TB / 32; ++k) v = threadIdx.x < 3 ? lesser(v, red[threadIdx.x][k]) : greater(v, red[threadIdx.x][k]);
    part[6 * blockIdx.x + threadIdx.x] = v;
  }
}

// Root cube per system (the host build's arithmetic, operation for operation).
// One block per system.
__global__ void __launch_bounds__(TB) k_root(const double* __restrict__ part, const int* __restrict__ chunk0,
                                             SysGeo* __restrict__ sg) {
  const int s = blockIdx.x;
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = chunk0[s] + threadIdx.x; b < chunk0[s + 1]; b += TB)
    for (int d = 0; d < 3; ++d) {
      mn[d] = lesser(mn[d], part[6 * b + d]);
      mx[d] = greater(mx[d], part[6 * b + 3 + d]);
    }
  __shared__ double red[6][TB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o; o >>= 1) {
      mn[d] = lesser(mn[d], __shfl_xor_sync(FULL, mn[d], o));
      mx[d] = greater(mx[d], __shfl_xor_sync(FULL, mx[d], o));
    }
    if (lane == 0) {
      red[d][w] = mn[d];
      red[3 + d][w] = mx[d];
    }
  }
  __syncthreads();
  if (threadIdx.x) return;
  for (int k = 1; k < TB / 32; ++k)
    for (int d = 0; d < 3; ++d) {
      red[d][0] = lesser(red[d][0], red[d][k]);
      red[3 + d][0] = greater(red[3 + d][0], red[3 + d][k]);
    }
  for (int d = 0; d < 3; ++d) {
    mn[d] = red[d][0];
    mx[d] = red[3 + d][0];
  }
  double ext = mx[0] - mn[0];
  if (mx[1] - mn[1] > ext) ext = mx[1] - mn[1];
  if (mx[2] - mn[2] > ext) ext = mx[2] - mn[2];
  if (!(ext > 0)) ext = 1.0;
  const double side = ext * (1.0 + 1.0 / 1048576.0);
  for (int d = 0; d < 3; ++d) sg[s].lo[d] = (mn[d] + mx[d]) * 0.5 - side * 0.5;
  sg[s].side = side;
  sg[s].rscale = (1.0 / side) * 2097152.0;
}

__global__ void __launch_bounds__(TB) k_morton(const double* __restrict__ pos, const Chunk* __restrict__ ch,
                                               const SysGeo* __restrict__ sg, uint64_t* __restrict__ key,
                                               uint32_t* __restrict__ val) {
  const Chunk c = ch[blockIdx.x];
  const SysGeo g = sg[c.sys];
  const double* lo = g.lo;
  const double side = g.side;
  const double scale = 2097152.0;  // 2^21
  const uint64_t qmax = (1ull << MAXD) - 1;
  for (int k = threadIdx.x; k < c.count; k += TB) {
    const int64_t i = c.first + k;
    uint64_t q[3];
    for (int d = 0; d < 3; ++d) {
      // The quantised coordinate is floor(fl(fl(x - lo) / side) * 2^21) =
      // floor(fl(fl(x - lo) * 2^21 / side)). a = fl(x - lo) * g.rscale is
      // within 4 ulp (< 2^-29 for a <= 2^21) of fl(fl(x - lo) * 2^21 / side),
      // so whenever no integer lies within 2^-28 of a the floors agree; the
      // rare remaining cases take the division.
      const double dx = pos[3 * i + d] - lo[d];
      const double a = dx * g.rscale;
      double v = floor(a - 0x1p-28);
      if (v != floor(a + 0x1p-28)) v = floor((dx / side) * scale);
      q[d] = v <= 0 ? 0 : (v >= static_cast<double>(qmax) ? qmax : static_cast<uint64_t>(v));
    }
    key[i] = spread21(q[0]) | (spread21(q[1]) << 1) | (spread21(q[2]) << 2);
    val[i] = static_cast<uint32_t>(i);
  }
}

// Digit histogram of one chunk, stored at (system, digit, chunk within the
// system): the scan over a (system, digit) row is then contiguous.
__global__ void __launch_bounds__(TB) k_upsweep(const uint64_t* __restrict__ key, const Chunk* __restrict__ ch,
                                                int shift, int* __restrict__ cnt) {
  __shared__ int h[256];
  const Chunk c = ch[blockIdx.x];
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < c.count; k += TB)
    atomicAdd(&h[(key[c.first + k] >> shift) & 255], 1);
  __syncthreads();
  cnt[256 * c.cs + threadIdx.x * c.nbs + (blockIdx.x - c.cs)] = h[threadIdx.x];
}

// Exclusive scan of a[0..m) in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_single(int* __restrict__ a, const int* __restrict__ m_dev, int m_max,
                                                      int* __restrict__ total) {
  const int m = m_dev ? min(*m_dev, m_max) : m_max;
  __shared__ int ws[32];
  const int per = (m + 1023) / 1024;
  const int lo = min(m, threadIdx.x * per), hi = min(m, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += a[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = s;
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = ws[lane];
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(FULL, t, d);
      if (lane >= d) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  int run = (w ? ws[w - 1] : 0) + x - s;
  for (int i = lo; i < hi; ++i) {
    const int v = a[i];
    a[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023 && total) *total = ws[31];
}

// Per (system, digit): exclusive scan over the system's chunks in place, and
// the digit's total. One warp per (system, digit).
__global__ void __launch_bounds__(TB) k_scan_digits(int* __restrict__ cnt, const int* __restrict__ chunk0, int n_sys,
                                                    int* __restrict__ dtot) {
  const int seg = static_cast<int>((blockIdx.x * static_cast<int64_t>(TB) + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (seg >= 256 * n_sys) return;
  const int s = seg >> 8, d = seg & 255;
  const int cs = chunk0[s], nbs = chunk0[s + 1] - cs;
  int* a = cnt + 256 * static_cast<int64_t>(cs) + static_cast<int64_t>(d) * nbs;
  int run = 0;
  for (int base = 0; base < nbs; base += 32) {
    const int v = base + lane < nbs ? a[base + lane] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (base + lane < nbs) a[base + lane] = run + x - v;
    run += __shfl_sync(FULL, x, 31);
  }
  if (lane == 0) dtot[seg] = run;
}

// Stable scatter of one chunk by the digit at `shift`: warp w ranks its 512
// elements round by round (32 at a time, in order), the warps' counts are
// combined in warp order, and the chunk's offsets come from the scan.
__global__ void __launch_bounds__(TB) k_downsweep(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                  uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                  const Chunk* __restrict__ ch, int shift,
                                                  const int* __restrict__ cnt, const int* __restrict__ dtot) {
  __shared__ int wc[TB / 32][257];  // per-warp digit counters (+ one for empty slots)
  __shared__ int goff[256];
  const Chunk c = ch[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < (TB / 32) * 257; k += TB) (&wc[0][0])[k] = 0;
  {  // destination of this chunk's first element of each digit
    int unused;
    const int dbase = block_scan_excl(dtot[256 * c.sys + threadIdx.x], &unused);
    goff[threadIdx.x] = ch[c.cs].first + dbase + cnt[256 * c.cs + threadIdx.x * c.nbs + (blockIdx.x - c.cs)];
  }
  __syncthreads();
  uint64_t kk[IPT];
  uint32_t vv[IPT];
  int rk[IPT];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const int e = w * (32 * IPT) + r * 32 + lane;
    const bool ok = e < c.count;
    kk[r] = ok ? kin[c.first + e] : 0ull;
    vv[r] = ok ? vin[c.first + e] : 0u;
    const int d = ok ? static_cast<int>((kk[r] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(FULL, d);
    const int before = wc[w][d];
    rk[r] = before + __popc(peers & lt);
    __syncwarp();
    if (lane == __ffs(peers) - 1) wc[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // warp offsets per digit
    const int d = threadIdx.x;
    int run = 0;
    for (int q = 0; q < TB / 32; ++q) {
      const int t = wc[q][d];
      wc[q][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const int e = w * (32 * IPT) + r * 32 + lane;
    if (e < c.count) {
      const int d = static_cast<int>((kk[r] >> shift) & 255);
      const int dst = goff[d] + wc[w][d] + rk[r];
      kout[dst] = kk[r];
      vout[dst] = vv[r];
    }
  }
}

// Particles in tree order: FP64 copies for the moments, hi/lo FP32 records
// for the walk kernel, and the permutation.
__global__ void k_gather(const uint32_t* __restrict__ val, const double* __restrict__ pos,
                         const double* __restrict__ mass, int64_t n, double* __restrict__ xs,
                         double* __restrict__ ms, float4* __restrict__ parts, int* __restrict__ perm) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = val[t];
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], m = mass[i];
    xs[3 * t] = x;
    xs[3 * t + 1] = y;
    xs[3 * t + 2] = z;
    ms[t] = m;
    const float hx = static_cast<float>(x), hy = static_cast<float>(y), hz = static_cast<float>(z);
    parts[2 * t] = make_float4(hx, hy, hz, static_cast<float>(m));
    parts[2 * t + 1] = make_float4(static_cast<float>(x - static_cast<double>(hx)),
                                   static_cast<float>(y - static_cast<double>(hy)),
                                   static_cast<float>(z - static_cast<double>(hz)), 0.f);
    perm[t] = static_cast<int>(i);
  }
}

// ---------------------------------------------------------------- levels

struct Cells {
  uint64_t* key;
  int *par, *pf, *pc, *sys, *fc, *nc;
};

__global__ void k_roots(int n_sys, const int64_t* __restrict__ offs, Cells C, int* __restrict__ lvl) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n_sys) {
    C.key[s] = 1;
    C.par[s] = -1;
    C.pf[s] = static_cast<int>(offs[s]);
    C.pc[s] = static_cast<int>(offs[s + 1] - offs[s]);
    C.sys[s] = s;
    C.fc[s] = -1;
    C.nc[s] = 0;
  }
  if (s <= NLEV + 1) lvl[s] = s == 0 ? 0 : n_sys;
}

// Block b of GL takes a contiguous range of the level's cells.
__device__ __forceinline__ void level_range(const int* lvl, int L, int& lb, int& le, int& c0, int& c1) {
  lb = lvl[L];
  le = lvl[L + 1];
  const int nl = le - lb;
  const int chunk = (nl + GL - 1) / GL;
  c0 = min(le, lb + static_cast<int>(blockIdx.x) * chunk);
  c1 = min(le, c0 + chunk);
}

// First position p in [a, b) whose child octant at depth D is >= o (b if
// none); octants ascend inside a cell. The warp probes 32 evenly spaced
// positions per round (all lanes get the same answer).
__device__ int warp_partition(const uint64_t* __restrict__ code, int a, int b, int D, int o, int lane) {
  // invariant: the answer lies in [a, b], and b is the end or a known hit
  while (b - a > 32) {
    const int64_t span = b - a;
    const int p = a + static_cast<int>((lane + 1) * span / 33);
    const unsigned m = __ballot_sync(FULL, octant_at(code[p], D) >= o);
    const int k = m ? __ffs(m) - 1 : 32;
    const int lo = k == 0 ? a : a + static_cast<int>(k * span / 33) + 1;
    const int hi = k == 32 ? b : a + static_cast<int>((k + 1) * span / 33);
    a = lo;
    b = hi;
  }
  const int p = a + lane;
  const unsigned m = __ballot_sync(FULL, p < b && octant_at(code[p], D) >= o);
  return m ? a + __ffs(m) - 1 : b;
}

// Split points of a cell holding particles [f, f + cnt): sp[o] = the first
// position whose child octant at depth D is >= o, sp[0] = f, sp[8] = f + cnt.
// One warp; a cell of at most 32 particles takes a single round of loads.
// Every lane returns the same sp.
__device__ void warp_split(const uint64_t* __restrict__ code, int f, int cnt, int D, int lane, int* sp) {
  sp[0] = f;
  sp[8] = f + cnt;
  if (cnt <= 32) {  // one probe per particle
    const int oc = lane < cnt ? octant_at(code[f + lane], D) : 8;
    for (int o = 1; o < 8; ++o) {
      const unsigned m = __ballot_sync(FULL, oc >= o);
      sp[o] = m ? f + __ffs(m) - 1 : f + cnt;
    }
    return;
  }
  for (int o = 1; o < 8; ++o) sp[o] = warp_partition(code, sp[o - 1], f + cnt, D, o, lane);
}

// Split points of every cell of level L (the host's partition points; one
// warp per cell), and the block-local exclusive prefix of the children counts.
__global__ void __launch_bounds__(TB) k_split(int L, const uint64_t* __restrict__ code, Cells C, int n_leaf,
                                              const int* __restrict__ lvl, int* __restrict__ spl,
                                              int* __restrict__ lpre, int* __restrict__ bsum) {
  constexpr int W = TB / 32;
  __shared__ int sn[W];
  __shared__ int carry;
  int lb, le, c0, c1;
  level_range(lvl, L, lb, le, c0, c1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  for (int base = c0; base < c1; base += W) {
    const int c = base + w;
    int nch = 0;
    if (c < c1) {  // warp-uniform
      const int f = C.pf[c], cnt = C.pc[c];
      int sp[9];
      if (cnt <= n_leaf || L >= MAXD) {
        for (int o = 0; o < 9; ++o) sp[o] = f;
      } else {
        warp_split(code, f, cnt, L + 1, lane, sp);
        for (int o = 0; o < 8; ++o) nch += sp[o + 1] > sp[o];
      }
      if (lane == 0) {
        int* d = &spl[9 * static_cast<int64_t>(c - lb)];
        for (int o = 0; o < 9; ++o) d[o] = sp[o];
      }
    }
    if (lane == 0) sn[w] = nch;
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = carry;
      for (int k = 0; k < W && base + k < c1; ++k) {
        lpre[base + k - lb] = run;
        run += sn[k];
      }
      carry = run;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = carry;
}

// Offsets of the blocks' children and the end of level L + 1; a level that
// does not fit the cell capacity stops the build (status overflow).
__global__ void __launch_bounds__(GLT) k_scan_level(int L, int* __restrict__ bsum, int* __restrict__ lvl, int cap,
                                                    int* __restrict__ misc) {
  constexpr int PER = GL / GLT;
  __shared__ int ws[32];
  int e[PER], v = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    e[k] = bsum[PER * threadIdx.x + k];
    v += e[k];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = ws[lane];
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(FULL, t, d);
      if (lane >= d) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  int run = (w ? ws[w - 1] : 0) + x - v;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    bsum[PER * threadIdx.x + k] = run;
    run += e[k];
  }
  if (threadIdx.x == 0) {
    const int le = lvl[L + 1];
    const int64_t next = static_cast<int64_t>(le) + ws[31];
    if (next > cap) {
      atomicOr(&misc[M_STATUS], GPU_BUILD_OVERFLOW);
      lvl[L + 2] = le;
    } else {
      lvl[L + 2] = static_cast<int>(next);
    }
  }
}

__global__ void __launch_bounds__(TB) k_emit(int L, Cells C, const int* __restrict__ lvl, const int* __restrict__ spl,
                                             const int* __restrict__ lpre, const int* __restrict__ boff,
                                             const int* __restrict__ misc) {
  if (misc[M_STATUS] & GPU_BUILD_OVERFLOW) return;
  int lb, le, c0, c1;
  level_range(lvl, L, lb, le, c0, c1);
  for (int c = c0 + threadIdx.x; c < c1; c += TB) {
    const int* sp = &spl[9 * static_cast<int64_t>(c - lb)];
    int nch = 0;
    for (int o = 0; o < 8; ++o) nch += sp[o + 1] > sp[o];
    if (!nch) continue;
    int w = le + boff[blockIdx.x] + lpre[c - lb];
    C.fc[c] = w;
    C.nc[c] = nch;
    const uint64_t k = C.key[c];
    const int s = C.sys[c];
    for (int o = 0; o < 8; ++o) {
      if (sp[o + 1] <= sp[o]) continue;
      C.key[w] = (k << 3) | static_cast<uint64_t>(o);
      C.par[w] = c;
      C.pf[w] = sp[o];
      C.pc[w] = sp[o + 1] - sp[o];
      C.sys[w] = s;
      C.fc[w] = -1;
      C.nc[w] = 0;
      ++w;
    }
  }
}

// After a level loop capped at max_level < MAXD: flag a cell of level
// max_level that still needs splitting (the caller rebuilds without the cap),
// and close the level table so that lvl[NLEV] is the cell count.
__global__ void k_depth_check(int max_level, Cells C, int* __restrict__ lvl, int n_leaf, int* __restrict__ misc) {
  const int lb = lvl[max_level], le = lvl[max_level + 1];
  bool deeper = false;
  for (int c = lb + blockIdx.x * blockDim.x + threadIdx.x; c < le; c += gridDim.x * blockDim.x)
    deeper |= C.pc[c] > n_leaf;
  if (__syncthreads_or(deeper) && threadIdx.x == 0) atomicOr(&misc[M_STATUS], GPU_BUILD_DEEPER);
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int L = max_level + 2; L <= NLEV; ++L) lvl[L] = le;
}

// Level of cell c: the last L with lvl[L] <= c.
__device__ __forceinline__ int level_of(const int* lvl, int c) {
  int L = 0;
  while (L + 1 < NLEV && lvl[L + 1] <= c) ++L;
  return L;
}

// ---------------------------------------------------------------- system-major order (batches)

__global__ void k_sys_bounds(const int* __restrict__ lvl, const int* __restrict__ csys, int* __restrict__ sstart,
                             int* __restrict__ send) {
  const int nc = lvl[NLEV];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const int L = level_of(lvl, c), s = csys[c];
    if (c == lvl[L] || csys[c - 1] != s) sstart[s * NLEV + L] = c;
    if (c == lvl[L + 1] - 1 || csys[c + 1] != s) send[s * NLEV + L] = c + 1;
  }
}

// Per system: its first cell in the final order and the final position of
// its first cell of every level.
__global__ void __launch_bounds__(1024) k_sys_offsets(int n_sys, const int* __restrict__ sstart,
                                                      const int* __restrict__ send, int* __restrict__ lofs,
                                                      int64_t* __restrict__ cell_off) {
  __shared__ int ws[32];
  const int per = (n_sys + 1023) / 1024;
  const int lo = min(n_sys, static_cast<int>(threadIdx.x) * per), hi = min(n_sys, lo + per);
  int sum = 0;
  for (int s = lo; s < hi; ++s)
    for (int L = 0; L < NLEV; ++L) sum += send[s * NLEV + L] - sstart[s * NLEV + L];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = sum;
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(FULL, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = ws[lane];
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(FULL, t, d);
      if (lane >= d) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  int run = (w ? ws[w - 1] : 0) + x - sum;
  for (int s = lo; s < hi; ++s) {
    cell_off[s] = run;
    for (int L = 0; L < NLEV; ++L) {
      lofs[s * NLEV + L] = run;
      run += send[s * NLEV + L] - sstart[s * NLEV + L];
    }
  }
  if (threadIdx.x == 1023) cell_off[n_sys] = ws[31];
}

__global__ void k_new_index(const int* __restrict__ lvl, const int* __restrict__ csys, const int* __restrict__ sstart,
                            const int* __restrict__ lofs, int* __restrict__ ni) {
  const int nc = lvl[NLEV];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const int L = level_of(lvl, c), k = csys[c] * NLEV + L;
    ni[c] = lofs[k] + (c - sstart[k]);
  }
}

__global__ void k_one_system_offsets(const int* __restrict__ lvl, int64_t* __restrict__ cell_off) {
  cell_off[0] = 0;
  cell_off[1] = lvl[NLEV];
}

// ---------------------------------------------------------------- cell properties

struct Props {  // final-order FP64 arrays and records
  double *bmin, *bmax, *cube, *M, *com, *S;
  uint64_t* key;
  float4* geo;
  int2* link;
  float4* mp;
  int *pcount, *cfirst;
};

__device__ __forceinline__ int final_index(const int* ni, int c) { return ni ? ni[c] : c; }

// Tight box, boundary cube, mass, centre of mass and second moments of cell
// c (a leaf from its particles, a node from its children with the
// parallel-axis shift, in the host build's operation order), then its records.
template <bool LEAF>
__device__ __forceinline__ void cell_props(int c, Cells C, const int* __restrict__ ni, const double* __restrict__ xs,
                                           const double* __restrict__ ms, const Props& P) {
  const int j = final_index(ni, c);
  double bn[3] = {INFINITY, INFINITY, INFINITY}, bx[3] = {-INFINITY, -INFINITY, -INFINITY};
  double Mc = 0, sx = 0, sy = 0, sz = 0;
  const int f = C.pf[c], cnt = C.pc[c], nch = LEAF ? 0 : C.nc[c];
  const int jc = LEAF ? 0 : final_index(ni, C.fc[c]);  // children are contiguous in both orders
  if (LEAF) {
    for (int t = f; t < f + cnt; ++t) {
      const double* xp = &xs[3 * static_cast<int64_t>(t)];
      const double x0 = xp[0], x1 = xp[1], x2 = xp[2], m = ms[t];
      bn[0] = lesser(bn[0], x0);
      bn[1] = lesser(bn[1], x1);
      bn[2] = lesser(bn[2], x2);
      bx[0] = greater(bx[0], x0);
      bx[1] = greater(bx[1], x1);
      bx[2] = greater(bx[2], x2);
      Mc += m;
      sx = fma(m, x0, sx);
      sy = fma(m, x1, sy);
      sz = fma(m, x2, sz);
    }
  } else {
    for (int q = jc; q < jc + nch; ++q) {
      for (int d = 0; d < 3; ++d) {
        bn[d] = lesser(bn[d], P.bmin[3 * q + d]);
        bx[d] = greater(bx[d], P.bmax[3 * q + d]);
      }
      const double m = P.M[q];
      Mc += m;
      sx = fma(m, P.com[3 * q], sx);
      sy = fma(m, P.com[3 * q + 1], sy);
      sz = fma(m, P.com[3 * q + 2], sz);
    }
  }
  double cu[4], cm[3], s6[6] = {0, 0, 0, 0, 0, 0};
  for (int d = 0; d < 3; ++d) cu[d] = (bn[d] + bx[d]) * 0.5;
  double e = bx[0] - bn[0];
  if (bx[1] - bn[1] > e) e = bx[1] - bn[1];
  if (bx[2] - bn[2] > e) e = bx[2] - bn[2];
  cu[3] = 0.5 * e;
  if (Mc > 0) {
    cm[0] = sx / Mc;
    cm[1] = sy / Mc;
    cm[2] = sz / Mc;
  } else {
    cm[0] = cu[0];
    cm[1] = cu[1];
    cm[2] = cu[2];
  }
  auto add_outer = [&](double wt, double y0, double y1, double y2) {
    const double w0 = wt * y0, w1 = wt * y1, w2 = wt * y2;
    s6[0] = fma(w0, y0, s6[0]);
    s6[1] = fma(w1, y1, s6[1]);
    s6[2] = fma(w2, y2, s6[2]);
    s6[3] = fma(w0, y1, s6[3]);
    s6[4] = fma(w0, y2, s6[4]);
    s6[5] = fma(w1, y2, s6[5]);
  };
  if (LEAF) {
    for (int t = f; t < f + cnt; ++t) {
      const double* xp = &xs[3 * static_cast<int64_t>(t)];
      add_outer(ms[t], xp[0] - cm[0], xp[1] - cm[1], xp[2] - cm[2]);
    }
  } else {
    for (int q = jc; q < jc + nch; ++q) {
      for (int k = 0; k < 6; ++k) s6[k] += P.S[6 * q + k];
      add_outer(P.M[q], P.com[3 * q] - cm[0], P.com[3 * q + 1] - cm[1], P.com[3 * q + 2] - cm[2]);
    }
  }
  for (int d = 0; d < 3; ++d) {
    P.bmin[3 * j + d] = bn[d];
    P.bmax[3 * j + d] = bx[d];
    P.com[3 * j + d] = cm[d];
  }
  for (int d = 0; d < 4; ++d) P.cube[4 * j + d] = cu[d];
  for (int k = 0; k < 6; ++k) P.S[6 * j + k] = s6[k];
  P.M[j] = Mc;
  // records read by the walk kernel
  P.key[j] = C.key[c];
  P.geo[j] = make_float4(static_cast<float>(cu[0]), static_cast<float>(cu[1]), static_cast<float>(cu[2]),
                         static_cast<float>(cu[3]));
  P.link[j] = LEAF ? make_int2(f, -cnt) : make_int2(jc, nch);
  float chi[3], clo[3];
  for (int d = 0; d < 3; ++d) {
    chi[d] = static_cast<float>(cm[d]);
    clo[d] = static_cast<float>(cm[d] - static_cast<double>(chi[d]));
  }
  const double tr = s6[0] + s6[1] + s6[2];
  P.mp[4 * j] = make_float4(chi[0], chi[1], chi[2], static_cast<float>(Mc));
  P.mp[4 * j + 1] = make_float4(clo[0], clo[1], clo[2], static_cast<float>(cnt));
  P.mp[4 * j + 2] = make_float4(static_cast<float>(3.0 * s6[0]), static_cast<float>(3.0 * s6[1]),
                                static_cast<float>(3.0 * s6[2]), static_cast<float>(3.0 * s6[3]));
  P.mp[4 * j + 3] = make_float4(static_cast<float>(3.0 * s6[4]), static_cast<float>(3.0 * s6[5]),
                                static_cast<float>(1.5 * tr), static_cast<float>(0.5 * tr));
  P.pcount[j] = cnt;
  P.cfirst[j] = f;
}

// Leaves (of every level) bucketed by particle count, largest first, so that
// the lanes of a warp loop over equally many particles: histogram, then
// scatter of the cell indices into lorder.
__device__ __forceinline__ int leaf_bin(int cnt) { return LBINS - min(cnt, LBINS); }  // 32+ -> bin 0

__global__ void __launch_bounds__(TB) k_leaf_hist(Cells C, const int* __restrict__ lvl, int* __restrict__ lhist,
                                                  int* __restrict__ misc) {
  __shared__ int h[LBINS];
  if (threadIdx.x < LBINS) h[threadIdx.x] = 0;
  __syncthreads();
  const int nc = lvl[NLEV];
  int leaves = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
    if (C.nc[c] == 0) {
      atomicAdd(&h[leaf_bin(C.pc[c])], 1);
      ++leaves;
    }
  for (int s = 16; s; s >>= 1) leaves += __shfl_xor_sync(FULL, leaves, s);
  if ((threadIdx.x & 31) == 0 && leaves) atomicAdd(&misc[M_NLEAVES], leaves);
  __syncthreads();
  if (threadIdx.x < LBINS && h[threadIdx.x]) atomicAdd(&lhist[threadIdx.x], h[threadIdx.x]);
}

__global__ void __launch_bounds__(TB) k_leaf_scatter(Cells C, const int* __restrict__ lvl,
                                                     const int* __restrict__ lhist, int* __restrict__ lfill,
                                                     int* __restrict__ lorder) {
  __shared__ int base[LBINS], h[LBINS];
  if (threadIdx.x < 32) {
    const int v = lhist[threadIdx.x];
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, x, o);
      if (threadIdx.x >= o) x += y;
    }
    base[threadIdx.x] = x - v;
  }
  const int nc = lvl[NLEV];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t c0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; c0 < nc; c0 += stride) {
    if (threadIdx.x < LBINS) h[threadIdx.x] = 0;
    __syncthreads();
    const int c = static_cast<int>(c0) + threadIdx.x;
    const bool leaf = c < nc && C.nc[c] == 0;
    const int b = leaf ? leaf_bin(C.pc[c]) : 0;
    const int r = leaf ? atomicAdd(&h[b], 1) : 0;  // rank within the block's bin
    __syncthreads();
    if (threadIdx.x < LBINS && h[threadIdx.x]) h[threadIdx.x] = atomicAdd(&lfill[threadIdx.x], h[threadIdx.x]);
    __syncthreads();
    if (leaf) lorder[base[b] + h[b] + r] = c;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(TB) k_leaf_props(Cells C, const int* __restrict__ lorder,
                                                   const int* __restrict__ misc, const int* __restrict__ ni,
                                                   const double* __restrict__ xs, const double* __restrict__ ms,
                                                   Props P) {
  const int nl = misc[M_NLEAVES];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nl; k += gridDim.x * blockDim.x)
    cell_props<true>(lorder[k], C, ni, xs, ms, P);
}

// Nodes of level L (their children, one level deeper, are done).
__global__ void __launch_bounds__(TB) k_node_props(int L, Cells C, const int* __restrict__ lvl,
                                                   const int* __restrict__ ni, Props P) {
  const int lb = lvl[L], le = lvl[L + 1];
  for (int c = lb + blockIdx.x * blockDim.x + threadIdx.x; c < le; c += gridDim.x * blockDim.x)
    if (C.nc[c] > 0) cell_props<false>(c, C, ni, nullptr, nullptr, P);
}

// ---------------------------------------------------------------- groups and items

// A group is a cell that is a leaf or holds <= n_group particles while its
// parent does not (the property is inherited by descendants, so "the first
// such cell from the root" is exactly this). Marked at its first particle.
__global__ void k_group_mark(Cells C, const int* __restrict__ lvl, int n_group, int* __restrict__ gmark,
                             int* __restrict__ gcell) {
  const int nc = lvl[NLEV];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const bool elig = C.nc[c] == 0 || C.pc[c] <= n_group;
    const int p = C.par[c];
    const bool pelig = p >= 0 && C.pc[p] <= n_group;  // a parent is never a leaf
    if (elig && !pelig) {
      gmark[C.pf[c]] = 1;
      gcell[C.pf[c]] = c;
    }
  }
}

// Block sums of in[0..n) in chunks of TILE.
__global__ void __launch_bounds__(TB) k_scan_reduce(const int* __restrict__ in, const int* __restrict__ n_dev, int n_max,
                                                    int* __restrict__ sblk) {
  const int n = n_dev ? min(*n_dev, n_max) : n_max;
  const int64_t lo = static_cast<int64_t>(blockIdx.x) * TILE;
  int s = 0;
  for (int64_t i = lo + threadIdx.x; i < min(static_cast<int64_t>(n), lo + TILE); i += TB) s += in[i];
  int tot;
  block_scan_excl(s, &tot);
  if (threadIdx.x == 0) sblk[blockIdx.x] = tot;
}

// out = exclusive prefix of in (chunk offsets from the scanned block sums).
__global__ void __launch_bounds__(TB) k_scan_down(const int* __restrict__ in, const int* __restrict__ n_dev, int n_max,
                                                  const int* __restrict__ sblk, int* __restrict__ out) {
  const int n = n_dev ? min(*n_dev, n_max) : n_max;
  const int64_t lo = static_cast<int64_t>(blockIdx.x) * TILE + static_cast<int64_t>(threadIdx.x) * IPT;
  int v[IPT], s = 0;
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    v[k] = lo + k < n ? in[lo + k] : 0;
    s += v[k];
  }
  int tot;
  int run = sblk[blockIdx.x] + block_scan_excl(s, &tot);
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    if (lo + k < n) out[lo + k] = run;
    run += v[k];
  }
}

__global__ void k_group_emit(int64_t n, const int* __restrict__ gmark, const int* __restrict__ gidx,
                             const int* __restrict__ gcell, Cells C, const int* __restrict__ ni,
                             int* __restrict__ group_cell, int* __restrict__ group_sys, int* __restrict__ misc) {
  int mg = 0;
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (!gmark[t]) continue;
    const int g = gidx[t], c = gcell[t];
    group_cell[g] = final_index(ni, c);
    group_sys[g] = C.sys[c];
    mg = max(mg, C.pc[c]);
  }
  for (int s = 16; s; s >>= 1) mg = max(mg, __shfl_xor_sync(FULL, mg, s));
  if ((threadIdx.x & 31) == 0 && mg) atomicMax(&misc[M_MAXGROUP], mg);
}

__global__ void k_item_count(const int* __restrict__ n_groups, const int* __restrict__ group_cell,
                             const int* __restrict__ pcount, int item_max, int split, int* __restrict__ nitem) {
  const int ng = *n_groups;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
    nitem[g] = item_count(pcount[group_cell[g]], item_max, split != 0);
}

// Work items of every group, cut by next_item_size (at most item_max
// particles each), all with the group's box, centre (hi/lo) and particle range.
__global__ void k_items(const int* __restrict__ n_groups, const int* __restrict__ group_cell,
                        const int* __restrict__ group_sys, const int* __restrict__ ioff, const int64_t* __restrict__ cell_off,
                        Props P, int item_max, int split, int4* __restrict__ items, float4* __restrict__ ibox,
                        uint64_t* __restrict__ item_key, int* __restrict__ group_item) {
  const int ng = *n_groups;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    const int c = group_cell[g], s = group_sys[g];
    const int pf = P.cfirst[c], cnt = P.pcount[c];
    float chi[3], clo[3];
    for (int d = 0; d < 3; ++d) {
      const double C0 = P.cube[4 * c + d];
      chi[d] = static_cast<float>(C0);
      clo[d] = static_cast<float>(C0 - static_cast<double>(chi[d]));
    }
    const float4 b0 = make_float4(static_cast<float>(P.bmin[3 * c]), static_cast<float>(P.bmin[3 * c + 1]),
                                  static_cast<float>(P.bmin[3 * c + 2]), chi[0]);
    const float4 b1 = make_float4(static_cast<float>(P.bmax[3 * c]), static_cast<float>(P.bmax[3 * c + 1]),
                                  static_cast<float>(P.bmax[3 * c + 2]), chi[1]);
    const float4 b2 = make_float4(clo[0], clo[1], clo[2], chi[2]);
    const float4 b3 = make_float4(__int_as_float(pf), __int_as_float(cnt), 0.f, 0.f);
    const int root = static_cast<int>(cell_off[s]);
    int k = ioff[g];
    group_item[g] = k;
    for (int off = 0, sz; off < cnt; off += sz, ++k) {
      sz = next_item_size(cnt - off, item_max, split != 0);
      items[k] = make_int4(root, pf + off, sz, s);
      ibox[4 * static_cast<int64_t>(k)] = b0;
      ibox[4 * static_cast<int64_t>(k) + 1] = b1;
      ibox[4 * static_cast<int64_t>(k) + 2] = b2;
      ibox[4 * static_cast<int64_t>(k) + 3] = b3;
      item_key[k] = P.key[c];
    }
  }
}

// Default processing order of the work items: most particles first (a
// counting sort on the item size; the order inside a size is arbitrary and
// does not affect any result).
__global__ void __launch_bounds__(TB) k_item_hist(const int* __restrict__ n_items, const int4* __restrict__ items,
                                                  int* __restrict__ ihist) {
  __shared__ int h[IBINS];
  for (int k = threadIdx.x; k < IBINS; k += TB) h[k] = 0;
  __syncthreads();
  const int ni = *n_items;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ni; k += gridDim.x * blockDim.x)
    atomicAdd(&h[IBINS - min(items[k].z, IBINS)], 1);
  __syncthreads();
  for (int k = threadIdx.x; k < IBINS; k += TB)
    if (h[k]) atomicAdd(&ihist[k], h[k]);
}

__global__ void __launch_bounds__(TB) k_item_scatter(const int* __restrict__ n_items, const int4* __restrict__ items,
                                                     const int* __restrict__ ihist, int* __restrict__ ifill,
                                                     int* __restrict__ order) {
  __shared__ int base[IBINS], h[IBINS];
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < IBINS; ++k) {
      base[k] = run;
      run += ihist[k];
    }
  }
  const int ni = *n_items;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t k0 = static_cast<int64_t>(blockIdx.x) * blockDim.x; k0 < ni; k0 += stride) {
    for (int k = threadIdx.x; k < IBINS; k += TB) h[k] = 0;
    __syncthreads();
    const int k = static_cast<int>(k0) + threadIdx.x;
    const bool live = k < ni;
    const int b = live ? IBINS - min(items[k].z, IBINS) : 0;
    const int r = live ? atomicAdd(&h[b], 1) : 0;
    __syncthreads();
    for (int q = threadIdx.x; q < IBINS; q += TB)
      if (h[q]) h[q] = atomicAdd(&ifill[q], h[q]);
    __syncthreads();
    if (live) order[base[b] + h[b] + r] = k;
    __syncthreads();
  }
}

__global__ void k_clear_status(int* __restrict__ misc) { misc[M_STATUS] = 0; }

__global__ void k_finish(const int* __restrict__ lvl, const int* __restrict__ misc, int64_t* __restrict__ res) {
  int depth = 0;
  for (int L = 0; L < NLEV; ++L)
    if (lvl[L + 1] > lvl[L]) depth = L;
  res[GB_NCELLS] = lvl[NLEV];
  res[GB_NGROUPS] = misc[M_NGROUPS];
  res[GB_NITEMS] = misc[M_NITEMS];
  res[GB_DEPTH] = depth;
  res[GB_NLEAVES] = misc[M_NLEAVES];
  res[GB_MAXGROUP] = misc[M_MAXGROUP];
  res[GB_STATUS] = misc[M_STATUS];
}

__global__ void k_unpermute(const float4* __restrict__ out, const int* __restrict__ perm, int64_t n,
                            double* __restrict__ acc, double* __restrict__ pot) {
  for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float4 a = out[t];
    const int64_t i = perm[t];
    acc[3 * i] = a.x;
    acc[3 * i + 1] = a.y;
    acc[3 * i + 2] = a.z;
    if (pot) pot[i] = a.w;
  }
}

int grid_for(int64_t n, int per_block) {
  const int64_t b = (n + per_block - 1) / per_block;
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16)));
}

// Items from the groups (group_cell, group_sys and the cell arrays in P).
cudaError_t enqueue_items(const GpuBuild& a, const Layout& Lo, int item_max, cudaStream_t st) {
  int* misc = at<int>(a.scratch, Lo.misc);
  int* nitem = at<int>(a.scratch, Lo.nitem);
  int* ioff = at<int>(a.scratch, Lo.ioff);
  int* sblk = at<int>(a.scratch, Lo.sblk);
  const int nmax = static_cast<int>(a.n);
  const int nb = static_cast<int>((a.n + TILE - 1) / TILE);
  Props P{a.bmin, a.bmax, a.cube, a.M, a.com, a.S, a.key, a.geo, a.link, a.mp, a.pcount, a.cfirst};
  k_item_count<<<grid_for(a.n, TB), TB, 0, st>>>(&misc[M_NGROUPS], a.group_cell, a.pcount, item_max, a.item_split,
                                                 nitem);
  k_scan_reduce<<<nb, TB, 0, st>>>(nitem, &misc[M_NGROUPS], nmax, sblk);
  k_scan_single<<<1, 1024, 0, st>>>(sblk, nullptr, nb, &misc[M_NITEMS]);
  k_scan_down<<<nb, TB, 0, st>>>(nitem, &misc[M_NGROUPS], nmax, sblk, ioff);
  k_items<<<grid_for(a.n, TB), TB, 0, st>>>(&misc[M_NGROUPS], a.group_cell, a.group_sys, ioff, a.cell_off, P,
                                            item_max, a.item_split, a.items, a.ibox, a.item_key, a.group_item);
  int* ihist = at<int>(a.scratch, Lo.ihist);
  cudaError_t e = cudaMemsetAsync(ihist, 0, 4 * 2 * IBINS, st);
  if (e != cudaSuccess) return e;
  k_item_hist<<<grid_for(a.n, TB), TB, 0, st>>>(&misc[M_NITEMS], a.items, ihist);
  k_item_scatter<<<grid_for(a.n, TB), TB, 0, st>>>(&misc[M_NITEMS], a.items, ihist, ihist + IBINS, a.order);
  return cudaGetLastError();
}

std::vector<Chunk> make_chunks(const int64_t* offsets, int n_sys, std::vector<int>& chunk0) {
  std::vector<Chunk> ch;
  chunk0.assign(n_sys + 1, 0);
  for (int s = 0; s < n_sys; ++s) {
    chunk0[s] = static_cast<int>(ch.size());
    const int64_t p0 = offsets[s], ns = offsets[s + 1] - p0;
    const int nbs = static_cast<int>((ns + TILE - 1) / TILE);
    for (int k = 0; k < nbs; ++k) {
      Chunk c{};
      c.sys = s;
      c.first = static_cast<int>(p0 + static_cast<int64_t>(k) * TILE);
      c.count = static_cast<int>(std::min<int64_t>(TILE, ns - static_cast<int64_t>(k) * TILE));
      c.cs = chunk0[s];
      c.nbs = nbs;
      ch.push_back(c);
    }
  }
  chunk0[n_sys] = static_cast<int>(ch.size());
  return ch;
}

}  // namespace

size_t gpu_build_scratch_bytes(int64_t n, int n_sys, int64_t cap) {
  const int64_t chunks = (n + TILE - 1) / TILE + n_sys;
  return layout(n, n_sys, chunks, cap).total;
}

cudaError_t gpu_build_tables(const GpuBuild& a, cudaStream_t st) {
  std::vector<int> chunk0;
  const std::vector<Chunk> ch = make_chunks(a.offsets, a.n_sys, chunk0);
  const Layout Lo = layout(a.n, a.n_sys, (a.n + TILE - 1) / TILE + a.n_sys, a.cap);
  if (Lo.total > a.scratch_bytes) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(at<Chunk>(a.scratch, Lo.chunks), ch.data(), sizeof(Chunk) * ch.size(),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(at<int64_t>(a.scratch, Lo.offs), a.offsets, 8 * (a.n_sys + 1), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(at<int>(a.scratch, Lo.chunk0), chunk0.data(), 4 * (a.n_sys + 1), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

cudaError_t gpu_build(const GpuBuild& a, cudaStream_t st) {
  cudaError_t e = gpu_build_tables(a, st);
  return e != cudaSuccess ? e : gpu_build_kernels(a, st);
}

cudaError_t gpu_build_kernels(const GpuBuild& a, cudaStream_t st) {
  int nch = 0;
  for (int s = 0; s < a.n_sys; ++s) nch += static_cast<int>((a.offsets[s + 1] - a.offsets[s] + TILE - 1) / TILE);
  const Layout Lo = layout(a.n, a.n_sys, (a.n + TILE - 1) / TILE + a.n_sys, a.cap);
  if (Lo.total > a.scratch_bytes) return cudaErrorInvalidValue;
  void* S = a.scratch;
  uint64_t* keyA = at<uint64_t>(S, Lo.keyA);
  uint64_t* keyB = at<uint64_t>(S, Lo.keyB);
  uint32_t* valA = at<uint32_t>(S, Lo.valA);
  uint32_t* valB = at<uint32_t>(S, Lo.valB);
  int* cnt = at<int>(S, Lo.cnt);
  double* part = at<double>(S, Lo.part);
  SysGeo* sg = at<SysGeo>(S, Lo.sg);
  double* xs = at<double>(S, Lo.xs);
  double* ms = at<double>(S, Lo.ms);
  Chunk* dch = at<Chunk>(S, Lo.chunks);
  int64_t* doffs = at<int64_t>(S, Lo.offs);
  int* dchunk0 = at<int>(S, Lo.chunk0);
  int* lvl = at<int>(S, Lo.lvl);
  int* misc = at<int>(S, Lo.misc);
  int* spl = at<int>(S, Lo.spl);
  int* lpre = at<int>(S, Lo.lpre);
  int* bsum = at<int>(S, Lo.bsum);
  Cells C{at<uint64_t>(S, Lo.ckey), at<int>(S, Lo.cpar), at<int>(S, Lo.cpf), at<int>(S, Lo.cpc),
          at<int>(S, Lo.csys),      at<int>(S, Lo.cfc),  at<int>(S, Lo.cnc)};
  Props P{a.bmin, a.bmax, a.cube, a.M, a.com, a.S, a.key, a.geo, a.link, a.mp, a.pcount, a.cfirst};
  cudaError_t e;
#define OG_TRY(x)                       \
  do {                                  \
    if ((e = (x)) != cudaSuccess) return e; \
  } while (0)
  OG_TRY(cudaMemsetAsync(misc, 0, 4 * 16, st));

  // ---- keys and the stable sort (8 passes of 8 bits over the 63-bit keys)
  k_bbox<<<nch, TB, 0, st>>>(a.pos, a.mass, dch, part, misc);
  k_root<<<a.n_sys, TB, 0, st>>>(part, dchunk0, sg);
  k_morton<<<nch, TB, 0, st>>>(a.pos, dch, sg, keyA, valA);
  int* dtot = at<int>(S, Lo.dtot);
  const int segblocks = (256 * a.n_sys + TB / 32 - 1) / (TB / 32);
  for (int pass = 0; pass < 8; ++pass) {
    const int sh = 8 * pass;
    const bool even = (pass & 1) == 0;
    k_upsweep<<<nch, TB, 0, st>>>(even ? keyA : keyB, dch, sh, cnt);
    k_scan_digits<<<segblocks, TB, 0, st>>>(cnt, dchunk0, a.n_sys, dtot);
    k_downsweep<<<nch, TB, 0, st>>>(even ? keyA : keyB, even ? valA : valB, even ? keyB : keyA,
                                    even ? valB : valA, dch, sh, cnt, dtot);
  }
  OG_TRY(cudaGetLastError());
  k_gather<<<grid_for(a.n, TB), TB, 0, st>>>(valA, a.pos, a.mass, a.n, xs, ms, a.parts, a.perm);

  // ---- cells, level by level (sizes live in lvl[] on the device)
  k_roots<<<(std::max(a.n_sys, NLEV + 2) + 127) / 128, 128, 0, st>>>(a.n_sys, doffs, C, lvl);
  const int top = std::min(std::max(a.max_level, 1), MAXD);  // deepest level built
  for (int L = 0; L < top; ++L) {
    k_split<<<GL, TB, 0, st>>>(L, keyA, C, a.n_leaf, lvl, spl, lpre, bsum);
    k_scan_level<<<1, GLT, 0, st>>>(L, bsum, lvl, static_cast<int>(a.cap), misc);
    k_emit<<<GL, TB, 0, st>>>(L, C, lvl, spl, lpre, bsum, misc);
  }
  if (top < MAXD) k_depth_check<<<grid_for(a.n, TB), TB, 0, st>>>(top, C, lvl, a.n_leaf, misc);
  OG_TRY(cudaGetLastError());

  // ---- final (system-major) cell order
  const int gc = grid_for(a.cap, TB);
  int* ni = nullptr;
  if (a.n_sys > 1) {
    int* sstart = at<int>(S, Lo.sstart);
    int* send = at<int>(S, Lo.send);
    int* lofs = at<int>(S, Lo.lofs);
    ni = at<int>(S, Lo.ni);
    OG_TRY(cudaMemsetAsync(sstart, 0, 4 * static_cast<size_t>(a.n_sys) * NLEV, st));
    OG_TRY(cudaMemsetAsync(send, 0, 4 * static_cast<size_t>(a.n_sys) * NLEV, st));
    k_sys_bounds<<<gc, TB, 0, st>>>(lvl, C.sys, sstart, send);
    k_sys_offsets<<<1, 1024, 0, st>>>(a.n_sys, sstart, send, lofs, a.cell_off);
    k_new_index<<<gc, TB, 0, st>>>(lvl, C.sys, sstart, lofs, ni);
  } else {
    k_one_system_offsets<<<1, 1, 0, st>>>(lvl, a.cell_off);
  }

  // ---- properties: every leaf at once, then the nodes deepest level first
  int* lorder = at<int>(S, Lo.lorder);
  int* lhist = at<int>(S, Lo.lhist);
  OG_TRY(cudaMemsetAsync(lhist, 0, 4 * 2 * LBINS, st));
  k_leaf_hist<<<gc, TB, 0, st>>>(C, lvl, lhist, misc);
  k_leaf_scatter<<<gc, TB, 0, st>>>(C, lvl, lhist, lhist + LBINS, lorder);
  k_leaf_props<<<gc, TB, 0, st>>>(C, lorder, misc, ni, xs, ms, P);
  for (int L = top - 1; L >= 0; --L) k_node_props<<<gc, TB, 0, st>>>(L, C, lvl, ni, P);
  OG_TRY(cudaGetLastError());

  // ---- groups (ordered by first particle) and work items
  int* gmark = at<int>(S, Lo.gmark);
  int* gidx = at<int>(S, Lo.gidx);
  int* gcell = at<int>(S, Lo.gcell);
  int* sblk = at<int>(S, Lo.sblk);
  const int nb = static_cast<int>((a.n + TILE - 1) / TILE);
  OG_TRY(cudaMemsetAsync(gmark, 0, 4 * a.n, st));
  k_group_mark<<<gc, TB, 0, st>>>(C, lvl, a.n_group, gmark, gcell);
  k_scan_reduce<<<nb, TB, 0, st>>>(gmark, nullptr, static_cast<int>(a.n), sblk);
  k_scan_single<<<1, 1024, 0, st>>>(sblk, nullptr, nb, &misc[M_NGROUPS]);
  k_scan_down<<<nb, TB, 0, st>>>(gmark, nullptr, static_cast<int>(a.n), sblk, gidx);
  k_group_emit<<<grid_for(a.n, TB), TB, 0, st>>>(a.n, gmark, gidx, gcell, C, ni, a.group_cell, a.group_sys, misc);
  OG_TRY(enqueue_items(a, Lo, a.item_max, st));
  k_finish<<<1, 1, 0, st>>>(lvl, misc, a.result);
#undef OG_TRY
  return cudaGetLastError();
}

cudaError_t gpu_refit(const GpuBuild& a, cudaStream_t st) {
  const Layout Lo = layout(a.n, a.n_sys, (a.n + TILE - 1) / TILE + a.n_sys, a.cap);
  if (Lo.total > a.scratch_bytes) return cudaErrorInvalidValue;
  void* S = a.scratch;
  int nch = 0;
  for (int s = 0; s < a.n_sys; ++s) nch += static_cast<int>((a.offsets[s + 1] - a.offsets[s] + TILE - 1) / TILE);
  int* misc = at<int>(S, Lo.misc);
  const int* lvl = at<int>(S, Lo.lvl);
  Cells C{at<uint64_t>(S, Lo.ckey), at<int>(S, Lo.cpar), at<int>(S, Lo.cpf), at<int>(S, Lo.cpc),
          at<int>(S, Lo.csys),      at<int>(S, Lo.cfc),  at<int>(S, Lo.cnc)};
  Props P{a.bmin, a.bmax, a.cube, a.M, a.com, a.S, a.key, a.geo, a.link, a.mp, a.pcount, a.cfirst};
  const int* ni = a.n_sys > 1 ? at<int>(S, Lo.ni) : nullptr;
  const int gc = grid_for(a.cap, TB);
  cudaError_t e;
  // the status bits only: the counts of the build stay
  k_clear_status<<<1, 1, 0, st>>>(misc);
  k_bbox<<<nch, TB, 0, st>>>(a.pos, a.mass, at<Chunk>(S, Lo.chunks), at<double>(S, Lo.part), misc);
  k_gather<<<grid_for(a.n, TB), TB, 0, st>>>(at<uint32_t>(S, Lo.valA), a.pos, a.mass, a.n, at<double>(S, Lo.xs),
                                             at<double>(S, Lo.ms), a.parts, a.perm);
  k_leaf_props<<<gc, TB, 0, st>>>(C, at<int>(S, Lo.lorder), misc, ni, at<double>(S, Lo.xs), at<double>(S, Lo.ms), P);
  for (int L = MAXD - 1; L >= 0; --L) k_node_props<<<gc, TB, 0, st>>>(L, C, lvl, ni, P);
  k_items<<<grid_for(a.n, TB), TB, 0, st>>>(&misc[M_NGROUPS], a.group_cell, a.group_sys, at<int>(S, Lo.ioff),
                                            a.cell_off, P, a.item_max, a.item_split, a.items, a.ibox, a.item_key,
                                            a.group_item);
  k_finish<<<1, 1, 0, st>>>(lvl, misc, a.result);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t gpu_build_items(const GpuBuild& a, cudaStream_t st) {
  const Layout Lo = layout(a.n, a.n_sys, (a.n + TILE - 1) / TILE + a.n_sys, a.cap);
  if (Lo.total > a.scratch_bytes) return cudaErrorInvalidValue;
  cudaError_t e = enqueue_items(a, Lo, a.item_max, st);
  if (e != cudaSuccess) return e;
  int* misc = at<int>(a.scratch, Lo.misc);
  const int* lvl = at<int>(a.scratch, Lo.lvl);
  k_finish<<<1, 1, 0, st>>>(lvl, misc, a.result);
  return cudaGetLastError();
}

__global__ void k_pull(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n16;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

cudaError_t pull_host(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | bytes) & 15u) return cudaErrorInvalidValue;
  const int64_t n16 = static_cast<int64_t>(bytes / 16);
  if (n16 == 0) return cudaSuccess;
  k_pull<<<grid_for(n16, TB * 4), TB, 0, st>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), n16);
  return cudaGetLastError();
}

cudaError_t gpu_unpermute(const float4* out, const int* perm, int64_t n, double* acc, double* pot, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_unpermute<<<grid_for(n, TB), TB, 0, st>>>(out, perm, n, acc, pot);
  return cudaGetLastError();
}

}  // namespace og
