// octgrav_kernels.cu -- fused tree walk + interaction-list evaluation for sm_103a.
//
// One warp owns one work item (a group of at most 32*R particles, Sec. 2.2:
// particles of a group share one interaction list). It walks the octree from
// the root with a node stack in shared memory (Listing 1), applies the opening
// test to the children of up to four popped nodes at once (one lane per child,
// Listing 2), and compacts the three outcomes with warp ballots:
//   accepted cell -> cell list: its 64-byte multipole record is fetched into a
//                    shared-memory ring by an asynchronous copy issued right
//                    after the step that accepted it (STAGE selects the copy:
//                    TMA tile::gather4 of 4 records per instruction with
//                    mbarrier completion, per-lane 16-byte cp.async, or one
//                    cp.async.bulk per record);
//   opened leaf   -> leaf queue (first particle, count);
//   opened node   -> pushed on the stack as (first child, number of children).
// Full tiles of 32 cell records are evaluated one walk step after their copies
// were issued, by all particles of the group (Listing 3); the leaf queue is
// evaluated in double-buffered chunks of 32 source particles (Listing 4). The paper's two
// walks (count, then write) and the host prefix sum between them (Sec. 2.2)
// are gone: lists never leave the SM.
//
// Lane mapping: the n_g particles of the item are spread over w = ceil(n_g/R)
// lanes (R particles per lane); the warp holds s = 32/w such slices, and slice
// k evaluates list entries k, k+s, k+2s, ... . Partial sums of the slices are
// combined with shuffles at the end, so small groups still fill the warp (the
// paper lost ~70% of its threads to part-filled groups, Sec. 3.3). Every
// arithmetic op is a packed FP32x2 op: with R = 2 its halves are the lane's two
// particles and the cell or source fields are broadcast; with R = 1 its halves
// are two records.
//
// Precision: positions are group-relative FP32, x' = (x_hi - C_hi) + (x_lo - C_lo)
// with C the group centre kept as a hi/lo float pair; sums are accumulated in
// FP32 and folded into a compensated (TwoSum) accumulator every ~32 terms.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>

#include "../../include/octgrav.h"
#include "octgrav_internal.h"
#include "octgrav_mlp.h"

namespace og {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARPS = 8;          // warps per CTA
constexpr int TILE = 32;          // cell records per tile
constexpr int NTILE = 3;          // tiles in the ring (copies run one step ahead)
// Staging of accepted cell records into the shared-memory ring.
constexpr int STAGE_BULK = 0;     // one cp.async.bulk (64 B) per record, issued by its lane
constexpr int STAGE_ASYNC = 1;    // four 16-byte cp.async per record, issued by its lane
constexpr int STAGE_GATHER4 = 2;  // TMA tile::gather4: 4 records per instruction, lane 0 issues
template <int STAGE>
struct RingStride {               // float4 per ring slot
  static constexpr int v = STAGE == STAGE_GATHER4 ? 4 : 5;  // 64 B rows / 64 B + 16 B pad
};
constexpr int STACK = 512;        // node-stack entries per warp
constexpr int CPAIR = 7;          // float4 per cell pair in the evaluated tile (6 = 96 B, 7 = 112 B)
constexpr int SPAIR = 3;          // float4 per source pair in a particle chunk (2 = 32 B, 3 = 48 B)
constexpr int FOLD_EVERY = 4;     // fold partial sums every FOLD_EVERY * (slices) tiles/chunks
constexpr int PCH = 32;           // source particles per particle-particle chunk
constexpr int LQ = 64;            // leaf-queue entries (flushed at >= 32)
constexpr long long WAIT_LIMIT = 1ll << 31;  // cycles (~1 s) before a wait gives up

constexpr int STACK_MLP = 384;    // node-stack entries per warp in the learned-criterion kernel
constexpr int MQ = 64;            // deferred candidates awaiting the network (flushed at >= 32)

template <bool GATHER, bool MLP>
struct __align__(128) WarpSmemT {
  float4 ring[NTILE * TILE * 5];    // 7680 B; stride 80 B keeps 8 slots on 8 bank quads
  float4 pbuf[2][2 * PCH];          // 2048 B: two chunks of source particles (hi, lo records),
                                    // rewritten in place into pairs; also the network's input
                                    // tile (32 rows x 16 bf16) during a network step
  int2 leafq[LQ];                   // 512 B: (first particle, count)
  int lpref[LQ];                    // 256 B: inclusive prefix of counts
  int stack[MLP ? STACK_MLP : STACK];  // packed (first child << 3 | n_child - 1)
  int cidx[GATHER ? NTILE * TILE : 1]; // cell index per ring slot (gather4 staging)
  int mq[MLP ? MQ : 1];             // deferred candidate cells
  unsigned long long bar[NTILE];    // one mbarrier per ring tile
};

static_assert(16 * CPAIR * (TILE / 2) <= 64 * TILE, "cell pairs must fit the tile's ring slots");
static_assert(16 * SPAIR * (PCH / 2) + 4 * PCH <= 32 * PCH, "source pairs and indices must fit a chunk");

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Raise the barrier's expected transaction bytes (no arrival).
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bulk asynchronous copy global -> shared; completion is signalled on bar.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// TMA gather of 4 rows (64-byte cell records) of a 2-D tensor map into
// 256 contiguous bytes of shared memory; completion on bar.
__device__ __forceinline__ void gather4_g2s(uint32_t dst, const void* tmap, int r0, int r1, int r2, int r3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tmap), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}
// Per-thread 16-byte asynchronous copy global -> shared (L1-allocating).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Hardware reciprocal square root (MUFU), denormal inputs flushed; every
// argument here is >= eps^2 > 0.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) writes to the same locations.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-level tensor-core MMA: D(16x8 f32) += A(16x16 bf16, row) * B(16x8 bf16, col).
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}
__device__ __forceinline__ void ldmatrix_x4(uint32_t* r, uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// The learned criterion's network on the first 16 * n16 rows of X (one
// candidate per lane; 16 bf16 inputs per row, the last 4 zero): 12 -> 64 -> 64
// -> 1 with ReLU, bf16 weights and inputs, FP32 accumulation on the tensor
// cores. Returns the prediction for row `lane` (rows >= 16 * n16 are not
// evaluated). Layer-1 accumulators become layer-2 A fragments in registers
// (the C and A fragment layouts line up pairwise).
__device__ float mlp_eval(const MlpDevice& W, uint32_t x_smem, int lane, int n16) {
  float y00 = 0.f, y01 = 0.f, y10 = 0.f, y11 = 0.f;
  const int q = 2 * (lane & 3);
#pragma unroll 1
  for (int t = 0; t < n16; ++t) {
    uint32_t a[4];
    ldmatrix_x4(a, x_smem + 2u * ((16 * t + (lane & 15)) * 16 + (lane >> 4) * 8));
    uint32_t a2[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(c0, a, W.w1f[2 * kk][lane]);
      mma_bf16(c1, a, W.w1f[2 * kk + 1][lane]);
      const int u0 = 16 * kk + q, u1 = u0 + 8;
      a2[kk][0] = pack_bf16(fmaxf(c0[0] + W.b1[u0], 0.f), fmaxf(c0[1] + W.b1[u0 + 1], 0.f));
      a2[kk][1] = pack_bf16(fmaxf(c0[2] + W.b1[u0], 0.f), fmaxf(c0[3] + W.b1[u0 + 1], 0.f));
      a2[kk][2] = pack_bf16(fmaxf(c1[0] + W.b1[u1], 0.f), fmaxf(c1[1] + W.b1[u1 + 1], 0.f));
      a2[kk][3] = pack_bf16(fmaxf(c1[2] + W.b1[u1], 0.f), fmaxf(c1[3] + W.b1[u1 + 1], 0.f));
    }
    float r0 = 0.f, r1 = 0.f;
#pragma unroll 1
    for (int j = 0; j < 8; ++j) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_bf16(acc, a2[kk], W.w2f[kk][j][lane]);
      const int u = 8 * j + q;
      r0 = fmaf(fmaxf(acc[0] + W.b2[u], 0.f), W.w3[u], r0);
      r0 = fmaf(fmaxf(acc[1] + W.b2[u + 1], 0.f), W.w3[u + 1], r0);
      r1 = fmaf(fmaxf(acc[2] + W.b2[u], 0.f), W.w3[u], r1);
      r1 = fmaf(fmaxf(acc[3] + W.b2[u + 1], 0.f), W.w3[u + 1], r1);
    }
    r0 += __shfl_xor_sync(FULL, r0, 1);
    r0 += __shfl_xor_sync(FULL, r0, 2);
    r1 += __shfl_xor_sync(FULL, r1, 1);
    r1 += __shfl_xor_sync(FULL, r1, 2);
    if (t == 0) {
      y00 = r0;  // row lane/4 of tile 0
      y01 = r1;  // row lane/4 + 8
    } else {
      y10 = r0;
      y11 = r1;
    }
  }
  const int r = lane & 15, src = 4 * (r & 7);
  const float v00 = __shfl_sync(FULL, y00, src), v01 = __shfl_sync(FULL, y01, src);
  const float v10 = __shfl_sync(FULL, y10, src), v11 = __shfl_sync(FULL, y11, src);
  const float v = lane < 16 ? (r < 8 ? v00 : v01) : (r < 8 ? v10 : v11);
  return v + W.b3;
}

// Bounded wait for the phase of parity `parity`; false after ~1 s.
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  bool ok = mbar_try_wait(bar, parity);
  if (!ok) {
    const long long t0 = clock64();
    while (!(ok = mbar_try_wait(bar, parity))) {
      if (clock64() - t0 > WAIT_LIMIT) break;
    }
  }
  return __all_sync(FULL, ok);
}

// ---------------------------------------------------------------- arithmetic

// Opening test (Sec. 2.2, Listing 2): open iff (2h)^2 >= theta^2 d^2, d the
// distance from the group's tight box to the cell's boundary cube. Every
// operation is an explicitly rounded FP32 op (no contraction), so the
// decision is reproducible bit for bit by a CPU implementation.
__device__ __forceinline__ bool must_open(float4 g, float3 gmin, float3 gmax, float theta2) {
  const float h = g.w;
  const float bx = __fsub_rn(gmin.x, __fadd_rn(g.x, h)), tx = __fsub_rn(__fsub_rn(g.x, h), gmax.x);
  const float by = __fsub_rn(gmin.y, __fadd_rn(g.y, h)), ty = __fsub_rn(__fsub_rn(g.y, h), gmax.y);
  const float bz = __fsub_rn(gmin.z, __fadd_rn(g.z, h)), tz = __fsub_rn(__fsub_rn(g.z, h), gmax.z);
  const float dx = fmaxf(0.f, fmaxf(bx, tx));
  const float dy = fmaxf(0.f, fmaxf(by, ty));
  const float dz = fmaxf(0.f, fmaxf(bz, tz));
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  return __fmul_rn(4.0f, __fmul_rn(h, h)) >= __fmul_rn(theta2, d2);
}

struct Acc4 {
  float x, y, z, p;
};

// ---- packed FP32x2 arithmetic (Blackwell FFMA2 / FMUL2 / FADD2): every op
// below evaluates two interactions at once, halving the issued instructions.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrt_ftz(a.x), rsqrt_ftz(a.y)); }

struct Acc2 {  // partial sums of the two halves of a pair
  float2 x, y, z, p;
};

// Two cell records side by side (each field holds record a in .x, record b
// in .y): centre of mass relative to the group centre and negated (nc), -M,
// S3 = 3 S, T3 = 3T and T = tr(S)/2. 96 bytes = six 16-byte loads.
struct CellPair {
  float2 ncx, ncy, ncz, nM, sxx, syy, szz, sxy, sxz, syz, t3, t;
};

// Particle-cell interaction: second-order Taylor expansion of the Plummer
// kernel about the cell's centre of mass (monopole + quadrupole). With
// d = x_i - com, r^2 = |d|^2 + eps^2, S3 = 3S, q = d.S3.d, T = trS/2:
//   a   += d (-M + (3T - 2.5 q/r^2)/r^2) / r^3 + S3 d / r^5
//   phi -= (M + (q/(2 r^2) - T)/r^2) / r
__device__ __forceinline__ void body_cell2(float2 X, float2 Y, float2 Z, float2 eps2, const CellPair& c,
                                           Acc2& a) {
  const float2 dx = add2(X, c.ncx), dy = add2(Y, c.ncy), dz = add2(Z, c.ncz);
  const float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
  const float2 rinv = rsqrt2(r2);
  const float2 rinv2 = mul2(rinv, rinv);
  const float2 rinv3 = mul2(rinv, rinv2);
  const float2 rinv5 = mul2(rinv3, rinv2);
  const float2 sx = fma2(c.sxx, dx, fma2(c.sxy, dy, mul2(c.sxz, dz)));
  const float2 sy = fma2(c.sxy, dx, fma2(c.syy, dy, mul2(c.syz, dz)));
  const float2 sz = fma2(c.sxz, dx, fma2(c.syz, dy, mul2(c.szz, dz)));
  const float2 q = fma2(dx, sx, fma2(dy, sy, mul2(dz, sz)));
  const float2 t1 = mul2(q, rinv2);
  const float2 t2 = fma2(f2(-2.5f), t1, c.t3);
  const float2 cd = mul2(fma2(t2, rinv2, c.nM), rinv3);
  a.x = fma2(cd, dx, fma2(rinv5, sx, a.x));
  a.y = fma2(cd, dy, fma2(rinv5, sy, a.y));
  a.z = fma2(cd, dz, fma2(rinv5, sz, a.z));
  const float2 np2 = fma2(fma2(f2(-0.5f), t1, c.t), rinv2, c.nM);  // -(M + (q/(2r^2) - T)/r^2)
  a.p = fma2(np2, rinv, a.p);
}

// Two source particles side by side: negated positions (relative to the group
// centre) and negated masses. 32 bytes = two 16-byte loads.
struct SrcPair {
  float2 nx, ny, nz, nm;
};

// Particle-particle interaction with Plummer softening; nm = -m_j (0 drops a term).
__device__ __forceinline__ void body_body2(float2 X, float2 Y, float2 Z, float2 eps2, const SrcPair& s,
                                           float2 nm, Acc2& a) {
  const float2 dx = add2(X, s.nx), dy = add2(Y, s.ny), dz = add2(Z, s.nz);  // x_i - x_j
  const float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
  const float2 rinv = rsqrt2(r2);
  const float2 nmr = mul2(nm, rinv);
  const float2 nmr3 = mul2(nmr, mul2(rinv, rinv));
  a.x = fma2(nmr3, dx, a.x);  // += m_j (x_j - x_i) / r^3
  a.y = fma2(nmr3, dy, a.y);
  a.z = fma2(nmr3, dz, a.z);
  a.p = add2(a.p, nmr);       // -= m_j / r
}

// ---- particle-packed evaluation (two particles per lane): the halves of
// every packed operation are two particles of the group, and the cell or
// source quantities enter as one value broadcast to both halves.

// One cell record for the particle-packed layout (48 bytes = three 16-byte
// loads): centre of mass relative to the group centre, negated, -M, S3 = 3S
// (xx, yy, zz, xy, xz, yz), 3T and T = tr(S)/2.
struct CellRec {
  float ncx, ncy, ncz, nM, sxx, syy, szz, sxy, sxz, syz, t3, t;
};
constexpr int CREC = 3;  // float4 per cell record in the evaluated tile
static_assert(16 * CREC <= 64, "packed cell records must fit the tile's ring slots");
static_assert(16 * 32 + 4 * 32 <= 32 * 32, "packed sources and indices must fit a chunk");

// Particle-cell interaction of two particles (X, Y, Z halves) with one cell:
// the same expansion as body_cell2, with the monopole folded into the bracket,
//   a += (S3 d + (3T - 2.5 q/r^2 - M r^2) d) / r^5
// (33 packed operations for two interactions).
__device__ __forceinline__ void body_cellP(float2 X, float2 Y, float2 Z, float2 eps2, const CellRec& c,
                                           Acc2& a) {
  const float2 dx = add2(X, f2(c.ncx)), dy = add2(Y, f2(c.ncy)), dz = add2(Z, f2(c.ncz));
  const float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
  const float2 rinv = rsqrt2(r2);
  const float2 rinv2 = mul2(rinv, rinv);
  const float2 rinv5 = mul2(mul2(rinv, rinv2), rinv2);
  const float2 sx = fma2(f2(c.sxx), dx, fma2(f2(c.sxy), dy, mul2(f2(c.sxz), dz)));
  const float2 sy = fma2(f2(c.sxy), dx, fma2(f2(c.syy), dy, mul2(f2(c.syz), dz)));
  const float2 sz = fma2(f2(c.sxz), dx, fma2(f2(c.syz), dy, mul2(f2(c.szz), dz)));
  const float2 q = fma2(dx, sx, fma2(dy, sy, mul2(dz, sz)));
  const float2 t1 = mul2(q, rinv2);
  const float2 cb = fma2(f2(c.nM), r2, fma2(f2(-2.5f), t1, f2(c.t3)));  // 3T - 2.5 q/r^2 - M r^2
  a.x = fma2(rinv5, fma2(cb, dx, sx), a.x);
  a.y = fma2(rinv5, fma2(cb, dy, sy), a.y);
  a.z = fma2(rinv5, fma2(cb, dz, sz), a.z);
  const float2 np2 = fma2(fma2(f2(-0.5f), t1, f2(c.t)), rinv2, f2(c.nM));
  a.p = fma2(np2, rinv, a.p);
}

// Particle-particle interaction of two particles with one source (negated
// relative position sx, sy, sz); nm = -m_j per half (0 drops a term).
__device__ __forceinline__ void body_bodyP(float2 X, float2 Y, float2 Z, float2 eps2, float sx, float sy, float sz,
                                           float2 nm, Acc2& a) {
  const float2 dx = add2(X, f2(sx)), dy = add2(Y, f2(sy)), dz = add2(Z, f2(sz));
  const float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2)));
  const float2 rinv = rsqrt2(r2);
  const float2 nmr = mul2(nm, rinv);
  const float2 nmr3 = mul2(nmr, mul2(rinv, rinv));
  a.x = fma2(nmr3, dx, a.x);
  a.y = fma2(nmr3, dy, a.y);
  a.z = fma2(nmr3, dz, a.z);
  a.p = add2(a.p, nmr);
}

// Error-free transformation: hi + t = s + e exactly.
__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float t) {
  const float s = hi + t;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (t - bp);
  hi = s;
  lo += e;
}

template <int R>
struct Particles {
  float2 X[R], Y[R], Z[R];  // group-relative position, broadcast to both halves
  int idx[R];               // tree position, -1 for an empty slot
  Acc2 part[R];             // plain FP32 partial sums since the last fold
  Acc4 hi[R];               // compensated accumulator: value = hi + lo
  Acc4 lo[R];

  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      two_sum_into(hi[r].x, lo[r].x, part[r].x.x + part[r].x.y);
      two_sum_into(hi[r].y, lo[r].y, part[r].y.x + part[r].y.y);
      two_sum_into(hi[r].z, lo[r].z, part[r].z.x + part[r].z.y);
      two_sum_into(hi[r].p, lo[r].p, part[r].p.x + part[r].p.y);
      part[r].x = part[r].y = part[r].z = part[r].p = f2(0.f);
    }
  }
};

// Packed TwoSum of both halves: hi + t = s + e exactly in each half.
__device__ __forceinline__ void two_sum_into2(float2& hi, float2& lo, float2 t) {
  const float2 s = add2(hi, t);
  const float2 bp = sub2(s, hi);
  const float2 e = add2(sub2(hi, sub2(s, bp)), sub2(t, bp));
  hi = s;
  lo = add2(lo, e);
}

// Two particles per lane in the halves of every register (particle-packed
// layout): positions, partial sums since the last fold and compensated
// accumulators (value = hi + lo), each half one particle.
struct ParticlesP {
  float2 X, Y, Z;
  int idx[2];  // tree positions, -1 for an empty slot
  Acc2 part;
  Acc2 hi, lo;

  __device__ __forceinline__ void fold() {
    two_sum_into2(hi.x, lo.x, part.x);
    two_sum_into2(hi.y, lo.y, part.y);
    two_sum_into2(hi.z, lo.z, part.z);
    two_sum_into2(hi.p, lo.p, part.p);
    part.x = part.y = part.z = part.p = f2(0.f);
  }
};

__device__ __forceinline__ CellRec load_cell_rec(const float4* q) {
  const float4 a = q[0], b = q[1], c = q[2];
  return CellRec{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
}

__device__ __forceinline__ CellPair load_cell_pair(const float4* q) {
  const float4 a = q[0], b = q[1], c = q[2], d = q[3], e = q[4], f = q[5];
  return CellPair{make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y), make_float2(b.z, b.w),
                  make_float2(c.x, c.y), make_float2(c.z, c.w), make_float2(d.x, d.y), make_float2(d.z, d.w),
                  make_float2(e.x, e.y), make_float2(e.z, e.w), make_float2(f.x, f.y), make_float2(f.z, f.w)};
}
__device__ __forceinline__ SrcPair load_src_pair(const float4* q) {
  const float4 a = q[0], b = q[1];
  return SrcPair{make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y), make_float2(b.z, b.w)};
}

// ---------------------------------------------------------------- the kernel

// The learned-criterion kernel runs one CTA of 16 warps per SM (at most 128
// registers per thread, as the plain kernel's two CTAs of 8 warps): its
// network fragments and feature inputs fit, and its larger shared memory
// (the network, a candidate queue per warp) needs one CTA.
constexpr int WARPS_MLP = 16;

template <bool MLP>
struct CtaWarps {
  static constexpr int v = MLP ? WARPS_MLP : WARPS;
};

template <int R, int STAGE, bool CAPTURE, bool MLP, bool SPLIT = false>
__global__ void __launch_bounds__(CtaWarps<MLP>::v * 32, MLP ? 1 : 2) walk_eval_kernel(const __grid_constant__ KParams p) {
  constexpr int REC = RingStride<STAGE>::v;
  using WarpSmem = WarpSmemT<STAGE == STAGE_GATHER4, MLP>;
  constexpr int STK = MLP ? STACK_MLP : STACK;
  constexpr bool PK = (R == 2);  // particle-packed evaluation
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  // align to 128 B by offsetting the shared array itself (keeps the
  // shared address space visible to the compiler: LDS, not generic LD)
  unsigned char* smem_base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  WarpSmem& S = reinterpret_cast<WarpSmem*>(smem_base)[threadIdx.x >> 5];
  MlpDevice& NW = *reinterpret_cast<MlpDevice*>(smem_base + sizeof(WarpSmem) * CtaWarps<MLP>::v);
  if (MLP) {  // the network, shared by the CTA's warps
    const uint4* src = reinterpret_cast<const uint4*>(p.mlp);
    uint4* dst = reinterpret_cast<uint4*>(&NW);
    for (int k = threadIdx.x; k < static_cast<int>(sizeof(MlpDevice) / 16); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
  }
  const uint32_t bar0 = smem_u32(&S.bar[0]);
  if (lane == 0) {
    for (int t = 0; t < NTILE; ++t) mbar_init(bar0 + 8 * t, 1);
    fence_mbar_init();
  }
  __syncwarp();
  const unsigned lt = lanemask_lt();

  // Ring counters, warp-uniform and persistent across items: `app` counts
  // cell entries whose copies were issued, `done` those evaluated. Tile
  // (e / TILE) % NTILE holds entry e; its k-th use completes phase k.
  uint32_t app = 0, done = 0;
  uint32_t iss = 0;  // gather4 staging: entries whose copies were issued (multiple of 4)
  int status = 0;

  for (;;) {
    int item = 0, part = 0;
    if (lane == 0) {
      item = static_cast<int>(atomicAdd(p.work, 1u));
      if (SPLIT) {  // the parts of one item are consecutive work indices
        part = item % p.nparts;
        item /= p.nparts;
      }
      if (p.order && item < p.n_items) item = __ldg(p.order + item);  // longest first
    }
    item = __shfl_sync(FULL, item, 0);
    if (SPLIT) part = __shfl_sync(FULL, part, 0);
    if (item >= p.n_items) break;

    // capture mode: the row this item's lists go to (-1: not captured)
    const int slot = CAPTURE ? (p.dbg_slot ? __ldg(p.dbg_slot + item) : item) : -1;
    const int4 it = __ldg(p.items + item);
    const float4 b0 = __ldg(p.ibox + 4 * item);
    const float4 b1 = __ldg(p.ibox + 4 * item + 1);
    const float4 b2 = __ldg(p.ibox + 4 * item + 2);
    const float4 b3 = __ldg(p.ibox + 4 * item + 3);
    const int gfirst = __float_as_int(b3.x), gcount = __float_as_int(b3.y);  // the whole group
    const float4 sp = p.sysp ? __ldg(p.sysp + it.w) : p.sys0;
    const float theta2 = sp.x, G = p.sys0.z;
    const float2 E2 = f2(sp.y);
    float f10 = 0.f, f11 = 0.f;  // learned criterion: group size and distance from the system's CoM
    if (MLP) {
      const float4 r0 = __ldg(p.mp + 4 * it.x), r1 = __ldg(p.mp + 4 * it.x + 1);
      const float ox = (b0.w - r0.x) + (b2.x - r1.x), oy = (b1.w - r0.y) + (b2.y - r1.y),
                  oz = (b2.w - r0.z) + (b2.z - r1.z);
      f10 = static_cast<float>(gcount) / static_cast<float>(p.n_group);
      f11 = mlp_lg2(sqrtf(ox * ox + oy * oy + oz * oz));
    }
    const float3 gmin = make_float3(b0.x, b0.y, b0.z);
    const float3 gmax = make_float3(b1.x, b1.y, b1.z);
    const float3 chi = make_float3(b0.w, b1.w, b2.w);
    const float3 clo = make_float3(b2.x, b2.y, b2.z);
    // The item's body runs as a one-iteration loop, left by `break` in the
    // plain kernel and by `goto` in the learned one. Only code generation
    // differs: timed in one session against the same body without the loop,
    // the plain kernel is 0.7 % faster on the 1M Plummer sphere and 1.1 % on
    // the 4M clustered system (the compiler gives it 128 registers instead of
    // 123), the learned kernel within 0.3 %.
    bool stop = false;
    for (int once = 0; once < 1; ++once) {
    const int pf = it.y, np = it.z;

    // lane -> (slice, particles)
    const int w = (np + R - 1) / R;
    const int s = 32 / w;
    const int sl = lane / w;
    const int wl = lane - sl * w;
    const bool act = sl < s;

    // two particles per lane are packed into the halves of every operation
    // (PK); one particle per lane takes the records in pairs instead
    std::conditional_t<PK, ParticlesP, Particles<R>> P;
    float px[R], py[R], pz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = wl + r * w;
      const bool v = act && k < np;
      P.idx[r] = v ? pf + k : -1;
      float x = 0.f, y = 0.f, z = 0.f;
      if (v) {
        const float4 h4 = __ldg(p.parts + 2 * (pf + k));
        const float4 l4 = __ldg(p.parts + 2 * (pf + k) + 1);
        x = (h4.x - chi.x) + (l4.x - clo.x);
        y = (h4.y - chi.y) + (l4.y - clo.y);
        z = (h4.z - chi.z) + (l4.z - clo.z);
      }
      px[r] = x;
      py[r] = y;
      pz[r] = z;
    }
    if constexpr (PK) {
      P.X = make_float2(px[0], px[1]);
      P.Y = make_float2(py[0], py[1]);
      P.Z = make_float2(pz[0], pz[1]);
      P.part.x = P.part.y = P.part.z = P.part.p = f2(0.f);
      P.hi = P.part;
      P.lo = P.part;
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        P.X[r] = f2(px[r]);
        P.Y[r] = f2(py[r]);
        P.Z[r] = f2(pz[r]);
        P.part[r].x = P.part[r].y = P.part[r].z = P.part[r].p = f2(0.f);
        P.hi[r] = P.lo[r] = Acc4{0.f, 0.f, 0.f, 0.f};
      }
    }
    int nsince = 0;  // tiles since the last fold

    // ---- evaluation of one ring tile holding n records
    auto eval_tile = [&](int n) -> bool {
      const uint32_t tile = (done / TILE) % NTILE;
      const uint32_t parity = (done / (TILE * NTILE)) & 1u;
      if (STAGE == STAGE_ASYNC) {
        __syncwarp();  // the lanes' completed copies (waited by the caller) are visible
      } else if (!mbar_wait_bounded(bar0 + 8 * tile, parity)) {
        return false;
      }
      float4* base = &S.ring[tile * TILE * REC];
      // Rewrite the tile in place into the pair layout: record e becomes half
      // (e & 1) of pair e >> 1; an odd last record is paired with zeros.
      float v[12];
#pragma unroll
      for (int f = 0; f < 12; ++f) v[f] = 0.f;
      if (lane < n) {
        const float4 q0 = base[lane * REC], q1 = base[lane * REC + 1];
        const float4 q2 = base[lane * REC + 2], q3 = base[lane * REC + 3];
        v[0] = -((q0.x - chi.x) + (q1.x - clo.x));
        v[1] = -((q0.y - chi.y) + (q1.y - clo.y));
        v[2] = -((q0.z - chi.z) + (q1.z - clo.z));
        v[3] = -q0.w;
        v[4] = q2.x; v[5] = q2.y; v[6] = q2.z; v[7] = q2.w;
        v[8] = q3.x; v[9] = q3.y; v[10] = q3.z; v[11] = q3.w;
      }
      __syncwarp();
      const int npad = (n + 1) & ~1;
      if constexpr (PK) {
        // record e -> three float4 at 48-byte stride; an odd last record is
        // followed by a zero record (M = 0, S = 0: no contribution)
        if (lane < npad) {
          float4* dst = base + CREC * lane;
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], v[6], v[7]);
          dst[2] = make_float4(v[8], v[9], v[10], v[11]);
        }
        __syncwarp();
        if (act) {
          const float4* pb = base;
          for (int k = sl; k < npad / 2; k += s) {  // records 2k and 2k+1
            const CellRec c0 = load_cell_rec(pb + CREC * (2 * k));
            const CellRec c1 = load_cell_rec(pb + CREC * (2 * k + 1));
            body_cellP(P.X, P.Y, P.Z, E2, c0, P.part);
            body_cellP(P.X, P.Y, P.Z, E2, c1, P.part);
          }
        }
      } else {
        if (lane < npad) {
          float* dst = reinterpret_cast<float*>(base) + 4 * CPAIR * (lane >> 1) + (lane & 1);
#pragma unroll
          for (int f = 0; f < 12; ++f) dst[2 * f] = v[f];
        }
        __syncwarp();
        if (act) {
          const float4* pb = base;
          for (int k = sl; k < npad / 2; k += s) {
            const CellPair c = load_cell_pair(pb + CPAIR * k);
#pragma unroll
            for (int r = 0; r < R; ++r) body_cell2(P.X[r], P.Y[r], P.Z[r], E2, c, P.part[r]);
          }
        }
      }
      if (++nsince >= FOLD_EVERY * s) {
        P.fold();
        nsince = 0;
      }
      if (STAGE != STAGE_ASYNC) fence_proxy_async();
      __syncwarp();
      done += TILE;
      return true;
    };

    // ---- particle-particle evaluation in chunks of PCH sources (Listing 4).
    // Chunk k+1 is copied asynchronously while chunk k is evaluated. The
    // sources are either the particles of the queued leaves (rank -> particle
    // through the prefix of leaf counts) or, with `own`, the item's whole
    // group, whose pass excludes the self term.
    int n_pp = 0;
    auto pp_pass = [&](int total, int nq, bool own) {
      const int nchunk = (total + PCH - 1) / PCH;
      auto stage = [&](int k) -> int {
        const int rk = k * PCH + lane;
        int j = -1;
        if (rk < total) {
          if (own) {
            j = gfirst + rk;
          } else {
            int lo = 0, hi = nq - 1;  // first entry whose inclusive prefix exceeds rk
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (S.lpref[mid] > rk) hi = mid; else lo = mid + 1;
            }
            const int start = lo ? S.lpref[lo - 1] : 0;
            j = S.leafq[lo].x + (rk - start);
          }
          const uint32_t dst = smem_u32(&S.pbuf[k & 1][2 * lane]);
          cp_async16(dst, p.parts + 2 * j);
          cp_async16(dst + 16, p.parts + 2 * j + 1);
        }
        cp_async_commit();
        return j;
      };
      int j_cur = nchunk > 0 ? stage(0) : -1;
      for (int k = 0; k < nchunk; ++k) {
        int j_next = -1;
        if (k + 1 < nchunk) {
          j_next = stage(k + 1);
          cp_async_wait_1();
        } else {
          cp_async_wait_all();
        }
        float4* buf = S.pbuf[k & 1];
        const int nloc = min(PCH, total - k * PCH);
        const int npad = (nloc + 1) & ~1;
        // this lane's own copy -> negated relative position and mass, pair layout
        float nx = 0.f, ny = 0.f, nz = 0.f, nm = 0.f;
        if (j_cur >= 0) {
          const float4 h4 = buf[2 * lane];
          const float4 l4 = buf[2 * lane + 1];
          nx = -((h4.x - chi.x) + (l4.x - clo.x));
          ny = -((h4.y - chi.y) + (l4.y - clo.y));
          nz = -((h4.z - chi.z) + (l4.z - clo.z));
          nm = -h4.w;
        }
        __syncwarp();
        if constexpr (PK) {
          // source e -> one float4 (negated relative position, negated mass);
          // an odd last source is followed by zeros (no contribution)
          if (lane < npad) {
            buf[lane] = make_float4(nx, ny, nz, nm);
            if (own) reinterpret_cast<int*>(buf)[4 * PCH + lane] = j_cur;  // source index
          }
          __syncwarp();
          if (act) {
            if (own) {
              const int* jj = reinterpret_cast<const int*>(buf) + 4 * PCH;
              for (int e = sl; e < npad / 2; e += s) {
                const float4 q0 = buf[2 * e], q1 = buf[2 * e + 1];
                const int ja = jj[2 * e], jb = jj[2 * e + 1];
                const float2 m0 = make_float2(ja == P.idx[0] ? 0.f : q0.w, ja == P.idx[1] ? 0.f : q0.w);
                const float2 m1 = make_float2(jb == P.idx[0] ? 0.f : q1.w, jb == P.idx[1] ? 0.f : q1.w);
                body_bodyP(P.X, P.Y, P.Z, E2, q0.x, q0.y, q0.z, m0, P.part);
                body_bodyP(P.X, P.Y, P.Z, E2, q1.x, q1.y, q1.z, m1, P.part);
              }
            } else {
              for (int e = sl; e < npad / 2; e += s) {
                const float4 q0 = buf[2 * e], q1 = buf[2 * e + 1];
                body_bodyP(P.X, P.Y, P.Z, E2, q0.x, q0.y, q0.z, f2(q0.w), P.part);
                body_bodyP(P.X, P.Y, P.Z, E2, q1.x, q1.y, q1.z, f2(q1.w), P.part);
              }
            }
          }
        } else {
        if (lane < npad) {
          float* dst = reinterpret_cast<float*>(buf) + 4 * SPAIR * (lane >> 1) + (lane & 1);
          dst[0] = nx;
          dst[2] = ny;
          dst[4] = nz;
          dst[6] = nm;
          if (own) reinterpret_cast<int*>(buf)[4 * SPAIR * 16 + lane] = j_cur;  // source index per half
        }
        __syncwarp();
        if (act) {
          if (own) {
            const int* jj = reinterpret_cast<const int*>(buf) + 4 * SPAIR * 16;
            for (int e = sl; e < npad / 2; e += s) {
              const SrcPair q = load_src_pair(buf + SPAIR * e);
              const int ja = jj[2 * e], jb = jj[2 * e + 1];
#pragma unroll
              for (int r = 0; r < R; ++r) {
                const float2 nm2 = make_float2(ja == P.idx[r] ? 0.f : q.nm.x, jb == P.idx[r] ? 0.f : q.nm.y);
                body_body2(P.X[r], P.Y[r], P.Z[r], E2, q, nm2, P.part[r]);
              }
            }
          } else {
            for (int e = sl; e < npad / 2; e += s) {
              const SrcPair q = load_src_pair(buf + SPAIR * e);
#pragma unroll
              for (int r = 0; r < R; ++r) body_body2(P.X[r], P.Y[r], P.Z[r], E2, q, q.nm, P.part[r]);
            }
          }
        }
        }
        if (++nsince >= FOLD_EVERY * s) {
          P.fold();
          nsince = 0;
        }
        __syncwarp();  // chunk k's buffer is free for chunk k+2
        j_cur = j_next;
      }
    };
    auto eval_leaves = [&](int nq) {
      const int c0 = lane < nq ? S.leafq[lane].y : 0;
      const int c1 = lane + 32 < nq ? S.leafq[lane + 32].y : 0;
      int s0 = c0, s1 = c1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u0 = __shfl_up_sync(FULL, s0, o);
        const int u1 = __shfl_up_sync(FULL, s1, o);
        if (lane >= o) {
          s0 += u0;
          s1 += u1;
        }
      }
      const int tot0 = __shfl_sync(FULL, s0, 31);
      const int total = tot0 + __shfl_sync(FULL, s1, 31);
      S.lpref[lane] = s0;
      S.lpref[lane + 32] = s1 + tot0;
      __syncwarp();
      n_pp += total;
      pp_pass(total, nq, false);
    };

    // The group's own particles: they sit in the group's own leaves, which are
    // always opened (distance 0) and are evaluated here, with the self term
    // left out, instead of through the leaf queue.
    if (!SPLIT || part == 0) {
      n_pp += gcount;
      pp_pass(gcount, 0, true);
    }

    // ---- walk (Listing 1): root opened; children of up to 4 nodes per step
    int top = 0, nlq = 0, n_pc = 0, n_leafent = 0;
    int nlq_all = 0;  // leaves queued by every part (SPLIT: their sequence numbers)
    bool ok = true;
    // failure injection: the first tile of this item is never requested
    const uint32_t drop_end = (STAGE == STAGE_GATHER4 && item + 1 == p.drop_item) ? app + TILE : 0u;
    {
      const int2 rl = __ldg(p.link + it.x);
      if (rl.y < 0) {  // the root is a leaf: it is the group itself (own pass above)
        if (CAPTURE && slot >= 0 && lane == 0 && p.dbg_cap > 0) p.dbg_leaf[(size_t)slot * p.dbg_cap] = it.x;
        n_leafent = 1;
      } else {
        if (lane == 0) S.stack[0] = (rl.x << 3) | (rl.y - 1);
        top = 1;
      }
      __syncwarp();
    }
    // The children tested in the next step are known as soon as a step has
    // pushed its nodes (the stack is LIFO and nothing else touches it), so
    // their cube and link records are loaded one step ahead: the loads are in
    // flight while this warp evaluates tiles and leaves.
    bool nx_valid = false;
    int nx_c = 0;
    float4 nx_g = make_float4(0.f, 0.f, 0.f, 0.f);
    int2 nx_lk = make_int2(0, 0);
    auto prefetch = [&]() {
      const int npop = min(4, top);
      const int k = lane >> 3, slot = lane & 7;
      const int packed = k < npop ? S.stack[top - npop + k] : 0;
      const int nch = (packed & 7) + 1;
      nx_valid = (k < npop) && (slot < nch);
      nx_c = (packed >> 3) + slot;
      if (nx_valid && static_cast<unsigned>(nx_c) >= static_cast<unsigned>(p.n_cells)) {
        status |= ST_INDEX;
        nx_valid = false;
      }
      nx_g = make_float4(0.f, 0.f, 0.f, 0.f);
      nx_lk = make_int2(0, 0);
      if (nx_valid) {
        nx_g = __ldg(p.geo + nx_c);
        nx_lk = __ldg(p.link + nx_c);
      }
      __syncwarp();  // stack reads precede the next step's pushes
    };
    // Learned criterion: the opening test with theta_hi opens, with theta_lo
    // accepts; the candidates in between (with h > 0) are deferred to a queue
    // that the network classifies 32 at a time. A network step takes the place
    // of a stack step; its outcomes are handled like the test's.
    int mq = 0;
    int n_net = 0;  // capture mode: network candidates recorded for this item
    auto network_step_next = [&]() { return MLP && (mq >= 32 || (top == 0 && mq > 0)); };
    if (top > 0 && !network_step_next()) prefetch();
    while (top > 0 || (MLP && mq > 0)) {
      if (app - done >= 2 * TILE) {
        // the oldest tile is complete and its copies were issued at least one step ago
        if (STAGE == STAGE_ASYNC) cp_async_wait_1();
        if (!eval_tile(TILE)) { ok = false; break; }
      }
      bool valid, open, defer = false;
      int c;
      float4 g;
      int2 lk;
      if (network_step_next()) {
        const int nb = min(32, mq);
        valid = lane < nb;
        c = valid ? S.mq[mq - nb + lane] : 0;
        mq -= nb;
        __syncwarp();
        g = valid ? __ldg(p.geo + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        lk = valid ? __ldg(p.link + c) : make_int2(0, 0);
        float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0, q2 = q0, q3 = q0;
        if (valid) {
          q0 = __ldg(p.mp + 4 * c);
          q1 = __ldg(p.mp + 4 * c + 1);
          q2 = __ldg(p.mp + 4 * c + 2);
          q3 = __ldg(p.mp + 4 * c + 3);
        }
        float f[MLP_NF];
        mlp_features(g, q0, q1, q2, q3, gmin, gmax, chi, clo, f10, f11, f);
        bool in_range = valid;
        uint32_t xw[8];
#pragma unroll
        for (int i = 0; i < MLP_NF; i += 2) {
          const float xa = (f[i] - NW.mu[i]) * NW.isig[i], xb = (f[i + 1] - NW.mu[i + 1]) * NW.isig[i + 1];
          in_range = in_range && xa >= NW.xmin[i] && xa <= NW.xmax[i] && xb >= NW.xmin[i + 1] &&
                     xb <= NW.xmax[i + 1];
          xw[i / 2] = pack_bf16(xa, xb);
        }
        xw[6] = xw[7] = 0u;
        if (!in_range) {
#pragma unroll
          for (int i = 0; i < 6; ++i) xw[i] = 0u;
        }
        uint4* xrow = reinterpret_cast<uint4*>(&S.pbuf[0][0]) + 2 * lane;
        xrow[0] = make_uint4(xw[0], xw[1], xw[2], xw[3]);
        xrow[1] = make_uint4(xw[4], xw[5], xw[6], xw[7]);
        __syncwarp();
        const float y = mlp_eval(NW, smem_u32(&S.pbuf[0][0]), lane, nb > 16 ? 2 : 1);
        __syncwarp();
        open = valid && (in_range ? !(y < NW.tau) : must_open(g, gmin, gmax, p.theta_fb2));
        if (CAPTURE) {  // the valid candidates are lanes 0 .. nb-1
          if (slot >= 0 && p.dbg_net && valid && n_net + lane < p.dbg_net_cap)
            p.dbg_net[(size_t)slot * p.dbg_net_cap + n_net + lane] =
                in_range ? make_int2(c, __float_as_int(y)) : make_int2(~c, 0);
          n_net += nb;
        }
      } else {
        top -= min(4, top);
        valid = nx_valid;
        c = nx_c;
        g = nx_g;
        lk = nx_lk;
        if (MLP) {
          const bool open_hi = valid && must_open(g, gmin, gmax, p.theta_hi2);
          const bool open_lo = valid && must_open(g, gmin, gmax, p.theta_lo2);
          defer = valid && !open_hi && open_lo && g.w > 0.f;
          open = open_hi;
        } else {
          open = valid && must_open(g, gmin, gmax, theta2);
        }
      }
      if (MLP) {
        const unsigned m_def = __ballot_sync(FULL, defer);
        if (defer) S.mq[mq + __popc(m_def & lt)] = c;
        mq += __popc(m_def);
        valid = valid && !defer;
      }
      const bool leaf = lk.y < 0;
      // leaves of the own group are evaluated by the own pass, not queued
      const bool own_leaf = open && leaf && lk.x >= gfirst && lk.x < gfirst + gcount;
      const unsigned m_acc = __ballot_sync(FULL, valid && !open);
      const unsigned m_leaf = __ballot_sync(FULL, open && leaf);
      const unsigned m_lq = __ballot_sync(FULL, open && leaf && !own_leaf);
      const unsigned m_node = __ballot_sync(FULL, open && !leaf);
      const int nn = __popc(m_node);
      if (top + nn > p.stack_cap) {
        status |= ST_STACK;
        break;
      }
      if (open && !leaf) S.stack[top + __popc(m_node & lt)] = (lk.x << 3) | (lk.y - 1);
      top += nn;
      unsigned m_lq_use = m_lq;  // the queued leaves this warp evaluates
      if (SPLIT) {
        const bool mine = (nlq_all + __popc(m_lq & lt)) % p.nparts == part;
        m_lq_use = __ballot_sync(FULL, open && leaf && !own_leaf && mine);
        nlq_all += __popc(m_lq);
      }
      if ((m_lq_use >> lane) & 1u) S.leafq[nlq + __popc(m_lq_use & lt)] = make_int2(lk.x, -lk.y);
      if (CAPTURE && slot >= 0 && open && leaf && n_leafent + __popc(m_leaf & lt) < p.dbg_cap)
        p.dbg_leaf[(size_t)slot * p.dbg_cap + n_leafent + __popc(m_leaf & lt)] = c;
      nlq += __popc(m_lq_use);
      n_leafent += __popc(m_leaf);
      unsigned m_stage = m_acc;  // the accepted cells this warp evaluates
      if (SPLIT) m_stage = __ballot_sync(FULL, valid && !open && (n_pc + __popc(m_acc & lt)) % p.nparts == part);
      if ((m_stage >> lane) & 1u) {
        const uint32_t e = app + __popc(m_stage & lt);
        const uint32_t se = e % (NTILE * TILE);
        if (STAGE == STAGE_BULK) {
          const uint32_t bar = bar0 + 8 * (se / TILE);
          mbar_expect_tx(bar, 64);
          bulk_g2s(smem_u32(&S.ring[se * REC]), p.mp + 4 * (size_t)c, 64, bar);
        } else if (STAGE == STAGE_ASYNC) {
          const uint32_t dst = smem_u32(&S.ring[se * REC]);
          const float4* src = p.mp + 4 * (size_t)c;
#pragma unroll
          for (int q = 0; q < 4; ++q) cp_async16(dst + 16 * q, src + q);
        } else {
          S.cidx[se] = c;
        }
        if (CAPTURE && slot >= 0 && n_pc + __popc(m_acc & lt) < p.dbg_cap)
          p.dbg_cell[(size_t)slot * p.dbg_cap + n_pc + __popc(m_acc & lt)] = c;
      }
      const int na = __popc(m_stage);
      const uint32_t old = app;
      app += na;
      n_pc += __popc(m_acc);
      if (STAGE == STAGE_ASYNC) cp_async_commit();
      __syncwarp();  // all expect_tx / index writes of this step are done
      if (STAGE == STAGE_BULK && lane == 0) {
        for (uint32_t b = (old / TILE + 1) * TILE; b <= app; b += TILE)
          mbar_arrive(bar0 + 8 * (((b - 1) / TILE) % NTILE));
      }
      if (STAGE == STAGE_GATHER4) {
        const uint32_t upto = app & ~3u;
        if (lane == 0) {
          for (uint32_t k = iss; k < upto; k += 4) {
            if (k < drop_end) continue;  // failure injection: this tile never arrives
            const uint32_t sk = k % (NTILE * TILE);
            const uint32_t bar = bar0 + 8 * (sk / TILE);
            const int4 r4 = *reinterpret_cast<const int4*>(&S.cidx[sk]);
            mbar_expect_tx(bar, 256);
            gather4_g2s(smem_u32(&S.ring[sk * REC]), &p.mp_map, r4.x, r4.y, r4.z, r4.w, bar);
            if ((k + 4) % TILE == 0) mbar_arrive(bar);
          }
        }
        iss = upto;
      }
      __syncwarp();
      if (top > 0 && !network_step_next()) prefetch();
      if (nlq >= TILE) {
        eval_leaves(nlq);
        nlq = 0;
      }
    }
    // ---- drain: close the partial tile, evaluate what is pending
    {
      const uint32_t rem = app % TILE;
      const uint32_t real_end = app;
      if (STAGE == STAGE_ASYNC) {
        cp_async_wait_all();
        __syncwarp();
        if (rem) app += TILE - rem;
      } else if (rem) {
        __syncwarp();
        if (lane == 0 && app >= drop_end) {
          const uint32_t bar = bar0 + 8 * ((app / TILE) % NTILE);
          if (STAGE == STAGE_GATHER4 && iss < app) {
            // last partial group of 4: pad with the first index; the padded
            // slots lie beyond the item's last entry and are never read
            const uint32_t sk = iss % (NTILE * TILE);
            int4 r4 = *reinterpret_cast<const int4*>(&S.cidx[sk]);
            if (app - iss < 2) r4.y = r4.x;
            if (app - iss < 3) r4.z = r4.x;
            r4.w = r4.x;
            mbar_expect_tx(bar, 256);
            gather4_g2s(smem_u32(&S.ring[sk * REC]), &p.mp_map, r4.x, r4.y, r4.z, r4.w, bar);
          }
          mbar_arrive(bar);
        }
        app += TILE - rem;
        iss = app;
      }
      while (done < app) {
        const int n = static_cast<int>(min(static_cast<uint32_t>(TILE), real_end - done));
        if (!ok) {
          // a wait already failed: give the rest one bounded wait each, then stop
          const uint32_t tile = (done / TILE) % NTILE;
          if (STAGE != STAGE_ASYNC) mbar_wait_bounded(bar0 + 8 * tile, (done / (TILE * NTILE)) & 1u);
          done += TILE;
          continue;
        }
        if (!eval_tile(n)) ok = false;
      }
    }
    if (!ok) {
      status |= ST_TIMEOUT;  // barrier phases are no longer trustworthy in this warp
      if constexpr (MLP) goto items_done;
      stop = true;
      break;
    }
    if (nlq > 0) eval_leaves(nlq);
    P.fold();

    // ---- per-particle compensated sums (value = hi + lo)
    Acc4 H[R], L[R];
    if constexpr (PK) {
      H[0] = Acc4{P.hi.x.x, P.hi.y.x, P.hi.z.x, P.hi.p.x};
      L[0] = Acc4{P.lo.x.x, P.lo.y.x, P.lo.z.x, P.lo.p.x};
      H[1] = Acc4{P.hi.x.y, P.hi.y.y, P.hi.z.y, P.hi.p.y};
      L[1] = Acc4{P.lo.x.y, P.lo.y.y, P.lo.z.y, P.lo.p.y};
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        H[r] = P.hi[r];
        L[r] = P.lo[r];
      }
    }
    // ---- combine the slices (lane wl of slice 0 gathers lanes wl + k*w)
    for (int kk = 1; kk < s; ++kk) {
      const int src = min(31, lane + kk * w);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float hx = __shfl_sync(FULL, H[r].x, src), lx = __shfl_sync(FULL, L[r].x, src);
        const float hy = __shfl_sync(FULL, H[r].y, src), ly = __shfl_sync(FULL, L[r].y, src);
        const float hz = __shfl_sync(FULL, H[r].z, src), lz = __shfl_sync(FULL, L[r].z, src);
        const float hp = __shfl_sync(FULL, H[r].p, src), lp = __shfl_sync(FULL, L[r].p, src);
        if (sl == 0) {
          two_sum_into(H[r].x, L[r].x, hx);
          L[r].x += lx;
          two_sum_into(H[r].y, L[r].y, hy);
          L[r].y += ly;
          two_sum_into(H[r].z, L[r].z, hz);
          L[r].z += lz;
          two_sum_into(H[r].p, L[r].p, hp);
          L[r].p += lp;
        }
      }
    }
    if (sl == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (P.idx[r] >= 0) {
          const float4 v = make_float4(G * (H[r].x + L[r].x), G * (H[r].y + L[r].y),
                                       G * (H[r].z + L[r].z), G * (H[r].p + L[r].p));
          if (SPLIT)
            p.part_out[static_cast<size_t>(part) * p.n + P.idx[r]] = v;
          else
            p.out[P.idx[r]] = v;
        }
      }
    }
    if (lane == 0) {
      if (SPLIT) {  // zeroed before the launch; every part walked all of the lists
        if (part == 0) atomicAdd(&p.counts[item].x, n_pc);
        atomicAdd(&p.counts[item].y, n_pp);
      } else {
        p.counts[item] = make_int2(n_pc, n_pp);
      }
      if (CAPTURE && slot >= 0) {
        p.dbg_n[slot] = make_int2(n_pc, n_leafent);
        if (MLP && p.dbg_net_n) p.dbg_net_n[slot] = n_net;
      }
    }
    if (status & ST_STACK) {
      if constexpr (MLP) goto items_done;
      stop = true;
      break;
    }
    }
    if (stop) break;
  }
items_done:
  status = static_cast<int>(__reduce_or_sync(FULL, static_cast<unsigned>(status)));
  if (status && lane == 0) atomicOr(p.status, status);
}

// Launch configuration per kernel instance and device, computed once (so a
// launch inside stream capture makes no attribute or occupancy calls).
struct LaunchCache {
  std::mutex mu;
  int grid_per_sm[64] = {};
  int sms[64] = {};
};

template <int R, int STAGE, bool CAPTURE, bool MLP = false, bool SPLIT = false>
cudaError_t launch_t(const KParams& p, int ctas_per_sm, cudaStream_t stream, LaunchInfo* info, bool dry) {
  constexpr int NW = CtaWarps<MLP>::v;
  const size_t smem = sizeof(WarpSmemT<STAGE == STAGE_GATHER4, MLP>) * NW + (MLP ? sizeof(MlpDevice) : 0) + 128;
  auto kern = walk_eval_kernel<R, STAGE, CAPTURE, MLP, SPLIT>;
  static LaunchCache cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int occ = 0, sms = 0;
  {
    std::lock_guard<std::mutex> lock(cache.mu);
    if (!cache.grid_per_sm[dev]) {
      if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem))) !=
          cudaSuccess)
        return e;
      if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NW * 32, smem)) != cudaSuccess) return e;
      if (occ < 1) return cudaErrorInvalidConfiguration;
      cache.grid_per_sm[dev] = occ;
      cache.sms[dev] = sms;
    }
    occ = cache.grid_per_sm[dev];
    sms = cache.sms[dev];
  }
  const int per_sm = ctas_per_sm > 0 ? min(ctas_per_sm, occ) : occ;
  const int grid = sms * per_sm;
  if (info) {
    info->grid = grid;
    info->block = NW * 32;
    info->smem = smem;
  }
  if (dry) return cudaSuccess;
  KParams q = p;
  constexpr int STK = MLP ? STACK_MLP : STACK;
  q.stack_cap = (p.stack_cap > 0 && p.stack_cap < STK) ? p.stack_cap : STK;
  kern<<<grid, NW * 32, smem, stream>>>(q);
  return cudaGetLastError();
}

}  // namespace

cudaError_t encode_mp_map(CUtensorMap* map, const void* mp, int n_cells) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static const EncodeFn fn = []() -> EncodeFn {  // looked up once, thread-safe
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeFn>(f);
  }();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {16, static_cast<cuuint64_t>(n_cells > 0 ? n_cells : 1)};
  const cuuint64_t strides[1] = {64};
  const cuuint32_t box[2] = {16, 1};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(mp), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t walk_eval_smem_bytes() { return sizeof(WarpSmemT<false, false>) * WARPS + 128; }

template <int STAGE>
cudaError_t launch_s(const KParams& p, int ppl, int ctas_per_sm, bool capture, cudaStream_t stream,
                     LaunchInfo* info, bool dry) {
  if (ppl == 1) {
    return capture ? launch_t<1, STAGE, true>(p, ctas_per_sm, stream, info, dry)
                   : launch_t<1, STAGE, false>(p, ctas_per_sm, stream, info, dry);
  }
  return capture ? launch_t<2, STAGE, true>(p, ctas_per_sm, stream, info, dry)
                 : launch_t<2, STAGE, false>(p, ctas_per_sm, stream, info, dry);
}

cudaError_t launch_dispatch(const KParams& p, int ppl, int ctas_per_sm, bool capture, cudaStream_t stream,
                            LaunchInfo* info, bool dry) {
  if (p.mlp) {  // learned criterion: one variant (2 particles per lane, cp.async staging)
    return capture ? launch_t<2, STAGE_ASYNC, true, true>(p, ctas_per_sm, stream, info, dry)
                   : launch_t<2, STAGE_ASYNC, false, true>(p, ctas_per_sm, stream, info, dry);
  }
  if (p.nparts > 1 && !capture && p.stage == STAGE_ASYNC) {  // list split (small systems)
    return ppl == 1 ? launch_t<1, STAGE_ASYNC, false, false, true>(p, ctas_per_sm, stream, info, dry)
                    : launch_t<2, STAGE_ASYNC, false, false, true>(p, ctas_per_sm, stream, info, dry);
  }
  switch (p.stage) {
    case STAGE_BULK: return launch_s<STAGE_BULK>(p, ppl, ctas_per_sm, capture, stream, info, dry);
    case STAGE_ASYNC: return launch_s<STAGE_ASYNC>(p, ppl, ctas_per_sm, capture, stream, info, dry);
    default: return launch_s<STAGE_GATHER4>(p, ppl, ctas_per_sm, capture, stream, info, dry);
  }
}

cudaError_t launch_walk_eval(const KParams& p, int ppl, int ctas_per_sm, bool capture,
                             cudaStream_t stream, LaunchInfo* info) {
  return launch_dispatch(p, ppl, ctas_per_sm, capture, stream, info, false);
}

namespace {
__global__ void k_split_sum(const float4* __restrict__ part_out, int nparts, int n, float4* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float4 s = part_out[i];
    for (int k = 1; k < nparts; ++k) {  // in part order: the same sum on every launch
      const float4 v = part_out[static_cast<size_t>(k) * n + i];
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    out[i] = s;
  }
}
}  // namespace

cudaError_t split_sum(const float4* part_out, int nparts, int n, float4* out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = min((n + 255) / 256, 152 * 8);
  k_split_sum<<<grid, 256, 0, stream>>>(part_out, nparts, n, out);
  return cudaGetLastError();
}

cudaError_t prepare_walk_eval(int ppl, int stage, int ctas_per_sm, LaunchInfo* info) {
  KParams p{};
  p.stage = stage;
  return launch_dispatch(p, ppl, ctas_per_sm, false, nullptr, info, true);
}

// ---------------------------------------------------------------- allocation-free launch
//
// Scratch of octgrav_forces_noalloc, for callers that must not allocate device
// memory themselves or have the library do it (see include/octgrav.h).
// Layout: bytes 0..3 status word, 4..7 work-queue counter, 256.. per-item
// interaction counts (int2) for at most OCTGRAV_NOALLOC_MAX_ITEMS items
// (2 MiB + 256 B in total). Every GPU that loads the library keeps this array
// until the process exits. All calls share it: calls that overlap on the GPU
// (two streams, or two threads) race on it and give wrong results.
namespace {
constexpr size_t kNoAllocHeader = 256;
constexpr size_t kNoAllocBytes = kNoAllocHeader + sizeof(int2) * OCTGRAV_NOALLOC_MAX_ITEMS;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
CUcontext g_noalloc_ctx[kMaxDevices] = {};

// The calling thread's current CUDA context (driver entry point looked up once).
cudaError_t current_context(CUcontext* ctx) {
  using GetFn = CUresult (*)(CUcontext*);
  static const GetFn fn = []() -> GetFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<GetFn>(f);
  }();
  if (!fn) return cudaErrorNotSupported;
  return fn(ctx) == CUDA_SUCCESS ? cudaSuccess : cudaErrorContextIsDestroyed;
}

// Device address of the scratch array on the current device. The first call on
// a device looks it up (cudaGetSymbolAddress) with that device current; later
// calls reuse the address while the device's context is the same one (a
// context created anew, e.g. after cudaDeviceReset, is looked up again).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  CUcontext ctx = nullptr;  // null until the runtime has made the device's context current
  if ((e = current_context(&ctx)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev] || !ctx || g_noalloc_ctx[dev] != ctx) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);  // initialises the primary context if needed
    if (e != cudaSuccess) return e;
    if ((e = current_context(&ctx)) != cudaSuccess) return e;
    g_noalloc_ptr[dev] = ptr;
    g_noalloc_ctx[dev] = ctx;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_walk_eval_noalloc(KParams p, int ppl, int ctas_per_sm, cudaStream_t stream,
                                     int* status_bits) {
  if (p.n_items < 0 || p.n_items > OCTGRAV_NOALLOC_MAX_ITEMS) return cudaErrorInvalidValue;
  void* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) return e;
  char* b = static_cast<char*>(base);
  p.status = reinterpret_cast<int*>(b);
  p.work = reinterpret_cast<unsigned*>(b + 4);
  p.counts = reinterpret_cast<int2*>(b + kNoAllocHeader);
  // the array keeps the previous call's contents: the status word and the
  // work counter must start at zero
  if ((e = cudaMemsetAsync(b, 0, 8, stream)) != cudaSuccess) return e;
  if (p.n_items > 0 && (e = launch_walk_eval(p, ppl, ctas_per_sm, false, stream, nullptr)) != cudaSuccess)
    return e;
  int h = 0;
  if ((e = cudaMemcpyAsync(&h, b, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return e;
  *status_bits = h;
  return cudaSuccess;
}

}  // namespace og
