// octgrav_internal.h -- shared between the host library (octgrav_host.cpp) and
// the CUDA kernels (octgrav_kernels.cu). Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace og {

struct MlpDevice;

#ifdef __CUDACC__
#define OG_HD __host__ __device__
#else
#define OG_HD
#endif

// Particles of the next work item of a group with `rest` particles left:
// item_max, or all of them when fewer. With `split` (item_max 64, two
// particles per lane) a rest of 33..48 particles becomes an item of 32 (two
// list slices of 16 lanes) followed by one of rest - 32 <= 16 (four or more
// slices): a single item of that size leaves 8..15 lanes of its warp idle
// during the whole evaluation, which costs more than the second item's walk.
// (A rest of 49..56 would leave a second item of two or three slices and gains
// less than that walk costs.) Host and GPU builds both cut with this rule.
OG_HD inline int next_item_size(int rest, int item_max, bool split) {
  if (split && item_max == 64 && rest > 32 && rest <= 48) return 32;
  return rest < item_max ? rest : item_max;
}
// Number of items next_item_size cuts a group of cnt particles into: the full
// items first, then the rest r = cnt mod item_max as one item or two.
OG_HD inline int item_count(int cnt, int item_max, bool split) {
  const int r = cnt % item_max;
  return cnt / item_max + (r > 0) + (r > 0 && next_item_size(r, item_max, split) < r);
}

// Device status bits (OR-ed into the status word by the kernel).
enum : int {
  ST_STACK = 1,    // node stack overflow in a walk
  ST_INDEX = 2,    // child index outside the cell array
  ST_TIMEOUT = 4,  // bounded mbarrier wait expired
};

// Kernel arguments. Array layouts (all in tree order):
//   parts [2*n]  float4: hi = (x_hi, y_hi, z_hi, m), lo = (x - x_hi, ..., 0)
//   geo   [nc]   float4: boundary cube centre (FP32-rounded) and half side h
//   link  [nc]   int2:   node -> (first child, number of children 1..8),
//                        leaf -> (first particle, -count)
//   mp    [4*nc] float4: q0 = (com_hi.xyz, M), q1 = (com_lo.xyz, T = trS/2),
//                        q2 = (3Sxx, 3Syy, 3Szz, 3Sxy), q3 = (3Sxz, 3Syz, 3T, 0)
//   items [ni]   int4:   (root cell of the system, first particle, count, system)
//   ibox  [4*ni] float4: (gmin.xyz, C_hi.x), (gmax.xyz, C_hi.y), (C_lo.xyz, C_hi.z),
//                        (first particle, count of the whole group as int bits, 0, 0):
//                        group tight box (FP32-rounded), group centre C (hi/lo), group range
//   sysp  [nsys] float4: (fl32(theta^2), fl32(eps^2), -, -) (optional; G is sys0.z)
// Staging of accepted cell records (KParams::stage).
enum : int {
  STAGING_BULK = 0,     // cp.async.bulk per record
  STAGING_ASYNC = 1,    // 4 x 16-byte cp.async per record
  STAGING_GATHER4 = 2,  // TMA tile::gather4, 4 records per instruction (needs mp_map)
};

struct KParams {
  CUtensorMap mp_map;    // 2-D map of mp: rows = cells, 16 floats per row (gather4 staging)
  const float4* parts;
  const float4* geo;
  const int2* link;
  const float4* mp;
  const int4* items;
  const float4* ibox;
  const float4* sysp;    // per-system parameters, or nullptr to use sys0
  float4 sys0;           // (fl32(theta^2), fl32(eps^2), G, 0) for every system
  float4* out;           // [n] (a_x, a_y, a_z, phi), tree order
  int2* counts;          // [ni] (n_pc, n_pp sources incl. self)
  int* status;           // device status word
  unsigned* work;        // work-queue counter (zeroed before the launch)
  const int* order;      // [ni] processing order of the work items, or nullptr for 0, 1, ...
  int n_items;
  int n_cells;
  int stage;             // STAGING_*
  // learned opening criterion (mlp != nullptr): network and band thresholds
  const struct MlpDevice* mlp;
  float theta_lo2, theta_hi2, theta_fb2;  // fl32(theta^2) of the band and the fallback
  int n_group;
  // failure injection (tests; nothing faults; zero = off): stack_cap =
  // node-stack entries a walk may use (0: all; launches clamp it to the
  // stack's size), so that a walk overflows and reports ST_STACK; drop_item =
  // 1 + the index of a work item whose first tile of cell records is never
  // requested in gather4 staging, so that the bounded wait for it runs out and
  // reports ST_TIMEOUT
  int stack_cap;
  int drop_item;
  // list split (small systems; 1 = off): work item k is walked by nparts warps,
  // part j evaluating the accepted cells and queued leaves whose sequence
  // number is j modulo nparts (part 0 also the group's own particles) into
  // part_out[j * n + particle]; counts are accumulated with atomics
  int nparts;
  int n;                 // particles (rows of one part_out slice)
  float4* part_out;
  // capture mode (tests): per captured item up to dbg_cap cell indices. Item k
  // is captured into row dbg_slot[k] (-1: not captured; dbg_slot == nullptr:
  // row k for every item). The learned criterion's network steps also record,
  // per captured item, up to dbg_net_cap candidates as (cell, prediction bits),
  // or (~cell, 0) for a candidate whose inputs left the training range.
  int* dbg_cell;
  int* dbg_leaf;
  int2* dbg_n;
  int dbg_cap;
  const int* dbg_slot;
  int2* dbg_net;
  int* dbg_net_n;
  int dbg_net_cap;
};

struct LaunchInfo {
  int grid;
  int block;
  size_t smem;
};

// Launch the fused walk + evaluation kernel. ppl = particles per lane (1 or 2),
// ctas_per_sm = 0 for the occupancy maximum. Returns a cudaError_t.
cudaError_t launch_walk_eval(const KParams& p, int ppl, int ctas_per_sm, bool capture,
                             cudaStream_t stream, LaunchInfo* info);

// Compute (and cache) the launch configuration of a kernel variant without
// launching it; call before stream capture.
cudaError_t prepare_walk_eval(int ppl, int stage, int ctas_per_sm, LaunchInfo* info);
// out[i] = sum over k of part_out[k * n + i], k = 0 .. nparts - 1 in order
// (the parts of a list-split launch).
cudaError_t split_sum(const float4* part_out, int nparts, int n, float4* out, cudaStream_t stream);

// Shared memory per CTA of the fused kernel.
size_t walk_eval_smem_bytes();

// Training samples of the learned criterion (octgrav_mlp.cu).
struct MlpSampleArgs {
  int n;                        // samples
  int chunks;                   // ceil(largest group / 32)
  const int* item;              // [n] work item of the sample's group (box, centre, range)
  const int* cell;              // [n] candidate cell
  const int4* items;
  const float4* ibox;
  const float4* geo;
  const float4* mp;
  const float4* parts;
  const int2* link_first_count; // [nc] (first particle, count) of every cell
  const double* com64;          // [3 nc] FP64 moments
  const double* M64;
  const double* S64;            // [6 nc]
  const float4* aref;           // [n_particles] reference acceleration (tree order)
  double eps2;
  int n_group;
  float* feat;                  // [n * 12]
  double* label64;              // [n], zeroed before the label kernel
};
cudaError_t mlp_sample_features(const MlpSampleArgs& a, cudaStream_t st);
cudaError_t mlp_sample_labels(const MlpSampleArgs& a, cudaStream_t st);
// One training step's gradient (grad and loss accumulated, zero them first);
// use_all: the B samples are X[0..B) instead of B counter-based draws.
cudaError_t mlp_grad(const float* w, const float* X, const float* t, int n_total, int B, int step, uint64_t seed,
                     bool use_all, float* grad, float* loss, cudaStream_t st);
cudaError_t mlp_adam(float* w, float* m, float* v, const float* g, float lr, int step, cudaStream_t st);

// Encode the 2-D tensor map over a cell-record array (n_cells rows of 64 B)
// used by the gather4 staging. Returns cudaSuccess or an error.
cudaError_t encode_mp_map(CUtensorMap* map, const void* mp, int n_cells);

// Allocation-free launch: like launch_walk_eval, but the status word, the
// work-queue counter and the per-item counts live in a file-scope device
// array (no cudaMalloc). p.status, p.work and p.counts are ignored; p.n_items
// must not exceed OCTGRAV_NOALLOC_MAX_ITEMS. Waits for the stream and returns
// the device status bits in *status_bits.
cudaError_t launch_walk_eval_noalloc(KParams p, int ppl, int ctas_per_sm, cudaStream_t stream,
                                     int* status_bits);

// ---- GPU tree build (octgrav_build.cu)

// Status bits of a GPU build (result[GB_STATUS]).
enum : int {
  GPU_BUILD_OVERFLOW = 1,  // more cells than the capacity: enlarge and build again
  GPU_BUILD_BADINPUT = 2,  // non-finite coordinate or mass, or a negative mass
  GPU_BUILD_DEEPER = 4,    // the level cap was too low: build again without it
};
// Entries of the result block (int64) the build writes at the end.
enum : int { GB_NCELLS = 0, GB_NGROUPS, GB_NITEMS, GB_DEPTH, GB_NLEAVES, GB_MAXGROUP, GB_STATUS, GB_COUNT };

// Arguments of the GPU build. Inputs: pos (3n) and mass (n) on the device,
// offsets (n_sys + 1) on the host. Outputs (device, capacity-sized: cells
// `cap`, particles / groups / items n): the arrays of the walk kernel in the
// layout of KParams, the FP64 cell properties in final cell order (bmin,
// bmax 3, cube 4, M 1, com 3, S 6 per cell), per cell the particle count and
// first particle, per group its cell, system and first work item, per item
// its group key, per system its root cell (cell_off, n_sys + 1), and the
// result block.
struct GpuBuild {
  const double* pos;
  const double* mass;
  int64_t n;
  int n_sys;
  const int64_t* offsets;
  int n_leaf, n_group, item_max;
  int item_split;  // cut items with next_item_size(..., split = item_split != 0)
  int max_level;  // deepest level the level loop builds (21 = no cap)
  int64_t cap;
  void* scratch;
  size_t scratch_bytes;
  float4* parts;
  int* perm;
  uint64_t* key;
  float4* geo;
  int2* link;
  float4* mp;
  double *bmin, *bmax, *cube, *M, *com, *S;
  int *pcount, *cfirst;
  int *group_cell, *group_sys, *group_item;
  int4* items;
  float4* ibox;
  uint64_t* item_key;
  int* order;         // [n] default processing order of the items: most particles first
  int64_t* cell_off;
  int64_t* result;
};

// Scratch bytes of a build of n particles in n_sys systems with `cap` cells.
size_t gpu_build_scratch_bytes(int64_t n, int n_sys, int64_t cap);
// Enqueue the whole build on `stream` (no host synchronisation inside):
// gpu_build_tables (host-made chunk tables copied into the scratch, from
// pageable memory) followed by gpu_build_kernels (device work only, so it can
// be captured into a CUDA graph and replayed while the tables and buffers
// stay the same).
cudaError_t gpu_build(const GpuBuild& a, cudaStream_t stream);
cudaError_t gpu_build_tables(const GpuBuild& a, cudaStream_t stream);
cudaError_t gpu_build_kernels(const GpuBuild& a, cudaStream_t stream);
// Refit the tree of the last gpu_build on this scratch to new positions and
// masses of the same particles (pos / mass in a): membership, order, groups
// and items stay; particle records, every cell's box, cube, moments and
// records, and the items' group boxes are recomputed. The result block gets
// the build's counts and the status of the new inputs.
cudaError_t gpu_refit(const GpuBuild& a, cudaStream_t stream);
// Rebuild the work items (another item_max) of a tree built by gpu_build with
// the same arguments and scratch.
cudaError_t gpu_build_items(const GpuBuild& a, cudaStream_t stream);
// acc[3 perm[t] + k] = out[t].xyz, pot[perm[t]] = out[t].w (pot may be NULL).
cudaError_t gpu_unpermute(const float4* out, const int* perm, int64_t n, double* acc, double* pot,
                          cudaStream_t stream);

// Copy `bytes` from pageable host memory to the device by a kernel that reads
// the host memory itself (devices with cudaDevAttrPageableMemoryAccess, e.g.
// over NVLink-C2C): asynchronous for the host, unlike cudaMemcpyAsync from
// pageable memory. Both pointers 16-byte aligned and bytes a multiple of 16
// (else cudaErrorInvalidValue). The source must stay valid and unchanged until
// the stream passes the copy.
cudaError_t pull_host(void* dst, const void* src, size_t bytes, cudaStream_t stream);

// ---- time integration (octgrav_sim.cu)

constexpr int SIM_EBLOCKS = 256;  // blocks (and partial-sum pairs) of the energy reduction
// v += a h; then x += v dt when drift (all arrays n x 3, FP64).
cudaError_t sim_kick_drift(double* x, double* v, const double* a, int64_t n, double h, double dt, bool drift,
                           cudaStream_t stream);
// part[2 b], part[2 b + 1] = block b's sums of m |v|^2 / 2 and m phi / 2.
cudaError_t sim_energy_partials(const double* v, const double* m, const double* pot, int64_t n, double* part,
                                cudaStream_t stream);

// ---- direct summation (octgrav_direct.cu)

// Source chunks of a direct sum over n sources (the partial-sum buffer holds
// 4 * chunks * nt doubles).
int64_t direct_chunks(int64_t n);
// FP64 direct sum at nt targets (indices into pos/mass, or the first nt
// particles when targets is NULL): acc (nt x 3), pot (nt), self excluded.
cudaError_t direct_sum(const double* pos, const double* mass, int64_t n, const int64_t* targets, int64_t nt,
                       double eps, double G, double* part, double* acc, double* pot, cudaStream_t stream);

}  // namespace og
