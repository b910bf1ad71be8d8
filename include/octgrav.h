/*
 * octgrav.h -- C ABI of the GB300 (sm_103a) grouped Barnes-Hut force library.
 *
 * Method: Gaburov, Bedorf & Portegies Zwart (2010), "Gravitational tree-code
 * on graphics processing units: implementation in CUDA". The octree, the
 * tight boxes, boundary cubes and multipole moments are built in FP64
 * (Sec. 2.1) on the host or, with a byte-identical result, on the GPU; the
 * per-group tree walk that sorts cells into an interaction list (Sec. 2.2,
 * Listings 1-2) and the evaluation of that list (Sec. 2.3, Listings 3-4) run
 * on the GPU in one fused CUDA kernel; a leapfrog integrator keeps an N-body
 * state on the device.
 *
 * Conventions shared by every entry point:
 *  - Positions are xyz-interleaved FP64 arrays of length 3*n, masses FP64 of
 *    length n, both in the caller's ("input") order and owned by the caller.
 *    Outputs named acc/pot are caller-owned host arrays in input order:
 *    acc[3*i+k] = a_k of particle i, pot[i] = its potential.
 *  - Plummer softening eps > 0, gravitational constant G (1 by default);
 *    the self term is excluded; potentials are negative.
 *  - Opening test (Sec. 2.2): a cell whose boundary-cube side l satisfies
 *    l < theta * d, with d the distance between the group's tight box and
 *    the cell's cube, is accepted as a multipole; otherwise it is opened.
 *  - Every call returns an octgrav status (0 = OK, negative = error) and never
 *    aborts or throws. On error, octgrav_last_error() gives a message (per
 *    calling thread).
 *  - stream arguments are a cudaStream_t passed as void* (NULL = the legacy
 *    default stream). Device memory owned by a tree is allocated by the
 *    library (cudaMalloc) on the current CUDA device and freed by
 *    octgrav_free_tree.
 *  - Thread safety: distinct trees may be used from distinct threads; one tree
 *    must not be used by two threads at once. The one-shot calls keep their
 *    buffers per calling thread and may run concurrently.
 *  - Environment (read at first use): OCTGRAV_THREADS = host build threads (default:
 *    all hardware threads); OCTGRAV_HOST_PULL=0 makes a thread's one-shot host-build
 *    call upload with cudaMemcpyAsync only (no copy kernel reading pageable
 *    memory); OCTGRAV_GPU_CELL_CAP = initial cell capacity of a GPU build.
 */
#ifndef OCTGRAV_H
#define OCTGRAV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OCTGRAV_OK 0
#define OCTGRAV_ERR_ARG (-1)       /* invalid argument (sizes, eps <= 0, theta < 0, ...) */
#define OCTGRAV_ERR_CUDA (-2)      /* a CUDA runtime call failed (message has the name) */
#define OCTGRAV_ERR_OOM (-3)       /* host or device allocation failed */
#define OCTGRAV_ERR_STACK (-4)     /* a walk overflowed its on-chip node stack */
#define OCTGRAV_ERR_LIST (-5)      /* a capture buffer (debug lists) was too small */
#define OCTGRAV_ERR_TIMEOUT (-6)   /* a bounded device-side wait ran out; results invalid */
#define OCTGRAV_ERR_NONFINITE (-7) /* NaN/Inf in positions or masses, or a negative mass */
#define OCTGRAV_ERR_STATE (-8)     /* call order violated (e.g. counts before any launch) */
#define OCTGRAV_ERR_INDEX (-9)     /* a walk met a cell index outside the tree (corrupt tree) */

#define OCTGRAV_MAX_DEPTH 21       /* octree depth limit (Morton keys fit one 64-bit word) */
#define OCTGRAV_MAX_ITEM 64        /* particles evaluated by one warp (larger groups are split) */

typedef struct octgrav_tree octgrav_tree; /* opaque, library-owned */
typedef struct octgrav_sim octgrav_sim;   /* opaque, library-owned integrator state */

/* Build the octree of one system on the host in FP64 (Sec. 2.1).
 *   pos[3n], mass[n]: input order, caller-owned, only read during the call.
 *   n >= 1; 1 <= n_leaf (a leaf holds at most n_leaf particles unless it sits
 *   at depth OCTGRAV_MAX_DEPTH); n_group >= n_leaf (groups are the largest
 *   cells holding at most n_group particles, Sec. 2.1-2.2).
 *   *out receives a new tree; free it with octgrav_free_tree.
 * No device work is done. Errors: ERR_ARG, ERR_NONFINITE, ERR_OOM. */
int octgrav_build_tree(const double *pos, const double *mass, int64_t n, int n_leaf,
                       int n_group, octgrav_tree **out);

/* Build one tree holding n_sys independent systems (the batched form).
 * System s owns particles offsets[s] .. offsets[s+1]-1 of pos/mass
 * (offsets has n_sys+1 entries, offsets[0] = 0, strictly increasing).
 * Each system gets its own octree; all systems share one set of device
 * arrays and are walked by one kernel launch. Errors as octgrav_build_tree. */
int octgrav_build_batch(int n_sys, const int64_t *offsets, const double *pos,
                        const double *mass, int n_leaf, int n_group, octgrav_tree **out);

/* Copy the tree's device arrays to the current CUDA device (library-owned
 * memory), asynchronously on stream. Called implicitly by the force calls
 * when needed. Errors: ERR_CUDA, ERR_OOM. */
int octgrav_tree_upload(octgrav_tree *t, void *stream);

/* Tree walk + evaluation on the GPU, asynchronous on stream (Sec. 2.2-2.3).
 *   acc4_dev: device array of 4*n floats (caller-owned, e.g. a torch tensor),
 *   written in TREE order: (a_x, a_y, a_z, phi) per particle; map to input
 *   order with octgrav_tree_perm.
 *   eps > 0, theta >= 0, G finite. For a batched tree the values apply to every
 *   system unless octgrav_set_system_params was called.
 * Launches exactly one kernel. Device-side failures (stack overflow, timeout)
 * are recorded in a status word read by octgrav_status. Errors: ERR_ARG,
 * ERR_CUDA. */
int octgrav_forces_device(octgrav_tree *t, double eps, double theta, double G, float *acc4_dev,
                          void *stream);

/* Per-system eps and theta for a batched tree (arrays of n_sys entries);
 * used by later octgrav_forces_device / octgrav_forces_tree calls, whose
 * scalar eps/theta arguments are then ignored. Pass NULL to clear.
 * Errors: ERR_ARG. */
int octgrav_set_system_params(octgrav_tree *t, const double *eps, const double *theta);

/* Forces with host outputs in input order: uploads if needed, launches,
 * copies the result back, waits for the stream and checks the device status.
 *   acc[3n], pot[n] (pot may be NULL). Errors: ERR_ARG, ERR_CUDA, ERR_STACK,
 *   ERR_TIMEOUT, ERR_INDEX. */
int octgrav_forces_tree(octgrav_tree *t, double eps, double theta, double G, double *acc,
                        double *pot, void *stream);

/* One-shot call (the paper's split, Sec. 2): FP64 tree build on the host
 * (n_group = n_leaf), upload, forces, free, on the default stream with G = 1.
 * Outputs in input order: acc[3n], pot[n] (pot may be NULL), unpermuted on the
 * device and copied into these arrays. Device buffers and the host build's
 * arrays are cached between calls of the calling thread (on its current
 * device). Where the device reads pageable host memory
 * (cudaDevAttrPageableMemoryAccess), the tree arrays are pulled by a copy
 * kernel, the particle records while the host still builds the cells; the
 * call returns only after the stream is done. Inputs are read, never written.
 * Errors: ERR_ARG, ERR_NONFINITE (checked before any device call), ERR_OOM,
 * ERR_CUDA, and the device statuses of octgrav_forces_tree. */
int octgrav_forces(const double *pos, const double *mass, int64_t n, double eps, double theta,
                   int n_leaf, double *acc, double *pot);

/* octgrav_forces with every knob: G, n_group and stream. */
int octgrav_forces_ex(const double *pos, const double *mass, int64_t n, double eps, double theta,
                      double G, int n_leaf, int n_group, double *acc, double *pot, void *stream);

/* Where the calling thread's last successful octgrav_forces_ex call spent its
 * time, in ms: host build phases 0 bounding box with the input check, 1 Morton
 * keys, 2 radix sort, 3 gather with the particle records (and the start of
 * their upload), 4 levels, 5 cell properties, 6 groups, 7 cell records and
 * work items, 8 the whole host build; device time between CUDA events on the
 * call's stream: 9 the remaining upload, 10 the walk-and-evaluate launch,
 * 11 unpermute and the FP64 copies out; 12 the whole call (host clock).
 * Writes min(n_out, OCTGRAV_ONESHOT_PHASES) values and returns that count.
 * Errors: ERR_ARG, ERR_STATE (no completed call on this thread). */
#define OCTGRAV_ONESHOT_PHASES 13
int octgrav_oneshot_phases(double *ms, int n_out);

/* ---- Tree build on the GPU (Sec. 2.1 run as CUDA kernels).
 *
 * The same tree as octgrav_build_tree / octgrav_build_batch of the same data,
 * byte for byte: Morton keys from the root cube, a stable radix sort, cells
 * split level by level, FP64 tight boxes, boundary cubes, masses, centres of
 * mass and second moments combined bottom-up in the host build's operation
 * order, the same groups and work items. The arrays are written on the
 * device in place; host copies of the tree (for the introspection calls
 * below) are made only when one of those calls asks. The whole build is
 * enqueued on `stream`; the call returns after reading one result block, so
 * the inputs may be freed or overwritten afterwards. */

/* One system from DEVICE arrays on the current device: pos_dev (n x 3 FP64,
 * xyz interleaved), mass_dev (n FP64). Errors: ERR_ARG (NULL, n < 1,
 * n_leaf < 1, n_group < n_leaf, too many particles or cells), ERR_NONFINITE
 * (non-finite coordinate or mass, negative mass; found on the device),
 * ERR_OOM, ERR_CUDA. */
int octgrav_build_tree_gpu(const double *pos_dev, const double *mass_dev, int64_t n, int n_leaf,
                           int n_group, void *stream, octgrav_tree **out);

/* n_sys systems concatenated as for octgrav_build_batch: offsets is a HOST
 * array (n_sys + 1, offsets[0] = 0, strictly increasing); pos_dev / mass_dev
 * are device arrays. Errors as octgrav_build_tree_gpu. */
int octgrav_build_batch_gpu(int n_sys, const int64_t *offsets, const double *pos_dev,
                            const double *mass_dev, int n_leaf, int n_group, void *stream,
                            octgrav_tree **out);

/* Refit a tree from octgrav_build_tree_gpu / octgrav_build_batch_gpu to new
 * positions and masses of the same particles (DEVICE arrays, input order, as
 * for the build): the cells keep their particles, order, groups and work
 * items; the particle records and every cell's tight box, boundary cube,
 * mass, centre of mass, second moments and the groups' boxes are recomputed
 * in FP64 exactly as a build does from those particles (a refit at unchanged
 * positions reproduces the tree bit for bit). Waits for the stream. Errors:
 * ERR_ARG, ERR_STATE (not a GPU-built tree), ERR_NONFINITE, ERR_CUDA. */
int octgrav_refit_tree_gpu(octgrav_tree *t, const double *pos_dev, const double *mass_dev,
                           void *stream);

/* Forces in INPUT order into DEVICE FP64 arrays: acc_dev (n x 3) and pot_dev
 * (n, may be NULL), for any tree (host- or GPU-built). Enqueued on stream and
 * not waited for: read the launch status with octgrav_status. Errors: ERR_ARG
 * (NULL tree/acc_dev, bad eps/theta/G), ERR_OOM, ERR_CUDA. */
int octgrav_forces_tree_device64(octgrav_tree *t, double eps, double theta, double G,
                                 double *acc_dev, double *pot_dev, void *stream);

/* One-shot call like octgrav_forces_ex with the tree built on the GPU: HOST
 * arrays pos (n x 3), mass (n) in, acc (n x 3) and pot (n, may be NULL) out,
 * both in input order. Copies the inputs to the device (at link speed when the
 * host arrays are pinned), builds the tree, evaluates, unpermutes on the
 * device and copies the FP64 results back; returns after the copies. Device
 * buffers are cached between calls on the calling thread's current device.
 * Errors as octgrav_build_tree_gpu plus the launch status (ERR_STACK,
 * ERR_TIMEOUT, ERR_INDEX). */
int octgrav_forces_gpu(const double *pos, const double *mass, int64_t n, double eps, double theta,
                       double G, int n_leaf, int n_group, double *acc, double *pot, void *stream);

/* One-shot call for many independent systems (the paper's "convenient user
 * interface", Sec. 1 and the abstract, in its batched form): HOST arrays in,
 * HOST FP64 results out, both in input order. System s owns particles
 * offsets[s] .. offsets[s+1]-1 of pos (n x 3) and mass (n), n = offsets[n_sys]
 * (offsets: n_sys + 1 entries, offsets[0] = 0, strictly increasing), and is
 * evaluated with its own softening eps[s] > 0 and opening parameter
 * theta[s] >= 0 (arrays of n_sys entries). acc (n x 3) and pot (n, may be NULL)
 * receive the results. The systems are copied to the device, their octrees
 * built on the GPU (octgrav_build_batch_gpu), walked and evaluated by one
 * persistent launch, unpermuted on the device and copied back; the call
 * returns after the copies. Device buffers are cached per calling thread (its
 * current device), as in octgrav_forces_gpu. Defaults: G = 1, N_leaf = 16,
 * N_group = 256 (the group size the autotuner picks for systems of 10^3 to
 * 10^5 particles); octgrav_forces_batched_ex takes every knob. Errors: ERR_ARG
 * (NULL, offsets, a bad eps/theta), ERR_NONFINITE (found on the device),
 * ERR_OOM, ERR_CUDA and the launch statuses. */
int octgrav_forces_batched(int n_sys, const int64_t *offsets, const double *pos, const double *mass,
                           const double *eps, const double *theta, double *acc, double *pot,
                           void *stream);
int octgrav_forces_batched_ex(int n_sys, const int64_t *offsets, const double *pos,
                              const double *mass, const double *eps, const double *theta, double G,
                              int n_leaf, int n_group, double *acc, double *pot, void *stream);

/* Direct Plummer-softened summation in FP64 on the GPU at nt target
 * particles (the exact reference of the error measure Delta a / a, Sec. 3.1):
 * targets[k] indexes pos/mass (HOST arrays, n particles); NULL targets means
 * the first nt particles. acc (nt x 3) and pot (nt) are HOST outputs; the
 * self term is excluded; eps >= 0. O(n * nt) work, deterministic order.
 * Returns after the copies. Errors: ERR_ARG (NULL, n < 1, nt < 0, target
 * out of range, bad eps/G), ERR_OOM, ERR_CUDA. */
int octgrav_direct(const double *pos, const double *mass, int64_t n, const int64_t *targets,
                   int64_t nt, double eps, double G, double *acc, double *pot, void *stream);

/* ---- Time integration on the device.
 *
 * The paper integrates on the host and does not name its scheme; this is the
 * standard kick-drift-kick leapfrog with one shared step dt, with the whole
 * state (FP64 positions, velocities, masses, accelerations, potentials, input
 * order) resident on the current device. Every force evaluation builds the
 * tree on the GPU (octgrav_build_tree_gpu) and runs the walk kernel; buffers
 * are reused from step to step. */

/* Create the integrator from HOST arrays pos, vel (n x 3) and mass (n), copied
 * to the device, and evaluate the initial forces. eps, theta, G, n_leaf and
 * n_group as for octgrav_forces_ex. Returns after the first force
 * evaluation. Errors: ERR_ARG, ERR_NONFINITE (non-finite input, negative
 * mass), ERR_OOM, ERR_CUDA and the launch status codes. */
int octgrav_sim_create(const double *pos, const double *vel, const double *mass, int64_t n,
                       double eps, double theta, double G, int n_leaf, int n_group, void *stream,
                       octgrav_sim **out);

/* Advance n_steps steps: v += a dt/2, x += v dt, forces, v += a dt/2 (each
 * update one rounded product and one rounded sum per component). dt may be
 * negative (the scheme is time-reversible). Returns when the steps are done.
 * Errors: ERR_ARG (NULL, non-finite dt, n_steps < 0) and those of a force
 * evaluation. */
int octgrav_sim_step(octgrav_sim *s, double dt, int n_steps, void *stream);

/* Kinetic energy sum m |v|^2 / 2 and potential energy sum m phi / 2 (phi of
 * the last force evaluation, self term excluded), FP64, in a fixed
 * summation order. Errors: ERR_ARG, ERR_CUDA. */
int octgrav_sim_energy(octgrav_sim *s, double *kinetic, double *potential, void *stream);

/* Copy the state to HOST arrays (any may be NULL): pos, vel, acc (n x 3),
 * pot (n), input order. Errors: ERR_ARG, ERR_CUDA. */
int octgrav_sim_state(octgrav_sim *s, double *pos, double *vel, double *acc, double *pot,
                      void *stream);

/* Release the integrator and its device memory (NULL is a no-op). */
void octgrav_sim_free(octgrav_sim *s);

/* Rebuild the tree every `every` force evaluations (1, the default, rebuilds
 * every step); in between the last tree is refitted (octgrav_refit_tree_gpu):
 * cheaper, and still exact in its boxes and moments, but its cells loosen as
 * particles move. Errors: ERR_ARG. */
int octgrav_sim_set_rebuild(octgrav_sim *s, int every);

/* Wait for stream and return the status of the last launch on this tree:
 * OK, ERR_STACK, ERR_TIMEOUT or ERR_INDEX. Clears nothing. */
int octgrav_status(octgrav_tree *t, void *stream);

/* Tree statistics: out[0..n_out) receives, in this order, n (particles),
 * n_cells, n_leaves, n_groups, n_items (warp work items), depth reached,
 * n_sys, max group size. */
int octgrav_tree_stats(const octgrav_tree *t, int64_t *out, int n_out);

/* perm[k] = input index of the particle at tree position k (n entries). */
int octgrav_tree_perm(const octgrav_tree *t, int64_t *perm);

/* Layout-independent cell keys: key = (1 << 3*depth) | octant path, in the
 * library's cell order (n_cells entries). In a batched tree keys restart in
 * every system; octgrav_item_info's sys field tells the systems apart. */
int octgrav_tree_cell_keys(const octgrav_tree *t, uint64_t *keys);

/* FP64 cell properties in the library's cell order (n_cells entries each;
 * any pointer may be NULL): tight box bmin[3], bmax[3], boundary cube
 * cube[4] = (centre xyz, half side), mass, centre of mass com[3], second
 * moments S[6] = (xx, yy, zz, xy, xz, yz) about the centre of mass, and the
 * particle count (Sec. 2.1, Fig. 1). */
int octgrav_tree_cell_props(const octgrav_tree *t, double *bmin, double *bmax, double *cube,
                            double *mass, double *com, double *S, int64_t *count);

/* Per work item: key of its group cell, first tree position, particle count,
 * system index (arrays of n_items entries; any may be NULL). A group of c
 * particles is cut into items of 32*ppl particles (octgrav_set_launch) and one
 * item for the rest r = c mod 32*ppl; with two particles per lane and the
 * plain criterion a rest of 33..48 becomes two items, 32 and r - 32
 * (a 33..48-particle item would leave lanes of its warp idle). Under a learned
 * criterion (octgrav_set_criterion) the rest stays whole: the network step
 * would run for both pieces. The host and the GPU build cut the same items. */
int octgrav_item_info(const octgrav_tree *t, uint64_t *group_key, int64_t *first,
                      int32_t *count, int32_t *sys);

/* Interaction counts of the last launch (waits for stream):
 * out[0] = sum over particles of particle-particle interactions (n_pp),
 * out[1] = sum over particles of particle-cell interactions (n_pc),
 * out[2] = flops by the paper's convention, 38 n_pp + 70 n_pc (Sec. 3.3). */
int octgrav_interaction_counts(octgrav_tree *t, int64_t *out, void *stream);

/* Test hook: run the fused kernel once in capture mode and return each work
 * item's interaction lists as cell keys. cell_keys/leaf_keys are host arrays
 * of n_items*cap entries (row = item); n_cell/n_leaf receive the true list
 * lengths. A list longer than cap is truncated and the call returns
 * ERR_LIST. Synchronous. */
int octgrav_debug_lists(octgrav_tree *t, double theta, int cap, uint64_t *cell_keys,
                        int32_t *n_cell, uint64_t *leaf_keys, int32_t *n_leaf, void *stream);

/* Test hook with a choice of work items, for trees too large to capture whole:
 * like octgrav_debug_lists, but row r of every output belongs to work item
 * items[r] (n_sel distinct indices in [0, n_items); items == NULL captures
 * every item, row = item). With the learned criterion (octgrav_set_criterion)
 * and net_cap > 0 it also records, per row, every candidate that reached the
 * network step (Sec. 2.2's opening test replaced by the network inside the
 * band): net_keys[r*net_cap + e] = the cell's key, net_y[...] = the network's
 * FP32 prediction, or NaN where a standardised input left the training range
 * and the theta_fb test decided; n_net[r] = their number. Candidates are
 * recorded in the order the walk met them. net_cap = 0 records none (net_*
 * may then be NULL). Truncation (a list or a candidate record longer than its
 * cap) returns ERR_LIST after filling what fits. Synchronous. Errors: ERR_ARG,
 * ERR_LIST, ERR_OOM, ERR_CUDA and the launch statuses. */
int octgrav_debug_walk(octgrav_tree *t, double theta, int64_t n_sel, const int64_t *items, int cap,
                       uint64_t *cell_keys, int32_t *n_cell, uint64_t *leaf_keys, int32_t *n_leaf,
                       int net_cap, uint64_t *net_keys, float *net_y, int32_t *n_net, void *stream);

/* Order in which later launches on this tree take the work items (the
 * persistent kernel's tail is shorter when the biggest items go first).
 * Every new tree (and every octgrav_set_launch or octgrav_set_criterion call
 * that cuts the items again) starts with mode 2. mode 2: most particles first. mode 1: longest first by
 * the cost of each item in the last launch (its particles times 70 n_pc +
 * 38 n_pp, that launch's interaction counts) -- an N-body code evaluating
 * the same tree again, or reusing the previous step's costs. mode 0: tree
 * order. Waits for the stream. A captured graph keeps the order it was
 * captured with. Results do not depend on the order.
 * Errors: ERR_ARG, ERR_STATE (mode 1 before any launch), ERR_CUDA. */
int octgrav_balance(octgrav_tree *t, int mode, void *stream);

/* Choose the kernel variant: particles per lane (1 or 2; work items hold at
 * most 32*ppl particles, cut as octgrav_item_info says) and CTAs per SM
 * (0 = as many as fit). Applies to later launches on this tree; a change of
 * ppl cuts the work items again (n_items may change, the order returns to
 * mode 2 of octgrav_balance, a captured graph is dropped).
 * Errors: ERR_ARG, ERR_CUDA (GPU-built tree). */
int octgrav_set_launch(octgrav_tree *t, int particles_per_lane, int ctas_per_sm);

/* Capture one octgrav_forces_device call (status reset + the persistent
 * walk/evaluation kernel) into a CUDA graph owned by the tree, for replay
 * with octgrav_graph_launch. Uploads the tree first if needed. stream must
 * be a non-default stream; acc4_dev is baked into the graph. The arguments
 * follow octgrav_forces_device. A call that cuts the work items again
 * (octgrav_set_launch, octgrav_set_criterion) drops the graph.
 * Errors: ERR_ARG, ERR_CUDA. */
int octgrav_graph_capture(octgrav_tree *t, double eps, double theta, double G, float *acc4_dev,
                          void *stream);

/* Replay the captured graph on stream (asynchronous). Status and interaction
 * counts are read as after octgrav_forces_device. Errors: ERR_STATE if
 * nothing was captured, ERR_CUDA. */
int octgrav_graph_launch(octgrav_tree *t, void *stream);

/* Autotuner: for the given systems (layout as octgrav_build_batch) times the
 * fused kernel for every group size in n_group_cand[0..n_cand) (values below
 * n_leaf are skipped), particles-per-lane 1 and 2 and, where the work items
 * are too few to fill the GPU (fewer than 4 per warp slot), list splits of
 * 1, 2, 4 and 8 (octgrav_set_split), and returns the fastest in best[0] =
 * n_group, best[1] = particles per lane, best[2] = list split, with its
 * median time in *best_ms (may be NULL).
 * Results are cached in-process (see octgrav_autotune_ex for the key). Builds
 * temporary trees and device buffers. Synchronous.
 * Errors: as octgrav_build_batch and octgrav_forces_device. */
int octgrav_autotune(int n_sys, const int64_t *offsets, const double *pos, const double *mass,
                     int n_leaf, double eps, double theta, const int *n_group_cand, int n_cand,
                     int *best, double *best_ms, void *stream);

/* The autotuner with every tuned dimension. First as octgrav_autotune: group
 * size, particles per lane (the particle side of the evaluated tile: a warp
 * covers 32 x particles-per-lane particles against slices of each 32-record
 * tile of the list; the record side is the warp width) and list split; then,
 * for the fastest of those without a split, the staging of the accepted cell
 * records (octgrav_set_staging: 0 cp.async.bulk, 1 per-lane cp.async, 2 TMA
 * tile::gather4), each timed the same way (median of three launches, items
 * longest first). Writes min(n_best, 4) values: best[0] n_group, best[1]
 * particles per lane, best[2] list split, best[3] staging mode. Both
 * autotuners cache their results in-process per (n_sys, log2 N, theta, eps,
 * n_leaf, candidates) and a coarse descriptor of the input distribution
 * (quartiles of the particles' distances from their system's box centre over
 * its half diagonal, log2 in halves, from up to 4096 particles). Synchronous.
 * Errors: ERR_ARG (also n_best < 1), and those of octgrav_autotune. */
int octgrav_autotune_ex(int n_sys, const int64_t *offsets, const double *pos, const double *mass,
                        int n_leaf, double eps, double theta, const int *n_group_cand, int n_cand,
                        int *best, int n_best, double *best_ms, void *stream);

/* ---- Learned opening criterion (a small network consulted inside the walk).
 * Record layout (OCTGRAV_MLP_RECORD floats): input mean[12], standard
 * deviation[12], standardised-input range min[12] and max[12], then the
 * network W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3. The network maps
 * the 12 inputs of a (group, cell) pair -- log2 l, log2 d, log2 |com - C_g|,
 * l/d, log2 M, |S|_F/(M l^2), log2 count, the group's half extents / l (3),
 * group count / N_group, log2 |C_g - com_root| -- to a prediction of log10 of
 * the relative force error of accepting the cell. */
#define OCTGRAV_MLP_RECORD 5105
#define OCTGRAV_MLP_NPARAM 5057

/* Training samples for the criterion, computed on the GPU: for each listed
 * group (index in tree order, 0 .. n_groups-1 of octgrav_tree_stats), every
 * child tested by a walk with theta_walk whose cube has h > 0 and lies apart
 * from the group box gives one sample: features[12] (FP32) and the label =
 * max over the group's particles of |a_multipole - a_direct(members)| /
 * |a_ref| (FP64 direct sums; a_ref from this tree at theta = 0.3), and
 * pairs[2] = (group, cell index). *n_out = number of samples; at most cap
 * are written (features == NULL: count only). Synchronous. */
int octgrav_mlp_samples(octgrav_tree *t, const int64_t *groups, int64_t n_groups, double theta_walk,
                        double eps, float *features, float *labels, int64_t *pairs, int64_t cap,
                        int64_t *n_out, void *stream);

/* Train the criterion's network on the GPU (FP32 forward/backward, Adam, mini-
 * batches drawn by a counter-based generator from seed) on log10 of the
 * labels, with inputs standardised over the samples. Writes the record
 * (OCTGRAV_MLP_RECORD floats; its input range is that of the standardised
 * samples widened by 1e-3 on each side, so that inputs equal to a training
 * extreme count as in range however they are rounded) and the last
 * mini-batch loss. Synchronous. */
int octgrav_mlp_train(const float *features, const float *labels, int64_t n, int steps, int batch,
                      double lr, uint64_t seed, float *record, float *final_loss, void *stream);

/* Gradient of L = sum (y - t)^2 / (2n) over n standardised inputs x[n][12]
 * and targets t[n] at params (OCTGRAV_MLP_NPARAM floats) -> grad, *loss.
 * Test hook for the training kernels. Synchronous. */
int octgrav_mlp_grad(const float *params, const float *x, const float *t, int64_t n, float *grad,
                     float *loss, void *stream);

/* Use the learned criterion in later launches on this tree (record == NULL
 * restores the plain test). A child is opened when the plain test with
 * theta_hi opens it, accepted when the plain test with theta_lo accepts it,
 * accepted when its cube has h = 0, and otherwise accepted iff the network's
 * prediction is below tau; a child whose standardised inputs leave the
 * training range falls back to the plain test with theta_fb. The launch's own
 * theta argument is then unused. Switching between the plain and the learned
 * criterion cuts the work items again (see octgrav_item_info; as after a
 * change of ppl in octgrav_set_launch); a new record on a tree that already
 * has one keeps them. Errors: ERR_ARG, ERR_CUDA. */
int octgrav_set_criterion(octgrav_tree *t, const float *record, double tau, double theta_lo,
                          double theta_hi, double theta_fb);

/* How the fused kernel stages accepted cell records into shared memory:
 *   0 = one cp.async.bulk (64 B) per record, issued by the accepting lane;
 *   1 = four 16-byte cp.async per record, issued by the accepting lane (default);
 *   2 = TMA tile::gather4, four records per instruction.
 * All modes compute identical results. Errors: ERR_ARG. */
int octgrav_set_staging(octgrav_tree *t, int mode);

/* Failure injection for tests (nothing faults or hangs): later launches of t
 * give each walk only stack_cap node-stack entries (0 = the whole stack), so
 * that a deep walk reports OCTGRAV_ERR_STACK; and, in staging mode 2, never
 * request the first tile of cell records of work item drop_item (-1 = none),
 * so that its bounded wait (~1 s) runs out and the launch reports
 * OCTGRAV_ERR_TIMEOUT; the warp then waits for its other copies and stops.
 * The context stays usable; octgrav_set_fault(t, 0, -1) restores normal
 * launches. A graph captured before the call keeps the old settings.
 * Errors: ERR_ARG (stack_cap < 0, drop_item outside [-1, n_items)). */
int octgrav_set_fault(octgrav_tree *t, int stack_cap, int64_t drop_item);

/* List split for systems too small to fill the GPU: later launches of t walk
 * every work item with nparts warps (1 = off, up to 16); part j evaluates the
 * accepted cells and queued leaves whose sequence numbers are j modulo nparts
 * (part 0 also the group's own particles), and the parts' results are summed
 * in part order by a second kernel, so a launch is deterministic but rounds
 * differently from an unsplit one (FP32 sums of nparts partial results).
 * Applies to launches with the plain opening test and staging mode 1 that
 * capture no lists; others run unsplit. Errors: ERR_ARG. */
int octgrav_set_split(octgrav_tree *t, int nparts);

void octgrav_free_tree(octgrav_tree *t);

#define OCTGRAV_NOALLOC_MAX_ITEMS 262144 /* work items accepted by octgrav_forces_noalloc */

/* Allocation-free variant of octgrav_forces_device. The paper has no
 * counterpart; it exists for callers that cannot allocate device memory at
 * this point: a code whose own allocator (for instance PyTorch's caching
 * allocator) owns every device byte, or a time-step loop that must not suffer
 * the device-wide synchronisation that cudaMalloc/cudaFree can cause. The
 * call makes no cudaMalloc, cudaFree or other allocating call.
 *   arena: caller-allocated device memory (256-byte aligned) that receives the
 *     tree's device arrays, copied on stream: device to device from a
 *     GPU-built tree (which must live on the current device), from the host
 *     images of a host-built one. Call once with arena = NULL to get the size
 *     needed in *arena_bytes; otherwise *arena_bytes is the arena's size and
 *     must be at least that.
 *   acc4_dev, eps, theta, G, stream: as octgrav_forces_device (tree order).
 * The tree's settings apply as in octgrav_forces_device -- staging mode,
 * particles per lane, per-system parameters and the learned criterion (whose
 * network stays in the tree's device memory; set it on the current device) --
 * except the list split of octgrav_set_split, which needs a per-part output
 * buffer: these launches run unsplit and round like an unsplit launch.
 * The status word, work-queue counter and per-item counts live in a
 * fixed-size array inside the library (2 MiB + 256 B per GPU, kept until the
 * process exits), so the tree may have at most OCTGRAV_NOALLOC_MAX_ITEMS work
 * items (octgrav_tree_stats out[4]); larger trees get ERR_ARG. The first call
 * on a device looks up that array's address with the device current; make it
 * before any stream capture. All calls share the array: calls that overlap on
 * the GPU race and give wrong results. The call waits for the stream and
 * returns OK, ERR_STACK, ERR_TIMEOUT or ERR_INDEX like octgrav_status.
 * octgrav_interaction_counts does not see these launches. */
int octgrav_forces_noalloc(octgrav_tree *t, void *arena, size_t *arena_bytes, double eps,
                           double theta, double G, float *acc4_dev, void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *octgrav_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int octgrav_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OCTGRAV_H */
