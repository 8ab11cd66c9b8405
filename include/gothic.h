/*
 * gothic.h -- C ABI of a GB300 (sm_103a) library for the block-time-step
 * oct-tree gravity method of Miki & Umemura, "GOTHIC: Gravitational oct-tree
 * code accelerated by hierarchical time step controlling" (arXiv:1610.07279).
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: GT_OK (0) or a negative GT_E* code.
 *     Nothing throws across the ABI.
 *   - Device work is enqueued on the caller's stream and is asynchronous unless
 *     the comment says "synchronises".  Errors found on the device (overflow of
 *     a fixed-size buffer, a bounded wait that ran out) are latched in a device
 *     error word; gt_sync_status() or gt_get_stats() reports them.
 *   - The caller owns all memory.  A system lives inside one workspace the caller
 *     allocates (gt_workspace_bytes) and hands over; the library never calls
 *     cudaMalloc/cudaFree for a system (only gt_block_step's look-ahead takes 16
 *     bytes of pinned host memory, once per system).  Pointers named d_* must be device
 *     pointers; pointers named p_* may be host (pageable or pinned) or device
 *     pointers (copied with cudaMemcpyAsync, kind inferred from the address).
 *   - Particle order: the library keeps particles sorted by their space-filling
 *     key ("internal index").  Arrays passed to gt_set_state are in the caller's
 *     order; gt_get_state returns the internal order together with id[] (the
 *     caller's index of each internal slot).
 *   - One stream at a time per system; systems are independent.
 *   - Precision: positions and velocities are FP64; the tree, the MAC and the
 *     force sums are FP32; centre-of-mass sums are FP64.
 */
#ifndef GOTHIC_H
#define GOTHIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every entry point is exported from the shared library (built with hidden
 * visibility otherwise). */
#if defined(__GNUC__)
#define GT_API __attribute__((visibility("default")))
#else
#define GT_API
#endif

/* ---- status codes ---------------------------------------------------------- */
#define GT_OK 0
#define GT_EINVAL (-1)    /* bad argument */
#define GT_ENOMEM (-2)    /* workspace too small */
#define GT_EOVERFLOW (-3) /* a fixed-size device buffer (nodes, walk queue) overflowed */
#define GT_ETIMEOUT (-4)  /* a bounded device wait ran out */
#define GT_ECUDA (-5)     /* a CUDA runtime call failed */
#define GT_EAGAIN (-6)    /* server: no slot or memory free now; retry later */
#define GT_EPENDING (-7)  /* server: the request has not finished yet */
#define GT_ENOTIMPL (-8)  /* option not implemented */
#define GT_ESTATE (-9)    /* call out of order (e.g. block step before start) */

/* ---- multipole acceptance criteria (Sec. 2.2) -------------------------------- */
#define GT_MAC_OPENING_ANGLE 0 /* Eq. (2), Barnes & Hut 1986: b_J / d <= theta   */
#define GT_MAC_ACCELERATION 1  /* Eq. (5), Springel 2005: d >= (G m_J b_J^2 /
                                  (Delta_acc |a_old|))^(1/4)                    */
#define GT_MAC_MULTIPOLE 2     /* Warren & Salmon 1993 (Sec. 2.2): d >= b_J/2 +
                                  sqrt(b_J^2/4 + sqrt(3 B_2 / Delta_mul)), B_2 =
                                  sum of m |r - r_J|^2 over the cell; Delta_mul is
                                  taken from delta_acc                          */

typedef struct CUstream_st *gt_stream; /* identical to cudaStream_t */

/* Method parameters.  gt_default_params fills the paper's fiducial values. */
typedef struct gt_params {
    int32_t mac;        /* GT_MAC_*; the paper's fiducial choice is ACCELERATION   */
    float theta;        /* opening angle of Eq. (2); also the bootstrap pass's     */
    float delta_acc;    /* Delta_acc of Eq. (5); fiducial 2^-7 (Sec. 3.3)          */
    float eps;          /* Plummer softening of Eq. (1)                            */
    float G;            /* gravitational constant of Eq. (1)                       */
    int32_t leaf_max;   /* a cell with more particles than this is split (<= 21 levels) */
    int32_t group_max;  /* at most this many i-particles share one walk (Sec. 2.3):
                           <= 32 / S for S > 1, else <= 64 (a group of more than 32
                           gives each lane of the warp two i-particles)            */
    int32_t ij_share;   /* S: threads sharing one i-particle (Sec. 2.5): 1..32, a power of
                           2; or 0 = per group, 32 / (members rounded up to a power of
                           two), one lane per two members above 32                 */
    int32_t levels;     /* L: number of block-step levels, 1..30 (Sec. 1)          */
    int32_t rebuild_every; /* rebuild the tree every n block steps (Sec. 2.6); 1 = always;
                              0 = automatic: the interval model of gt_rebuild_interval fed
                              with the measured walk and rebuild times (synchronises the
                              stream once per block step)                             */
    int32_t walk_queue; /* per-warp cell queue capacity, power of 2 (Sec. 2.3); >= 8192
                           leaves room for the depth-first fallback that bounds it */
    int32_t node_factor;   /* tree-cell capacity = node_factor * n + 2048 (>= 1); tight
                              clumps of more than leaf_max particles form chains down to
                              level 21 and may need more than the default 2 */
    double eta;         /* step accuracy: dt_i = sqrt(2 eta eps / |a_i|)           */
    double dt_max;      /* longest step, a power of two; <= 0: derived at gt_start */
    int32_t group_mode; /* GT_GROUP_CELLS (default): a group is the actives of one tree
                           cell holding at most group_max of them, so it never straddles
                           distant regions (Sec. 2.4); GT_GROUP_CELLS_TUNED: the same with
                           the size tuned per class of step (below); GT_GROUP_RUNS:
                           consecutive runs of group_max actives in the given order */
    float r_crit;       /* critical separation of a group (Sec. 2.4), cell grouping only:
                           a cell whose enclosing radius b_J exceeds it is split into its
                           children even when it holds few actives (leaves are kept).
                           0 = no limit (default); > 0 = this value; < 0 = tuned on line
                           by Brent's method from |r_crit| on, one search per class of
                           block step (the coarsest active level), minimising the walk
                           time per active particle (gt_block_step with the automatic
                           rebuild interval only; elsewhere |r_crit| is used)       */
    int32_t key_curve;  /* GT_KEY_MORTON (default) or GT_KEY_HILBERT (Sec. 2.1, App. A:
                           the paper's Peano-Hilbert order); either way the first 3l bits
                           of a key name the level-l cube, so the tree holds the same
                           cells                                                    */
    int32_t reserved2;
} gt_params;

#define GT_KEY_MORTON 0
#define GT_KEY_HILBERT 1

#define GT_GROUP_RUNS 0
#define GT_GROUP_CELLS 1
/* Cell groups whose size is tuned on line (gt_block_step with the automatic rebuild
 * interval): for every class of block step (the coarsest active level) the walk time
 * per active particle is measured once with group_max, / 2 and / 4, the fastest is
 * kept, and the three are measured again every 64 steps of the class.  Elsewhere it
 * acts as GT_GROUP_CELLS. */
#define GT_GROUP_CELLS_TUNED 2
/* Flag added to group_mode: the pseudo i-particle of a group is centred on Ritter's
 * efficient bounding sphere of its members (Appendix B; the paper's choice on its
 * newest GPU) instead of the centre of their bounding box (GEO, the default); the
 * radius is the largest member distance either way. */
#define GT_SPHERE_EBS 0x100

/* Counters and state read back by gt_get_stats (synchronises the stream). */
typedef struct gt_stats {
    int64_t n;              /* particles                                           */
    int64_t T;              /* current block time in ticks of the finest step      */
    int64_t n_active;       /* i-particles of the last force evaluation            */
    int64_t n_groups;       /* groups of the last force evaluation                 */
    int64_t n_nodes;        /* tree cells                                          */
    int64_t depth;          /* deepest tree level + 1                              */
    int64_t interactions;   /* cumulative i-j interactions evaluated               */
    int64_t mac_tests;      /* cumulative MAC evaluations                          */
    int64_t block_steps;    /* block steps taken since gt_start                    */
    int64_t rebuilds;       /* tree builds since create                            */
    double dt_max;          /* longest step in use                                 */
    int32_t err;            /* latched device error (GT_OK if none)                */
    int32_t err_where;      /* kernel that latched it (diagnostic)                 */
} gt_stats;

typedef struct gt_system gt_system;

/* Human-readable name of a status code (static string). */
GT_API const char *gt_strerror(int status);

/* The paper's fiducial parameters: acceleration MAC with Delta_acc = 2^-7
 * (Sec. 3.3), theta = 0.5 for the bootstrap pass, G = 1, eps = 1/64,
 * leaf_max = 16, group_max = 64, S = 0 (per group), L = 8, eta = 0.025,
 * queue 16384, node_factor 2, cell grouping with the size tuned per class of step
 * (GT_GROUP_CELLS_TUNED), r_crit 0, automatic rebuild interval. */
GT_API int gt_default_params(gt_params *prm);

/* Bytes of device workspace a system of n particles needs (0 <= n < 2^30; GT_EINVAL
 * otherwise -- the sort's look-back counts hold 30 bits). */
GT_API int gt_workspace_bytes(int64_t n, const gt_params *prm, size_t *bytes);

/* Create a system of n particles inside the caller's workspace d_ws (at least
 * gt_workspace_bytes, 256-byte aligned, on the current device).  The workspace
 * must outlive the system.  Host-side bookkeeping is malloc'ed here and freed by
 * gt_system_destroy.  GT_ENOMEM if ws_bytes is too small. */
GT_API int gt_system_create(gt_system **sys, int64_t n, const gt_params *prm, void *d_ws,
                     size_t ws_bytes);
GT_API int gt_system_destroy(gt_system *sys);

/* Replace the parameters (same n; leaf_max/group_max/ij_share/walk_queue may
 * change; levels and dt_max only before gt_start). */
GT_API int gt_set_params(gt_system *sys, const gt_params *prm);

/* Load particles in the caller's order: p_pos, p_vel n x 3 FP64 (row-major),
 * p_mass n FP32 (> 0).  Positions are also rounded to FP32 for the tree.  Resets
 * time to 0 and the internal order to the caller's order.  Any p_* may be host
 * or device memory. */
GT_API int gt_set_state(gt_system *sys, const double *p_pos, const double *p_vel, const float *p_mass,
                 gt_stream stream);

/* Steps A1-A5 of the method on the current FP32 positions (Sec. 2.1):
 * bounding cube and 63-bit Morton keys (Appendix A), a stable radix sort of
 * (key, index), permutation of every particle array into key order, the
 * breadth-first octree (cells split into up to eight children by key digit,
 * numbered level by level with prefix sums) and the pseudo j-particles
 * (mass, FP64-accumulated centre of mass, enclosing radius b_J; Fig. 1). */
GT_API int gt_build_tree(gt_system *sys, gt_stream stream);

/* Steps A6-A7: accelerations of the listed i-particles from the current tree
 * (Sec. 2.3-2.4): the i-particles are cut into groups that share one walk -- with
 * cell grouping (the default) the listed particles of one tree cell holding at most
 * group_max of them, with run grouping consecutive runs of group_max entries of
 * d_active; each group's pseudo i-particle is the sphere about the centre of its
 * bounding box (Appendix B, GEO; or Ritter's sphere with GT_SPHERE_EBS); cells are
 * tested with the MAC at distance
 * lambda r_JI (Eqs. 6-7) and the Plummer-softened sums of Eq. (1) run over the
 * accepted cells and the particles of opened leaves.
 *   d_active  n_active internal indices (uint32), or NULL for all particles
 *             (then n_active must be n).  With cell grouping the list must be
 *             strictly increasing (else GT_EINVAL is latched); with run grouping
 *             groups follow the given order.
 *   d_aold    n FP32 |a_old| by internal index (the acceleration MAC needs it),
 *             or NULL to use the system's own.
 *   d_acc     n_active x 4 FP32 output (ax, ay, az, potential), in d_active order.
 * Uses the current parameters' mac.  Requires a built tree. */
GT_API int gt_accel_active(gt_system *sys, const uint32_t *d_active, int64_t n_active,
                    const float *d_aold, float *d_acc, gt_stream stream);

/* Start the block-step integration at t = 0 (Sec. 2.7): build the tree, run
 * an opening-angle bootstrap pass (theta) whose |a| seeds a_old (the paper has
 * no a_old at t = 0), an acceleration-MAC pass, choose dt_max (if not given) as
 * the largest power of two not above max dt_i, assign each particle the level
 * of the smallest step dt_max 2^-k <= dt_i = sqrt(2 eta eps/|a|), and give
 * every particle its first half kick v^{1/2} = v + (dt/2) a.
 *   p_aold_boot  optional n FP32 |a_old| in the caller's order; if given the
 *                bootstrap pass is skipped and these values are used. */
GT_API int gt_start(gt_system *sys, const float *p_aold_boot, gt_stream stream);

/* One block step (Sec. 1; Sec. 2.7, Eqs. 15-17): advance to the next tick T
 * at which some particle's step ends; predict every particle to T; rebuild
 * the tree (every rebuild_every steps, else refresh the pseudo j-particles on
 * the old topology, Sec. 2.6); select the active particles (t0 + ticks(level)
 * == T); walk them; correct their velocities, assign new levels (a shorter
 * step at once, a longer one by one level when T is aligned to it) and give
 * the next half kick.  With a fixed rebuild interval it is fully asynchronous
 * (no host synchronisation).  With the automatic interval (rebuild_every = 0)
 * the on-line tuners read the previous step's times and counts, so it first
 * waits for that step to finish; to keep the device busy meanwhile, every such
 * step ends by enqueuing the prediction (A8) of the next one (a look-ahead into
 * the system's scratch positions, with the control words the next call reads
 * copied to 16 bytes of mapped pinned host memory, allocated once per system).
 * The next gt_block_step on the same stream uses it; any call that changes the
 * state or the tree drops it.  Results are the same bit for bit either way. */
GT_API int gt_block_step(gt_system *sys, gt_stream stream);

/* Resume a block-step integration (checkpoint/restart, or a caller-driven
 * integration): after gt_set_state, whose velocities are then taken as the
 * stored half-step velocities v^{1/2}, set per particle (caller's order) the
 * level p_level (uint8, < L), the tick of the last correction p_t0 (int64,
 * multiple of the level's span), |a_old| p_aold (FP32) and optionally the last
 * acceleration p_acc (n x 4 FP32, may be NULL), together with dt_max (a power of
 * two) and the current tick T.  Afterwards gt_block_step continues from there.
 * Does not build a tree (gt_block_step or gt_build_tree will). */
GT_API int gt_set_integrator_state(gt_system *sys, const uint8_t *p_level, const int64_t *p_t0,
                                   const float *p_aold, const float *p_acc, double dt_max, int64_t T,
                                   gt_stream stream);

/* Step A8 alone (Eq. 16 with the elapsed time): positions of every particle at
 * tick T, r(T) = r0 + ((T - t0) dt_min) v^{1/2}, rounded to FP32, written as
 * n x 4 FP32 (x, y, z, m) in internal order to d_posm (device).  Requires a
 * started or resumed integration. */
GT_API int gt_predict(gt_system *sys, int64_t T, float *d_posm, gt_stream stream);

/* Step A9 alone (Eq. 17): correct the listed particles (internal indices) at
 * tick T with the caller's accelerations d_acc (n_active x 4 FP32, device), give
 * them their new level and next half kick, exactly as gt_block_step does. */
GT_API int gt_correct(gt_system *sys, const uint32_t *d_active, int64_t n_active, const float *d_acc,
                      int64_t T, gt_stream stream);

/* Run block steps until the next block time would exceed T_end (ticks of the
 * finest step); *steps (may be NULL) receives the number taken.  Reads the
 * next block time back after every step (waits for every step: for the words
 * the look-ahead of gt_block_step mirrors to the host, or else for the stream).
 * One full block-step cycle is T_end = the next multiple of 2^(L-1). */
GT_API int gt_advance(gt_system *sys, int64_t T_end, int64_t *steps, gt_stream stream);

/* Per-phase device timers (CUDA events around each phase of gt_block_step and
 * the passes of gt_start; the paper monitors per-function times on the fly,
 * Sec. 1, Sec. 2.4, Sec. 2.6).  Phases: 0 predict, 1 keys+sort, 2 permute,
 * 3 tree build, 4 pseudo j-particles, 5 active set, 6 walk, 7 correct.
 * gt_profile(sys, 1) enables and zeroes them; timing is read at the waits of
 * gt_block_step (automatic interval; with a fixed interval and timers on, each
 * step waits for the previous one to read them), gt_advance and gt_get_timers.
 * A prediction enqueued ahead of its step counts once it has run.  ms_out[8]
 * total milliseconds, launches_out[8] number of timed phase executions. */
#define GT_NPHASES 8
GT_API int gt_profile(gt_system *sys, int enable);
GT_API int gt_get_timers(gt_system *sys, double *ms_out, int64_t *launches_out, gt_stream stream);

/* Kernels launched by this library since load (all systems). */
GT_API int gt_kernel_launches(int64_t *count);

/* Tree-rebuild interval model (Sec. 2.6, Eqs. 8-14; Appendix C).  Host only.
 * t_walk[0..n-1]: measured walk times of the n block steps since the last
 * rebuild (n >= 3); t_make: the rebuild's time.  Fits the linear, power-law and
 * parabolic growth models by least squares, keeps the one with the smallest
 * reduced chi^2 (sigma_i = 1) in *model (0 linear, 1 power law, 2 parabolic),
 * its coefficients in coef[3] (may be NULL: t1, dt | t1, r | t1, b, a), and the
 * interval that minimises the mean time per step in *n_opt (1e6 when the model
 * has no minimum, i.e. no rebuild is due). */
/* Brent's minimisation of f over [lo, hi] to a relative tolerance tol, at most max_evals
 * evaluations (host only): the search the library runs on line for r_crit (Sec. 2.4).
 * Writes the abscissa and value of the minimum found and the evaluations used. */
GT_API int gt_brent_minimize(double (*f)(double x, void *ctx), void *ctx, double lo, double hi, double tol,
                             int max_evals, double *x_min, double *f_min, int *evals);
GT_API int gt_rebuild_interval(const double *t_walk, int n, double t_make, int *model, double *n_opt,
                               double *coef);

/* Copy the state out in internal order.  Any pointer may be NULL to skip it;
 * any may be host or device memory.  p_pos, p_vel n x 3 FP64 (velocity is the
 * half-step velocity v^{1/2} that the scheme stores), p_mass n FP32, p_acc n x 4 FP32 (the
 * last acceleration and potential), p_aold n FP32 (|a_old| used by the
 * acceleration MAC), p_level n uint8, p_t0 n int64 (tick of the
 * last correction), p_id n uint32 (caller's index). */
GT_API int gt_get_state(gt_system *sys, double *p_pos, double *p_vel, float *p_mass, float *p_acc,
                        float *p_aold, uint8_t *p_level, int64_t *p_t0, uint32_t *p_id, gt_stream stream);

/* Copy the tree out.  p_keys n uint64 sorted keys; p_order n uint32 (the
 * caller's index of each internal slot, same as id); p_nodes n_nodes x 4 uint32
 * (first particle, count, first child or 0xffffffff for a leaf, number of
 * children); p_jpos n_nodes x 4 FP32 (x, y, z, m); p_bj n_nodes FP32.  Pass
 * *n_nodes_inout = capacity (entries) on entry; it returns the node count
 * (synchronises; GT_EOVERFLOW if the capacity is short). */
GT_API int gt_get_tree(gt_system *sys, uint64_t *p_keys, uint32_t *p_order, uint32_t *p_nodes,
                float *p_jpos, float *p_bj, int64_t *n_nodes_inout, gt_stream stream);

/* The i-particles selected by the last block step (internal indices, in
 * order).  *n_inout = capacity on entry, count on return (synchronises). */
GT_API int gt_get_active(gt_system *sys, uint32_t *p_active, int64_t *n_inout, gt_stream stream);

/* Synchronise the stream and report the latched device error (and clear it). */
GT_API int gt_sync_status(gt_system *sys, gt_stream stream);

/* Synchronise and read counters (see gt_stats). */
GT_API int gt_get_stats(gt_system *sys, gt_stats *out, gt_stream stream);

/* Bound of every spin-wait of this system's kernels (the decoupled look-backs of the
 * sort, the tree build and the active-set compaction, the level waits of the pseudo
 * j-particle pass), in polling iterations of a few tens of nanoseconds each; 0 restores
 * the default 2^22.  A wait that runs out latches GT_ETIMEOUT in the error word and its
 * kernel returns, so the context stays usable (the results of that call are not).  On
 * the stream, asynchronous. */
GT_API int gt_set_wait_limit(gt_system *sys, uint32_t iterations, gt_stream stream);

/* Failure-detection check: runs, with the bound `iterations`, the same warp look-back
 * the build and the compaction use, for a tile whose predecessor never publishes, so the
 * wait must run out.  Synchronises and returns the latched status (GT_ETIMEOUT when the
 * bounded wait works) and clears it, like gt_sync_status; the system's own bound is put
 * back afterwards.  Uses two of the system's look-back status words, so call it between
 * the system's other calls, not during them. */
GT_API int gt_probe_bounded_wait(gt_system *sys, uint32_t iterations, gt_stream stream);

/* Measure the device's FP32 FMA throughput (FLOP/s, FMA = 2 flops) with a
 * dependent-FMA-chain kernel on all SMs.  Synchronises; ~10 ms. */
GT_API int gt_measure_fp32_peak(double *flops, gt_stream stream);

/* FP32 instruction throughputs of the device, each from chains of one instruction
 * form on every SM (lane operations per second).  The walk's force loop issues the
 * packed form (f32x2: two FMAs, adds or multiplies per lane and instruction) and the
 * special-function reciprocal square root.  peak_flops = 2 x the larger of the two FMA
 * rates: the FP32 roofline of the walk.  rsqrt_flops = the larger of the add and
 * multiply rates / the rsqrt rate: the flops one rsqrt counts for under the paper's
 * convention (Sec. 4 and the note to Table 3: 8, 6 and 4 on its three GPUs, so that
 * one interaction is 20 + rsqrt_flops flops).  Synchronises; ~50 ms. */
typedef struct gt_fp32_rates {
    double fma_per_s;    /* scalar FMA */
    double fma2_per_s;   /* packed FMA, counted per lane operation (two per instruction) */
    double add_per_s;    /* scalar add */
    double mul_per_s;    /* scalar multiply */
    double rsqrt_per_s;  /* rsqrt.approx.ftz.f32 */
    double peak_flops;
    double rsqrt_flops;
    double fp64_fma_per_s; /* FP64 FMA, for the FP64 sums of the pseudo j-particles and the
                              integration (not part of the walk's roofline)  */
} gt_fp32_rates;
GT_API int gt_measure_fp32_rates(gt_fp32_rates *out, gt_stream stream);

/* ---- sort without allocation ------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory when they need the sort: code running inside
 * another framework's memory budget, loops that must not pay cudaMalloc's
 * implicit device synchronisation, or host code that cannot own CUDA
 * allocations at all.
 *
 * Sorts n (key, value) pairs in place by key, stably (equal keys keep their
 * order), with the same radix-sort kernels gt_build_tree uses.  d_keys (n
 * uint64) and d_vals (n uint32) are device arrays owned by the caller; they
 * receive the sorted pairs.  The scratch the sort needs (the alternate key and
 * value buffers, per-tile look-back status words, digit histograms and a control
 * block) lives in one file-scope device array of the library, sized for
 * GT_NOALLOC_SORT_MAX pairs (about 14 MiB, held on every GPU that loads the
 * library until the process exits); nothing is allocated or freed by the call.
 *   - n > GT_NOALLOC_SORT_MAX: rejected with GT_EINVAL before any device work.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any stream
 *     capture.
 *   - Every call uses the same array: calls that overlap on the GPU (on two
 *     streams, or from two threads) race and corrupt each other's results.
 *     Serialise them on one stream.
 * Asynchronous on the stream; GT_ECUDA if a launch fails; device-side errors are read
 * with gt_sort_noalloc_status. */
#define GT_NOALLOC_SORT_MAX (1 << 20)
GT_API int gt_sort_pairs_noalloc(uint64_t *d_keys, uint32_t *d_vals, int64_t n, gt_stream stream);
/* Device errors of the no-allocation sort on the current device: its look-back waits are
 * bounded, and a wait that runs out latches GT_ETIMEOUT in the sort's own static control
 * block (the sorted result of that call is then wrong).  Synchronises the stream, returns
 * the latched status (GT_OK if none, or if no sort has run on this device) and clears it.
 * Call it after the sorts whose results you use. */
GT_API int gt_sort_noalloc_status(gt_stream stream);

/* ---- batches: many independent systems, one walk launch (Sec. 2.3, 2.5) -------
 *
 * A batch holds nsys systems of any sizes in one caller workspace.  One force
 * evaluation of the batch rebuilds every system's tree (A1-A5), makes every particle
 * active and cuts the groups (A6), on forked streams so that the small systems'
 * kernels overlap, then walks the groups of ALL systems in one persistent launch
 * (A7): warps take global group numbers from one counter and find their system from
 * a device-side prefix of the systems' group counts.  Each system's forces are the
 * same, bit for bit, as gt_build_tree + gt_accel_active of that system alone with the
 * same parameters.  The whole evaluation can be captured once into a CUDA graph and
 * replayed.  Batch members share one walk queue and the batch's streams: their own
 * entry points (gt_set_state, gt_get_state, gt_accel_active, ...) may be called
 * between batch evaluations, one at a time.
 */
typedef struct gt_batch gt_batch;

/* Bytes of workspace for a batch of nsys systems of n[k] particles and parameters
 * prm[k] (prm may hold 1 entry used for all).  The queue depth of the batch is the
 * largest walk_queue. */
GT_API int gt_batch_workspace_bytes(int nsys, const int64_t *n, const gt_params *prm, int n_prm,
                                    size_t *bytes);
/* Create the batch inside d_ws (256-byte aligned, gt_batch_workspace_bytes long).
 * The library creates up to 32 streams of its own for the forked builds.  Every
 * system starts empty: load each with gt_set_state(gt_batch_system(...)). */
GT_API int gt_batch_create(gt_batch **batch, int nsys, const int64_t *n, const gt_params *prm, int n_prm,
                           void *d_ws, size_t ws_bytes);
GT_API int gt_batch_destroy(gt_batch *batch);
/* The k-th member (owned by the batch; do not destroy it). */
GT_API int gt_batch_system(gt_batch *batch, int k, gt_system **sys);
/* The walk's tuning knobs of every member: leaf_max (tree leaf size), group_max
 * (i-particles per group), walk_queue (node-queue depth per warp, a power of two no
 * larger than the depth fixed at create; 0 keeps each).  Drops a captured graph. */
GT_API int gt_batch_set_knobs(gt_batch *batch, int leaf_max, int group_max, int walk_queue);
/* One force evaluation of every member with all particles active, enqueued on
 * stream.  bootstrap != 0 first walks with the opening-angle MAC (theta of each
 * member) and takes |a| as a_old, then walks with each member's own MAC (the
 * acceleration MAC needs a_old, Sec. 2.2); bootstrap == 0 uses the a_old each member
 * already holds.  The accelerations stay in each member's force buffer: read them
 * with gt_batch_get_acc. */
GT_API int gt_batch_accel(gt_batch *batch, int bootstrap, gt_stream stream);
/* Capture the same evaluation into a CUDA graph (replaces a previous one);
 * gt_batch_launch replays it on stream. */
GT_API int gt_batch_capture(gt_batch *batch, int bootstrap, gt_stream stream);
GT_API int gt_batch_launch(gt_batch *batch, gt_stream stream);
/* Accelerations (x, y, z, potential; n x 4 FP32) of member k in internal order, and
 * optionally the original index of every internal slot (n uint32); host or device
 * pointers.  Synchronises stream. */
GT_API int gt_batch_get_acc(gt_batch *batch, int k, float *p_acc, uint32_t *p_id, gt_stream stream);
/* Error words of all members (the first non-zero status; each word is cleared) and
 * the interactions counted so far per member (n_out[k], may be NULL).  Synchronises. */
GT_API int gt_batch_sync_status(gt_batch *batch, int64_t *interactions_out, gt_stream stream);

/* Autotuner of the batch's walk knobs.  Every combination of the candidate leaf
 * sizes, group sizes and queue depths is run reps times as a captured evaluation
 * (bootstrap == 0, so every member must hold a_old, e.g. after one bootstrap
 * evaluation) and timed with CUDA events; the fastest is kept (set on the batch) and
 * returned with every candidate's mean time.  Zero-length candidate lists keep the
 * current value. */
typedef struct gt_tune_space {
    int32_t n_leaf, leaf_max[8];
    int32_t n_group, group_max[8];
    int32_t n_queue, walk_queue[4];
    int32_t reps;                 /* timed replays per candidate (>= 1) */
} gt_tune_space;
typedef struct gt_tune_result {
    int32_t leaf_max, group_max, walk_queue;
    int32_t n_tried;
    double best_ms;               /* mean time of one evaluation with the kept knobs */
    double ms[256];               /* per candidate, leaf-major, then group, then queue */
} gt_tune_result;
GT_API int gt_batch_autotune(gt_batch *batch, const gt_tune_space *space, gt_tune_result *result,
                             gt_stream stream);

/* ---- serving: continuous batching of block-step requests ----------------------
 *
 * A server keeps admitted systems resident in device memory and advances them with
 * iteration-level batching.  Each server tick enqueues, for every resident request, one
 * unit of work: the start-up (tree, opening-angle pass, a_old, first force, levels;
 * Sec. 2.2, 2.7) for a new request, one block step (predict, rebuild or pseudo j, active
 * set, correct; Sec. 2.6-2.7) for a running one.  The per-request parts run on forked
 * streams; the tree walks of all requests in the tick run in one persistent launch.
 * Requests join and leave at tick boundaries: one submitted while others are on the
 * GPU is admitted as soon as a slot and memory are free and its work overlaps theirs.
 * A request's result does not depend on the other requests (separate buffers, the
 * same kernels and order per system): it is the same bit for bit alone and in a mix.
 *
 * Memory comes from the caller's callbacks only: one region at create (the shared walk
 * queue and the per-tick tables) and one workspace per admitted request, returned
 * through free_fn when the request's result has been collected (or at destroy).
 * Admission keeps the sum of those blocks within hbm_cap bytes.  Not thread-safe: one
 * host thread drives a server (single producer).
 */
#define GT_SERVER_MAX_SLOTS 256
typedef void *(*gt_alloc_fn)(size_t bytes, void *ctx);  /* device memory, 256-byte aligned; NULL on failure */
typedef void (*gt_free_fn)(void *ptr, void *ctx);
typedef struct gt_server gt_server;

typedef struct gt_request {
    int64_t n;                 /* particles */
    const double *p_pos;       /* n x 3 FP64, host or device; copied in by gt_submit */
    const double *p_vel;       /* n x 3 FP64 */
    const float *p_mass;       /* n FP32 */
    gt_params params;          /* rebuild_every 0 means every 4 block steps here (the
                                  automatic interval needs a host sync per step) */
    int32_t nsteps;            /* block steps after the start-up (>= 0) */
    int32_t reserved;
} gt_request;

enum { GT_REQ_UNKNOWN = 0, GT_REQ_RUNNING = 1, GT_REQ_DONE = 2 };

typedef struct gt_server_stats {
    int64_t ticks;             /* ticks enqueued */
    int64_t admitted, completed;
    int64_t slots_used;
    int64_t hbm_used;          /* bytes held through alloc_fn */
    int64_t hbm_cap;
    int64_t walk_launches;     /* batched walk launches */
    int64_t reserved;
} gt_server_stats;

/* max_slots <= GT_SERVER_MAX_SLOTS resident requests; walk_queue: the per-warp walk
 * queue depth of the server (a power of two; requests asking for more are clamped). */
GT_API int gt_server_create(gt_server **srv, size_t hbm_cap, int max_slots, int walk_queue,
                            gt_alloc_fn alloc_fn, gt_free_fn free_fn, void *ctx);
/* Waits for the device, returns every block through free_fn. */
GT_API int gt_server_destroy(gt_server *srv);
/* Admit a request: GT_EAGAIN when no slot is free or its workspace would pass hbm_cap
 * (retry after collecting results), GT_EINVAL for bad arguments, GT_ENOMEM when
 * alloc_fn fails.  The inputs are copied before the call returns.  Non-blocking
 * otherwise; *ticket identifies the request. */
GT_API int gt_submit(gt_server *srv, const gt_request *req, uint64_t *ticket);
/* Enqueue ticks while there is work and fewer than two ticks are in flight; never
 * waits for the device.  *running = requests resident (may be NULL). */
GT_API int gt_server_progress(gt_server *srv, int *running);
/* Drive the server (as gt_server_progress) and report a request: GT_EPENDING while it
 * runs; GT_OK with *state = GT_REQ_DONE once finished, after writing its final state in
 * the caller's particle order -- positions at each particle's last correction and the
 * stored half-step velocities (Sec. 2.7), n x 3 FP64 each, host or device, either may be
 * NULL -- and releasing its slot (a later poll reports GT_REQ_UNKNOWN / GT_EINVAL).  A
 * device error of the request is returned instead of GT_OK (its slot is released). */
GT_API int gt_poll(gt_server *srv, uint64_t ticket, int *state, double *p_pos_out, double *p_vel_out);
GT_API int gt_server_get_stats(gt_server *srv, gt_server_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* GOTHIC_H */
