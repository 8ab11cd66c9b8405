// Internal declarations shared by the CUDA translation units of libgothic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gothic.h"

#define GT_KEY_LEVELS 21              // 21 bits per axis -> 63-bit Morton keys
#define GT_TREE_LEVELS 22             // tree levels 0..21
#define GT_LEAF_BUCKETS 17            // a level's leaves by particle count: 1..16, then larger
#define GT_LEVEL_BUCKETS (GT_LEAF_BUCKETS + 8)  // + its cells with children by number of children
#define GT_CELL_BUCKETS (GT_TREE_LEVELS * GT_LEVEL_BUCKETS)
#define GT_LEAF_FLAG 0x80000000u      // set in a node's second link word for a leaf
#define GT_SPIN_LIMIT (1u << 22)      // default bound on every device spin-wait (iterations)
// Enclosing radii computed in FP32 are widened by (1 + 2^-20): the few roundings of
// an FP32 distance (each <= 2^-24 relative) cannot then shrink a radius below the
// true one.
#define GT_RADIUS_MARGIN (1.0f + 0x1p-20f)

// The debug build (-DGT_DEBUG=1, a separate library) checks the node and particle
// indices that the walk and the pseudo j-particle pass read from the tree against the
// node and particle counts; a failed check latches GT_EINVAL with the kernel's tag and
// the access is skipped (no trap).  The release build compiles none of it.
#ifndef GT_DEBUG
#define GT_DEBUG 0
#endif

// Kernel ids recorded with a latched error (diagnostic only).
enum { GTK_NONE = 0, GTK_BUILD, GTK_PSEUDO, GTK_ACTIVE, GTK_WALK, GTK_SORT, GTK_CORRECT, GTK_PROBE };

// Small control block in device memory: counters, per-step scalars and the
// error word.  One per system, inside the workspace.
struct DevCtl {
    int err;                          // first latched GT_E* code
    int err_where;                    // GTK_* of the kernel that latched it
    unsigned int epoch;               // bumped once per tree build / compaction
    unsigned int n_active;            // i-particles of the current force evaluation
    unsigned int n_groups;            // groups of the current force evaluation (cell grouping)
    unsigned int seg[2 * GT_TREE_LEVELS + 1];  // cell list: level l's leaves start at seg[2l], its
                                               // cells with children at seg[2l + 1]; [44] = all
    unsigned int cell_bucket[GT_CELL_BUCKETS];  // bucket sizes, then fill cursors, of the cell list
    unsigned int group_next;          // dynamic group counter of the walk
    unsigned int tile_ticket[GT_TREE_LEVELS + 4];  // dynamic tile ids: levels, actives, groups, leaves, cells
    unsigned int level_start[GT_TREE_LEVELS + 2];  // first cell of each level; [22] = node count
    unsigned int sort_ticket[8];      // dynamic tile ids of the 8 sort passes
    unsigned int pl_ticket;           // chunk tickets of the pseudo j-particle cell pass
    unsigned int pl_done[GT_TREE_LEVELS];  // finished cell chunks per level of that pass
    unsigned long long interactions;  // cumulative
    unsigned long long mac_tests;     // cumulative
    unsigned long long tnext;         // block time of the current step
    unsigned long long tnext_acc;     // running minimum for the next step
    unsigned long long max_dt_bits;   // bit pattern of the largest dt_i (start only)
    double dt_max;                    // longest block step (a power of two)
    int M;                            // log2(dt_max)
    int levels_m1;                    // L - 1 (finest level)
    float bbox_min[3];
    float pad1;
    double side;                      // side of the bounding cube (FP64)
    double scale;                     // 2^21 / side
    unsigned int spin_limit;          // bound on every spin-wait of this system; 0: GT_SPIN_LIMIT
    unsigned int pad2;
};

// The bound of a spin-wait: the control block's own, or the default.
__device__ __forceinline__ unsigned int gt_spin_limit(const DevCtl *ctl) {
    const unsigned int v = *((const volatile unsigned int *)&ctl->spin_limit);
    return v ? v : GT_SPIN_LIMIT;
}

// Particle state, structure of arrays, in internal (key) order.
struct State {
    double *rx, *ry, *rz;  // position at t0 (FP64)
    double *vx, *vy, *vz;  // half-step velocity v^{1/2} (FP64); the velocity before gt_start
    long long *t0;         // tick of the last correction
    uint8_t *level;        // block-step level
    float *aold;           // |a| of the last force evaluation (FP32)
    float4 *acc;           // last acceleration and potential
    uint32_t *id;          // caller's index
    float *mass;
};

// Node arrays of the tree.
// FP64 sums of a cell: mass and the three first moments.
struct __align__(32) DSum4 {
    double m, x, y, z;
};

struct Nodes {
    uint32_t *first, *count;   // particle range
    int32_t *child;            // first child, -1 for a leaf
    uint32_t *nchild;
    int32_t *parent;
    float4 *jpos;              // pseudo j-particle (x, y, z, m) FP32
    float4 *walk;              // (b_J, link0, link1, B_2): link0 = first child or first particle,
                               // link1 = nchild, or count | GT_LEAF_FLAG for a leaf; B_2 the
                               // second moment of the multipole MAC
    DSum4 *sum;                // FP64 (m, m x, m y, m z)
    uint32_t *cells;           // every node once: the leaves bucketed by particle count, then
                               // the cells with children by level (deepest last) and, inside
                               // a level, by number of children
};

__device__ __forceinline__ void gt_set_error(DevCtl *ctl, int code, int where) {
    if (atomicCAS(&ctl->err, 0, code) == 0) ctl->err_where = where;
}

__device__ __forceinline__ unsigned int lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned int lanemask_lt() {
    unsigned int m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exact FP32 -> FP64 conversion of a normal float by its IEEE-754 fields, on the
// integer pipe (the FP64 pipe of this GPU is narrow); zero, subnormal, inf and nan
// take the hardware conversion.
__device__ __forceinline__ double f2d(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned long long d = ((unsigned long long)(b >> 31) << 63) |
                                 ((unsigned long long)(e + (1023u - 127u)) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// FP64 -> FP32 rounded to nearest (ties to even) by the IEEE-754 fields on the integer
// pipe, for results in the normal FP32 range; zero, subnormal, overflowing, inf and nan
// values take the hardware conversion.  Keeping the 23 leading fraction bits and rounding
// on the 29 dropped ones; a carry out of the fraction moves into the exponent, which is
// the correctly rounded result (up to infinity at the top of the range).
__device__ __forceinline__ float d2f(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
    if (e <= 0 || e >= 255) return __double2float_rn(d);
    const unsigned long long frac = b & 0xfffffffffffffull;
    unsigned int keep = (unsigned int)(frac >> 29);
    const unsigned int rest = (unsigned int)(frac & 0x1fffffffu);
    keep += (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) ? 1u : 0u;
    return __uint_as_float((unsigned int)(b >> 63) << 31 | ((unsigned int)e << 23) + keep);
}

// (double)d * 2^k for 0 <= d < 2^53 (exact, built from the bits; the FP64 pipe of this
// GPU is narrow); any other case, or an exponent out of range, takes the FP64 product.
__device__ __forceinline__ double i2d_scaled(long long d, int k) {
    if (d == 0) return 0.0;
    if (d < 0 || d >= (1ll << 53)) return __dmul_rn((double)d, ldexp(1.0, k));
    const int top = 63 - __clzll(d);
    const int e = top + k + 1023;
    if (e <= 0 || e >= 2047) return __dmul_rn((double)d, ldexp(1.0, k));
    const unsigned long long frac = ((unsigned long long)d << (52 - top)) & 0xfffffffffffffull;
    return __longlong_as_double((long long)(((unsigned long long)e << 52) | frac));
}

// Inclusive warp scan of 32-bit counts.
__device__ __forceinline__ unsigned int warp_incl_scan(unsigned int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane_id() >= (unsigned)o) v += t;
    }
    return v;
}

// Exclusive block scan for blockDim.x == NT (multiple of 32, <= 1024).
// Returns the exclusive prefix of v; *total receives the block sum.
template <int NT>
__device__ __forceinline__ unsigned int block_excl_scan(unsigned int v, unsigned int *total,
                                                        unsigned int *smem /* NT/32 + 1 */) {
    const unsigned int lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned int inc = warp_incl_scan(v);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned int w = lane < NT / 32 ? smem[lane] : 0u;
        unsigned int wi = warp_incl_scan(w);
        if (lane < NT / 32) smem[lane] = wi - w;
        if (lane == NT / 32 - 1) smem[NT / 32] = wi;
    }
    __syncthreads();
    const unsigned int r = smem[warp] + inc - v;
    *total = smem[NT / 32];
    __syncthreads();
    return r;
}

// Decoupled look-back, by one full warp: publish this tile's aggregate, gather the
// exclusive prefix from its predecessors, publish the inclusive prefix.  Status
// words pack (tag << 32 | value); tag = 4*epoch + {1: aggregate, 2: prefix}.  Lane
// i reads predecessor tile - 1 - i, so each step covers 32 tiles: once every tile
// up to the nearest published prefix has published at least its aggregate, the
// values up to and including that prefix are summed by shuffles; with no prefix in
// the window the 32 aggregates are added and the window moves back.  Tiles are taken
// in increasing order from a ticket, so every predecessor is held by a running block
// and the wait ends; it is still bounded (gt_spin_limit), and a wait that runs out
// latches GT_ETIMEOUT and returns the partial prefix.  Every lane gets the result.
__device__ __forceinline__ unsigned int lookback_warp(unsigned long long *status, unsigned int tile,
                                                      unsigned int aggregate, unsigned int epoch,
                                                      DevCtl *ctl, int where) {
    const unsigned long long tagA = (unsigned long long)(4u * epoch + 1u) << 32;
    const unsigned long long tagP = (unsigned long long)(4u * epoch + 2u) << 32;
    const int lane = (int)(threadIdx.x & 31u);
    if (tile == 0) {
        if (lane == 0) atomicExch(&status[0], tagP | aggregate);
        return 0u;
    }
    if (lane == 0) atomicExch(&status[tile], tagA | aggregate);
    unsigned int excl = 0;
    int base = (int)tile - 1;
    unsigned int spins = 0;
    const unsigned int limit = gt_spin_limit(ctl);
    for (;;) {
        const int t = base - lane;
        // a slot before tile 0 reads as a published prefix of 0
        const unsigned long long sv = t >= 0 ? *((volatile unsigned long long *)&status[t]) : tagP;
        const unsigned long long tag = sv & 0xffffffff00000000ull;
        const unsigned int pmask = __ballot_sync(0xffffffffu, tag == tagP);
        const unsigned int vmask = __ballot_sync(0xffffffffu, tag == tagP || tag == tagA);
        const int firstP = pmask ? __ffs(pmask) - 1 : 32;
        const unsigned int need = firstP >= 31 ? 0xffffffffu : ((1u << (firstP + 1)) - 1u);
        if ((vmask & need) != need) {
            if (++spins > limit) {
                if (lane == 0) gt_set_error(ctl, GT_ETIMEOUT, where);
                break;
            }
            __nanosleep(32);
            continue;
        }
        unsigned int v = lane <= firstP ? (unsigned int)sv : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (firstP < 32) break;
        base -= 32;
    }
    if (lane == 0) atomicExch(&status[tile], tagP | (unsigned long long)(excl + aggregate));
    return excl;
}

// ---- host-side launch helpers (defined in the .cu files) --------------------
// Every helper reports the kernels it launched (counted for gt_kernel_launches).
void gt_note_launches(int k);

struct SortBufs {
    uint64_t *key[2];
    uint32_t *val[2];
    uint32_t *status;            // look-back status of the 8 passes, 8 x tiles x RADIX
    uint32_t *hist;              // digit histograms of the 8 passes, 8 x RADIX
    uint32_t *digit_base;        // digit starts of the 8 passes, 8 x RADIX
};

// keys.cu
void gt_launch_bbox(const float4 *posm, int64_t n, float *partial, int nblk, DevCtl *ctl,
                    cudaStream_t st);
void gt_launch_keys(const float4 *posm, int64_t n, const DevCtl *ctl, int curve, uint64_t *key, uint32_t *idx,
                    cudaStream_t st);
// sort.cu: sorts (key, val) in buffers 0; result in buffers 0 (even passes).
int gt_sort_tiles(int64_t n);
size_t gt_sort_scratch_bytes(int64_t n);
void gt_launch_sort(SortBufs &b, int64_t n, DevCtl *ctl, cudaStream_t st);
void gt_sort_init();
// tree.cu
// scratch: gt_build_scratch_bytes(n) bytes (per-particle marks and per-tile counts)
size_t gt_build_scratch_bytes(int64_t n);
void gt_launch_build(const uint64_t *skey, int64_t n, int leaf_max, Nodes nd, int64_t cap,
                     unsigned long long *status, uint8_t *scratch, DevCtl *ctl, int nsm, cudaStream_t st);
void gt_launch_cell_lists(Nodes nd, int64_t cap, DevCtl *ctl, int nsm, cudaStream_t st);
// with_mass: form the FP64 mass sums (after a build); otherwise reuse the stored ones
void gt_launch_pseudo(Nodes nd, int64_t cap, const float4 *posm, DevCtl *ctl, int nsm, bool with_mass,
                      cudaStream_t st);
// integrate.cu
void gt_launch_prepare(DevCtl *ctl, int begin_step, cudaStream_t st);
void gt_launch_set_nactive(DevCtl *ctl, unsigned int n_active, cudaStream_t st);
// T of the prediction: the current step's block time, or (ahead) the next one, still
// in tnext_acc before k_prepare moves it
void gt_launch_predict(const State &s, int64_t n, const DevCtl *ctl, float4 *posm, cudaStream_t st,
                       bool ahead = false);
// The control words the host reads between block steps, copied by the device into
// (mapped, pinned) host memory.
struct StepMirror {
    unsigned long long tnext_acc;  // block time of the next step
    unsigned int n_active;         // i-particles of the step just finished
    int err;                       // latched device error
};
void gt_launch_mirror(const DevCtl *ctl, StepMirror *dst, cudaStream_t st);
void gt_launch_load(const State &s, float4 *posm, int64_t n, cudaStream_t st);
void gt_launch_permute(const State &src, const State &dst, const float4 *posm_in, float4 *posm_out,
                       const uint32_t *perm, int64_t n, cudaStream_t st);
void gt_launch_copy_state(const State &src, const State &dst, const float4 *posm_in, float4 *posm_out,
                          int64_t n, cudaStream_t st);
void gt_launch_deinterleave3(const double *in, int64_t n, double *x, double *y, double *z,
                             cudaStream_t st);
void gt_launch_interleave3(const double *x, const double *y, const double *z, int64_t n, double *out,
                           cudaStream_t st);
void gt_launch_state_out(const State &t, int64_t n, double *pos, double *vel, cudaStream_t st);
void gt_launch_gather_f(const float *in, const uint32_t *id, int64_t n, float *out, cudaStream_t st);
void gt_launch_active(const State &s, int64_t n, int L, int all, DevCtl *ctl, uint32_t *active,
                      uint32_t *prefix, unsigned long long *status, int nsm, cudaStream_t st);
void gt_launch_active_from_list(const uint32_t *list, int64_t n_list, int64_t n, uint8_t *flags, DevCtl *ctl,
                                uint32_t *active, uint32_t *prefix, unsigned long long *status, int nsm,
                                cudaStream_t st);
void gt_launch_groups(Nodes nd, int64_t cap, const uint32_t *prefix, int gmax, float r_crit, int64_t n,
                      uint8_t *marks, DevCtl *ctl, uint32_t *gstart, unsigned long long *status, int nsm,
                      cudaStream_t st);
void gt_launch_correct(const State &s, const uint32_t *active, const float4 *acc, DevCtl *ctl,
                       int64_t n, int L, double c2, int nsm, cudaStream_t st);
void gt_launch_aold(const float4 *acc, int64_t n, float *aold, cudaStream_t st);
void gt_launch_set_clock(DevCtl *ctl, int M, int L, long long T, cudaStream_t st);
void gt_launch_set_tnext(DevCtl *ctl, long long T, cudaStream_t st);
void gt_launch_set_u32(unsigned int *dst, unsigned int v, cudaStream_t st);
// api.cu: one warp's look-back over a predecessor that never publishes (bounded-wait probe)
void gt_launch_wait_probe(unsigned long long *status, DevCtl *ctl, cudaStream_t st);
void gt_launch_tnext_all(const State &s, int64_t n, int L, DevCtl *ctl, int nsm, cudaStream_t st);
void gt_launch_gather_resume(const uint8_t *lv, const long long *t0, const float *ao, const float4 *acc,
                             const State &s, int64_t n, cudaStream_t st);
void gt_launch_init_levels(const State &s, const float4 *acc, int64_t n, int L, double c2, int M_given,
                           int have_M, DevCtl *ctl, int nsm, cudaStream_t st);
// walk.cu
struct WalkArgs {
    const float4 *jpos;
    const float4 *walk;
    const float4 *posm;
    const uint32_t *active;  // null: identity
    const uint32_t *gstart;  // first active position of every group; null: runs of gmax
    const float *aold;
    float4 *acc;
    uint32_t *queue;
    DevCtl *ctl;
    uint32_t n;              // particles (bound of the indices in active)
    int gmax;
    int qcap;                // power of two
    int mac;
    int ij_share;            // lanes per i-particle; 0: 32 / (members rounded up to a power of two)
    int sphere;              // pseudo i-particle: 0 GEO centre, 1 Ritter's efficient bounding sphere
    float theta, delta_acc, eps2, G, inv_eps;
};
int gt_walk_blocks(int nsm);
// tuner.cu
// On-line Brent minimisation (one abscissa out, its cost back) for the critical
// separation of groups (Sec. 2.4).
struct BrentSearch {
    double a, b, x, w, v, fx, fw, fv, d, e, u, tol, abs_tol;
    int state;  // 0: first point pending, 1: searching, 2: converged
    int evals;
};
void gt_brent_start(BrentSearch *b, double lo, double hi, double tol, double abs_tol);
double gt_brent_next(BrentSearch *b);
void gt_brent_report(BrentSearch *b, double f);
bool gt_brent_done(const BrentSearch *b);
extern "C" int gt_rebuild_interval(const double *t_walk, int n, double t_make, int *model_out,
                                   double *n_opt_out, double *coef_out);
int gt_walk_warps_per_block();
void gt_launch_walk(const WalkArgs &a, int nblocks, cudaStream_t st);
// one launch over the groups of nsys systems (args, ctls: device arrays of nsys entries)
void gt_launch_walk_batch(DevCtl *const *ctls, const WalkArgs *args, int nsys, uint32_t *gprefix,
                          unsigned int *group_next, uint32_t *queue, int qcap, int mac, int nblocks,
                          cudaStream_t st);
