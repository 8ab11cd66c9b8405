// Block time step (Sec. 1; Sec. 2.7, Eqs. 15-17), active sets and groups, and the
// particle-array plumbing:
//   k_prepare      per-phase bookkeeping (epoch, tickets, the step's block time)
//   k_predict      A8: r(T) = fma((T - t0) dt_min, v^{1/2}, r0) for every particle, FP64,
//                  rounded to FP32 for the tree                    (HBM: 60 B read, 16 B written)
//   k_permute      A3: gather every particle array into key order  (HBM: ~100 B each way)
//   k_compact      A6: order-preserving compaction with a block scan and a bounded decoupled
//                  look-back; selects by block time (t0 + ticks(level) == T), by a flag array,
//                  or all, and writes the active prefix P[i] = #actives below i
//                  (HBM: 9 B read + 4 B prefix per particle, 4 B per active)
//   k_group_cells  A6: groups bounded by tree cells (Sec. 2.4): the actives of every maximal
//                  cell with at most group_max of them (or of a leaf, cut into runs)
//   k_correct      A9: Eq. (17), the new level, the next half kick; the active particles'
//                  new step ends are folded into the next block time
//   k_init_levels  start: dt_max, levels and the first half kick
// Level of a particle: the smallest k with dt_k = dt_max 2^-k <= dt_i = sqrt(c/|a|),
// c = 2 eta eps, clamped to [0, L-1]; equivalently 2^(4(M-k)) A2 <= c2 with
// A2 = (ax^2 + ay^2) + az^2 and c2 = c c in FP64, decided exactly on the exponents
// (no root, no division: FP64 throughput is low on this GPU).  A shorter step is taken
// at once; a longer one only by one level and only when T is a multiple of it.  Every
// FP64 operation carries an explicit rounding, so results are reproducible bit for bit.
#include "gt_internal.cuh"

namespace {

__global__ void k_prepare(DevCtl *ctl, int begin_step) {
    ctl->epoch += 1u;
    for (int l = 0; l < GT_TREE_LEVELS + 4; l++) ctl->tile_ticket[l] = 0;
    ctl->group_next = 0;
    if (begin_step) {
        ctl->tnext = ctl->tnext_acc;
        ctl->tnext_acc = ~0ull;
    }
}

__global__ void k_set_nactive(DevCtl *ctl, unsigned int n_active) { ctl->n_active = n_active; }

__global__ void k_mirror(const DevCtl *ctl, StepMirror *dst) {
    volatile StepMirror *d = dst;
    d->tnext_acc = ctl->tnext_acc;
    d->n_active = ctl->n_active;
    d->err = ctl->err;
    __threadfence_system();
}

// Two particles per thread with 16-byte loads (n even, so that every array of the state,
// and the second and third coordinate arrays inside its block, start 16-byte aligned).
__global__ __launch_bounds__(256) void k_predict2(State s, long long n, const DevCtl *__restrict__ ctl,
                                                  float4 *__restrict__ posm, int ahead) {
    const long long i = 2 * (blockIdx.x * 256ll + threadIdx.x);
    if (i >= n) return;
    const long long T = (long long)(ahead ? ctl->tnext_acc : ctl->tnext);
    const int k = (int)((__double_as_longlong(ctl->dt_max) >> 52) & 0x7ff) - 1023 - ctl->levels_m1;
    const longlong2 t0 = *(const longlong2 *)&s.t0[i];
    const double dt0 = ctl->dt_max > 0.0 ? i2d_scaled(T - t0.x, k) : 0.0;
    const double dt1 = ctl->dt_max > 0.0 ? i2d_scaled(T - t0.y, k) : 0.0;
    const double2 rx = *(const double2 *)&s.rx[i], ry = *(const double2 *)&s.ry[i], rz = *(const double2 *)&s.rz[i];
    const double2 vx = *(const double2 *)&s.vx[i], vy = *(const double2 *)&s.vy[i], vz = *(const double2 *)&s.vz[i];
    const float2 m = *(const float2 *)&s.mass[i];
    posm[i] = make_float4(d2f(__fma_rn(dt0, vx.x, rx.x)), d2f(__fma_rn(dt0, vy.x, ry.x)),
                          d2f(__fma_rn(dt0, vz.x, rz.x)), m.x);
    posm[i + 1] = make_float4(d2f(__fma_rn(dt1, vx.y, rx.y)), d2f(__fma_rn(dt1, vy.y, ry.y)),
                              d2f(__fma_rn(dt1, vz.y, rz.y)), m.y);
}

__global__ __launch_bounds__(256) void k_predict(State s, long long n, const DevCtl *__restrict__ ctl,
                                                 float4 *__restrict__ posm, int ahead) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    const long long T = (long long)(ahead ? ctl->tnext_acc : ctl->tnext);
    // dt = (T - t0) dt_min with dt_min = dt_max 2^-(L-1) a power of two: exact, so it is
    // built from the bits; only the three fused multiply-adds run on the FP64 pipe
    const int k = (int)((__double_as_longlong(ctl->dt_max) >> 52) & 0x7ff) - 1023 - ctl->levels_m1;
    const double dt = ctl->dt_max > 0.0 ? i2d_scaled(T - s.t0[i], k) : 0.0;
    const float x = d2f(__fma_rn(dt, s.vx[i], s.rx[i]));
    const float y = d2f(__fma_rn(dt, s.vy[i], s.ry[i]));
    const float z = d2f(__fma_rn(dt, s.vz[i], s.rz[i]));
    posm[i] = make_float4(x, y, z, s.mass[i]);
}

__global__ __launch_bounds__(256) void k_load(State s, long long n, float4 *__restrict__ posm) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    posm[i] = make_float4(d2f(s.rx[i]), d2f(s.ry[i]), d2f(s.rz[i]), s.mass[i]);
    s.id[i] = (uint32_t)i;
    s.t0[i] = 0;
    s.level[i] = 0;
    s.aold[i] = 0.0f;
    s.acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ __launch_bounds__(256) void k_permute(State src, State dst, const float4 *__restrict__ pin,
                                                 float4 *__restrict__ pout,
                                                 const uint32_t *__restrict__ perm, long long n) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = perm[i];
    dst.rx[i] = src.rx[k];
    dst.ry[i] = src.ry[k];
    dst.rz[i] = src.rz[k];
    dst.vx[i] = src.vx[k];
    dst.vy[i] = src.vy[k];
    dst.vz[i] = src.vz[k];
    dst.t0[i] = src.t0[k];
    dst.level[i] = src.level[k];
    dst.aold[i] = src.aold[k];
    dst.acc[i] = src.acc[k];
    dst.id[i] = src.id[k];
    dst.mass[i] = src.mass[k];
    pout[i] = pin[k];
}

// copy the permuted state back, so that buffer 0 always holds the current state
__global__ __launch_bounds__(256) void k_copy_state(State src, State dst, const float4 *__restrict__ pin,
                                                    float4 *__restrict__ pout, long long n) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    dst.rx[i] = src.rx[i];
    dst.ry[i] = src.ry[i];
    dst.rz[i] = src.rz[i];
    dst.vx[i] = src.vx[i];
    dst.vy[i] = src.vy[i];
    dst.vz[i] = src.vz[i];
    dst.t0[i] = src.t0[i];
    dst.level[i] = src.level[i];
    dst.aold[i] = src.aold[i];
    dst.acc[i] = src.acc[i];
    dst.id[i] = src.id[i];
    dst.mass[i] = src.mass[i];
    if (pin) pout[i] = pin[i];
}

// n x 3 row-major <-> three arrays
__global__ __launch_bounds__(256) void k_deinterleave3(const double *__restrict__ in, long long n,
                                                       double *__restrict__ x, double *__restrict__ y,
                                                       double *__restrict__ z) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    x[i] = in[3 * i];
    y[i] = in[3 * i + 1];
    z[i] = in[3 * i + 2];
}

__global__ __launch_bounds__(256) void k_interleave3(const double *__restrict__ x, const double *__restrict__ y,
                                                     const double *__restrict__ z, long long n,
                                                     double *__restrict__ out) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    out[3 * i] = x[i];
    out[3 * i + 1] = y[i];
    out[3 * i + 2] = z[i];
}

// state out in the caller's particle order: row id[i] of pos/vel (n x 3) <- slot i
__global__ __launch_bounds__(256) void k_state_out(State t, long long n, double *__restrict__ pos,
                                                   double *__restrict__ vel) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    const long long j = t.id[i];
    if (pos) {
        pos[3 * j] = t.rx[i];
        pos[3 * j + 1] = t.ry[i];
        pos[3 * j + 2] = t.rz[i];
    }
    if (vel) {
        vel[3 * j] = t.vx[i];
        vel[3 * j + 1] = t.vy[i];
        vel[3 * j + 2] = t.vz[i];
    }
}

__global__ __launch_bounds__(256) void k_gather_f(const float *__restrict__ in, const uint32_t *__restrict__ id,
                                                  long long n, float *__restrict__ out) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i < n) out[i] = in[id[i]];
}

// flags[active[k]] = 1 for a caller's list; a list that is not strictly increasing or
// holds an index >= n latches GT_EINVAL (the cell grouping needs key order)
__global__ __launch_bounds__(256) void k_scatter_flags(const uint32_t *__restrict__ active, long long na,
                                                       long long n, uint8_t *__restrict__ flags, DevCtl *ctl) {
    const long long k = blockIdx.x * 256ll + threadIdx.x;
    if (k >= na) return;
    const uint32_t i = active[k];
    if ((long long)i >= n || (k > 0 && active[k - 1] >= i)) {
        gt_set_error(ctl, GT_EINVAL, GTK_ACTIVE);
        return;
    }
    flags[i] = 1;
}

constexpr int AT = 256, AIPT = 16, ATILE = AT * AIPT;

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t < v ? t : v;
    }
    return v;
}

enum { CM_TIME = 0, CM_ALL = 1, CM_FLAGS = 2 };

// Order-preserving compaction of [0, n) (n from n_dev if given).  Writes the selected
// indices to out, the prefix P[i] = #selected below i (i = 0..n) if prefix != null,
// and the count to *count_out.  CM_TIME also folds the unselected particles' step
// ends into the next block time.
__global__ __launch_bounds__(AT) void k_compact(long long n_host, const unsigned int *n_dev, int mode,
                                                const long long *__restrict__ t0,
                                                const uint8_t *__restrict__ level, int L,
                                                const uint8_t *__restrict__ flags, DevCtl *ctl,
                                                int ticket, uint32_t tag_slot, uint32_t *__restrict__ out,
                                                uint32_t *__restrict__ prefix, unsigned int *count_out,
                                                unsigned long long *status) {
    __shared__ uint32_t tmp[AT / 32 + 1];
    __shared__ uint32_t tile_sh, excl_sh;
    const long long n = n_dev ? (long long)*n_dev : n_host;
    const unsigned long long T = ctl->tnext;
    const uint32_t tag = ctl->epoch * 32u + tag_slot;
    const uint32_t ntiles = (uint32_t)((n + ATILE - 1) / ATILE);
    unsigned long long tmin = ~0ull;
    if (n == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *count_out = 0;
            if (prefix) prefix[0] = 0;
        }
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) tile_sh = atomicAdd(&ctl->tile_ticket[ticket], 1u);
        __syncthreads();
        const uint32_t tile = tile_sh;
        __syncthreads();
        if (tile >= ntiles) break;
        // warp w owns items [wbase, wbase + 32 AIPT); row q is items wbase + 32 q + lane, so
        // every load and store of a row is one coalesced access, and rows then lanes
        // visit the items in index order (the compaction keeps it)
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const long long wbase = (long long)tile * ATILE + (long long)w * (32 * AIPT);
        unsigned int bal[AIPT];
        uint32_t wsel = 0;
#pragma unroll
        for (int q = 0; q < AIPT; q++) {
            const long long i = wbase + 32 * q + lane;
            bool on = false;
            if (i < n) {
                if (mode == CM_ALL) {
                    on = true;
                } else if (mode == CM_FLAGS) {
                    on = flags[i] != 0;
                } else {
                    const unsigned long long tend =
                        (unsigned long long)t0[i] + (1ull << (L - 1 - (int)level[i]));
                    on = tend == T;
                    if (!on) tmin = tend < tmin ? tend : tmin;
                }
            }
            bal[q] = __ballot_sync(0xffffffffu, on);
            wsel += (uint32_t)__popc(bal[q]);
        }
        // the warps' counts in order: one value per warp into the block scan
        uint32_t total;
        const uint32_t wexcl = block_excl_scan<AT>(lane == 31 ? wsel : 0u, &total, tmp);
        const uint32_t wstart = __shfl_sync(0xffffffffu, wexcl, 31);
        if (threadIdx.x < 32) {
            const uint32_t e = lookback_warp(status, tile, total, tag, ctl, GTK_ACTIVE);
            if (threadIdx.x == 0) excl_sh = e;
        }
        __syncthreads();
        uint32_t pos = excl_sh + wstart;
        const unsigned int lt = lanemask_lt();
#pragma unroll
        for (int q = 0; q < AIPT; q++) {
            const long long i = wbase + 32 * q + lane;
            const uint32_t at = pos + (uint32_t)__popc(bal[q] & lt);
            if (i < n && prefix) prefix[i] = at;
            if ((bal[q] >> lane) & 1u) out[at] = (uint32_t)i;
            pos += (uint32_t)__popc(bal[q]);
        }
        if (tile == ntiles - 1 && threadIdx.x == AT - 1) {
            *count_out = excl_sh + total;
            if (prefix) prefix[n] = excl_sh + total;
        }
    }
    if (mode == CM_TIME) {
        tmin = warp_min_u64(tmin);
        if (lane_id() == 0 && tmin != ~0ull) atomicMin(&ctl->tnext_acc, tmin);
    }
}

// Mark the first active position of every group (Sec. 2.4 reading: groups never
// straddle two tree cells).  A cell qualifies when it holds at most gmax actives and is
// a leaf or no wider than r_crit (b_J <= r_crit; r_crit <= 0: no radius limit).  Counts
// and radii only shrink from a cell to its children, so a group cell is a qualifying
// cell whose parent does not qualify (or the root), or a leaf under no qualifying cell;
// its actives are cut into runs of gmax.
__device__ __forceinline__ bool group_cell_ok(const Nodes &nd, const uint32_t *P, uint32_t c, int gmax,
                                              float r_crit) {
    const uint32_t f = nd.first[c];
    if (P[f + nd.count[c]] - P[f] > (uint32_t)gmax) return false;
    return nd.child[c] < 0 || r_crit <= 0.0f || nd.walk[c].x <= r_crit;
}

__global__ __launch_bounds__(256) void k_group_cells(Nodes nd, long long cap, const uint32_t *__restrict__ P,
                                                     int gmax, float r_crit, uint8_t *__restrict__ marks,
                                                     const DevCtl *ctl) {
    long long nn = ctl->level_start[GT_TREE_LEVELS];
    if (nn > cap) nn = cap;
    for (long long c = blockIdx.x * 256ll + threadIdx.x; c < nn; c += (long long)gridDim.x * 256) {
        const uint32_t f = nd.first[c];
        const uint32_t a0 = P[f], A = P[f + nd.count[c]] - a0;
        if (A == 0) continue;
        const int32_t p = nd.parent[c];
        if (p >= 0 && group_cell_ok(nd, P, (uint32_t)p, gmax, r_crit)) continue;  // inside a group cell
        if (nd.child[c] >= 0 && !group_cell_ok(nd, P, (uint32_t)c, gmax, r_crit)) continue;  // children decide
        for (uint32_t s = a0; s < a0 + A; s += (uint32_t)gmax) marks[s] = 1;
    }
}

__device__ __forceinline__ double a2_of(float4 a) {
    const double ax = f2d(a.x), ay = f2d(a.y), az = f2d(a.z);  // exact widenings, integer pipe
    // the squares are exact in FP64, so the fused forms round only at the additions
    return __fma_rn(az, az, __fma_rn(ay, ay, __dmul_rn(ax, ax)));
}

__device__ __forceinline__ long long floordiv4(long long d) { return d >= 0 ? d / 4 : -((-d + 3) / 4); }

__device__ __forceinline__ int level_from_a2(double a2, double c2, int M, int L) {
    if (!(a2 > 0.0) || !isfinite(a2)) return 0;
    int ea, ec;
    const double fa = frexp(a2, &ea), fc = frexp(c2, &ec);
    // level k qualifies iff 4k > D, or 4k == D and fa <= fc, with D = ea + 4M - ec
    const long long D = (long long)ea + 4ll * M - ec;
    const long long q = floordiv4(D);
    long long k = (4 * q == D && fa <= fc) ? q : q + 1;
    k = k < 0 ? 0 : k;
    k = k > L - 1 ? L - 1 : k;
    return (int)k;
}

__global__ __launch_bounds__(256) void k_correct(State s, const uint32_t *__restrict__ active,
                                                 const float4 *__restrict__ acc, DevCtl *ctl, long long n,
                                                 int L, double c2) {
    const uint32_t na = ctl->n_active;
    const long long T = (long long)ctl->tnext;
    const int M = ctl->M;  // dt_max = 2^M
    // the step's powers of two and the exact widenings are built on the integer pipe (the
    // FP64 pipe of this GPU is narrow); only the kicks, drifts and |a|^2 use it
    auto p2 = [](int e) {  // 2^e
        return (e > -1023 && e < 1024) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
    };
    unsigned long long tmin = ~0ull;
    for (uint32_t k = blockIdx.x * 256u + threadIdx.x; k < na; k += gridDim.x * 256u) {
        const uint32_t i = active[k];
        if ((long long)i >= n) {  // an index outside the system: report it and skip
            gt_set_error(ctl, GT_EINVAL, GTK_CORRECT);
            continue;
        }
        const float4 a = acc[k];
        const int kold = s.level[i];
        const double hold = p2(M - kold - 1);                  // dt(kold) / 2
        const double dtp = i2d_scaled(T - s.t0[i], M - (L - 1));  // (T - t0) dt_min, exact
        const double ax = f2d(a.x), ay = f2d(a.y), az = f2d(a.z);
        const double vx0 = s.vx[i], vy0 = s.vy[i], vz0 = s.vz[i];
        s.rx[i] = __fma_rn(dtp, vx0, s.rx[i]);
        s.ry[i] = __fma_rn(dtp, vy0, s.ry[i]);
        s.rz[i] = __fma_rn(dtp, vz0, s.rz[i]);
        const double vx = __fma_rn(hold, ax, vx0);
        const double vy = __fma_rn(hold, ay, vy0);
        const double vz = __fma_rn(hold, az, vz0);
        const double a2 = a2_of(a);
        const int kc = level_from_a2(a2, c2, M, L);
        int knew = kold;
        if (kc > kold) {
            knew = kc;
        } else if (kc < kold) {
            const long long span = 1ll << (L - 1 - (kold - 1));
            if (T % span == 0) knew = kold - 1;
        }
        const double hnew = p2(M - knew - 1);
        s.vx[i] = __fma_rn(hnew, ax, vx);
        s.vy[i] = __fma_rn(hnew, ay, vy);
        s.vz[i] = __fma_rn(hnew, az, vz);
        s.level[i] = (uint8_t)knew;
        s.t0[i] = T;
        s.aold[i] = __fsqrt_rn(d2f(a2));
        s.acc[i] = a;
        const unsigned long long tend = (unsigned long long)T + (1ull << (L - 1 - knew));
        tmin = tend < tmin ? tend : tmin;
    }
    tmin = warp_min_u64(tmin);
    if (lane_id() == 0 && tmin != ~0ull) atomicMin(&ctl->tnext_acc, tmin);
}

__global__ __launch_bounds__(256) void k_aold(const float4 *__restrict__ acc, long long n,
                                              float *__restrict__ aold) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i < n) aold[i] = __fsqrt_rn(__double2float_rn(a2_of(acc[i])));
}

// start, phase 1: the smallest positive A2 (bit pattern of a positive double)
__global__ __launch_bounds__(256) void k_min_a2(const float4 *__restrict__ acc, long long n, DevCtl *ctl) {
    unsigned long long best = ~0ull;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const double a2 = a2_of(acc[i]);
        if (!(a2 > 0.0) || !isfinite(a2)) continue;
        const unsigned long long b = (unsigned long long)__double_as_longlong(a2);
        best = b < best ? b : best;
    }
    best = warp_min_u64(best);
    if (lane_id() == 0 && best != ~0ull) atomicMin(&ctl->max_dt_bits, best);
}

// start, phase 2: dt_max (the largest 2^M with 2^(4M) A2min <= c2), levels, t0 = 0,
// first half kick v^{1/2} = fma(dt/2, a, v)
__global__ __launch_bounds__(256) void k_init_levels(State s, const float4 *__restrict__ acc, long long n,
                                                     int L, double c2, int M_given, int have_M, DevCtl *ctl) {
    int M = M_given;
    if (!have_M) {
        M = 0;
        if (ctl->max_dt_bits != ~0ull) {
            const double a2min = __longlong_as_double((long long)ctl->max_dt_bits);
            int ea, ec;
            const double fa = frexp(a2min, &ea), fc = frexp(c2, &ec);
            const long long D = (long long)ec - ea;  // M qualifies iff 4M < D, or 4M == D and fa <= fc
            const long long q = floordiv4(D);
            M = (int)(4 * q == D ? (fa <= fc ? q : q - 1) : q);
        }
    }
    const double dt_max = ldexp(1.0, M);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->M = M;
        ctl->dt_max = dt_max;
        ctl->levels_m1 = L - 1;
    }
    unsigned long long tmin = ~0ull;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float4 a = acc[i];
        const double a2 = a2_of(a);
        const int k = level_from_a2(a2, c2, M, L);
        const double h = 0.5 * ldexp(dt_max, -k);
        s.vx[i] = __fma_rn(h, (double)a.x, s.vx[i]);
        s.vy[i] = __fma_rn(h, (double)a.y, s.vy[i]);
        s.vz[i] = __fma_rn(h, (double)a.z, s.vz[i]);
        s.level[i] = (uint8_t)k;
        s.t0[i] = 0;
        s.aold[i] = __fsqrt_rn(__double2float_rn(a2));
        s.acc[i] = a;
        const unsigned long long tend = 1ull << (L - 1 - k);
        tmin = tend < tmin ? tend : tmin;
    }
    tmin = warp_min_u64(tmin);
    if (lane_id() == 0 && tmin != ~0ull) atomicMin(&ctl->tnext_acc, tmin);
}

// resume: scalars of the integration and the next block time over all particles
__global__ void k_set_clock(DevCtl *ctl, int M, int L, long long T) {
    ctl->M = M;
    ctl->dt_max = ldexp(1.0, M);
    ctl->levels_m1 = L - 1;
    ctl->tnext = (unsigned long long)T;
    ctl->tnext_acc = ~0ull;
}

__global__ void k_set_tnext(DevCtl *ctl, long long T) { ctl->tnext = (unsigned long long)T; }

__global__ void k_set_u32(unsigned int *dst, unsigned int v) { *dst = v; }

__global__ __launch_bounds__(256) void k_tnext_all(const long long *__restrict__ t0,
                                                   const uint8_t *__restrict__ level, long long n, int L,
                                                   DevCtl *ctl) {
    unsigned long long tmin = ~0ull;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const unsigned long long tend = (unsigned long long)t0[i] + (1ull << (L - 1 - (int)level[i]));
        tmin = tend < tmin ? tend : tmin;
    }
    tmin = warp_min_u64(tmin);
    if (lane_id() == 0 && tmin != ~0ull) atomicMin(&ctl->tnext_acc, tmin);
}

__global__ __launch_bounds__(256) void k_gather_resume(const uint8_t *__restrict__ lv, const long long *__restrict__ t0,
                                                       const float *__restrict__ ao, const float4 *__restrict__ acc,
                                                       const uint32_t *__restrict__ id, long long n, State s) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = id[i];
    s.level[i] = lv[k];
    s.t0[i] = t0[k];
    s.aold[i] = ao[k];
    s.acc[i] = acc ? acc[k] : make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_reset_start(DevCtl *ctl) {
    ctl->max_dt_bits = ~0ull;
    ctl->tnext_acc = ~0ull;
    ctl->tnext = 0;
}

inline unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void gt_launch_prepare(DevCtl *ctl, int begin_step, cudaStream_t st) {
    { k_prepare<<<1, 1, 0, st>>>(ctl, begin_step); gt_note_launches(1); }
}

void gt_launch_set_nactive(DevCtl *ctl, unsigned int n_active, cudaStream_t st) {
    { k_set_nactive<<<1, 1, 0, st>>>(ctl, n_active); gt_note_launches(1); }
}

void gt_launch_predict(const State &s, int64_t n, const DevCtl *ctl, float4 *posm, cudaStream_t st, bool ahead) {
    if (n <= 0) return;
    const bool aligned = ((uintptr_t)s.rx | (uintptr_t)s.ry | (uintptr_t)s.rz | (uintptr_t)s.vx | (uintptr_t)s.vy |
                          (uintptr_t)s.vz | (uintptr_t)s.t0 | (uintptr_t)s.mass) % 16 == 0;
    if (n % 2 == 0 && aligned) k_predict2<<<nblk(n / 2), 256, 0, st>>>(s, n, ctl, posm, ahead ? 1 : 0);
    else k_predict<<<nblk(n), 256, 0, st>>>(s, n, ctl, posm, ahead ? 1 : 0);
    gt_note_launches(1);
}

void gt_launch_mirror(const DevCtl *ctl, StepMirror *dst, cudaStream_t st) {
    { k_mirror<<<1, 1, 0, st>>>(ctl, dst); gt_note_launches(1); }
}

void gt_launch_load(const State &s, float4 *posm, int64_t n, cudaStream_t st) {
    if (n > 0) { k_load<<<nblk(n), 256, 0, st>>>(s, n, posm); gt_note_launches(1); }
}

void gt_launch_permute(const State &src, const State &dst, const float4 *posm_in, float4 *posm_out,
                       const uint32_t *perm, int64_t n, cudaStream_t st) {
    if (n > 0) { k_permute<<<nblk(n), 256, 0, st>>>(src, dst, posm_in, posm_out, perm, n); gt_note_launches(1); }
}

void gt_launch_copy_state(const State &src, const State &dst, const float4 *posm_in, float4 *posm_out,
                          int64_t n, cudaStream_t st) {
    if (n > 0) { k_copy_state<<<nblk(n), 256, 0, st>>>(src, dst, posm_in, posm_out, n); gt_note_launches(1); }
}

void gt_launch_deinterleave3(const double *in, int64_t n, double *x, double *y, double *z,
                             cudaStream_t st) {
    if (n > 0) { k_deinterleave3<<<nblk(n), 256, 0, st>>>(in, n, x, y, z); gt_note_launches(1); }
}

void gt_launch_interleave3(const double *x, const double *y, const double *z, int64_t n, double *out,
                           cudaStream_t st) {
    if (n > 0) { k_interleave3<<<nblk(n), 256, 0, st>>>(x, y, z, n, out); gt_note_launches(1); }
}

void gt_launch_state_out(const State &t, int64_t n, double *pos, double *vel, cudaStream_t st) {
    if (n > 0) { k_state_out<<<nblk(n), 256, 0, st>>>(t, n, pos, vel); gt_note_launches(1); }
}

void gt_launch_gather_f(const float *in, const uint32_t *id, int64_t n, float *out, cudaStream_t st) {
    if (n > 0) { k_gather_f<<<nblk(n), 256, 0, st>>>(in, id, n, out); gt_note_launches(1); }
}

void gt_launch_active(const State &s, int64_t n, int L, int all, DevCtl *ctl, uint32_t *active,
                      uint32_t *prefix, unsigned long long *status, int nsm, cudaStream_t st) {
    { k_compact<<<nsm * 4, AT, 0, st>>>(n, nullptr, all ? CM_ALL : CM_TIME, s.t0, s.level, L, nullptr, ctl,
                                        GT_TREE_LEVELS, 30u, active, prefix, &ctl->n_active, status);
      gt_note_launches(1); }
}

void gt_launch_active_from_list(const uint32_t *list, int64_t n_list, int64_t n, uint8_t *flags, DevCtl *ctl,
                                uint32_t *active, uint32_t *prefix, unsigned long long *status, int nsm,
                                cudaStream_t st) {
    if (n > 0) cudaMemsetAsync(flags, 0, (size_t)n, st);
    if (n_list > 0) { k_scatter_flags<<<nblk(n_list), 256, 0, st>>>(list, n_list, n, flags, ctl); gt_note_launches(1); }
    { k_compact<<<nsm * 4, AT, 0, st>>>(n, nullptr, CM_FLAGS, nullptr, nullptr, 0, flags, ctl, GT_TREE_LEVELS,
                                        30u, active, prefix, &ctl->n_active, status);
      gt_note_launches(1); }
}

void gt_launch_groups(Nodes nd, int64_t cap, const uint32_t *prefix, int gmax, float r_crit, int64_t n,
                      uint8_t *marks, DevCtl *ctl, uint32_t *gstart, unsigned long long *status, int nsm,
                      cudaStream_t st) {
    if (n > 0) cudaMemsetAsync(marks, 0, (size_t)n, st);
    { k_group_cells<<<nsm * 8, 256, 0, st>>>(nd, cap, prefix, gmax, r_crit, marks, ctl); gt_note_launches(1); }
    { k_compact<<<nsm * 4, AT, 0, st>>>(0, &ctl->n_active, CM_FLAGS, nullptr, nullptr, 0, marks, ctl,
                                        GT_TREE_LEVELS + 1, 31u, gstart, nullptr, &ctl->n_groups, status);
      gt_note_launches(1); }
}

void gt_launch_correct(const State &s, const uint32_t *active, const float4 *acc, DevCtl *ctl,
                       int64_t n, int L, double c2, int nsm, cudaStream_t st) {
    if (n > 0) { k_correct<<<nsm * 8, 256, 0, st>>>(s, active, acc, ctl, n, L, c2); gt_note_launches(1); }
}

void gt_launch_aold(const float4 *acc, int64_t n, float *aold, cudaStream_t st) {
    if (n > 0) { k_aold<<<nblk(n), 256, 0, st>>>(acc, n, aold); gt_note_launches(1); }
}

void gt_launch_set_clock(DevCtl *ctl, int M, int L, long long T, cudaStream_t st) {
    { k_set_clock<<<1, 1, 0, st>>>(ctl, M, L, T); gt_note_launches(1); }
}

void gt_launch_set_tnext(DevCtl *ctl, long long T, cudaStream_t st) {
    { k_set_tnext<<<1, 1, 0, st>>>(ctl, T); gt_note_launches(1); }
}

void gt_launch_set_u32(unsigned int *dst, unsigned int v, cudaStream_t st) {
    { k_set_u32<<<1, 1, 0, st>>>(dst, v); gt_note_launches(1); }
}

void gt_launch_tnext_all(const State &s, int64_t n, int L, DevCtl *ctl, int nsm, cudaStream_t st) {
    if (n > 0) { k_tnext_all<<<nsm * 4, 256, 0, st>>>(s.t0, s.level, n, L, ctl); gt_note_launches(1); }
}

void gt_launch_gather_resume(const uint8_t *lv, const long long *t0, const float *ao, const float4 *acc,
                             const State &s, int64_t n, cudaStream_t st) {
    if (n > 0) { k_gather_resume<<<nblk(n), 256, 0, st>>>(lv, t0, ao, acc, s.id, n, s); gt_note_launches(1); }
}

void gt_launch_init_levels(const State &s, const float4 *acc, int64_t n, int L, double c2, int M_given,
                           int have_M, DevCtl *ctl, int nsm, cudaStream_t st) {
    { k_reset_start<<<1, 1, 0, st>>>(ctl); gt_note_launches(1); }
    if (!have_M && n > 0) { k_min_a2<<<nsm * 4, 256, 0, st>>>(acc, n, ctl); gt_note_launches(1); }
    { k_init_levels<<<nsm * 8, 256, 0, st>>>(s, acc, n, L, c2, M_given, have_M, ctl); gt_note_launches(1); }
}
