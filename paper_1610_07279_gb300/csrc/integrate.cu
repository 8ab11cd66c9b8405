// Block time step (Sec. 1; Sec. 2.7, Eqs. 15-17) and the particle-array plumbing:
//   k_prepare      per-phase bookkeeping (epoch, tickets, the step's block time)
//   k_predict      A8: r(T) = r0 + ((T - t0) dt_min) v^{1/2} for every particle, FP64,
//                  rounded to FP32 for the tree                    (HBM: 60 B read, 16 B written)
//   k_permute      A3: gather every particle array into key order  (HBM: ~100 B each way)
//   k_active       A6: active = (t0 + ticks(level) == T), compacted in key order with a
//                  block scan and a bounded decoupled look-back; the inactive particles'
//                  next step ends are folded into the next block time (HBM: 9 B + 4 B/active)
//   k_correct      A9: Eq. (17), the new level, the next half kick; the active particles'
//                  new step ends are folded into the next block time
//   k_init_levels  start: dt_max, levels and the first half kick
// Level of a particle: the smallest k with dt_max 2^-k <= dt_i = sqrt(2 eta eps / |a|),
// clamped to [0, L-1]; with dt_i = f 2^e (f in [0.5, 1)) this is k = M - e + 1 where
// dt_max = 2^M.  A shorter step is taken at once; a longer one only by one level and
// only when T is a multiple of the longer step.  Every FP64 operation is written with
// an explicit rounding intrinsic (no contraction), so results are reproducible bit for bit.
#include "gt_internal.cuh"

namespace {

__global__ void k_prepare(DevCtl *ctl, int begin_step) {
    ctl->epoch += 1u;
    for (int l = 0; l < GT_TREE_LEVELS + 2; l++) ctl->tile_ticket[l] = 0;
    ctl->group_next = 0;
    if (begin_step) {
        ctl->tnext = ctl->tnext_acc;
        ctl->tnext_acc = ~0ull;
    }
}

__global__ void k_set_nactive(DevCtl *ctl, unsigned int n_active) { ctl->n_active = n_active; }

__global__ __launch_bounds__(256) void k_predict(State s, long long n, const DevCtl *__restrict__ ctl,
                                                 float4 *__restrict__ posm) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    const long long T = (long long)ctl->tnext;
    const double dt_min = ldexp(ctl->dt_max, -ctl->levels_m1);
    const double dt = __dmul_rn((double)(T - s.t0[i]), dt_min);
    const float x = __double2float_rn(__dadd_rn(s.rx[i], __dmul_rn(dt, s.vx[i])));
    const float y = __double2float_rn(__dadd_rn(s.ry[i], __dmul_rn(dt, s.vy[i])));
    const float z = __double2float_rn(__dadd_rn(s.rz[i], __dmul_rn(dt, s.vz[i])));
    posm[i] = make_float4(x, y, z, s.mass[i]);
}

__global__ __launch_bounds__(256) void k_load(State s, long long n, float4 *__restrict__ posm) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    posm[i] = make_float4(__double2float_rn(s.rx[i]), __double2float_rn(s.ry[i]),
                          __double2float_rn(s.rz[i]), s.mass[i]);
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

__global__ __launch_bounds__(256) void k_gather_f(const float *__restrict__ in, const uint32_t *__restrict__ id,
                                                  long long n, float *__restrict__ out) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i < n) out[i] = in[id[i]];
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

__global__ __launch_bounds__(AT) void k_active(long long n, const long long *__restrict__ t0,
                                               const uint8_t *__restrict__ level, int L, int all,
                                               DevCtl *ctl, uint32_t *__restrict__ active,
                                               unsigned long long *status) {
    __shared__ uint32_t tmp[AT / 32 + 1];
    __shared__ uint32_t tile_sh, excl_sh;
    const unsigned long long T = ctl->tnext;
    const uint32_t tag = ctl->epoch * 32u + 30u;
    const uint32_t ntiles = (uint32_t)((n + ATILE - 1) / ATILE);
    unsigned long long tmin = ~0ull;
    for (;;) {
        if (threadIdx.x == 0) tile_sh = atomicAdd(&ctl->tile_ticket[GT_TREE_LEVELS], 1u);
        __syncthreads();
        const uint32_t tile = tile_sh;
        __syncthreads();
        if (tile >= ntiles) break;
        const long long i0 = (long long)tile * ATILE + threadIdx.x * AIPT;
        uint32_t flags = 0;
#pragma unroll
        for (int q = 0; q < AIPT; q++) {
            const long long i = i0 + q;
            if (i < n) {
                if (all) {
                    flags |= 1u << q;
                } else {
                    const unsigned long long tend =
                        (unsigned long long)t0[i] + (1ull << (L - 1 - (int)level[i]));
                    if (tend == T) flags |= 1u << q;
                    else tmin = tend < tmin ? tend : tmin;
                }
            }
        }
        uint32_t total;
        const uint32_t excl = block_excl_scan<AT>((uint32_t)__popc(flags), &total, tmp);
        if (threadIdx.x == 0) excl_sh = lookback_prefix(status, tile, total, tag, ctl, GTK_ACTIVE);
        __syncthreads();
        uint32_t pos = excl_sh + excl;
#pragma unroll
        for (int q = 0; q < AIPT; q++)
            if (flags & (1u << q)) active[pos++] = (uint32_t)(i0 + q);
        if (tile == ntiles - 1 && threadIdx.x == AT - 1) ctl->n_active = excl_sh + total;
    }
    if (!all) {
        tmin = warp_min_u64(tmin);
        if (lane_id() == 0 && tmin != ~0ull) atomicMin(&ctl->tnext_acc, tmin);
    }
}

__device__ __forceinline__ double amag3(float4 a) {
    const double ax = a.x, ay = a.y, az = a.z;
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az)));
}

__device__ __forceinline__ double dt_crit(double am, double eta, double eps) {
    return __dsqrt_rn(__ddiv_rn(__dmul_rn(__dmul_rn(2.0, eta), eps), am));
}

__device__ __forceinline__ int level_from_amag(double am, double eta, double eps, int M, int L) {
    if (!(am > 0.0) || !isfinite(am)) return 0;
    const double dti = dt_crit(am, eta, eps);
    if (!isfinite(dti)) return 0;
    int e;
    (void)frexp(dti, &e);
    int k = M - e + 1;
    k = k < 0 ? 0 : k;
    k = k > L - 1 ? L - 1 : k;
    return k;
}

__global__ __launch_bounds__(256) void k_correct(State s, const uint32_t *__restrict__ active,
                                                 const float4 *__restrict__ acc, DevCtl *ctl, long long n,
                                                 int L, double eta, double eps) {
    const uint32_t na = ctl->n_active;
    const long long T = (long long)ctl->tnext;
    const double dt_max = ctl->dt_max;
    const int M = ctl->M;
    const double dt_min = ldexp(dt_max, -(L - 1));
    unsigned long long tmin = ~0ull;
    for (uint32_t k = blockIdx.x * 256u + threadIdx.x; k < na; k += gridDim.x * 256u) {
        const uint32_t i = active[k];
        if ((long long)i >= n) {  // an index outside the system: report it and skip
            gt_set_error(ctl, GT_EINVAL, GTK_CORRECT);
            continue;
        }
        const float4 a = acc[k];
        const int kold = s.level[i];
        const double hold = __dmul_rn(0.5, ldexp(dt_max, -kold));
        const double dtp = __dmul_rn((double)(T - s.t0[i]), dt_min);
        const double ax = a.x, ay = a.y, az = a.z;
        const double vx = __dadd_rn(s.vx[i], __dmul_rn(hold, ax));
        const double vy = __dadd_rn(s.vy[i], __dmul_rn(hold, ay));
        const double vz = __dadd_rn(s.vz[i], __dmul_rn(hold, az));
        s.rx[i] = __dadd_rn(s.rx[i], __dmul_rn(dtp, s.vx[i]));
        s.ry[i] = __dadd_rn(s.ry[i], __dmul_rn(dtp, s.vy[i]));
        s.rz[i] = __dadd_rn(s.rz[i], __dmul_rn(dtp, s.vz[i]));
        const double am = amag3(a);
        const int kc = level_from_amag(am, eta, eps, M, L);
        int knew = kold;
        if (kc > kold) {
            knew = kc;
        } else if (kc < kold) {
            const long long span = 1ll << (L - 1 - (kold - 1));
            if (T % span == 0) knew = kold - 1;
        }
        const double hnew = __dmul_rn(0.5, ldexp(dt_max, -knew));
        s.vx[i] = __dadd_rn(vx, __dmul_rn(hnew, ax));
        s.vy[i] = __dadd_rn(vy, __dmul_rn(hnew, ay));
        s.vz[i] = __dadd_rn(vz, __dmul_rn(hnew, az));
        s.level[i] = (uint8_t)knew;
        s.t0[i] = T;
        s.aold[i] = __double2float_rn(am);
        s.acc[i] = a;
        const unsigned long long tend = (unsigned long long)T + (1ull << (L - 1 - knew));
        tmin = tend < tmin ? tend : tmin;
    }
    tmin = warp_min_u64(tmin);
    if (lane_id() == 0 && tmin != ~0ull) atomicMin(&ctl->tnext_acc, tmin);
}

__global__ __launch_bounds__(256) void k_amag(const float4 *__restrict__ acc, long long n,
                                              float *__restrict__ aold) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i < n) aold[i] = __double2float_rn(amag3(acc[i]));
}

// start, phase 1: the largest dt_i over all particles (bit pattern of a positive double)
__global__ __launch_bounds__(256) void k_max_dt(const float4 *__restrict__ acc, long long n, double eta,
                                                double eps, DevCtl *ctl) {
    unsigned long long best = 0;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const double am = amag3(acc[i]);
        if (!(am > 0.0)) continue;
        const unsigned long long b = (unsigned long long)__double_as_longlong(dt_crit(am, eta, eps));
        best = b > best ? b : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
        best = t > best ? t : best;
    }
    if (lane_id() == 0 && best) atomicMax(&ctl->max_dt_bits, best);
}

// start, phase 2: dt_max, levels, t0 = 0, first half kick v^{1/2} = v + (dt/2) a
__global__ __launch_bounds__(256) void k_init_levels(State s, const float4 *__restrict__ acc, long long n,
                                                     int L, double eta, double eps, int M_given,
                                                     int have_M, DevCtl *ctl) {
    int M = M_given;
    if (!have_M) {
        const double best = __longlong_as_double((long long)ctl->max_dt_bits);
        M = 0;
        if (best > 0.0 && isfinite(best)) {
            int e;
            (void)frexp(best, &e);
            M = e - 1;
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
        const double am = amag3(a);
        const int k = level_from_amag(am, eta, eps, M, L);
        const double h = __dmul_rn(0.5, ldexp(dt_max, -k));
        s.vx[i] = __dadd_rn(s.vx[i], __dmul_rn(h, (double)a.x));
        s.vy[i] = __dadd_rn(s.vy[i], __dmul_rn(h, (double)a.y));
        s.vz[i] = __dadd_rn(s.vz[i], __dmul_rn(h, (double)a.z));
        s.level[i] = (uint8_t)k;
        s.t0[i] = 0;
        s.aold[i] = __double2float_rn(am);
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
    ctl->max_dt_bits = 0;
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

void gt_launch_predict(const State &s, int64_t n, const DevCtl *ctl, float4 *posm, cudaStream_t st) {
    if (n > 0) { k_predict<<<nblk(n), 256, 0, st>>>(s, n, ctl, posm); gt_note_launches(1); }
}

void gt_launch_load(const State &s, float4 *posm, int64_t n, cudaStream_t st) {
    if (n > 0) { k_load<<<nblk(n), 256, 0, st>>>(s, n, posm); gt_note_launches(1); }
}

void gt_launch_permute(const State &src, const State &dst, const float4 *posm_in, float4 *posm_out,
                       const uint32_t *perm, int64_t n, cudaStream_t st) {
    if (n > 0) { k_permute<<<nblk(n), 256, 0, st>>>(src, dst, posm_in, posm_out, perm, n); gt_note_launches(1); }
}

void gt_launch_deinterleave3(const double *in, int64_t n, double *x, double *y, double *z,
                             cudaStream_t st) {
    if (n > 0) { k_deinterleave3<<<nblk(n), 256, 0, st>>>(in, n, x, y, z); gt_note_launches(1); }
}

void gt_launch_interleave3(const double *x, const double *y, const double *z, int64_t n, double *out,
                           cudaStream_t st) {
    if (n > 0) { k_interleave3<<<nblk(n), 256, 0, st>>>(x, y, z, n, out); gt_note_launches(1); }
}

void gt_launch_gather_f(const float *in, const uint32_t *id, int64_t n, float *out, cudaStream_t st) {
    if (n > 0) { k_gather_f<<<nblk(n), 256, 0, st>>>(in, id, n, out); gt_note_launches(1); }
}

void gt_launch_active(const State &s, int64_t n, int L, int all, DevCtl *ctl, uint32_t *active,
                      unsigned long long *status, int nsm, cudaStream_t st) {
    if (n <= 0) {
        { k_set_nactive<<<1, 1, 0, st>>>(ctl, 0u); gt_note_launches(1); }
        return;
    }
    { k_active<<<nsm * 4, AT, 0, st>>>(n, s.t0, s.level, L, all, ctl, active, status); gt_note_launches(1); }
}

void gt_launch_correct(const State &s, const uint32_t *active, const float4 *acc, DevCtl *ctl,
                       int64_t n, int L, double eta, double eps, int nsm, cudaStream_t st) {
    if (n > 0) { k_correct<<<nsm * 8, 256, 0, st>>>(s, active, acc, ctl, n, L, eta, eps); gt_note_launches(1); }
}

void gt_launch_amag(const float4 *acc, int64_t n, float *aold, cudaStream_t st) {
    if (n > 0) { k_amag<<<nblk(n), 256, 0, st>>>(acc, n, aold); gt_note_launches(1); }
}

void gt_launch_set_clock(DevCtl *ctl, int M, int L, long long T, cudaStream_t st) {
    { k_set_clock<<<1, 1, 0, st>>>(ctl, M, L, T); gt_note_launches(1); }
}

void gt_launch_set_tnext(DevCtl *ctl, long long T, cudaStream_t st) { { k_set_tnext<<<1, 1, 0, st>>>(ctl, T); gt_note_launches(1); } }

void gt_launch_tnext_all(const State &s, int64_t n, int L, DevCtl *ctl, int nsm, cudaStream_t st) {
    if (n > 0) { k_tnext_all<<<nsm * 4, 256, 0, st>>>(s.t0, s.level, n, L, ctl); gt_note_launches(1); }
}

void gt_launch_gather_resume(const uint8_t *lv, const long long *t0, const float *ao, const float4 *acc,
                             const State &s, int64_t n, cudaStream_t st) {
    if (n > 0) { k_gather_resume<<<nblk(n), 256, 0, st>>>(lv, t0, ao, acc, s.id, n, s); gt_note_launches(1); }
}

void gt_launch_init_levels(const State &s, const float4 *acc, int64_t n, int L, double eta,
                           double eps, int M_given, int have_M, DevCtl *ctl, int nsm,
                           cudaStream_t st) {
    { k_reset_start<<<1, 1, 0, st>>>(ctl); gt_note_launches(1); }
    if (!have_M && n > 0) { k_max_dt<<<nsm * 4, 256, 0, st>>>(acc, n, eta, eps, ctl); gt_note_launches(1); }
    { k_init_levels<<<nsm * 8, 256, 0, st>>>(s, acc, n, L, eta, eps, M_given, have_M, ctl); gt_note_launches(1); }
}
