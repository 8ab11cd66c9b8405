// Steps A4-A5: breadth-first octree over the sorted keys and the pseudo
// j-particles (Sec. 2.1, Fig. 1).
//
// A4, one kernel per level (Sec. 2.1: cells are examined in parallel and their
// children numbered serially with prefix sums).  A cell at level l with more than
// leaf_max particles (and l < 21) splits into the non-empty ranges of the digit
// (key >> 3(20 - l)) & 7 -- the "seven partitions" of its key range, found by a
// lock-step 7-way binary search.  Children get consecutive numbers after the level,
// in the order of their parents and digits, via a block scan plus a decoupled
// look-back over tiles taken in ticket order (bounded wait).  Numbering is thus
// level by level and, inside a level, by first particle.
//
// A5: one lane per leaf sums its particles in FP64 (mass, m x, m y, m z), then one
// pass per level, deepest first, over the cells with children (a list compacted at
// build time) sums the children's FP64 sums in child order -- every FP64 instruction
// runs with full warps, which matters on this GPU's narrow FP64 pipe.  m_J = (float)M and
// r_J = (float)S / (float)M (a cell of one particle is that particle); b_J is the
// largest FP32 |r - r_J| of a leaf's particles, or the largest |r_c - r_J| + b_c
// over a cell's children, widened by (1 + 2^-20) so that FP32 rounding cannot
// shrink it below the true enclosing radius.  FP64 is kept to the four sums (FP64
// throughput is low on this GPU).  Every operation carries an explicit rounding,
// so the result is the same bit for bit on every run.
#include "gt_internal.cuh"

namespace {

constexpr int BT = 256;         // threads per build block
constexpr int NPT = 1;          // cells per thread
constexpr int BTILE = BT * NPT; // cells per tile

__global__ void k_build_init(long long n, Nodes nd, DevCtl *ctl) {
    // root = level 0, all particles; level_start[0..1]
    ctl->level_start[0] = 0;
    ctl->level_start[1] = n > 0 ? 1u : 0u;
    if (n > 0) {
        nd.first[0] = 0;
        nd.count[0] = (uint32_t)n;
        nd.parent[0] = -1;
    }
}

__global__ __launch_bounds__(BT) void k_build_level(int lvl, const unsigned long long *__restrict__ skey,
                                                    int leaf_max, Nodes nd, long long cap,
                                                    unsigned long long *status, DevCtl *ctl) {
    __shared__ uint32_t tmp[BT / 32 + 1];
    __shared__ uint32_t tile_sh, excl_sh;
    const uint32_t lo = ctl->level_start[lvl], hi = ctl->level_start[lvl + 1];
    const uint32_t cnt = hi - lo;
    if (cnt == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->level_start[lvl + 2] = hi;
        return;
    }
    const uint32_t ntiles = (cnt + BTILE - 1) / BTILE;
    const uint32_t tag = ctl->epoch * 32u + (uint32_t)lvl;
    const bool can_split = lvl < GT_KEY_LEVELS;
    const int shift = 3 * (GT_KEY_LEVELS - 1 - lvl);
    for (;;) {
        if (threadIdx.x == 0) tile_sh = atomicAdd(&ctl->tile_ticket[lvl], 1u);
        __syncthreads();
        const uint32_t tile = tile_sh;
        __syncthreads();
        if (tile >= ntiles) break;
        uint32_t bnd[NPT][9];
        uint32_t nc[NPT];
        uint32_t tsum = 0;
#pragma unroll
        for (int q = 0; q < NPT; q++) {
            const uint32_t c = lo + tile * BTILE + threadIdx.x * NPT + q;
            nc[q] = 0;
            if (c < hi) {
                const uint32_t f = nd.first[c], k = nd.count[c];
                if (can_split && k > (uint32_t)leaf_max) {
                    // smallest p in [f, f+k) with digit(p) >= d, for d = 1..7, in lock step
                    uint32_t l7[7], h7[7];
#pragma unroll
                    for (int d = 0; d < 7; d++) { l7[d] = f; h7[d] = f + k; }
                    const int iters = 32 - __clz(k);
                    for (int it = 0; it < iters; it++) {
#pragma unroll
                        for (int d = 0; d < 7; d++) {
                            if (l7[d] < h7[d]) {
                                const uint32_t mid = (l7[d] + h7[d]) >> 1;
                                const uint32_t dig = (uint32_t)((__ldg(&skey[mid]) >> shift) & 7ull);
                                if (dig < (uint32_t)(d + 1)) l7[d] = mid + 1; else h7[d] = mid;
                            }
                        }
                    }
                    bnd[q][0] = f;
#pragma unroll
                    for (int d = 0; d < 7; d++) bnd[q][d + 1] = l7[d];
                    bnd[q][8] = f + k;
#pragma unroll
                    for (int d = 0; d < 8; d++) nc[q] += bnd[q][d + 1] > bnd[q][d] ? 1u : 0u;
                }
            }
            tsum += nc[q];
        }
        uint32_t total;
        uint32_t excl = block_excl_scan<BT>(tsum, &total, tmp);
        if (threadIdx.x < 32) {
            const uint32_t e = lookback_warp(status, tile, total, tag, ctl, GTK_BUILD);
            if (threadIdx.x == 0) excl_sh = e;
        }
        __syncthreads();
        uint32_t next = hi + excl_sh + excl;  // node id of this thread's first child
#pragma unroll
        for (int q = 0; q < NPT; q++) {
            const uint32_t c = lo + tile * BTILE + threadIdx.x * NPT + q;
            if (c >= hi) continue;
            if (nc[q] == 0) {  // a leaf
                nd.child[c] = -1;
                nd.nchild[c] = 0;
                continue;
            }
            if ((long long)next + nc[q] > cap) {
                gt_set_error(ctl, GT_EOVERFLOW, GTK_BUILD);
                nd.child[c] = -1;
                nd.nchild[c] = 0;
                next += nc[q];
                continue;
            }
            nd.child[c] = (int32_t)next;
            nd.nchild[c] = nc[q];
#pragma unroll
            for (int d = 0; d < 8; d++) {
                if (bnd[q][d + 1] > bnd[q][d]) {
                    nd.first[next] = bnd[q][d];
                    nd.count[next] = bnd[q][d + 1] - bnd[q][d];
                    nd.parent[next] = (int32_t)c;
                    nd.child[next] = -1;
                    nd.nchild[next] = 0;
                    next++;
                }
            }
        }
        if (tile == ntiles - 1 && threadIdx.x == BT - 1) {
            unsigned long long end = (unsigned long long)hi + excl_sh + total;
            if (end > (unsigned long long)cap) {
                gt_set_error(ctl, GT_EOVERFLOW, GTK_BUILD);
                end = (unsigned long long)cap;
            }
            ctl->level_start[lvl + 2] = (uint32_t)end;
        }
    }
}

__device__ __forceinline__ float sq3f(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ---- cell lists for the per-step pseudo j-particle passes -----------------------
// Every node goes once into nd.cells: the leaves first, bucketed by particle count
// (1..16, then all larger), then the cells with children, level by level and inside a
// level by number of children.  A warp of the pseudo-j passes then takes cells of one
// size, so the FP64 sums run with all lanes busy.  The order inside a bucket is free:
// every cell's result depends on its own particles or children only.

// bucket of node p, given the level ranges ls[0..GT_TREE_LEVELS]
__device__ __forceinline__ int cell_bucket_of(const Nodes &nd, uint32_t p, const uint32_t *ls) {
    if (nd.child[p] < 0) {
        const uint32_t k = nd.count[p];
        return (k >= GT_LEAF_BUCKETS ? GT_LEAF_BUCKETS : (int)k) - 1;
    }
    int lvl = 0;  // the last level starting at or before p
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (lvl + step < GT_TREE_LEVELS && ls[lvl + step] <= p) lvl += step;
    return GT_LEAF_BUCKETS + lvl * 8 + (int)nd.nchild[p] - 1;
}

__global__ __launch_bounds__(256) void k_cell_count(Nodes nd, long long cap, DevCtl *ctl) {
    __shared__ uint32_t ls[GT_TREE_LEVELS + 1];
    __shared__ uint32_t h[GT_CELL_BUCKETS];
    for (int i = threadIdx.x; i <= GT_TREE_LEVELS; i += 256) ls[i] = ctl->level_start[i];
    for (int i = threadIdx.x; i < GT_CELL_BUCKETS; i += 256) h[i] = 0;
    __syncthreads();
    long long nn = ls[GT_TREE_LEVELS];
    if (nn > cap) nn = cap;
    for (long long p = blockIdx.x * 256ll + threadIdx.x; p < nn; p += (long long)gridDim.x * 256)
        atomicAdd(&h[cell_bucket_of(nd, (uint32_t)p, ls)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < GT_CELL_BUCKETS; i += 256)
        if (h[i]) atomicAdd(&ctl->cell_bucket[i], h[i]);
}

// one block: bucket sizes -> fill cursors; the leaf count and where every level starts
__global__ __launch_bounds__(256) void k_cell_scan(DevCtl *ctl) {
    static_assert(GT_CELL_BUCKETS <= 256, "one thread per bucket");
    __shared__ uint32_t tmp[256 / 32 + 1];
    const int b = threadIdx.x;
    const uint32_t v = b < GT_CELL_BUCKETS ? ctl->cell_bucket[b] : 0u;
    uint32_t total;
    const uint32_t start = block_excl_scan<256>(v, &total, tmp);
    if (b < GT_CELL_BUCKETS) ctl->cell_bucket[b] = start;
    if (b == GT_LEAF_BUCKETS) ctl->n_leaves = start;
    if (b >= GT_LEAF_BUCKETS && b < GT_CELL_BUCKETS && (b - GT_LEAF_BUCKETS) % 8 == 0)
        ctl->istart[(b - GT_LEAF_BUCKETS) / 8] = start;
    if (b == 0) ctl->istart[GT_TREE_LEVELS] = total;
}

__global__ __launch_bounds__(256) void k_cell_fill(Nodes nd, long long cap, DevCtl *ctl) {
    __shared__ uint32_t ls[GT_TREE_LEVELS + 1];
    for (int i = threadIdx.x; i <= GT_TREE_LEVELS; i += 256) ls[i] = ctl->level_start[i];
    __syncthreads();
    long long nn = ls[GT_TREE_LEVELS];
    if (nn > cap) nn = cap;
    const unsigned lt = lanemask_lt();
    // the loop bound is warp-uniform, so every lane takes part in the match
    for (long long p0 = blockIdx.x * 256ll + (threadIdx.x & ~31u); p0 < nn; p0 += (long long)gridDim.x * 256) {
        const long long p = p0 + (threadIdx.x & 31);
        const bool ok = p < nn;
        const int b = ok ? cell_bucket_of(nd, (uint32_t)p, ls) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t pos0 = 0;
        if (ok && (peers & lt) == 0) pos0 = atomicAdd(&ctl->cell_bucket[b], (uint32_t)__popc(peers));
        pos0 = __shfl_sync(0xffffffffu, pos0, leader);
        if (ok) nd.cells[pos0 + __popc(peers & lt)] = (uint32_t)p;
    }
}

// leaves: one lane per leaf, a warp's leaves of one particle count.  The masses and the
// cells' members do not change between tree builds, so the mass sums are formed at a
// build (with_mass) and read back at the other block steps: the same values, one FP64
// addition per particle fewer.
template <bool WITH_MASS>
__global__ __launch_bounds__(256) void k_pseudo_leaves(Nodes nd, const float4 *__restrict__ posm, DevCtl *ctl) {
    const long long nl = ctl->n_leaves;
    for (long long t = blockIdx.x * 256ll + threadIdx.x; t < nl; t += (long long)gridDim.x * 256) {
        const uint32_t c = nd.cells[t];
        const uint32_t f = nd.first[c];
        const uint32_t k = nd.count[c];
        double m = WITH_MASS ? 0.0 : nd.sum[c].m, sx = 0.0, sy = 0.0, sz = 0.0;
        for (uint32_t i = f; i < f + k; i++) {
            const float4 p = posm[i];
            const double mi = f2d(p.w);  // m x is exact in FP64, so the fused form rounds once like + does
            if (WITH_MASS) m = __dadd_rn(m, mi);
            sx = __fma_rn(mi, f2d(p.x), sx);
            sy = __fma_rn(mi, f2d(p.y), sy);
            sz = __fma_rn(mi, f2d(p.z), sz);
        }
        float jx, jy, jz;
        if (k == 1) {  // a cell of one particle is that particle
            const float4 p = posm[f];
            jx = p.x; jy = p.y; jz = p.z;
        } else {
            const float mf = d2f(m);
            jx = __fdiv_rn(d2f(sx), mf);
            jy = __fdiv_rn(d2f(sy), mf);
            jz = __fdiv_rn(d2f(sz), mf);
        }
        float d2max = 0.0f, b2 = 0.0f;  // b2: B_2 of the multipole MAC
        for (uint32_t i = f; i < f + k; i++) {
            const float4 p = posm[i];
            const float d2 = sq3f(__fsub_rn(p.x, jx), __fsub_rn(p.y, jy), __fsub_rn(p.z, jz));
            if (d2 > d2max) d2max = d2;
            b2 = __fadd_rn(b2, __fmul_rn(p.w, d2));
        }
        nd.sum[c] = DSum4{m, sx, sy, sz};
        nd.jpos[c] = make_float4(jx, jy, jz, d2f(m));
        nd.walk[c] = make_float4(__fmul_rn(__fsqrt_rn(d2max), GT_RADIUS_MARGIN), __uint_as_float(f),
                                 __uint_as_float(k | GT_LEAF_FLAG), b2);
    }
}

// Cells with children, all levels in one launch.  Every level's part of the cell list
// is cut into chunks of PL cells; chunks are handed out by a ticket counter, the deepest
// level first.  Before a chunk of level l is summed, its block waits until every chunk
// of level l + 1 is finished: those chunks hold smaller tickets, so the blocks holding
// them are running, and the wait ends (it is bounded all the same).  A cell adds its
// children's sums in child order.
constexpr int PL = 256;

template <bool WITH_MASS>
__global__ __launch_bounds__(PL) void k_pseudo_levels(Nodes nd, DevCtl *ctl) {
    __shared__ unsigned int cum[GT_TREE_LEVELS + 1];  // first ticket of every level
    __shared__ unsigned int t_sh;
    __shared__ int bad_sh;
    constexpr int TOP = GT_TREE_LEVELS - 2;           // the deepest level with children
    if (threadIdx.x == 0) {
        unsigned int c = 0;
        for (int l = TOP; l >= 0; l--) {
            cum[l] = c;
            c += (ctl->istart[l + 1] - ctl->istart[l] + PL - 1) / PL;
        }
        cum[GT_TREE_LEVELS] = c;  // total
        bad_sh = 0;
    }
    __syncthreads();
    const unsigned int total = cum[GT_TREE_LEVELS];
    for (;;) {
        if (threadIdx.x == 0) t_sh = atomicAdd(&ctl->pl_ticket, 1u);
        __syncthreads();
        const unsigned int t = t_sh;
        __syncthreads();
        if (t >= total || bad_sh) break;
        int lvl = 0;  // the level whose tickets hold t: cum decreases with the level
        while (lvl < TOP && cum[lvl] > t) lvl++;
        if (threadIdx.x == 0 && lvl < TOP) {
            const unsigned int need = cum[lvl] - cum[lvl + 1];  // chunks of level lvl + 1
            unsigned int spins = 0;
            while (*((volatile unsigned int *)&ctl->pl_done[lvl + 1]) < need) {
                if (++spins > GT_SPIN_LIMIT) {
                    gt_set_error(ctl, GT_ETIMEOUT, GTK_PSEUDO);
                    bad_sh = 1;
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
        }
        __syncthreads();
        if (bad_sh) break;
        const long long idx = (long long)ctl->istart[lvl] + (long long)(t - cum[lvl]) * PL + threadIdx.x;
        if (idx < (long long)ctl->istart[lvl + 1]) {
            const uint32_t p = nd.cells[idx];
            const int32_t ch0 = nd.child[p];
            const uint32_t nch = nd.nchild[p];
            // children written by other blocks of this launch: read through L2 (__ldcg), an SM's
            // L1 may hold a line of them from before they were written
            double m = WITH_MASS ? 0.0 : nd.sum[p].m, sx = 0.0, sy = 0.0, sz = 0.0;
            for (uint32_t q = 0; q < nch; q++) {
                const double2 *cs = (const double2 *)&nd.sum[ch0 + q];
                const double2 s0 = __ldcg(cs), s1 = __ldcg(cs + 1);  // (m, x), (y, z)
                if (WITH_MASS) m = __dadd_rn(m, s0.x);
                sx = __dadd_rn(sx, s0.y);
                sy = __dadd_rn(sy, s1.x);
                sz = __dadd_rn(sz, s1.y);
            }
            const float mf = d2f(m);
            const float jx = __fdiv_rn(d2f(sx), mf);
            const float jy = __fdiv_rn(d2f(sy), mf);
            const float jz = __fdiv_rn(d2f(sz), mf);
            float b = 0.0f, b2 = 0.0f;  // b2: B_2 by parallel axes
            for (uint32_t q = 0; q < nch; q++) {
                const float4 cj = __ldcg(&nd.jpos[ch0 + q]);
                const float4 cw = __ldcg(&nd.walk[ch0 + q]);
                const float d2 = sq3f(__fsub_rn(cj.x, jx), __fsub_rn(cj.y, jy), __fsub_rn(cj.z, jz));
                const float e = __fadd_rn(__fsqrt_rn(d2), cw.x);
                if (e > b) b = e;
                b2 = __fadd_rn(b2, __fadd_rn(cw.w, __fmul_rn(cj.w, d2)));
            }
            nd.sum[p] = DSum4{m, sx, sy, sz};
            nd.jpos[p] = make_float4(jx, jy, jz, mf);
            nd.walk[p] = make_float4(__fmul_rn(b, GT_RADIUS_MARGIN), __uint_as_float((uint32_t)ch0),
                                     __uint_as_float(nch), b2);
        }
        __threadfence();  // every thread's cell is visible device-wide before the chunk counts as done
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&ctl->pl_done[lvl], 1u);
    }
}

}  // namespace

void gt_launch_build(const uint64_t *skey, int64_t n, int leaf_max, Nodes nd, int64_t cap,
                     unsigned long long *status, DevCtl *ctl, int nsm, cudaStream_t st) {
    { k_build_init<<<1, 1, 0, st>>>(n, nd, ctl); gt_note_launches(1); }
    for (int l = 0; l < GT_TREE_LEVELS; l++)
        { k_build_level<<<nsm * 4, BT, 0, st>>>(l, (const unsigned long long *)skey, leaf_max, nd, cap,
                                              status, ctl); gt_note_launches(1); }
}

void gt_launch_cell_lists(Nodes nd, int64_t cap, DevCtl *ctl, int nsm, cudaStream_t st) {
    cudaMemsetAsync(ctl->cell_bucket, 0, sizeof(ctl->cell_bucket), st);
    { k_cell_count<<<nsm * 4, 256, 0, st>>>(nd, cap, ctl); gt_note_launches(1); }
    { k_cell_scan<<<1, 256, 0, st>>>(ctl); gt_note_launches(1); }
    { k_cell_fill<<<nsm * 4, 256, 0, st>>>(nd, cap, ctl); gt_note_launches(1); }
}

void gt_launch_pseudo(Nodes nd, int64_t cap, const float4 *posm, DevCtl *ctl, int nsm, bool with_mass,
                      cudaStream_t st) {
    (void)cap;
    if (with_mass) { k_pseudo_leaves<true><<<nsm * 8, 256, 0, st>>>(nd, posm, ctl); }
    else { k_pseudo_leaves<false><<<nsm * 8, 256, 0, st>>>(nd, posm, ctl); }
    gt_note_launches(1);
    // the level pass's ticket and per-level counters start at zero
    cudaMemsetAsync(&ctl->pl_ticket, 0, sizeof(ctl->pl_ticket) + sizeof(ctl->pl_done), st);
    if (with_mass) { k_pseudo_levels<true><<<nsm * 4, PL, 0, st>>>(nd, ctl); }
    else { k_pseudo_levels<false><<<nsm * 4, PL, 0, st>>>(nd, ctl); }
    gt_note_launches(1);
}
