// Steps A4-A5: breadth-first octree over the sorted keys and the pseudo
// j-particles (Sec. 2.1, Fig. 1).
//
// A4.  A cell at level l with more than leaf_max particles (and l < 21) splits into the
// non-empty ranges of its particles' level-(l + 1) digit; children are numbered after
// their level, level by level and, inside a level, by first particle.  With leaf_max up
// to 64 the whole tree comes from one sweep over the sorted keys (k_flat_*: every
// particle's leaf level from the digits in which its neighbours' keys differ, then the
// nodes' starts and ends counted, scanned and scattered by level); larger leaves take
// one kernel per level (k_build_level: the "seven partitions" of a cell's key range by a
// lock-step 7-way binary search, children numbered by a block scan plus a decoupled
// look-back over tiles taken in ticket order).  Both give the same numbering.
//
// A5, one launch over a cell list bucketed by level and size: a leaf's lane sums its
// particles in FP64 (mass, m x, m y, m z); a cell with children sums its children's FP64
// sums in child order once the level below is done -- every FP64 instruction runs with
// full warps, which matters on this GPU's narrow FP64 pipe.  m_J = (float)M and
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

// ---- A4 in one sweep over the sorted keys (leaf_max <= FLAT_LWIN) ------------------
// d(p), the index of the first 3-bit digit in which keys p - 1 and p differ (21 for equal
// keys; -1 at p = 0 and p = n), says at which levels a new cell begins at particle p: a
// run of particles between two positions with d < l shares its first l digits, so it is
// one level-l cell of the full octree.  The tree keeps a level-l run iff its parent run
// holds more than leaf_max particles, so particle i's leaf is at the first level whose
// run around i holds at most leaf_max -- found from the d values within leaf_max of i.
// Particle i then starts a node at every level l with d(i) < l <= leaf level(i), and ends
// one (as its last particle) at every l with d(i + 1) < l <= leaf level(i).  Counting
// those starts and ends per level and tile, scanning, and scattering them by rank gives
// the same numbering as the level-by-level split: level by level, and inside a level by
// first particle.  A node's first child starts at its own first particle; the others
// are the next nodes of the child level that start before its end.
constexpr int FLAT_LWIN = 64;              // the largest leaf_max of this build
constexpr int FT = 2048;                   // particles per tile
constexpr int FB = 256;                    // threads per block
constexpr int NREC = 2 * GT_TREE_LEVELS;   // start and end counters per level

__device__ __forceinline__ int key_diff_digit(unsigned long long a, unsigned long long b) {
    const unsigned long long x = a ^ b;  // keys use bits 0..62, so clz >= 1
    return x ? (__clzll((long long)x) - 1) / 3 : GT_KEY_LEVELS;
}

// Leaf level of the particle at ds[j]: the run around it at level l holds at most M
// particles iff, for some a in [0, M), positions i - a .. i and i + 1 .. i + M - a both
// hold a d below l; so the leaf level is 1 + min over a of max(the smallest d of the
// first window, the smallest d of the second).  MT > 0: M = MT, unrolled in registers.
template <int MT>
__device__ __forceinline__ int leaf_level_of(const int8_t *ds, int j) {
    int mr[MT + 1];  // mr[b]: smallest d over i + 1 .. i + b
    int m = 127;
#pragma unroll
    for (int b = 1; b <= MT; b++) {
        m = min(m, (int)ds[j + b]);
        mr[b] = m;
    }
    int ml = 127, best = 127;
#pragma unroll
    for (int a = 0; a < MT; a++) {
        ml = min(ml, (int)ds[j - a]);
        best = min(best, max(ml, mr[MT - a]));
    }
    return min(best + 1, GT_KEY_LEVELS);
}

// d and the leaf level of every particle (packed (d + 1) | leaf << 8), and every tile's
// start and end counts per level (column-major: counter k of tile t at cnt[k * ntiles + t]).
// MT > 0: leaf_max == MT; MT == 0: any leaf_max up to FLAT_LWIN (running minima in shared memory).
template <int MT>
__global__ __launch_bounds__(FB) void k_flat_marks(const unsigned long long *__restrict__ skey, long long n,
                                                   int M, uint16_t *__restrict__ dl,
                                                   uint32_t *__restrict__ cnt, int ntiles) {
    constexpr int W = FLAT_LWIN;
    constexpr int MW = MT > 0 ? 1 : W;
    __shared__ int8_t ds[FT + 2 * W + 1];      // d of positions base - W .. base + FT + W
    __shared__ uint8_t mr[MW][FB];             // generic: 1 + smallest d over (i, i + b]
    __shared__ unsigned int c[NREC];
    const long long base = (long long)blockIdx.x * FT;
    for (int j = threadIdx.x; j < FT + 2 * W + 1; j += FB) {
        const long long p = base - W + j;
        ds[j] = (int8_t)((p > 0 && p < n) ? key_diff_digit(skey[p - 1], skey[p]) : -1);
    }
    for (int j = threadIdx.x; j < NREC; j += FB) c[j] = 0;
    __syncthreads();
    for (int r = 0; r < FT / FB; r++) {
        const int t = r * FB + threadIdx.x;
        const long long i = base + t;
        if (i >= n) break;
        const int j = t + W;  // position i in ds
        int leaf;
        if constexpr (MT > 0) {
            leaf = leaf_level_of<MT>(ds, j);
        } else {
            int m = 127;
            for (int b = 1; b <= M; b++) {
                m = min(m, (int)ds[j + b]);
                mr[b - 1][threadIdx.x] = (uint8_t)(m + 1);
            }
            int ml = 127, best = 127;
            for (int a = 0; a < M; a++) {
                ml = min(ml, (int)ds[j - a]);
                best = min(best, max(ml, (int)mr[M - a - 1][threadIdx.x] - 1));
            }
            leaf = min(best + 1, GT_KEY_LEVELS);
        }
        const int d0 = ds[j], d1 = ds[j + 1];
        dl[i] = (uint16_t)((d0 + 1) | (leaf << 8));
        for (int l = d0 + 1; l <= leaf; l++) atomicAdd(&c[l], 1u);
        for (int l = d1 + 1; l <= leaf; l++) atomicAdd(&c[GT_TREE_LEVELS + l], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NREC; k += FB) cnt[(size_t)k * ntiles + blockIdx.x] = c[k];
}

// one block per counter: exclusive scan over the tiles, the column total into tot[k]
__global__ __launch_bounds__(1024) void k_flat_scan(uint32_t *__restrict__ cnt, int ntiles,
                                                    uint32_t *__restrict__ tot) {
    __shared__ unsigned int tmp[1024 / 32 + 1];
    uint32_t *col = cnt + (size_t)blockIdx.x * ntiles;
    unsigned int carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += 1024) {
        const int t = b0 + (int)threadIdx.x;
        const unsigned int v = t < ntiles ? col[t] : 0u;
        unsigned int total;
        const unsigned int e = block_excl_scan<1024>(v, &total, tmp);
        if (t < ntiles) col[t] = carry + e;
        carry += total;
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// level starts from the per-level node counts (clamped to the node capacity)
__global__ void k_flat_levels(const uint32_t *__restrict__ tot, long long cap, DevCtl *ctl) {
    unsigned long long s = 0;
    for (int l = 0; l < GT_TREE_LEVELS; l++) {
        ctl->level_start[l] = (uint32_t)(s < (unsigned long long)cap ? s : (unsigned long long)cap);
        s += tot[l];
    }
    if (s > (unsigned long long)cap) {
        gt_set_error(ctl, GT_EOVERFLOW, GTK_BUILD);
        s = (unsigned long long)cap;
    }
    ctl->level_start[GT_TREE_LEVELS] = (uint32_t)s;
    ctl->level_start[GT_TREE_LEVELS + 1] = (uint32_t)s;
}

// every start and end to its node: first, the first child and the parent along a
// particle's own chain of starts, leaves; an end goes to count (as the end position)
__global__ __launch_bounds__(FB) void k_flat_scatter(const uint16_t *__restrict__ dl, long long n,
                                                     const uint32_t *__restrict__ cnt, int ntiles,
                                                     long long cap, Nodes nd, const DevCtl *__restrict__ ctl) {
    __shared__ uint32_t lb[GT_TREE_LEVELS];
    __shared__ uint32_t run[NREC];
    __shared__ uint32_t wc[FB / 32][NREC];
    __shared__ uint16_t dls[FT + 1];
    const long long base = (long long)blockIdx.x * FT;
    for (int k = threadIdx.x; k < GT_TREE_LEVELS; k += FB) lb[k] = ctl->level_start[k];
    for (int k = threadIdx.x; k < NREC; k += FB) run[k] = cnt[(size_t)k * ntiles + blockIdx.x];
    for (int j = threadIdx.x; j <= FT; j += FB) dls[j] = base + j < n ? dl[base + j] : (uint16_t)0;  // d(n) = -1
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const unsigned int lt = lanemask_lt();
    for (int r = 0; r < FT / FB; r++) {
        const int t = r * FB + threadIdx.x;
        const long long i = base + t;
        const bool valid = i < n;
        const int v = dls[t];
        const int slo = valid ? (v & 0xff) : GT_TREE_LEVELS, leaf = v >> 8;
        const int elo = valid ? (dls[t + 1] & 0xff) : GT_TREE_LEVELS;
        // ranks inside the round: per-warp counts, then warps in order after the tile's
        // offset; a warp visits only the levels at which one of its lanes has a record
        const int has = slo <= leaf || elo <= leaf;
        const int lmin = __reduce_min_sync(0xffffffffu, has ? min(slo, elo) : GT_TREE_LEVELS);
        const int lmax = __reduce_max_sync(0xffffffffu, has ? leaf : -1);
        if ((threadIdx.x & 31) < GT_TREE_LEVELS) {
            wc[w][threadIdx.x & 31] = 0;
            wc[w][GT_TREE_LEVELS + (threadIdx.x & 31)] = 0;
        }
        __syncwarp();
        for (int l = lmin; l <= lmax; l++) {
            const unsigned int bs = __ballot_sync(0xffffffffu, slo <= l && l <= leaf);
            const unsigned int be = __ballot_sync(0xffffffffu, elo <= l && l <= leaf);
            if ((threadIdx.x & 31) == 0) {
                wc[w][l] = __popc(bs);
                wc[w][GT_TREE_LEVELS + l] = __popc(be);
            }
        }
        __syncthreads();
        if (threadIdx.x < NREC) {
            uint32_t s = run[threadIdx.x];
            for (int q = 0; q < FB / 32; q++) {
                const uint32_t x = wc[q][threadIdx.x];
                wc[q][threadIdx.x] = s;
                s += x;
            }
            run[threadIdx.x] = s;
        }
        __syncthreads();
        long long prev = -1;  // this particle's node one level up, when it starts one there
        for (int l = lmin; l <= lmax; l++) {
            const bool hs = slo <= l && l <= leaf, he = elo <= l && l <= leaf;
            const unsigned int bs = __ballot_sync(0xffffffffu, hs);
            const unsigned int be = __ballot_sync(0xffffffffu, he);
            if (hs) {
                const long long id = (long long)lb[l] + wc[w][l] + __popc(bs & lt);
                if (prev >= 0) nd.child[prev] = id < cap ? (int32_t)id : -1;
                if (id < cap) {
                    nd.first[id] = (uint32_t)i;
                    if (l == 0 || prev >= 0) nd.parent[id] = (int32_t)prev;  // else: the link pass
                    if (l == leaf) {
                        nd.child[id] = -1;
                        nd.nchild[id] = 0;
                    }
                }
                prev = id < cap ? id : -1;
            }
            if (he) {
                const long long id = (long long)lb[l] + wc[w][GT_TREE_LEVELS + l] + __popc(be & lt);
                if (id < cap) nd.count[id] = (uint32_t)(i + 1);
            }
        }
        __syncthreads();  // wc is rewritten by the next round
    }
}

// per node: count = end - first; a node with children counts them (the nodes of the
// next level from its first child on that start before its end) and is their parent
__global__ __launch_bounds__(256) void k_flat_link(Nodes nd, long long cap, const DevCtl *__restrict__ ctl) {
    __shared__ uint32_t ls[GT_TREE_LEVELS + 2];
    for (int i = threadIdx.x; i < GT_TREE_LEVELS + 2; i += 256) ls[i] = ctl->level_start[i];
    __syncthreads();
    const long long nn = ls[GT_TREE_LEVELS];
    for (long long p = blockIdx.x * 256ll + threadIdx.x; p < nn; p += (long long)gridDim.x * 256) {
        const uint32_t f = nd.first[p], e = nd.count[p];
        nd.count[p] = e - f;
        const int32_t c0 = nd.child[p];
        if (c0 < 0) continue;
        int lvl = 0;  // the last level starting at or before p
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (lvl + step < GT_TREE_LEVELS && ls[lvl + step] <= (uint32_t)p) lvl += step;
        long long hi = ls[lvl + 2];
        if (hi > cap) hi = cap;
        uint32_t nch = 1;
        for (int q = 1; q < 8; q++) {
            const long long c = (long long)c0 + q;
            if (c >= hi || nd.first[c] >= e) break;
            nd.parent[c] = (int32_t)p;
            nch++;
        }
        nd.nchild[p] = nch;
    }
}

__device__ __forceinline__ float sq3f(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// ---- cell lists for the per-step pseudo j-particle pass ---------------------------
// Every node goes once into nd.cells, level by level; inside a level the leaves come
// first, bucketed by particle count (1..16, then all larger), then the cells with
// children, bucketed by number of children.  A warp of the pseudo-j pass then takes
// cells of one size, so the FP64 sums run with all lanes busy.  The order inside a
// bucket is free: every cell's result depends on its own particles or children only.

// bucket of node p, given the level ranges ls[0..GT_TREE_LEVELS]
__device__ __forceinline__ int cell_bucket_of(const Nodes &nd, uint32_t p, const uint32_t *ls) {
    int lvl = 0;  // the last level starting at or before p
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (lvl + step < GT_TREE_LEVELS && ls[lvl + step] <= p) lvl += step;
    if (nd.child[p] < 0) {
        const uint32_t k = nd.count[p];
        return lvl * GT_LEVEL_BUCKETS + (k >= GT_LEAF_BUCKETS ? GT_LEAF_BUCKETS : (int)k) - 1;
    }
    return lvl * GT_LEVEL_BUCKETS + GT_LEAF_BUCKETS + (int)nd.nchild[p] - 1;
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

// one block: bucket sizes -> fill cursors, and where every level's leaves and cells
// with children start
__global__ __launch_bounds__(1024) void k_cell_scan(DevCtl *ctl) {
    static_assert(GT_CELL_BUCKETS <= 1024, "one thread per bucket");
    __shared__ unsigned int tmp[1024 / 32 + 1];
    const int b = threadIdx.x;
    const uint32_t v = b < GT_CELL_BUCKETS ? ctl->cell_bucket[b] : 0u;
    uint32_t total;
    const uint32_t start = block_excl_scan<1024>(v, &total, tmp);
    if (b < GT_CELL_BUCKETS) {
        ctl->cell_bucket[b] = start;
        const int q = b % GT_LEVEL_BUCKETS;
        if (q == 0) ctl->seg[2 * (b / GT_LEVEL_BUCKETS)] = start;
        if (q == GT_LEAF_BUCKETS) ctl->seg[2 * (b / GT_LEVEL_BUCKETS) + 1] = start;
    }
    if (b == 0) ctl->seg[2 * GT_TREE_LEVELS] = total;
}

// A block takes a contiguous range of nodes, counts them per bucket in shared memory,
// reserves its room in every bucket with one global atomic each, and fills it.
constexpr int CF_NODES = 4096;  // nodes per fill block

__global__ __launch_bounds__(256) void k_cell_fill(Nodes nd, long long cap, DevCtl *ctl) {
    __shared__ uint32_t ls[GT_TREE_LEVELS + 1];
    __shared__ uint32_t h[GT_CELL_BUCKETS];
    for (int i = threadIdx.x; i <= GT_TREE_LEVELS; i += 256) ls[i] = ctl->level_start[i];
    long long nn = ctl->level_start[GT_TREE_LEVELS];
    if (nn > cap) nn = cap;
    for (long long b0 = (long long)blockIdx.x * CF_NODES; b0 < nn; b0 += (long long)gridDim.x * CF_NODES) {
        __syncthreads();
        for (int i = threadIdx.x; i < GT_CELL_BUCKETS; i += 256) h[i] = 0;
        __syncthreads();
        const long long b1 = b0 + CF_NODES < nn ? b0 + CF_NODES : nn;
        for (long long p = b0 + threadIdx.x; p < b1; p += 256)
            atomicAdd(&h[cell_bucket_of(nd, (uint32_t)p, ls)], 1u);
        __syncthreads();
        for (int i = threadIdx.x; i < GT_CELL_BUCKETS; i += 256)
            if (h[i]) h[i] = atomicAdd(&ctl->cell_bucket[i], h[i]);
        __syncthreads();
        for (long long p = b0 + threadIdx.x; p < b1; p += 256)
            nd.cells[atomicAdd(&h[cell_bucket_of(nd, (uint32_t)p, ls)], 1u)] = (uint32_t)p;
    }
}

// ---- A5: pseudo j-particles, every node in one launch ------------------------------
// The cell list's segments (a level's leaves, a level's cells with children) are cut
// into chunks of PL nodes, handed out by a ticket counter in this order: the leaves of
// level 21; then, for l = 20 .. 0, the leaves of level l and the cells with children of
// level l + 1; the cells of level 0 last.  A chunk of cells of level l waits until every
// chunk of level l + 1 is finished: those hold smaller tickets, so the blocks holding
// them are running and the wait ends (it is bounded all the same).  Leaves wait for
// nothing, so their FP64 sums fill the time a level's cells wait for the one below.
#ifndef GT_PSEUDO_PU
#define GT_PSEUDO_PU 2  // a leaf's particles loaded per round
#endif
#ifndef GT_PSEUDO_CU
#define GT_PSEUDO_CU 2  // a cell's children loaded per round
#endif
#ifndef GT_PSEUDO_COOP
#define GT_PSEUDO_COOP 16384  // a level's cells with children taken eight lanes each when at most this many
#endif
#ifndef GT_PSEUDO_MINB
#define GT_PSEUDO_MINB 6  // resident blocks per SM (the grid) the register budget is sized for
#endif
constexpr int PL = 128;  // nodes per chunk, one per thread
constexpr uint32_t PU = GT_PSEUDO_PU, CU = GT_PSEUDO_CU;
constexpr int PSEUDO_LAG = 1;  // levels of leaves between a level's cells and the level below
constexpr int NSEG = 2 * GT_TREE_LEVELS;

// Leaf c: one lane sums its particles in FP64 (mass, m x, m y, m z) in particle order.
// The masses and the cells' members do not change between tree builds, so the mass
// sums are formed at a build (WITH_MASS) and read back at the other block steps: the
// same values, one FP64 addition per particle fewer.
template <bool WITH_MASS>
__device__ __forceinline__ void pseudo_leaf(const Nodes &nd, const float4 *__restrict__ posm, uint32_t c) {
    const uint32_t f = nd.first[c];
    const uint32_t k = nd.count[c];
    double m = WITH_MASS ? 0.0 : nd.sum[c].m, sx = 0.0, sy = 0.0, sz = 0.0;
    // in particle order; the loads of four particles go out before their sums
    // (m x is exact in FP64, so the fused form rounds once like + does)
    for (uint32_t i0 = f; i0 < f + k; i0 += PU) {
        float4 p[PU];
#pragma unroll
        for (uint32_t q = 0; q < PU; q++)
            if (i0 + q < f + k) p[q] = posm[i0 + q];
#pragma unroll
        for (uint32_t q = 0; q < PU; q++)
            if (i0 + q < f + k) {
                const double mi = f2d(p[q].w);
                if (WITH_MASS) m = __dadd_rn(m, mi);
                sx = __fma_rn(mi, f2d(p[q].x), sx);
                sy = __fma_rn(mi, f2d(p[q].y), sy);
                sz = __fma_rn(mi, f2d(p[q].z), sz);
            }
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
    for (uint32_t i0 = f; i0 < f + k; i0 += PU) {
        float4 p[PU];
#pragma unroll
        for (uint32_t q = 0; q < PU; q++)
            if (i0 + q < f + k) p[q] = posm[i0 + q];
#pragma unroll
        for (uint32_t q = 0; q < PU; q++)
            if (i0 + q < f + k) {
                const float d2 = sq3f(__fsub_rn(p[q].x, jx), __fsub_rn(p[q].y, jy), __fsub_rn(p[q].z, jz));
                if (d2 > d2max) d2max = d2;
                b2 = __fadd_rn(b2, __fmul_rn(p[q].w, d2));
            }
    }
    nd.sum[c] = DSum4{m, sx, sy, sz};
    nd.jpos[c] = make_float4(jx, jy, jz, d2f(m));
    nd.walk[c] = make_float4(__fmul_rn(__fsqrt_rn(d2max), GT_RADIUS_MARGIN), __uint_as_float(f),
                             __uint_as_float(k | GT_LEAF_FLAG), b2);
}

// Cell p with children: its children's FP64 sums added in child order.  The children
// were written by other blocks of this launch: they are read through L2 (__ldcg), an
// SM's L1 may hold a line of them from before they were written.  Loads go out four
// children at a time, so a level costs few L2 round trips.
template <bool WITH_MASS>
__device__ __forceinline__ void pseudo_cell(const Nodes &nd, uint32_t p) {
    const int32_t ch0 = nd.child[p];
    const uint32_t nch = nd.nchild[p];
    double m = WITH_MASS ? 0.0 : nd.sum[p].m, sx = 0.0, sy = 0.0, sz = 0.0;
    for (uint32_t q0 = 0; q0 < nch; q0 += CU) {
        double2 s0[CU], s1[CU];  // (m, x), (y, z)
#pragma unroll
        for (uint32_t q = 0; q < CU; q++)
            if (q0 + q < nch) {
                const double2 *cs = (const double2 *)&nd.sum[ch0 + q0 + q];
                s0[q] = __ldcg(cs);
                s1[q] = __ldcg(cs + 1);
            }
#pragma unroll
        for (uint32_t q = 0; q < CU; q++)
            if (q0 + q < nch) {
                if (WITH_MASS) m = __dadd_rn(m, s0[q].x);
                sx = __dadd_rn(sx, s0[q].y);
                sy = __dadd_rn(sy, s1[q].x);
                sz = __dadd_rn(sz, s1[q].y);
            }
    }
    const float mf = d2f(m);
    const float jx = __fdiv_rn(d2f(sx), mf);
    const float jy = __fdiv_rn(d2f(sy), mf);
    const float jz = __fdiv_rn(d2f(sz), mf);
    float b = 0.0f, b2 = 0.0f;  // b2: B_2 by parallel axes
    for (uint32_t q0 = 0; q0 < nch; q0 += CU) {
        float4 cj[CU], cw[CU];
#pragma unroll
        for (uint32_t q = 0; q < CU; q++)
            if (q0 + q < nch) {
                cj[q] = __ldcg(&nd.jpos[ch0 + q0 + q]);
                cw[q] = __ldcg(&nd.walk[ch0 + q0 + q]);
            }
#pragma unroll
        for (uint32_t q = 0; q < CU; q++)
            if (q0 + q < nch) {
                const float d2 = sq3f(__fsub_rn(cj[q].x, jx), __fsub_rn(cj[q].y, jy), __fsub_rn(cj[q].z, jz));
                const float e = __fadd_rn(__fsqrt_rn(d2), cw[q].x);
                if (e > b) b = e;
                b2 = __fadd_rn(b2, __fadd_rn(cw[q].w, __fmul_rn(cj[q].w, d2)));
            }
    }
    nd.sum[p] = DSum4{m, sx, sy, sz};
    nd.jpos[p] = make_float4(jx, jy, jz, mf);
    nd.walk[p] = make_float4(__fmul_rn(b, GT_RADIUS_MARGIN), __uint_as_float((uint32_t)ch0),
                             __uint_as_float(nch), b2);
}

// The same cell with eight lanes, one child each (lanes 8g .. 8g + 7 of the warp hold cell
// g of four): the children's records arrive in one round of loads instead of one per
// pair of children.  Every lane of the group forms the FP64 sums and the B_2 sum itself,
// in child order, from its neighbours' values (shuffles), so the operations and their
// order are those of pseudo_cell; the radius is a maximum, taken across the lanes.  For
// the levels near the root, whose few cells each wait for the level below.  Every lane
// of the warp must call it; `valid` marks groups that own a cell.
template <bool WITH_MASS>
__device__ __forceinline__ void pseudo_cell_coop(const Nodes &nd, uint32_t p, bool valid) {
    const unsigned FULL = 0xffffffffu;
    const uint32_t lane = threadIdx.x & 31u, j = lane & 7u, g0 = lane & ~7u;
    const int32_t ch0 = valid ? nd.child[p] : 0;
    const uint32_t nch = valid ? nd.nchild[p] : 0u;
    const bool has = j < nch;
    double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);  // (m, x), (y, z)
    float4 cj = make_float4(0.f, 0.f, 0.f, 0.f), cw = make_float4(0.f, 0.f, 0.f, 0.f);
    if (has) {
        const double2 *cs = (const double2 *)&nd.sum[ch0 + j];
        s0 = __ldcg(cs);
        s1 = __ldcg(cs + 1);
        cj = __ldcg(&nd.jpos[ch0 + j]);
        cw = __ldcg(&nd.walk[ch0 + j]);
    }
    double m = (WITH_MASS || !valid) ? 0.0 : nd.sum[p].m, sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
    for (uint32_t q = 0; q < 8; q++) {
        const double cm = __shfl_sync(FULL, s0.x, g0 + q), cx = __shfl_sync(FULL, s0.y, g0 + q);
        const double cy = __shfl_sync(FULL, s1.x, g0 + q), cz = __shfl_sync(FULL, s1.y, g0 + q);
        if (q < nch) {
            if (WITH_MASS) m = __dadd_rn(m, cm);
            sx = __dadd_rn(sx, cx);
            sy = __dadd_rn(sy, cy);
            sz = __dadd_rn(sz, cz);
        }
    }
    const float mf = d2f(m);
    const float jx = __fdiv_rn(d2f(sx), mf);
    const float jy = __fdiv_rn(d2f(sy), mf);
    const float jz = __fdiv_rn(d2f(sz), mf);
    const float d2 = sq3f(__fsub_rn(cj.x, jx), __fsub_rn(cj.y, jy), __fsub_rn(cj.z, jz));
    float b = 0.0f;
    if (has) {
        const float e = __fadd_rn(__fsqrt_rn(d2), cw.x);
        if (e > b) b = e;
    }
    const float t = __fadd_rn(cw.w, __fmul_rn(cj.w, d2));
    float b2 = 0.0f;
#pragma unroll
    for (uint32_t q = 0; q < 8; q++) {
        const float tq = __shfl_sync(FULL, t, g0 + q);
        if (q < nch) b2 = __fadd_rn(b2, tq);
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const float bo = __shfl_xor_sync(FULL, b, o);
        if (bo > b) b = bo;
    }
    if (valid && j == 0) {
        nd.sum[p] = DSum4{m, sx, sy, sz};
        nd.jpos[p] = make_float4(jx, jy, jz, mf);
        nd.walk[p] = make_float4(__fmul_rn(b, GT_RADIUS_MARGIN), __uint_as_float((uint32_t)ch0),
                                 __uint_as_float(nch), b2);
    }
}

template <bool WITH_MASS>
__global__ __launch_bounds__(PL, GT_PSEUDO_MINB) void k_pseudo(Nodes nd, const float4 *__restrict__ posm, DevCtl *ctl) {
    __shared__ uint32_t seg[NSEG + 1];
    __shared__ uint8_t olvl[NSEG], ocell[NSEG];      // ticket order: segment level and kind
    __shared__ uint32_t ocum[NSEG + 1];              // first ticket of every entry
    __shared__ uint32_t nchunk[NSEG];                // chunks of segment (2 l + kind)
    __shared__ uint8_t coop[NSEG];                   // cells of the segment taken eight lanes each
    __shared__ unsigned int t_sh;
    __shared__ int o_sh, bad_sh;
    for (int i = threadIdx.x; i <= NSEG; i += PL) seg[i] = ctl->seg[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NSEG; k++) {
            const uint32_t cnt = seg[k + 1] - seg[k];
            coop[k] = (k & 1) && cnt <= (uint32_t)GT_PSEUDO_COOP;
            const uint32_t per = coop[k] ? PL / 8 : PL;
            nchunk[k] = (cnt + per - 1) / per;
        }
        int o = 0;  // level l's cells go right after the leaves of level l - PSEUDO_LAG
        for (int s = 0; s < GT_TREE_LEVELS + PSEUDO_LAG; s++) {
            const int ll = GT_TREE_LEVELS - 1 - s, lc = GT_TREE_LEVELS - 1 + PSEUDO_LAG - s;
            if (ll >= 0) { olvl[o] = (uint8_t)ll; ocell[o] = 0; o++; }
            if (lc >= 0 && lc < GT_TREE_LEVELS - 1) { olvl[o] = (uint8_t)lc; ocell[o] = 1; o++; }
        }
        // o == NSEG - 1 (level 21 has no cells with children): the last entry is empty
        olvl[o] = 0; ocell[o] = 2;
        uint32_t c = 0;
        for (int k = 0; k < NSEG; k++) {
            ocum[k] = c;
            if (ocell[k] < 2) c += nchunk[2 * olvl[k] + ocell[k]];
        }
        ocum[NSEG] = c;
        bad_sh = 0;
    }
    __syncthreads();
    const uint32_t total = ocum[NSEG];
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned int t = atomicAdd(&ctl->pl_ticket, 1u);
            int o = 0;
            if (t < total)
                while (ocum[o + 1] <= t) o++;
            t_sh = t;
            o_sh = o;
            if (t < total && ocell[o] == 1 && olvl[o] + 1 < GT_TREE_LEVELS) {
                const int l1 = olvl[o] + 1;  // every chunk of that level first
                const unsigned int need = nchunk[2 * l1] + nchunk[2 * l1 + 1];
                unsigned int spins = 0;
                const unsigned int limit = gt_spin_limit(ctl);
                while (*((volatile unsigned int *)&ctl->pl_done[l1]) < need) {
                    if (++spins > limit) {
                        gt_set_error(ctl, GT_ETIMEOUT, GTK_PSEUDO);
                        bad_sh = 1;
                        break;
                    }
                    __nanosleep(64);
                }
                __threadfence();
            }
        }
        __syncthreads();
        const unsigned int t = t_sh;
        const int o = o_sh;
        if (t >= total || bad_sh) break;
        const int lvl = olvl[o], kind = ocell[o], sg = 2 * lvl + kind;
#if GT_DEBUG
        {   // every node of the chunk: its particle or child range inside the tree
            const uint32_t nn = ctl->level_start[GT_TREE_LEVELS], np = nd.count[0];
            const uint32_t per = coop[sg] ? PL / 8 : PL;
            const long long i0 = (long long)seg[sg] + (long long)(t - ocum[o]) * per;
            bool bad = false;
            for (long long i = i0 + threadIdx.x; i < i0 + per && i < (long long)seg[sg + 1]; i += PL) {
                const uint32_t c = nd.cells[i];
                if (c >= nn) { bad = true; continue; }
                bad |= kind == 0 ? ((unsigned long long)nd.first[c] + nd.count[c] > np)
                                 : (nd.child[c] < 0 || (unsigned long long)nd.child[c] + nd.nchild[c] > nn);
            }
            if (__syncthreads_or(bad)) {  // the whole chunk is skipped
                if (threadIdx.x == 0) {
                    gt_set_error(ctl, GT_EINVAL, GTK_PSEUDO);
                    atomicAdd(&ctl->pl_done[lvl], 1u);
                }
                continue;
            }
        }
#endif
        if (coop[sg]) {  // the whole block: PL / 8 cells, eight lanes each
            const long long idx = (long long)seg[sg] + (long long)(t - ocum[o]) * (PL / 8) + (threadIdx.x >> 3);
            const bool valid = idx < (long long)seg[sg + 1];
            pseudo_cell_coop<WITH_MASS>(nd, valid ? nd.cells[idx] : 0u, valid);
        } else {
            const long long idx = (long long)seg[sg] + (long long)(t - ocum[o]) * PL + threadIdx.x;
            if (idx < (long long)seg[sg + 1]) {
                if (kind == 0) pseudo_leaf<WITH_MASS>(nd, posm, nd.cells[idx]);
                else pseudo_cell<WITH_MASS>(nd, nd.cells[idx]);
            }
        }
        __threadfence();  // every thread's node is visible device-wide before the chunk counts as done
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&ctl->pl_done[lvl], 1u);
    }
}

}  // namespace

size_t gt_build_scratch_bytes(int64_t n) {
    const size_t N = (size_t)(n > 0 ? n : 1);
    const size_t tiles = (N + FT - 1) / FT;
    return (2 * N + 15) / 16 * 16 + 4 * (size_t)NREC * (tiles + 1);
}

void gt_launch_build(const uint64_t *skey, int64_t n, int leaf_max, Nodes nd, int64_t cap,
                     unsigned long long *status, uint8_t *scratch, DevCtl *ctl, int nsm, cudaStream_t st) {
    if (leaf_max <= FLAT_LWIN) {
        const int ntiles = (int)((n + FT - 1) / FT);
        uint16_t *dl = (uint16_t *)scratch;
        uint32_t *cnt = (uint32_t *)(scratch + (2 * (size_t)(n > 0 ? n : 1) + 15) / 16 * 16);
        uint32_t *tot = cnt + (size_t)NREC * ntiles;
        if (ntiles > 0) {
            const unsigned long long *k = (const unsigned long long *)skey;
            switch (leaf_max) {
            case 4: k_flat_marks<4><<<ntiles, FB, 0, st>>>(k, n, leaf_max, dl, cnt, ntiles); break;
            case 8: k_flat_marks<8><<<ntiles, FB, 0, st>>>(k, n, leaf_max, dl, cnt, ntiles); break;
            case 16: k_flat_marks<16><<<ntiles, FB, 0, st>>>(k, n, leaf_max, dl, cnt, ntiles); break;
            case 24: k_flat_marks<24><<<ntiles, FB, 0, st>>>(k, n, leaf_max, dl, cnt, ntiles); break;
            case 32: k_flat_marks<32><<<ntiles, FB, 0, st>>>(k, n, leaf_max, dl, cnt, ntiles); break;
            default: k_flat_marks<0><<<ntiles, FB, 0, st>>>(k, n, leaf_max, dl, cnt, ntiles); break;
            }
            gt_note_launches(1);
        }
        { k_flat_scan<<<NREC, 1024, 0, st>>>(cnt, ntiles, tot); gt_note_launches(1); }
        { k_flat_levels<<<1, 1, 0, st>>>(tot, cap, ctl); gt_note_launches(1); }
        if (ntiles > 0) {
            k_flat_scatter<<<ntiles, FB, 0, st>>>(dl, n, cnt, ntiles, cap, nd, ctl);
            { k_flat_link<<<nsm * 8, 256, 0, st>>>(nd, cap, ctl); }
            gt_note_launches(2);
        }
        return;
    }
    { k_build_init<<<1, 1, 0, st>>>(n, nd, ctl); gt_note_launches(1); }
    for (int l = 0; l < GT_TREE_LEVELS; l++)
        { k_build_level<<<nsm * 4, BT, 0, st>>>(l, (const unsigned long long *)skey, leaf_max, nd, cap,
                                              status, ctl); gt_note_launches(1); }
}

void gt_launch_cell_lists(Nodes nd, int64_t cap, DevCtl *ctl, int nsm, cudaStream_t st) {
    cudaMemsetAsync(ctl->cell_bucket, 0, sizeof(ctl->cell_bucket), st);
    { k_cell_count<<<nsm * 4, 256, 0, st>>>(nd, cap, ctl); gt_note_launches(1); }
    { k_cell_scan<<<1, 1024, 0, st>>>(ctl); gt_note_launches(1); }
    { k_cell_fill<<<nsm * 2, 256, 0, st>>>(nd, cap, ctl); gt_note_launches(1); }
}

void gt_launch_pseudo(Nodes nd, int64_t cap, const float4 *posm, DevCtl *ctl, int nsm, bool with_mass,
                      cudaStream_t st) {
    (void)cap;
    // the ticket and the per-level counters start at zero
    cudaMemsetAsync(&ctl->pl_ticket, 0, sizeof(ctl->pl_ticket) + sizeof(ctl->pl_done), st);
    if (with_mass) { k_pseudo<true><<<nsm * GT_PSEUDO_MINB, PL, 0, st>>>(nd, posm, ctl); }
    else { k_pseudo<false><<<nsm * GT_PSEUDO_MINB, PL, 0, st>>>(nd, posm, ctl); }
    gt_note_launches(1);
}
