// Step A2: stable LSD radix sort of (63-bit key, 32-bit index) pairs (Sec. 2.1: the
// particles are sorted by their space-filling key with a library radix sort).
//
// Eight passes of 8-bit digits, one kernel per pass after one histogram pass:
//   k_hist_all     all eight digit histograms in one read of the keys   (reads 8 B/key)
//   k_digit_bases  exclusive scans of the histograms -> where every digit starts
//   k_onesweep     per 4096-key tile (512 threads) taken in ticket order: a stable rank of
//                  every key inside the tile (warp-striped; a key's peers with the same
//                  digit from nine ballots, its rank by popc), the tile's per-digit counts
//                  published and each digit's exclusive prefix over earlier tiles found
//                  by a decoupled look-back (256 digits in parallel, a window of
//                  GT_SORT_LB earlier tiles per step, every wait bounded), a local sort in
//                  shared memory, then coalesced writes of each digit run
//                  (reads and writes 12 B/key; 4 B of status per digit and tile: two flag
//                  bits, aggregate or inclusive prefix, and a 30-bit count; every pass has
//                  its own status rows, all cleared once per sort)
// HBM-bound: ~25 B per key per pass.
#include <mutex>

#include "gt_internal.cuh"

namespace {

#ifndef GT_SORT_ST
#define GT_SORT_ST 512
#endif
#ifndef GT_SORT_IPT
#define GT_SORT_IPT 8
#endif
#ifndef GT_SORT_MINB
#define GT_SORT_MINB 3
#endif
#ifndef GT_SORT_LB
#define GT_SORT_LB 8               // earlier tiles read per look-back step
#endif
constexpr int RB = 8;              // digit bits
constexpr int R = 1 << RB;         // digits
constexpr int HT = R;              // threads of the histogram and digit-base kernels
constexpr int ST = GT_SORT_ST;     // threads per tile (the first R of them also own one digit each)
constexpr int IPT = GT_SORT_IPT;   // keys per thread
constexpr int TILE = ST * IPT;     // keys per tile
constexpr int NW = ST / 32;
constexpr int PASSES = 8;          // 64 / RB (bit 63 is always 0; the last pass is cheap)
constexpr uint32_t ST_AGG = 1u << 30;   // status word: the tile's own count of the digit
constexpr uint32_t ST_PRE = 2u << 30;   // status word: the inclusive count over tiles 0..t
constexpr uint32_t ST_VAL = ST_AGG - 1u;
constexpr size_t SCATTER_SMEM = TILE * sizeof(unsigned long long) + TILE * sizeof(uint32_t) +
                                (NW * R + 2 * R + NW + 1) * sizeof(uint32_t);
static_assert(ST >= R && ST % 32 == 0, "one thread per digit in the per-tile scans");

__global__ __launch_bounds__(HT) void k_hist_all(long long n, const unsigned long long *__restrict__ key,
                                                 uint32_t *__restrict__ hist /* PASSES x R */) {
    __shared__ uint32_t h[PASSES][R];
    for (int p = 0; p < PASSES; p++) h[p][threadIdx.x] = 0;
    __syncthreads();
    // the keys of a tree rebuild arrive nearly sorted (the particles are still in the
    // previous key order), so a warp's 32 neighbouring keys often share their high digits:
    // such a digit is counted once for the whole warp, the others by one atomic per lane
    for (long long i0 = (long long)blockIdx.x * HT; i0 < n; i0 += (long long)gridDim.x * HT) {
        const long long i = i0 + threadIdx.x;
        const bool ok = i < n;
        const unsigned long long k = ok ? key[i] : 0ull;
        const bool full = __all_sync(0xffffffffu, ok);
#pragma unroll
        for (int p = 0; p < PASSES; p++) {
            const unsigned int d = (unsigned int)((k >> (p * RB)) & (R - 1));
            const unsigned int d0 = __shfl_sync(0xffffffffu, d, 0);
            if (full && __all_sync(0xffffffffu, d == d0)) {
                if ((threadIdx.x & 31) == 0) atomicAdd(&h[p][d], 32u);
            } else if (ok) {
                atomicAdd(&h[p][d], 1u);
            }
        }
    }
    __syncthreads();
    for (int p = 0; p < PASSES; p++)
        if (h[p][threadIdx.x]) atomicAdd(&hist[p * R + threadIdx.x], h[p][threadIdx.x]);
}

// one block: digit starts of every pass; also resets the tile tickets
__global__ __launch_bounds__(HT) void k_digit_bases(const uint32_t *__restrict__ hist,
                                                    uint32_t *__restrict__ base, DevCtl *ctl) {
    __shared__ uint32_t tmp[HT / 32 + 1];
    for (int p = 0; p < PASSES; p++) {
        uint32_t tot;
        const uint32_t b = block_excl_scan<HT>(hist[p * R + threadIdx.x], &tot, tmp);
        base[p * R + threadIdx.x] = b;
    }
    if (threadIdx.x < PASSES) ctl->sort_ticket[threadIdx.x] = 0;
}

// Look-back of one digit: the count of digit d in all tiles before `tile`.  The status
// word of tile t, digit d sits at status[t * R + d], so the 256 threads of a tile read one
// contiguous row per predecessor; each step reads a window of LB rows at once and adds
// counts back to the first tile whose inclusive prefix is published.
__device__ __forceinline__ uint32_t lookback_digit(const uint32_t *status, int tile, int d, DevCtl *ctl) {
    constexpr int LB = GT_SORT_LB;
    uint32_t excl = 0;
    int t = tile - 1;
    unsigned int spins = 0;
    const unsigned int limit = gt_spin_limit(ctl);
    while (t >= 0) {
        uint32_t sv[LB];
#pragma unroll
        for (int j = 0; j < LB; j++)
            sv[j] = t - j >= 0 ? *((const volatile uint32_t *)&status[(size_t)(t - j) * R + d]) : ST_PRE;
        int used = 0;
        bool done = false, stalled = false;
#pragma unroll
        for (int j = 0; j < LB; j++) {
            if (done || stalled) continue;
            if (sv[j] & ST_PRE) {
                excl += sv[j] & ST_VAL;
                done = true;
            } else if (sv[j] & ST_AGG) {
                excl += sv[j] & ST_VAL;
                used = j + 1;
            } else {
                stalled = true;
            }
        }
        if (done) break;
        t -= used;
        if (stalled) {
            if (++spins > limit) {
                gt_set_error(ctl, GT_ETIMEOUT, GTK_SORT);
                break;
            }
            __nanosleep(32);
        }
    }
    return excl;
}

__global__ __launch_bounds__(ST, GT_SORT_MINB) void k_onesweep(long long n, int pass,
                                                 const unsigned long long *__restrict__ kin,
                                                 const uint32_t *__restrict__ vin,
                                                 unsigned long long *__restrict__ kout,
                                                 uint32_t *__restrict__ vout,
                                                 const uint32_t *__restrict__ digit_base,
                                                 uint32_t *status /* this pass: ntiles x R */, int ntiles,
                                                 DevCtl *ctl) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *skey = (unsigned long long *)smraw;
    uint32_t *sval = (uint32_t *)(skey + TILE);
    uint32_t *wcnt = sval + TILE;     // NW x R: per-warp digit counts, then offsets
    uint32_t *dstart = wcnt + NW * R; // R: tile-local start of every digit
    uint32_t *gbase = dstart + R;     // R: global slot of every digit's first key in this tile
    uint32_t *scantmp = gbase + R;    // NW + 1
    __shared__ uint32_t tile_sh;
    const int shift = pass * RB;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) tile_sh = atomicAdd(&ctl->sort_ticket[pass], 1u);
    for (int k = threadIdx.x; k < NW * R; k += ST) wcnt[k] = 0;
    __syncthreads();
    const int tile = (int)tile_sh;
    if (tile >= ntiles) return;

    // warp w owns keys [base, base + 32*IPT) of the tile, item j of lane l is base + 32 j + l:
    // visiting j in order and lanes in order visits the keys in index order (stability)
    const long long base = (long long)tile * TILE + w * (32 * IPT);
    unsigned long long k[IPT];
    uint32_t v[IPT], loc[IPT];
#pragma unroll
    for (int j = 0; j < IPT; j++) {
        const long long i = base + j * 32 + lane;
        k[j] = i < n ? kin[i] : 0ull;
        v[j] = i < n ? vin[i] : 0u;
    }
    const unsigned int lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < IPT; j++) {
        const bool ok = base + j * 32 + lane < n;
        const unsigned int d = ok ? (unsigned int)((k[j] >> shift) & (R - 1)) : (unsigned int)R;
        unsigned int peers = 0xffffffffu;  // lanes with the same digit (bit 8: past the end)
#pragma unroll
        for (int b = 0; b <= RB; b++) {
            const unsigned int bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
        const unsigned int rank = __popc(peers & lt);
        unsigned int prev = 0;
        if (ok) prev = wcnt[w * R + d];
        __syncwarp();
        if (ok && rank == 0) wcnt[w * R + d] = prev + __popc(peers);
        __syncwarp();
        loc[j] = prev + rank;
    }
    __syncthreads();
    // thread d < R: exclusive offsets of the warps for digit d, the tile's count of digit d
    const int d = threadIdx.x;
    const bool dig = d < R;
    uint32_t cnt = 0;
    if (dig)
        for (int ww = 0; ww < NW; ww++) {
            const uint32_t t = wcnt[ww * R + d];
            wcnt[ww * R + d] = cnt;
            cnt += t;
        }
    // publish this tile's count of digit d as early as possible
    uint32_t *own = status + (size_t)tile * R + (dig ? d : 0);
    if (dig) *((volatile uint32_t *)own) = (tile == 0 ? ST_PRE : ST_AGG) | cnt;
    uint32_t total;
    const uint32_t ds0 = block_excl_scan<ST>(cnt, &total, scantmp);
    if (dig) dstart[d] = ds0;
    __syncthreads();
    // local sort by digit in shared memory (stable: warp offset + rank inside the warp)
#pragma unroll
    for (int j = 0; j < IPT; j++) {
        const bool ok = base + j * 32 + lane < n;
        if (ok) {
            const unsigned int dj = (unsigned int)((k[j] >> shift) & (R - 1));
            const uint32_t pos = dstart[dj] + wcnt[w * R + dj] + loc[j];
            skey[pos] = k[j];
            sval[pos] = v[j];
        }
    }
    // count of digit d in all earlier tiles, then this tile's inclusive prefix
    if (dig) {
        uint32_t excl = 0;
        if (tile > 0) {
            excl = lookback_digit(status, tile, d, ctl);
            *((volatile uint32_t *)own) = ST_PRE | (excl + cnt);
        }
        gbase[d] = digit_base[pass * R + d] + excl - dstart[d];
    }
    __syncthreads();
    const long long rem = n - (long long)tile * TILE;
    const int m = rem < TILE ? (int)rem : TILE;
    for (int p = threadIdx.x; p < m; p += ST) {
        const unsigned long long kk = skey[p];
        const unsigned int dk = (unsigned int)((kk >> shift) & (R - 1));
        const uint32_t g = gbase[dk] + (uint32_t)p;
        kout[g] = kk;
        vout[g] = sval[p];
    }
}

}  // namespace

int gt_sort_tiles(int64_t n) { return (int)((n + TILE - 1) / TILE); }

size_t gt_sort_scratch_bytes(int64_t n) {
    // look-back status of every pass (PASSES x tiles x R x 4 B)
    return (size_t)PASSES * R * (size_t)(gt_sort_tiles(n) > 0 ? gt_sort_tiles(n) : 1) * sizeof(uint32_t);
}

void gt_sort_init() {
    cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SCATTER_SMEM);
}

void gt_launch_sort(SortBufs &b, int64_t n, DevCtl *ctl, cudaStream_t st) {
    if (n <= 1) return;
    const int ntiles = gt_sort_tiles(n);
    cudaMemsetAsync(b.hist, 0, PASSES * R * sizeof(uint32_t), st);
    cudaMemsetAsync(b.status, 0, (size_t)PASSES * R * ntiles * sizeof(uint32_t), st);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = (n + HT - 1) / HT;
    { k_hist_all<<<(unsigned)(blocks < nsm * 8 ? blocks : nsm * 8), HT, 0, st>>>(n, (const unsigned long long *)b.key[0], b.hist); gt_note_launches(1); }
    { k_digit_bases<<<1, HT, 0, st>>>(b.hist, b.digit_base, ctl); gt_note_launches(1); }
    for (int p = 0; p < PASSES; p++) {
        const int src = p & 1, dst = src ^ 1;
        { k_onesweep<<<ntiles, ST, SCATTER_SMEM, st>>>(n, p, (const unsigned long long *)b.key[src], b.val[src],
                                                       (unsigned long long *)b.key[dst], b.val[dst], b.digit_base,
                                                       b.status + (size_t)p * R * ntiles, ntiles, ctl);
          gt_note_launches(1); }
    }
}

// ---- sort without allocation (gt_sort_pairs_noalloc) -----------------------------
// All scratch of one sort of up to GT_NOALLOC_SORT_MAX pairs lives in this array:
// [control block | alternate keys | alternate values | look-back status | digit
// histograms | digit bases].  Host code must not use the symbol as an address: the device
// address is looked up once per device below.
namespace {

constexpr size_t NA_ALIGN = 256;
constexpr size_t na_up(size_t b) { return (b + NA_ALIGN - 1) / NA_ALIGN * NA_ALIGN; }
constexpr size_t NA_TILES = (GT_NOALLOC_SORT_MAX + TILE - 1) / TILE;
constexpr size_t NA_OFF_KEY = na_up(sizeof(DevCtl));
constexpr size_t NA_OFF_VAL = NA_OFF_KEY + na_up((size_t)GT_NOALLOC_SORT_MAX * sizeof(unsigned long long));
constexpr size_t NA_OFF_STATUS = NA_OFF_VAL + na_up((size_t)GT_NOALLOC_SORT_MAX * sizeof(uint32_t));
constexpr size_t NA_OFF_HIST = NA_OFF_STATUS + na_up(PASSES * R * NA_TILES * sizeof(uint32_t));
constexpr size_t NA_OFF_BASE = NA_OFF_HIST + na_up(PASSES * R * sizeof(uint32_t));
constexpr size_t NA_BYTES = NA_OFF_BASE + na_up(PASSES * R * sizeof(uint32_t));

__device__ __align__(256) unsigned char g_noalloc_sort_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 256;
std::mutex g_na_mu;
char *g_na_addr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
int noalloc_scratch(char **out, bool *first_use) {
    *first_use = false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GT_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return GT_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_sort_scratch) != cudaSuccess || !p) return GT_ECUDA;
        gt_sort_init();  // the sort kernel's shared-memory limit, on this device
        g_na_addr[dev] = (char *)p;
        *first_use = true;
    }
    *out = g_na_addr[dev];
    return GT_OK;
}

}  // namespace

extern "C" int gt_sort_pairs_noalloc(uint64_t *d_keys, uint32_t *d_vals, int64_t n, gt_stream stream) {
    if (n < 0 || (n > 0 && (!d_keys || !d_vals))) return GT_EINVAL;
    if (n > GT_NOALLOC_SORT_MAX) return GT_EINVAL;  // larger than the static scratch
    char *base = nullptr;
    bool first_use = false;
    const int rc = noalloc_scratch(&base, &first_use);
    if (rc != GT_OK) return rc;
    if (n <= 1) return GT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DevCtl *ctl = (DevCtl *)base;
    // the histograms and the look-back status words are cleared by the sort itself; the
    // control block (tickets, error word) starts at zero once, on the first call on a
    // device, after which every call leaves it consistent for the next
    if (first_use) {
        if (cudaMemsetAsync(ctl, 0, sizeof(DevCtl), st) != cudaSuccess) return GT_ECUDA;
    }
    SortBufs b;
    b.key[0] = d_keys;
    b.val[0] = d_vals;
    b.key[1] = (uint64_t *)(base + NA_OFF_KEY);
    b.val[1] = (uint32_t *)(base + NA_OFF_VAL);
    b.status = (uint32_t *)(base + NA_OFF_STATUS);
    b.hist = (uint32_t *)(base + NA_OFF_HIST);
    b.digit_base = (uint32_t *)(base + NA_OFF_BASE);
    gt_launch_sort(b, n, ctl, st);  // an even number of passes leaves the result in d_keys/d_vals
    return cudaGetLastError() == cudaSuccess ? GT_OK : GT_ECUDA;
}

extern "C" int gt_sort_noalloc_status(gt_stream stream) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GT_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return GT_EINVAL;
    char *base;
    {
        std::lock_guard<std::mutex> lock(g_na_mu);
        base = g_na_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GT_ECUDA;
    if (!base) return GT_OK;  // no sort has run on this device
    DevCtl *ctl = (DevCtl *)base;
    int err = 0;
    if (cudaMemcpyAsync(&err, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GT_ECUDA;
    if (err && (cudaMemsetAsync(&ctl->err, 0, 2 * sizeof(int), st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess))
        return GT_ECUDA;
    return err;
}
