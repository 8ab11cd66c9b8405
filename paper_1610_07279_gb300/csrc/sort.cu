// Step A2: stable LSD radix sort of (63-bit key, 32-bit index) pairs (Sec. 2.1: the
// particles are sorted by their space-filling key with a library radix sort).
//
// Eight passes of 8-bit digits.  Each pass runs three kernels:
//   tile_hist   per 4096-key tile, a histogram of the pass digit     (reads 8 B/key)
//   digit_scan  per digit, an exclusive scan over tiles; the last block to finish
//               turns the digit totals into digit bases (no waiting)
//   scatter     per tile, a stable rank of every key inside the tile (warp-striped
//               match/popc ranking), a local sort in shared memory, then coalesced
//               writes of each digit run to its global slot       (reads and writes 12 B/key)
// HBM-bound: 32 B per key per pass plus the small tile histograms.
#include <mutex>

#include "gt_internal.cuh"

namespace {

constexpr int ST = 256;            // threads per tile
constexpr int IPT = 16;            // keys per thread
constexpr int TILE = ST * IPT;     // keys per tile
constexpr int RB = 8;              // digit bits
constexpr int R = 1 << RB;         // digits
constexpr int NW = ST / 32;
constexpr int PASSES = 8;          // 64 / RB (bit 63 is always 0; the last pass is cheap)
constexpr size_t SCATTER_SMEM =
    TILE * sizeof(unsigned long long) + TILE * sizeof(uint32_t) + (NW * R + R + NW + 1) * sizeof(uint32_t);
static_assert(ST == R, "one thread per digit in the per-tile scans");

__global__ __launch_bounds__(ST) void k_tile_hist(long long n, int shift,
                                                  const unsigned long long *__restrict__ key,
                                                  uint32_t *__restrict__ tile_hist, int ntiles) {
    __shared__ uint32_t h[R];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * TILE;
#pragma unroll 4
    for (int j = 0; j < IPT; j++) {
        const long long i = base + j * ST + threadIdx.x;
        const bool ok = i < n;
        const unsigned int d = ok ? (unsigned int)((key[i] >> shift) & (R - 1)) : (unsigned int)R;
        const unsigned int peers = __match_any_sync(0xffffffffu, d);
        if (ok && (peers & lanemask_lt()) == 0) atomicAdd(&h[d], (unsigned int)__popc(peers));
    }
    __syncthreads();
    tile_hist[threadIdx.x * (long long)ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ __launch_bounds__(1024) void k_digit_scan(uint32_t *__restrict__ tile_hist, int ntiles,
                                                     uint32_t *__restrict__ digit_total,
                                                     uint32_t *__restrict__ digit_base, DevCtl *ctl) {
    __shared__ uint32_t tmp[1024 / 32 + 1];
    __shared__ bool last;
    uint32_t *row = tile_hist + (long long)blockIdx.x * ntiles;
    const int per = (ntiles + 1023) / 1024;
    const int t0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int k = 0; k < per; k++)
        if (t0 + k < ntiles) s += row[t0 + k];
    uint32_t total;
    uint32_t run = block_excl_scan<1024>(s, &total, tmp);
    for (int k = 0; k < per; k++)
        if (t0 + k < ntiles) {
            const uint32_t v = row[t0 + k];
            row[t0 + k] = run;
            run += v;
        }
    if (threadIdx.x == 0) {
        digit_total[blockIdx.x] = total;
        __threadfence();
        last = atomicAdd(&ctl->sort_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        const uint32_t v = threadIdx.x < R ? __ldcg(&digit_total[threadIdx.x]) : 0u;
        uint32_t tot;
        const uint32_t b = block_excl_scan<1024>(v, &tot, tmp);
        if (threadIdx.x < R) digit_base[threadIdx.x] = b;
        if (threadIdx.x == 0) ctl->sort_done = 0;
    }
}

__global__ __launch_bounds__(ST) void k_scatter(long long n, int shift,
                                                const unsigned long long *__restrict__ kin,
                                                const uint32_t *__restrict__ vin,
                                                unsigned long long *__restrict__ kout,
                                                uint32_t *__restrict__ vout,
                                                const uint32_t *__restrict__ tile_prefix,
                                                const uint32_t *__restrict__ digit_base, int ntiles) {
    extern __shared__ __align__(16) unsigned char smraw[];
    unsigned long long *skey = (unsigned long long *)smraw;
    uint32_t *sval = (uint32_t *)(skey + TILE);
    uint32_t *wcnt = sval + TILE;     // NW x R: per-warp digit counts, then offsets
    uint32_t *dstart = wcnt + NW * R; // R: tile-local start of every digit
    uint32_t *scantmp = dstart + R;   // NW + 1
    const int tile = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < NW * R; k += ST) wcnt[k] = 0;
    __syncthreads();

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
        const unsigned int peers = __match_any_sync(0xffffffffu, d);
        const unsigned int rank = __popc(peers & lt);
        unsigned int prev = 0;
        if (ok) prev = wcnt[w * R + d];
        __syncwarp();
        if (ok && rank == 0) wcnt[w * R + d] = prev + __popc(peers);
        __syncwarp();
        loc[j] = prev + rank;
    }
    __syncthreads();
    // per digit: exclusive offsets of the warps, then the digit's tile-local start
    uint32_t tot = 0;
    for (int ww = 0; ww < NW; ww++) {
        const uint32_t t = wcnt[ww * R + threadIdx.x];
        wcnt[ww * R + threadIdx.x] = tot;
        tot += t;
    }
    uint32_t total;
    const uint32_t ds = block_excl_scan<ST>(tot, &total, scantmp);
    dstart[threadIdx.x] = ds;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IPT; j++) {
        const bool ok = base + j * 32 + lane < n;
        if (ok) {
            const unsigned int d = (unsigned int)((k[j] >> shift) & (R - 1));
            const uint32_t pos = dstart[d] + wcnt[w * R + d] + loc[j];
            skey[pos] = k[j];
            sval[pos] = v[j];
        }
    }
    __syncthreads();
    const long long rem = n - (long long)tile * TILE;
    const int m = rem < TILE ? (int)rem : TILE;
    for (int p = threadIdx.x; p < m; p += ST) {
        const unsigned long long kk = skey[p];
        const unsigned int d = (unsigned int)((kk >> shift) & (R - 1));
        const uint32_t g = digit_base[d] + tile_prefix[d * (long long)ntiles + tile] + (uint32_t)(p - dstart[d]);
        kout[g] = kk;
        vout[g] = sval[p];
    }
}

}  // namespace

int gt_sort_tiles(int64_t n) { return (int)((n + TILE - 1) / TILE); }

size_t gt_sort_scratch_bytes(int64_t n) {
    return (size_t)R * (size_t)(gt_sort_tiles(n) > 0 ? gt_sort_tiles(n) : 1) * sizeof(uint32_t);
}

void gt_sort_init() {
    cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SCATTER_SMEM);
}

void gt_launch_sort(SortBufs &b, int64_t n, DevCtl *ctl, cudaStream_t st) {
    if (n <= 1) return;
    const int ntiles = gt_sort_tiles(n);
    for (int p = 0; p < PASSES; p++) {
        const int src = p & 1, dst = src ^ 1;
        const int shift = p * RB;
        { k_tile_hist<<<ntiles, ST, 0, st>>>(n, shift, (const unsigned long long *)b.key[src],
                                           b.tile_hist, ntiles); gt_note_launches(1); }
        { k_digit_scan<<<R, 1024, 0, st>>>(b.tile_hist, ntiles, b.digit_total, b.digit_base, ctl); gt_note_launches(1); }
        { k_scatter<<<ntiles, ST, SCATTER_SMEM, st>>>(n, shift, (const unsigned long long *)b.key[src],
                                                    b.val[src], (unsigned long long *)b.key[dst],
                                                    b.val[dst], b.tile_hist, b.digit_base, ntiles); gt_note_launches(1); }
    }
}

// ---- sort without allocation (gt_sort_pairs_noalloc) -----------------------------
// All scratch of one sort of up to GT_NOALLOC_SORT_MAX pairs lives in this array:
// [control block | alternate keys | alternate values | tile histograms | digit bases |
// digit totals].  Host code must not use the symbol as an address: the device
// address is looked up once per device below.
namespace {

constexpr size_t NA_ALIGN = 256;
constexpr size_t na_up(size_t b) { return (b + NA_ALIGN - 1) / NA_ALIGN * NA_ALIGN; }
constexpr size_t NA_TILES = (GT_NOALLOC_SORT_MAX + TILE - 1) / TILE;
constexpr size_t NA_OFF_KEY = na_up(sizeof(DevCtl));
constexpr size_t NA_OFF_VAL = NA_OFF_KEY + na_up((size_t)GT_NOALLOC_SORT_MAX * sizeof(unsigned long long));
constexpr size_t NA_OFF_HIST = NA_OFF_VAL + na_up((size_t)GT_NOALLOC_SORT_MAX * sizeof(uint32_t));
constexpr size_t NA_OFF_BASE = NA_OFF_HIST + na_up(R * NA_TILES * sizeof(uint32_t));
constexpr size_t NA_OFF_TOTAL = NA_OFF_BASE + na_up(R * sizeof(uint32_t));
constexpr size_t NA_BYTES = NA_OFF_TOTAL + na_up(R * sizeof(uint32_t));

__device__ __align__(256) unsigned char g_noalloc_sort_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 256;
std::mutex g_na_mu;
char *g_na_addr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
int noalloc_scratch(char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GT_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return GT_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_sort_scratch) != cudaSuccess || !p) return GT_ECUDA;
        gt_sort_init();  // the scatter kernel's shared-memory limit, on this device
        g_na_addr[dev] = (char *)p;
    }
    *out = g_na_addr[dev];
    return GT_OK;
}

}  // namespace

extern "C" int gt_sort_pairs_noalloc(uint64_t *d_keys, uint32_t *d_vals, int64_t n, gt_stream stream) {
    if (n < 0 || (n > 0 && (!d_keys || !d_vals))) return GT_EINVAL;
    if (n > GT_NOALLOC_SORT_MAX) return GT_EINVAL;  // larger than the static scratch
    char *base = nullptr;
    const int rc = noalloc_scratch(&base);
    if (rc != GT_OK) return rc;
    if (n <= 1) return GT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DevCtl *ctl = (DevCtl *)base;
    // the digit scan's last-block counter must start at zero (a previous call may
    // have been cut short); everything else is fully written before it is read
    if (cudaMemsetAsync(&ctl->sort_done, 0, sizeof(ctl->sort_done), st) != cudaSuccess) return GT_ECUDA;
    SortBufs b;
    b.key[0] = d_keys;
    b.val[0] = d_vals;
    b.key[1] = (uint64_t *)(base + NA_OFF_KEY);
    b.val[1] = (uint32_t *)(base + NA_OFF_VAL);
    b.tile_hist = (uint32_t *)(base + NA_OFF_HIST);
    b.digit_base = (uint32_t *)(base + NA_OFF_BASE);
    b.digit_total = (uint32_t *)(base + NA_OFF_TOTAL);
    gt_launch_sort(b, n, ctl, st);  // an even number of passes leaves the result in d_keys/d_vals
    return cudaGetLastError() == cudaSuccess ? GT_OK : GT_ECUDA;
}
