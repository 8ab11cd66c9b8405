// Step A1: bounding cube and 63-bit Morton keys (Sec. 2.1; Morton key layout of
// Appendix A: every 3-bit digit is (x, y, z) with x the most significant bit).
//
// The bounding box reads 16 B per particle, the key pass reads 16 B and writes 12 B
// (key + index); the key pass is bound by the exact quantisation's integer work, split
// with the FP64 pipe (one axis there, two on the integer pipe).
#include <float.h>

#include "gt_internal.cuh"
#include "keys_quant.cuh"

namespace {

constexpr int BBOX_THREADS = 256;

__global__ __launch_bounds__(BBOX_THREADS) void k_bbox_partial(const float4 *__restrict__ posm,
                                                               long long n,
                                                               float *__restrict__ partial) {
    float mn0 = FLT_MAX, mn1 = FLT_MAX, mn2 = FLT_MAX;
    float mx0 = -FLT_MAX, mx1 = -FLT_MAX, mx2 = -FLT_MAX;
    for (long long i = blockIdx.x * (long long)BBOX_THREADS + threadIdx.x; i < n;
         i += (long long)gridDim.x * BBOX_THREADS) {
        const float4 p = posm[i];
        mn0 = fminf(mn0, p.x); mx0 = fmaxf(mx0, p.x);
        mn1 = fminf(mn1, p.y); mx1 = fmaxf(mx1, p.y);
        mn2 = fminf(mn2, p.z); mx2 = fmaxf(mx2, p.z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn0 = fminf(mn0, __shfl_xor_sync(0xffffffffu, mn0, o));
        mn1 = fminf(mn1, __shfl_xor_sync(0xffffffffu, mn1, o));
        mn2 = fminf(mn2, __shfl_xor_sync(0xffffffffu, mn2, o));
        mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
        mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
        mx2 = fmaxf(mx2, __shfl_xor_sync(0xffffffffu, mx2, o));
    }
    __shared__ float s[BBOX_THREADS / 32][6];
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) {
        s[w][0] = mn0; s[w][1] = mn1; s[w][2] = mn2;
        s[w][3] = mx0; s[w][4] = mx1; s[w][5] = mx2;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = s[0][threadIdx.x];
        for (int k = 1; k < BBOX_THREADS / 32; k++)
            v = threadIdx.x < 3 ? fminf(v, s[k][threadIdx.x]) : fmaxf(v, s[k][threadIdx.x]);
        partial[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

__global__ void k_bbox_final(const float *__restrict__ partial, int nblk, long long n, DevCtl *ctl) {
    // one warp: reduce the per-block extrema, then the cube of Sec. 2.1's keys
    float v[6];
    for (int a = 0; a < 6; a++) v[a] = a < 3 ? FLT_MAX : -FLT_MAX;
    for (int b = lane_id(); b < nblk; b += 32)
        for (int a = 0; a < 6; a++)
            v[a] = a < 3 ? fminf(v[a], partial[b * 6 + a]) : fmaxf(v[a], partial[b * 6 + a]);
    for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 6; a++) {
            const float t = __shfl_xor_sync(0xffffffffu, v[a], o);
            v[a] = a < 3 ? fminf(v[a], t) : fmaxf(v[a], t);
        }
    if (lane_id() == 0) {
        double side = 0.0;
        if (n > 0)
            for (int a = 0; a < 3; a++) {
                const double ext = __dsub_rn((double)v[a + 3], (double)v[a]);
                if (ext > side) side = ext;
            }
        for (int a = 0; a < 3; a++) ctl->bbox_min[a] = n > 0 ? v[a] : 0.0f;
        ctl->side = side;
        ctl->scale = side > 0.0 ? __ddiv_rn((double)(1u << GT_KEY_LEVELS), side) : 0.0;
    }
}

// Spread the low 21 bits of v so that bit b lands on bit 3b.
__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x001f00000000ffffull;
    v = (v | (v << 16)) & 0x001f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

constexpr unsigned long long QMAX = (1ull << GT_KEY_LEVELS) - 1ull;

__device__ __forceinline__ unsigned long long quantise(float x, float xmin, double scale) {
    // floor((x - xmin) * 2^21/side) with FP64 roundings (RN difference, RN product, then
    // the floor), clamped to 2^21 - 1: in integer arithmetic (keys_quant.cuh), or for the
    // rare operands it does not take, on the FP64 pipe -- x widened exactly on the
    // integer pipe, the floor the round-down conversion (the product is >= 0).
    unsigned long long q;
    if (quantise_exact(x, xmin, (unsigned long long)__double_as_longlong(scale), QMAX, &q)) return q;
    q = __double2ull_rd(__dmul_rn(__dsub_rn(f2d(x), f2d(xmin)), scale));
    return q < QMAX ? q : QMAX;
}

// The same quantisation with the two roundings on the FP64 pipe (x and xmin widened
// exactly on the integer pipe; the floor of the non-negative product taken from its
// bits).  k_keys runs one axis this way and two through quantise(): the FP64 pipe is
// narrow on this GPU, the integer pipe bounds the pass, so the two share the work.
__device__ __forceinline__ unsigned long long quantise_fp64(float x, float xmin, double scale) {
    const double p = __dmul_rn(__dsub_rn(f2d(x), f2d(xmin)), scale);
    const unsigned long long b = (unsigned long long)__double_as_longlong(p);
    if (b >> 63) return 0ull;                    // negative (x below xmin: not produced by the bounding box)
    const int e = (int)(b >> 52) - 1023;         // p = 1.f 2^e
    if (e < 0) return 0ull;                      // p < 1, zero included
    if (e >= GT_KEY_LEVELS) return QMAX;         // p >= 2^21 (and inf, nan)
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    return m >> (52 - e);
}

// Peano-Hilbert order (Sec. 2.1, App. A), Skilling's transpose method on the three
// 21-bit integers: the rotations and reflections are undone from the top bit down, a
// Gray code runs across the axes, and the transposed bits are interleaved like a Morton
// key (axis 0 the most significant of every triplet).
__device__ __forceinline__ void hilbert_transpose(uint32_t &x0, uint32_t &x1, uint32_t &x2) {
#pragma unroll 4
    for (uint32_t q = 1u << (GT_KEY_LEVELS - 1); q > 1u; q >>= 1) {
        const uint32_t p = q - 1u;
        if (x0 & q) x0 ^= p;  // axis 0 against itself: a reflection or nothing
        if (x1 & q) { x0 ^= p; } else { const uint32_t t = (x0 ^ x1) & p; x0 ^= t; x1 ^= t; }
        if (x2 & q) { x0 ^= p; } else { const uint32_t t = (x0 ^ x2) & p; x0 ^= t; x2 ^= t; }
    }
    x1 ^= x0;
    x2 ^= x1;
    uint32_t t = 0u;
#pragma unroll 4
    for (uint32_t q = 1u << (GT_KEY_LEVELS - 1); q > 1u; q >>= 1)
        if (x2 & q) t ^= q - 1u;
    x0 ^= t;
    x1 ^= t;
    x2 ^= t;
}

__global__ __launch_bounds__(256) void k_keys(const float4 *__restrict__ posm, long long n,
                                              const DevCtl *__restrict__ ctl, int curve,
                                              unsigned long long *__restrict__ key,
                                              uint32_t *__restrict__ idx) {
    const long long i = blockIdx.x * 256ll + threadIdx.x;
    if (i >= n) return;
    const double side = ctl->side, scale = ctl->scale;
    unsigned long long k = 0;
    if (side > 0.0) {
        const float4 p = posm[i];
        const unsigned long long qx = quantise_fp64(p.x, ctl->bbox_min[0], scale);
        const unsigned long long qy = quantise(p.y, ctl->bbox_min[1], scale);
        const unsigned long long qz = quantise(p.z, ctl->bbox_min[2], scale);
        if (curve == GT_KEY_HILBERT) {
            uint32_t x0 = (uint32_t)qx, x1 = (uint32_t)qy, x2 = (uint32_t)qz;
            hilbert_transpose(x0, x1, x2);
            k = (spread3(x0) << 2) | (spread3(x1) << 1) | spread3(x2);
        } else {
            k = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
        }
    }
    key[i] = k;
    idx[i] = (uint32_t)i;
}

}  // namespace

void gt_launch_bbox(const float4 *posm, int64_t n, float *partial, int nblk, DevCtl *ctl,
                    cudaStream_t st) {
    { k_bbox_partial<<<nblk, BBOX_THREADS, 0, st>>>(posm, n, partial); gt_note_launches(1); }
    { k_bbox_final<<<1, 32, 0, st>>>(partial, nblk, n, ctl); gt_note_launches(1); }
}

void gt_launch_keys(const float4 *posm, int64_t n, const DevCtl *ctl, int curve, uint64_t *key, uint32_t *idx,
                    cudaStream_t st) {
    if (n <= 0) return;
    { k_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(posm, n, ctl, curve, (unsigned long long *)key, idx); gt_note_launches(1); }
}
