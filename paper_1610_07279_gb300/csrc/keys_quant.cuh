// Exact integer evaluation of the key quantisation q = floor(RN(RN(x - xmin) * scale))
// (Sec. 2.1: positions mapped onto the 2^21 grid of the bounding cube), where x, xmin
// are FP32, the difference and the product are rounded to nearest-even in FP64, and
// scale is a normal FP64 number.  Both roundings are carried out on integers: the
// difference exactly in 64 bits, the product exactly in 128 bits, each then rounded to
// 53 significant bits -- the same result as the FP64 instructions, without the FP64
// pipe (slow on this GPU).  Callers take the FP64 route for the rare operands outside
// the handled range (see quantise_exact).
#pragma once

#include <stdint.h>
#include <string.h>

__host__ __device__ __forceinline__ int gtq_clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

__host__ __device__ __forceinline__ unsigned long long gtq_mulhi64(unsigned long long a, unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ uint32_t gtq_bits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}

// v (bit length nb > 53) rounded to nearest-even at bit r = nb - 53: the kept high
// part (at most 2^53), to be scaled by 2^r
__host__ __device__ __forceinline__ unsigned long long gtq_rne64(unsigned long long v, int r) {
    const unsigned long long kept = v >> r, rem = v & ((1ull << r) - 1ull), half = 1ull << (r - 1);
    return kept + ((rem > half || (rem == half && (kept & 1ull))) ? 1ull : 0ull);
}

// On success *q = min(floor(RN(RN(x - xmin) * scale)), qmax) and true.  Returns false
// for operands it does not handle: a non-finite x or xmin, x < xmin, the two
// exponents more than 38 apart, or a scale that is not a normal number.
__host__ __device__ __forceinline__ bool quantise_exact(float x, float xmin, unsigned long long scale_bits,
                                                       unsigned long long qmax, unsigned long long *q) {
    const uint32_t bx = gtq_bits(x), by = gtq_bits(xmin);
    const int ex8 = (int)((bx >> 23) & 0xffu), ey8 = (int)((by >> 23) & 0xffu);
    const int es11 = (int)((scale_bits >> 52) & 0x7ffu);
    if (ex8 == 0xff || ey8 == 0xff || es11 == 0 || es11 == 0x7ff) return false;
    // x = mx 2^ex, xmin = my 2^ey with integer significands (subnormals: no hidden bit)
    const long long mx = (long long)((bx & 0x7fffffu) | (ex8 ? 0x800000u : 0u));
    const long long my = (long long)((by & 0x7fffffu) | (ey8 ? 0x800000u : 0u));
    int ex = (ex8 ? ex8 : 1) - 150, ey = (ey8 ? ey8 : 1) - 150;
    if (mx == 0) ex = ey;  // a zero takes the other operand's scale
    if (my == 0) ey = ex;
    const int e0 = ex < ey ? ex : ey;
    if (ex - e0 > 38 || ey - e0 > 38) return false;
    long long X = mx << (ex - e0), Y = my << (ey - e0);  // both below 2^62
    if (bx >> 31) X = -X;
    if (by >> 31) Y = -Y;
    const long long D = X - Y;  // x - xmin = D 2^e0, exactly
    if (D < 0) return false;
    if (D == 0) {
        *q = 0;
        return true;
    }
    // RN(x - xmin) = dm 2^ed
    unsigned long long dm = (unsigned long long)D;
    int ed = e0;
    int nb = 64 - gtq_clz64(dm);
    if (nb > 53) {
        dm = gtq_rne64(dm, nb - 53);
        ed += nb - 53;
    }
    // the product with scale = sm 2^es, exact in 128 bits, then rounded to 53 bits
    const unsigned long long sm = (scale_bits & ((1ull << 52) - 1ull)) | (1ull << 52);
    int e = ed + es11 - 1075;
    const unsigned long long lo = dm * sm, hi = gtq_mulhi64(dm, sm);
    nb = hi ? 128 - gtq_clz64(hi) : 64 - gtq_clz64(lo);
    unsigned long long m = lo;  // the rounded product is m 2^e
    if (nb > 53) {
        const int r = nb - 53;  // 1 .. 54
        const unsigned long long kept = r < 64 ? ((lo >> r) | (hi << (64 - r))) : (hi >> (r - 64));
        const unsigned long long rem = lo & ((1ull << r) - 1ull), half = 1ull << (r - 1);
        m = kept + ((rem > half || (rem == half && (kept & 1ull))) ? 1ull : 0ull);
        e += r;
    }
    // floor(m 2^e), clamped
    unsigned long long v;
    if (e >= 0)
        v = (e > 63 || m > (0xffffffffffffffffull >> e)) ? qmax : (m << e);
    else
        v = -e >= 64 ? 0ull : (m >> -e);
    *q = v < qmax ? v : qmax;
    return true;
}
