// Host check of the key quantisation's integer evaluation (keys_quant.cuh) against the
// same expression evaluated with FP64 arithmetic: floor((double)(x) - (double)(xmin)) *
// scale) on random and adversarial operands (wide exponent ranges, neighbours one ulp
// apart, subnormals, zeros, products with few significant bits, i.e. rounding ties).
// Prints the counts and exits non-zero on a mismatch.
#define __host__
#define __device__
#define __forceinline__ inline
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <random>
#include "keys_quant.cuh"
static unsigned long long ref(float x, float xmin, double scale, unsigned long long qmax) {
    volatile double d = (double)x - (double)xmin;
    volatile double t = d * scale;
    double f = std::floor(t);
    unsigned long long q = f >= 18446744073709551616.0 ? ~0ull : (unsigned long long)f;
    return q < qmax ? q : qmax;
}
static float rf(std::mt19937_64 &g, int emin, int emax) {
    std::uniform_int_distribution<int> E(emin, emax);
    uint32_t m = (uint32_t)(g() & 0x7fffff);
    int e = E(g);
    float v = std::ldexp((float)(m | 0x800000) / 8388608.0f, e);
    if (g() & 1) v = -v;
    if ((g() & 63) == 0) v = 0.0f;
    if ((g() & 255) == 0) { uint32_t b = (uint32_t)(g() & 0x807fffff); memcpy(&v, &b, 4); }  // subnormal
    return v;
}
int main() {
    std::mt19937_64 g(12345);
    const unsigned long long QMAX = (1ull << 21) - 1;
    long long n = 0, handled = 0, bad = 0;
    for (long long it = 0; it < 3000000; it++) {
        int mode = (int)(it % 5);
        float x, xmin;
        if (mode == 0) { x = rf(g, -30, 30); xmin = rf(g, -30, 30); }
        else if (mode == 1) { xmin = rf(g, -3, 9); x = xmin + std::ldexp((float)(g() % 1000000) / 1e6f, (int)(g() % 12)); }
        else if (mode == 2) { x = rf(g, -149, 127); xmin = rf(g, -149, 127); }
        else if (mode == 3) { xmin = -200.0f + (float)(g() % 1000) * 0.01f; x = rf(g, -40, 8); }
        else { xmin = rf(g, -2, 2); x = std::nextafterf(xmin, 1e30f); for (int k = (int)(g() % 8); k > 0; k--) x = std::nextafterf(x, 1e30f); }
        if (x < xmin) { float t = x; x = xmin; xmin = t; }
        if (!std::isfinite(x) || !std::isfinite(xmin)) continue;
        double side;
        int sm = (int)(g() % 4);
        if (sm == 0) side = (double)x - (double)xmin;
        else if (sm == 1) side = std::ldexp(1.0 + (double)(g() >> 11) / 9007199254740992.0, (int)(g() % 60) - 30);
        else if (sm == 2) side = ((double)x - (double)xmin) * (1.0 + (double)(g() % 1000) / 1000.0);
        else side = std::ldexp(1.0, (int)(g() % 40) - 20) * 3.0;
        if (!(side > 0.0)) continue;
        double scale = 2097152.0 / side;
        unsigned long long sb; memcpy(&sb, &scale, 8);
        unsigned long long q = 0;
        n++;
        if (quantise_exact(x, xmin, sb, QMAX, &q)) {
            handled++;
            unsigned long long r = ref(x, xmin, scale, QMAX);
            if (q != r) { if (bad < 10) printf("MISMATCH x=%a xmin=%a scale=%a q=%llu ref=%llu\n", x, xmin, scale, q, r); bad++; }
        }
    }
    // products with few bits: ties at the rounding position
    for (long long it = 0; it < 1000000; it++) {
        float xmin = 0.0f;
        uint32_t m = (uint32_t)(g() & 0xffffff) | 1u;
        float x = std::ldexp((float)m, (int)(g() % 40) - 30);
        double scale = std::ldexp((double)((g() >> 11) | 1ull), -(int)(g() % 60) - 10);
        unsigned long long sb; memcpy(&sb, &scale, 8);
        unsigned long long q = 0;
        n++;
        if (quantise_exact(x, xmin, sb, ~0ull >> 1, &q)) {
            handled++;
            unsigned long long r = ref(x, xmin, scale, ~0ull >> 1);
            if (q != r) { if (bad < 20) printf("MISMATCH2 x=%a scale=%a q=%llu ref=%llu\n", x, scale, q, r); bad++; }
        }
    }
    long long ties = 0;
    for (long long it = 0; it < 1000000; it++) {
        uint32_t m = (uint32_t)(g() & 0xffffff) | 0x800000u;
        float x = std::ldexp((float)m, (int)(g() % 20) - 30);
        const int sbits = 29 + (int)(g() % 4);  // product of 53..57 bits: ties at the rounding bit
        double scale = std::ldexp((double)((g() >> (64 - sbits)) | (1ull << (sbits - 1)) | 1ull), -(int)(g() % 30) - 5);
        unsigned long long sb; memcpy(&sb, &scale, 8);
        unsigned long long q = 0;
        n++;
        if (quantise_exact(x, 0.0f, sb, ~0ull >> 1, &q)) {
            handled++;
            unsigned long long r = ref(x, 0.0f, scale, ~0ull >> 1);
            volatile double t = (double)x * scale; double e = (double)x; long double ex = (long double)e * (long double)scale;
            if ((long double)t != ex) ties++;
            if (q != r) { if (bad < 30) printf("MISMATCH3 x=%a scale=%a q=%llu ref=%llu\n", x, scale, q, r); bad++; }
        }
    }
    printf("inexact products in the third set: %lld\n", ties);
    printf("cases %lld handled %lld mismatches %lld\n", n, handled, bad);
    return bad != 0;
}
