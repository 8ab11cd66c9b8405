// Step A7: the tree walk for groups of active i-particles (Sec. 2.3) with the
// ij-parallelisation of Sec. 2.5.
//
// One warp walks one group at a time (a persistent grid; groups are taken from an
// atomic counter, so slow groups do not hold a fixed share of the GPU).  A group is a
// range of the active list: the actives of one tree cell (Sec. 2.4 reading) or a run
// of group_max.  Per group:
//   * S lanes per member (Sec. 2.5): fixed, or 32 / (members rounded up to a power of
//     two) so that small groups still fill the warp;
//   * pseudo i-particle: the sphere about the centre of the members' bounding box
//     (Appendix B, "GEO"), the FP32 radius widened by (1 + 2^-20); |a_old| of the
//     group is the smallest of its members';
//   * breadth-first traversal: a ring-buffer queue of cells in a per-warp slice of
//     global memory (when the queue fills up, the newest cells are taken first, i.e.
//     depth-first, which bounds its size; the order of the interactions does not change
//     the set of interactions); 32 queued cells are tested at once, one per lane, with the MAC at
//     distance lambda r_JI (Eqs. 2, 5-7) in FP32 with explicit rounding (so the decision
//     is reproducible); accepted cells join the shared-memory interaction list,
//     rejected cells push their children, rejected leaves copy their particles into the
//     list with asynchronous global-to-shared copies (cp.async), waited for only when the
//     list is flushed -- both spread over the whole warp (a warp prefix sum, then each
//     lane finds the owner of its entry by a binary search over the lanes);
//   * the list is kept as structure of arrays (x, y, z, m), so two consecutive entries
//     load as packed pairs; it is flushed through Eq. (1) whenever it fills: each
//     i-particle is held by S lanes that take every S-th pair of entries on the packed
//     FP32 pipe (f32x2 add, mul and fma: two interactions per instruction; rsqrt on the
//     SFU), the two halves and the S lanes summed at the end (an odd list gets a
//     massless last entry).  The potential is accumulated too; the member's own term
//     -G m_i/eps is removed at the end (Eq. 1 excludes j = i).
// Bound: FP32 ALU (the force loop: 3 FADD, 3 FMUL, 7 FFMA and one MUFU rsqrt per
// interaction); the node records (32 B per cell) stay resident in L2.
#include <math.h>

#include "gt_internal.cuh"

namespace {

#ifndef GT_WALK_MINB
#define GT_WALK_MINB 3            // resident blocks per SM the register budget is sized for
#endif
constexpr int WT = 256;           // threads per block
constexpr int NWARP = WT / 32;
constexpr int LIST_CAP = 384;     // interaction-list entries per warp
constexpr int FLUSH_AT = 256;     // flush once the list holds this many
// Depth-first reserve of the queue: popping the newest 32 cells and pushing at most
// 8 children each grows the queue by <= 224 per tree level, <= ~22 x 256 in all.
constexpr int LIFO_ROOM = 6144;

__device__ __forceinline__ bool mac_accept(int mac, float theta, float dacc_amin, float delta, float G, float cx,
                                           float cy, float cz, float bI, float4 jp, float bJ, float B2) {
    const float dx = __fsub_rn(jp.x, cx);
    const float dy = __fsub_rn(jp.y, cy);
    const float dz = __fsub_rn(jp.z, cz);
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const float r = __fsqrt_rn(r2);
    const float d = (bI < r) ? __fsub_rn(r, bI) : 0.0f;   // lambda r_JI, Eqs. (6)-(7)
    if (mac == GT_MAC_OPENING_ANGLE) return bJ <= __fmul_rn(theta, d);  // Eq. (2)
    if (mac == GT_MAC_MULTIPOLE)  // Warren & Salmon: d >= b/2 + sqrt(b^2/4 + sqrt(3 B_2 / Delta_mul))
        return d >= __fadd_rn(__fmul_rn(0.5f, bJ),
                              __fsqrt_rn(__fadd_rn(__fmul_rn(__fmul_rn(0.25f, bJ), bJ),
                                                   __fsqrt_rn(__fdiv_rn(__fmul_rn(3.0f, B2), delta)))));
    const float d2 = __fmul_rn(d, d);                                   // Eq. (5), raised to the 4th power
    return __fmul_rn(__fmul_rn(d2, d2), dacc_amin) >= __fmul_rn(__fmul_rn(G, jp.w), __fmul_rn(bJ, bJ));
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// 1/sqrt(r2) on the special-function unit; r2 >= eps^2 > 0 is never subnormal, so the
// flush-to-zero form needs no range handling
__device__ __forceinline__ float rsqrt_sfu(float r2) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
    return r;
}

// Two list entries (packed: x = (x_e, x_e+1), ...) against one i-particle (negated
// coordinates nx, ny, nz) on the packed FP32 pipe; the sums keep the two entries' shares
// in their two halves.
__device__ __forceinline__ void interact_pairs(float2 X, float2 Y, float2 Z, float2 W, float2 nx, float2 ny,
                                               float2 nz, float2 e2, float2 &ax, float2 &ay, float2 &az,
                                               float2 &ph) {
    const float2 dx = __fadd2_rn(X, nx), dy = __fadd2_rn(Y, ny), dz = __fadd2_rn(Z, nz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, e2)));
    const float2 rinv = make_float2(rsqrt_sfu(r2.x), rsqrt_sfu(r2.y));
    const float2 mr = __fmul2_rn(W, rinv);
    const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, rinv), rinv);
    ax = __ffma2_rn(mr3, dx, ax);
    ay = __ffma2_rn(mr3, dy, ay);
    az = __ffma2_rn(mr3, dz, az);
    ph = __fadd2_rn(ph, mr);
}

// (value, member) of the extreme member on one axis: the smallest (want_max false) or
// largest value, the lowest member index on ties
__device__ __forceinline__ void warp_arg_ext(float &v, int &m, bool want_max) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int m2 = __shfl_xor_sync(0xffffffffu, m, o);
        const bool take = want_max ? (v2 > v || (v2 == v && m2 < m)) : (v2 < v || (v2 == v && m2 < m));
        if (take) { v = v2; m = m2; }
    }
}

// Centre of Ritter's efficient bounding sphere of the group's members (Appendix B): the
// first diameter joins the extreme members of the axis whose pair is farthest apart; the
// sphere then grows towards the first member outside it (member order) until none is,
// at most cnt times.  FP32, every operation rounded as written.  Member k < 32 is the
// first member of the lane holding slot k (pi), member 32 + l the second of lane l (pi2).
__device__ __forceinline__ void ebs_centre(float4 pi, float4 pi2, bool mine1, bool mine2, int slot, int lane,
                                           int logS, uint32_t cnt, float &cx, float &cy, float &cz) {
    const unsigned FULL = 0xffffffffu;
    const float INF = __int_as_float(0x7f800000);
    auto coord = [](const float4 &p, int a) { return a == 0 ? p.x : (a == 1 ? p.y : p.z); };
    // the member's position, fetched from the lane that holds it
    auto fetch = [&](int m, float &x, float &y, float &z) {
        const bool second = m >= 32;
        const int src = second ? m - 32 : (m << logS);
        const float4 a1 = make_float4(__shfl_sync(FULL, pi.x, src), __shfl_sync(FULL, pi.y, src),
                                      __shfl_sync(FULL, pi.z, src), 0.f);
        const float4 a2 = make_float4(__shfl_sync(FULL, pi2.x, src), __shfl_sync(FULL, pi2.y, src),
                                      __shfl_sync(FULL, pi2.z, src), 0.f);
        x = second ? a2.x : a1.x; y = second ? a2.y : a1.y; z = second ? a2.z : a1.z;
    };
    float bd2 = -1.0f, lx = 0.f, ly = 0.f, lz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
    for (int ax = 0; ax < 3; ax++) {
        float vmin = mine1 ? coord(pi, ax) : INF, vmax = mine1 ? coord(pi, ax) : -INF;
        int mmin = mine1 ? slot : 1 << 20, mmax = mmin;
        if (mine2) {
            const float v2 = coord(pi2, ax);
            if (v2 < vmin) { vmin = v2; mmin = lane + 32; }  // the second member has the larger index
            if (v2 > vmax) { vmax = v2; mmax = lane + 32; }
        }
        warp_arg_ext(vmin, mmin, false);
        warp_arg_ext(vmax, mmax, true);
        float ax0, ay0, az0, ax1, ay1, az1;
        fetch(mmin, ax0, ay0, az0);
        fetch(mmax, ax1, ay1, az1);
        const float dx = __fsub_rn(ax1, ax0), dy = __fsub_rn(ay1, ay0), dz = __fsub_rn(az1, az0);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        if (d2 > bd2) { bd2 = d2; lx = ax0; ly = ay0; lz = az0; hx = ax1; hy = ay1; hz = az1; }
    }
    cx = __fmul_rn(0.5f, __fadd_rn(lx, hx));
    cy = __fmul_rn(0.5f, __fadd_rn(ly, hy));
    cz = __fmul_rn(0.5f, __fadd_rn(lz, hz));
    float r = __fmul_rn(0.5f, __fsqrt_rn(bd2));
    for (uint32_t it = 0; it < cnt; it++) {
        const float r2 = __fmul_rn(r, r);
        auto outside = [&](const float4 &p) {
            const float dx = __fsub_rn(p.x, cx), dy = __fsub_rn(p.y, cy), dz = __fsub_rn(p.z, cz);
            return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) > r2;
        };
        const unsigned b1 = __ballot_sync(FULL, mine1 && outside(pi));
        const unsigned b2 = __ballot_sync(FULL, mine2 && outside(pi2));
        int m;
        if (b1) m = (__ffs(b1) - 1) >> logS;
        else if (b2) m = 32 + __ffs(b2) - 1;
        else break;
        float px, py, pz;
        fetch(m, px, py, pz);
        const float dx = __fsub_rn(px, cx), dy = __fsub_rn(py, cy), dz = __fsub_rn(pz, cz);
        const float d = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
        const float rn = __fmul_rn(0.5f, __fadd_rn(r, d));
        const float f = __fdiv_rn(__fsub_rn(d, rn), d);
        cx = __fadd_rn(cx, __fmul_rn(f, dx));
        cy = __fadd_rn(cy, __fmul_rn(f, dy));
        cz = __fadd_rn(cz, __fmul_rn(f, dz));
        r = rn;
    }
}

// One group g of system a (Sec. 2.3): pseudo i-particle, traversal, force loop.  The
// warp's interaction and MAC-test counts are added to n_inter and n_tests.
__device__ __forceinline__ void walk_group(const WalkArgs &a, uint32_t g, uint32_t ngroups, float *lx,
                                           uint32_t *q, unsigned long long &n_inter,
                                           unsigned long long &n_tests) {
    const int lane = threadIdx.x & 31;
    const uint32_t qmask = (uint32_t)a.qcap - 1u;
    const int lifo_at = a.qcap - LIFO_ROOM;
    const uint32_t na = a.ctl->n_active;
    const uint32_t gmax = (uint32_t)a.gmax;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = lanemask_lt();
    uint32_t a0, a1;
    if (a.gstart) {
        a0 = a.gstart[g];
        a1 = g + 1 < ngroups ? a.gstart[g + 1] : na;
    } else {
        a0 = g * gmax;
        a1 = min(a0 + gmax, na);
    }
    const uint32_t cnt = a1 - a0;
    // a group of more than 32 gives every lane a second member (lane + 32), one lane each
    const bool two = cnt > 32u;
    if (cnt == 0u || cnt > 64u || (two && a.ij_share > 1)) {  // a malformed group: report it, skip
        if (lane == 0) gt_set_error(a.ctl, GT_EINVAL, GTK_WALK);
        return;
    }
    const int S = two ? 1 : (a.ij_share ? a.ij_share : 32 >> (cnt <= 1 ? 0 : 32 - __clz(cnt - 1)));
    const int logS = __ffs(S) - 1;
    const int slot = lane >> logS, sub = lane & (S - 1);
    const bool have = (uint32_t)slot < cnt;
    const bool have2 = two && (uint32_t)(lane + 32) < cnt;
    const uint32_t kk = a0 + (have ? (uint32_t)slot : 0u);
    const uint32_t kk2 = a0 + (have2 ? (uint32_t)(lane + 32) : 0u);
    uint32_t i = a.active ? a.active[kk] : kk;
    uint32_t i2 = have2 ? (a.active ? a.active[kk2] : kk2) : i;
    if (i >= a.n || i2 >= a.n) {  // an index outside the system: report it, walk particle 0 instead
        gt_set_error(a.ctl, GT_EINVAL, GTK_WALK);
        i = i >= a.n ? 0u : i;
        i2 = i2 >= a.n ? 0u : i2;
    }
    const float4 pi = a.posm[i];
    const float4 pi2 = have2 ? a.posm[i2] : pi;
    float ao = have ? (a.aold ? a.aold[i] : 0.0f) : INFINITY;
    if (have2) ao = fminf(ao, a.aold ? a.aold[i2] : 0.0f);

    // pseudo i-particle (lanes without a member repeat member 0: no effect on the box)
    float mnx = fminf(pi.x, pi2.x), mny = fminf(pi.y, pi2.y), mnz = fminf(pi.z, pi2.z);
    float mxx = fmaxf(pi.x, pi2.x), mxy = fmaxf(pi.y, pi2.y), mxz = fmaxf(pi.z, pi2.z);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(FULL, mnx, o));
        mny = fminf(mny, __shfl_xor_sync(FULL, mny, o));
        mnz = fminf(mnz, __shfl_xor_sync(FULL, mnz, o));
        mxx = fmaxf(mxx, __shfl_xor_sync(FULL, mxx, o));
        mxy = fmaxf(mxy, __shfl_xor_sync(FULL, mxy, o));
        mxz = fmaxf(mxz, __shfl_xor_sync(FULL, mxz, o));
        ao = fminf(ao, __shfl_xor_sync(FULL, ao, o));
    }
    float cx = __fmul_rn(0.5f, __fadd_rn(mnx, mxx));
    float cy = __fmul_rn(0.5f, __fadd_rn(mny, mxy));
    float cz = __fmul_rn(0.5f, __fadd_rn(mnz, mxz));
    if (a.sphere == 1) ebs_centre(pi, pi2, have && sub == 0, have2, slot, lane, logS, cnt, cx, cy, cz);
    const float ddx = __fsub_rn(pi.x, cx), ddy = __fsub_rn(pi.y, cy), ddz = __fsub_rn(pi.z, cz);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy)), __fmul_rn(ddz, ddz));
    {
        const float ex = __fsub_rn(pi2.x, cx), ey = __fsub_rn(pi2.y, cy), ez = __fsub_rn(pi2.z, cz);
        d2 = fmaxf(d2, __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(FULL, d2, o));
    const float bI = __fmul_rn(__fsqrt_rn(d2), GT_RADIUS_MARGIN);
    const float dacc_amin = __fmul_rn(a.delta_acc, ao);

    float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
    float bx = 0.f, by = 0.f, bz = 0.f, qh = 0.f;  // the second member's sums
    int list_n = 0;
    // the list, structure of arrays: x, y, z, m of entry e at lx[e], ly[e], lz[e], lw[e]
    float *ly = lx + LIST_CAP, *lz = lx + 2 * LIST_CAP, *lw = lx + 3 * LIST_CAP;
    auto flush = [&]() {
        cp_async_wait_all();
        __syncwarp();
        // entries are taken four at a time (one 16-byte load per coordinate), as the pairs
        // (e, e + 1) and (e + 2, e + 3); the list is padded with massless entries to a
        // multiple of four, which add exactly nothing
        const int pad = (-list_n) & 3;
        if (pad) {
            if (lane < pad) {
                lx[list_n + lane] = 0.f; ly[list_n + lane] = 0.f; lz[list_n + lane] = 0.f; lw[list_n + lane] = 0.f;
            }
            __syncwarp();
        }
        const int nquad = (list_n + 3) >> 2;
        const float4 *px = (const float4 *)lx, *py = (const float4 *)ly, *pz = (const float4 *)lz,
                     *pw = (const float4 *)lw;
        // one i-particle against quads k0, k0 + step, ... (its sums carried in and out)
        auto run = [&](const float4 &p, float &sx_, float &sy_, float &sz_, float &sp_, int k0, int step) {
            const float2 e2 = make_float2(a.eps2, a.eps2);
            const float2 nx = make_float2(-p.x, -p.x), ny = make_float2(-p.y, -p.y), nz = make_float2(-p.z, -p.z);
            float2 sx = make_float2(sx_, 0.f), sy = make_float2(sy_, 0.f), sz = make_float2(sz_, 0.f);
            float2 sp = make_float2(-sp_, 0.f);
            for (int k = k0; k < nquad; k += step) {
                const float4 X = px[k], Y = py[k], Z = pz[k], W = pw[k];
                interact_pairs(make_float2(X.x, X.y), make_float2(Y.x, Y.y), make_float2(Z.x, Z.y),
                               make_float2(W.x, W.y), nx, ny, nz, e2, sx, sy, sz, sp);
                interact_pairs(make_float2(X.z, X.w), make_float2(Y.z, Y.w), make_float2(Z.z, Z.w),
                               make_float2(W.z, W.w), nx, ny, nz, e2, sx, sy, sz, sp);
            }
            sx_ = __fadd_rn(sx.x, sx.y); sy_ = __fadd_rn(sy.x, sy.y); sz_ = __fadd_rn(sz.x, sz.y);
            sp_ = -__fadd_rn(sp.x, sp.y);
        };
        if (two) {  // both members of the lane over every pair, one after the other
            run(pi, ax, ay, az, ph, 0, 1);
            run(pi2, bx, by, bz, qh, 0, 1);
        } else {  // S lanes per i-particle: lane sub takes quads sub, sub + S, ...
            run(pi, ax, ay, az, ph, sub, S);
        }
        n_inter += (unsigned long long)list_n * cnt;
        list_n = 0;
        __syncwarp();
    };

#if GT_DEBUG
    const uint32_t nnodes = a.ctl->level_start[GT_TREE_LEVELS];
#endif
    uint32_t head = 0, tail = 1;
    if (lane == 0) q[0] = 0u;  // the root
    __syncwarp();
    bool overflow = false;
    while (head != tail) {
        const uint32_t live = tail - head;
        const uint32_t nb = min(live, 32u);
#if !GT_DEBUG
        const bool valid = (uint32_t)lane < nb;
#endif
        // breadth-first from the head while there is room, depth-first from the tail after
        uint32_t base;
        if ((int)live > lifo_at) {
            tail -= nb;
            base = tail;
        } else {
            base = head;
            head += nb;
        }
        float4 jp = make_float4(0.f, 0.f, 0.f, 0.f), wk = make_float4(0.f, 0.f, 0.f, 0.f);
#if GT_DEBUG
        bool valid = (uint32_t)lane < nb;
        if (valid) {
            const uint32_t node = q[(base + lane) & qmask];
            if (node >= nnodes) {
                gt_set_error(a.ctl, GT_EINVAL, GTK_WALK);
                valid = false;
            } else {
                jp = a.jpos[node];
                wk = a.walk[node];
                const uint32_t c = __float_as_uint(wk.z), f = __float_as_uint(wk.y);
                const bool lf = (c & GT_LEAF_FLAG) != 0u;
                if ((unsigned long long)f + (lf ? (c & ~GT_LEAF_FLAG) : c) > (lf ? a.n : nnodes)) {
                    gt_set_error(a.ctl, GT_EINVAL, GTK_WALK);
                    valid = false;
                }
            }
        }
#else
        if (valid) {
            const uint32_t node = q[(base + lane) & qmask];
            jp = a.jpos[node];
            wk = a.walk[node];
        }
#endif
        n_tests += nb;
        const bool ok = valid && mac_accept(a.mac, a.theta, dacc_amin, a.delta_acc, a.G, cx, cy, cz, bI, jp,
                                            wk.x, wk.w);
        const uint32_t l0 = __float_as_uint(wk.y), l1 = __float_as_uint(wk.z);
        const bool leaf = (l1 & GT_LEAF_FLAG) != 0u;
        // accepted cells -> list
        const unsigned am = __ballot_sync(FULL, ok);
        if (am) {
            const int nacc = __popc(am);
            if (list_n + nacc > LIST_CAP) flush();
            if (ok) {
                const int e = list_n + __popc(am & lt);
                lx[e] = jp.x; ly[e] = jp.y; lz[e] = jp.z; lw[e] = jp.w;
            }
            list_n += nacc;
        }
        // opened cells -> their children into the queue; opened leaves -> their particles
        // into the list (asynchronous copies).  One warp scan counts both (children in the
        // low 16 bits, particles in the high 16: they fit while every leaf of the batch holds
        // fewer than 2048 particles) and one loop writes both: entry e of the batch belongs
        // to the first lane whose inclusive count exceeds e (a binary search over the lanes
        // by shuffles); each lane's entries are its cell's children or its leaf's particles.
        const uint32_t nch = (valid && !ok && !leaf) ? l1 : 0u;
        const uint32_t lc = (valid && !ok && leaf) ? (l1 & ~GT_LEAF_FLAG) : 0u;
        if (__all_sync(FULL, lc < 2048u)) {
            const uint32_t mine = nch | (lc << 16);
            const uint32_t incl = warp_incl_scan(mine);
            const uint32_t tot = __shfl_sync(FULL, incl, 31);
            const uint32_t tc = tot & 0xffffu, tp = tot >> 16;
            if (tail - head + tc > (uint32_t)a.qcap) {
                overflow = true;
                break;
            }
            const uint32_t inclm = (incl & 0xffffu) + (incl >> 16);  // entries up to this lane
            int pbase = list_n;  // list slot of the batch's first particle
            uint32_t pdone = 0;  // particles written by earlier rounds
            for (uint32_t r = 0; r < tc + tp; r += 32) {
                const uint32_t e = r + (uint32_t)lane;
                int own = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(FULL, inclm, own + step - 1) <= e) own += step;
                const uint32_t oi = __shfl_sync(FULL, incl, own);
                const uint32_t om = __shfl_sync(FULL, mine, own);
                const uint32_t ol = __shfl_sync(FULL, l0, own);
                const uint32_t ec = (oi & 0xffffu) - (om & 0xffffu), ep = (oi >> 16) - (om >> 16);
                const bool in = e < tc + tp;
                const bool isp = in && (om >> 16) != 0u;
                const uint32_t off = e - ec - ep;
                const unsigned pm = __ballot_sync(FULL, isp);
                if (pm && pbase + (int)pdone + __popc(pm) > LIST_CAP) {
                    list_n = pbase + (int)pdone;
                    flush();
                    pbase = -(int)pdone;
                }
                if (in && !isp) q[(tail + ec + off) & qmask] = ol + off;
                if (isp) {
                    const int slot = pbase + (int)(ep + off);
                    const float *src = (const float *)&a.posm[ol + off];
                    cp_async4(&lx[slot], src);
                    cp_async4(&ly[slot], src + 1);
                    cp_async4(&lz[slot], src + 2);
                    cp_async4(&lw[slot], src + 3);
                }
                pdone += (uint32_t)__popc(pm);
            }
            tail += tc;
            list_n = pbase + (int)pdone;
        } else {
            // a leaf of 2048 or more particles (coincident particles chained to level 21)
            const uint32_t incl = warp_incl_scan(nch);
            const uint32_t tot = __shfl_sync(FULL, incl, 31);
            if (tot) {
                if (tail - head + tot > (uint32_t)a.qcap) {
                    overflow = true;
                    break;
                }
                // the warp writes the children together: entry e belongs to the first lane whose
                // inclusive count exceeds e (a binary search over the lanes by shuffles)
                const uint32_t cbase = l0 - (incl - nch);
                for (uint32_t r = 0; r < tot; r += 32) {
                    const uint32_t e = r + (uint32_t)lane;
                    int own = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (__shfl_sync(FULL, incl, own + step - 1) <= e) own += step;
                    const uint32_t cb = __shfl_sync(FULL, cbase, own);
                    if (e < tot) q[(tail + e) & qmask] = cb + e;
                }
                tail += tot;
            }
            // opened leaves -> their particles into the list (asynchronous copies)
            const uint32_t lincl = warp_incl_scan(lc);
            const uint32_t ltot = __shfl_sync(FULL, lincl, 31);
            if (ltot) {
                if (list_n + (int)ltot > LIST_CAP) flush();
                if (ltot <= (uint32_t)LIST_CAP) {
                    const uint32_t pbase = l0 - (lincl - lc);
                    for (uint32_t r = 0; r < ltot; r += 32) {
                        const uint32_t e = r + (uint32_t)lane;
                        int own = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1)
                            if (__shfl_sync(FULL, lincl, own + step - 1) <= e) own += step;
                        const uint32_t pb = __shfl_sync(FULL, pbase, own);
                        if (e < ltot) {
                            const float *src = (const float *)&a.posm[pb + e];
                            cp_async4(&lx[list_n + e], src);
                            cp_async4(&ly[list_n + e], src + 1);
                            cp_async4(&lz[list_n + e], src + 2);
                            cp_async4(&lw[list_n + e], src + 3);
                        }
                    }
                    list_n += (int)ltot;
                } else {  // leaves holding more particles than the list: one at a time, in chunks
                    unsigned lm = __ballot_sync(FULL, lc != 0u);
                    while (lm) {
                        const int src = __ffs(lm) - 1;
                        lm &= lm - 1;
                        const uint32_t lf = __shfl_sync(FULL, l0, src);
                        const uint32_t lcount = __shfl_sync(FULL, lc, src);
                        uint32_t done = 0;
                        while (done < lcount) {
                            if (list_n == LIST_CAP) flush();
                            const uint32_t take = min(lcount - done, (uint32_t)(LIST_CAP - list_n));
                            for (uint32_t k = lane; k < take; k += 32) {
                                const float *src = (const float *)&a.posm[lf + done + k];
                                cp_async4(&lx[list_n + k], src);
                                cp_async4(&ly[list_n + k], src + 1);
                                cp_async4(&lz[list_n + k], src + 2);
                                cp_async4(&lw[list_n + k], src + 3);
                            }
                            list_n += (int)take;
                            done += take;
                        }
                    }
                }
            }
        }
        if (list_n >= FLUSH_AT) flush();
        __syncwarp();
    }
    if (overflow) {
        if (lane == 0) gt_set_error(a.ctl, GT_EOVERFLOW, GTK_WALK);
        cp_async_wait_all();
        list_n = 0;
        if (sub == 0 && have) a.acc[kk] = make_float4(NAN, NAN, NAN, NAN);
        if (have2) a.acc[kk2] = make_float4(NAN, NAN, NAN, NAN);
        __syncwarp();
        return;
    }
    flush();
    for (int o = 1; o < S; o <<= 1) {
        ax += __shfl_xor_sync(FULL, ax, o);
        ay += __shfl_xor_sync(FULL, ay, o);
        az += __shfl_xor_sync(FULL, az, o);
        ph += __shfl_xor_sync(FULL, ph, o);
    }
    if (sub == 0 && have) {
        const float phi = fmaf(pi.w, a.inv_eps, ph);
        a.acc[kk] = make_float4(a.G * ax, a.G * ay, a.G * az, a.G * phi);
    }
    if (have2) {
        const float phi = fmaf(pi2.w, a.inv_eps, qh);
        a.acc[kk2] = make_float4(a.G * bx, a.G * by, a.G * bz, a.G * phi);
    }
}

// groups of one system in a list of the systems' group counts: gprefix[s] is the first
// global group of system s, gprefix[nsys] the total
__device__ __forceinline__ int system_of(const uint32_t *gprefix, int nsys, uint32_t gg) {
    int lo = 0, hi = nsys - 1;  // the last s with gprefix[s] <= gg
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gprefix[mid] <= gg) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ __launch_bounds__(WT, GT_WALK_MINB) void k_walk(WalkArgs a) {
    __shared__ __align__(16) float list_sm[NWARP][4 * LIST_CAP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *list = list_sm[warp];
    uint32_t *q = a.queue + (size_t)(blockIdx.x * NWARP + warp) * (size_t)a.qcap;
    const uint32_t na = a.ctl->n_active;
    const uint32_t gmax = (uint32_t)a.gmax;
    const uint32_t ngroups = a.gstart ? a.ctl->n_groups : (na + gmax - 1) / gmax;
    unsigned long long n_inter = 0, n_tests = 0;
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&a.ctl->group_next, 1u);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        walk_group(a, g, ngroups, list, q, n_inter, n_tests);
    }
    if (lane == 0) {
        if (n_inter) atomicAdd(&a.ctl->interactions, n_inter);
        if (n_tests) atomicAdd(&a.ctl->mac_tests, n_tests);
    }
}

// Many systems in one persistent launch: global group numbers run over the systems
// in order (gprefix), every warp takes the next one from one counter and walks it
// with that system's arguments (copied to shared memory).  mac >= 0 overrides every
// system's MAC (the opening-angle start-up pass).
__global__ __launch_bounds__(WT, 3) void k_walk_batch(const WalkArgs *__restrict__ args, int nsys,
                                                      const uint32_t *__restrict__ gprefix,
                                                      unsigned int *group_next, uint32_t *queue, int qcap,
                                                      int mac) {
    __shared__ __align__(16) float list_sm[NWARP][4 * LIST_CAP];
    __shared__ WalkArgs sargs[NWARP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *list = list_sm[warp];
    uint32_t *q = queue + (size_t)(blockIdx.x * NWARP + warp) * (size_t)qcap;
    const uint32_t total = gprefix[nsys];
    for (;;) {
        uint32_t gg = 0;
        if (lane == 0) gg = atomicAdd(group_next, 1u);
        gg = __shfl_sync(0xffffffffu, gg, 0);
        if (gg >= total) break;
        int sys = 0;
        if (lane == 0) sys = system_of(gprefix, nsys, gg);
        sys = __shfl_sync(0xffffffffu, sys, 0);
        static_assert(sizeof(WalkArgs) % 4 == 0, "copied as words");
        const uint32_t *src = (const uint32_t *)&args[sys];
        uint32_t *dst = (uint32_t *)&sargs[warp];
        for (int w = lane; w < (int)(sizeof(WalkArgs) / 4); w += 32) dst[w] = src[w];
        __syncwarp();
        if (mac >= 0 && lane == 0) sargs[warp].mac = mac;
        __syncwarp();
        const WalkArgs &a = sargs[warp];
        const uint32_t g = gg - gprefix[sys];
        const uint32_t ngroups = gprefix[sys + 1] - gprefix[sys];
        unsigned long long n_inter = 0, n_tests = 0;
        // the batch queue replaces the system's own
        walk_group(a, g, ngroups, list, q, n_inter, n_tests);
        if (lane == 0) {
            if (n_inter) atomicAdd(&a.ctl->interactions, n_inter);
            if (n_tests) atomicAdd(&a.ctl->mac_tests, n_tests);
        }
        __syncwarp();
    }
}

// gprefix over the systems' group counts (one warp; also resets the batch counter)
__global__ void k_batch_prefix(DevCtl *const *__restrict__ ctls, const WalkArgs *__restrict__ args, int nsys,
                               uint32_t *gprefix, unsigned int *group_next) {
    uint32_t carry = 0;
    for (int s0 = 0; s0 < nsys; s0 += 32) {
        const int s = s0 + (int)threadIdx.x;
        uint32_t ng = 0;
        if (s < nsys) {
            const DevCtl *c = ctls[s];
            const uint32_t na = c->n_active;
            const uint32_t gm = (uint32_t)args[s].gmax;
            ng = args[s].gstart ? c->n_groups : (na + gm - 1) / gm;
        }
        const uint32_t incl = warp_incl_scan(ng);
        if (s < nsys) gprefix[s] = carry + incl - ng;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (threadIdx.x == 0) {
        gprefix[nsys] = carry;
        *group_next = 0u;
    }
}

}  // namespace

int gt_walk_blocks(int nsm) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk, WT, 0);
    if (per < 1) per = 1;
    return per * nsm;
}

int gt_walk_warps_per_block() { return NWARP; }

void gt_launch_walk(const WalkArgs &a, int nblocks, cudaStream_t st) {
    { k_walk<<<nblocks, WT, 0, st>>>(a); gt_note_launches(1); }
}

void gt_launch_walk_batch(DevCtl *const *ctls, const WalkArgs *args, int nsys, uint32_t *gprefix,
                          unsigned int *group_next, uint32_t *queue, int qcap, int mac, int nblocks,
                          cudaStream_t st) {
    if (nsys <= 0) return;
    { k_batch_prefix<<<1, 32, 0, st>>>(ctls, args, nsys, gprefix, group_next); gt_note_launches(1); }
    { k_walk_batch<<<nblocks, WT, 0, st>>>(args, nsys, gprefix, group_next, queue, qcap, mac); gt_note_launches(1); }
}
