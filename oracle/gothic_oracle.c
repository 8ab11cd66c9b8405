/*
 * CPU oracle for the block-step oct-tree gravity method of Miki & Umemura,
 * "GOTHIC: Gravitational oct-tree code accelerated by hierarchical time step
 * controlling" (New Astronomy; arXiv:1610.07279).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference against which
 * the CUDA path is checked.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it; the product never does.  It shares no
 * code, header, table or constant with the CUDA sources.
 *
 * Precision: FP64 everywhere the method has a plain definition (direct sums,
 * centre of mass, integration).  Two decisions are taken in FP32 because the
 * method takes them in FP32 on the GPU and both sides must decide identically:
 * the multipole acceptance test and the pseudo i-particle centre.
 * Build with -ffp-contract=off so that no multiply-add is fused behind our back.
 *
 * Index spaces: every tree routine works on particles already sorted by key
 * ("sorted index").  Callers permute their arrays with or_sort's order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define KEY_LEVELS 21 /* 21 bits per axis -> 63-bit keys (Appendix A) */

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops that follow (timing of the oracle on one core or all). */
void or_set_num_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

/* Enclosing radii are evaluated in FP32 and widened by (1 + 2^-20): an FP32
 * distance carries a few roundings of at most 2^-24 each, so the widened radius
 * still holds every particle (Sec. 2.1 asks only for a sphere that contains them). */
#define RADIUS_MARGIN (1.0f + 0x1p-20f)

/* ------------------------------------------------------------------------- */
/* O1. Direct summation, Eq. (1): a_i = sum_{j != i} G m_j (r_j - r_i) /     */
/* (|r_j - r_i|^2 + eps^2)^{3/2}.  The potential phi_i = -sum_{j != i} G m_j  */
/* / (|r_j - r_i|^2 + eps^2)^{1/2} is returned as the fourth component (the   */
/* paper's force kernel also returns the potential, Sec. 4 flop count).      */
/* p4: n x (x, y, z, m) in FP32.  Evaluated for the ni particles listed in   */
/* iidx (all if iidx == NULL and ni == n).  out: ni x 4 doubles.             */
/* ------------------------------------------------------------------------- */
void or_direct(int64_t n, const float *p4, double eps, double G, int64_t ni,
               const int64_t *iidx, double *out) {
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < ni; k++) {
        const int64_t i = iidx ? iidx[k] : k;
        const double xi = p4[4 * i + 0], yi = p4[4 * i + 1], zi = p4[4 * i + 2];
        double ax = 0.0, ay = 0.0, az = 0.0, phi = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            const double dx = (double)p4[4 * j + 0] - xi;
            const double dy = (double)p4[4 * j + 1] - yi;
            const double dz = (double)p4[4 * j + 2] - zi;
            const double r2 = dx * dx + dy * dy + dz * dz + eps2;
            const double rinv = 1.0 / sqrt(r2);
            const double mr = (double)p4[4 * j + 3] * rinv;
            const double mr3 = mr * rinv * rinv;
            ax += mr3 * dx;
            ay += mr3 * dy;
            az += mr3 * dz;
            phi -= mr;
        }
        out[4 * k + 0] = G * ax;
        out[4 * k + 1] = G * ay;
        out[4 * k + 2] = G * az;
        out[4 * k + 3] = G * phi;
    }
}

/* ------------------------------------------------------------------------- */
/* A1. Bounding cube and Morton keys (Sec. 2.1; Morton curve, Appendix A).   */
/* The cube is anchored at the per-axis minima of the FP32 positions; its    */
/* side is the largest per-axis extent, taken in FP64.  Each coordinate is   */
/* quantised to 21 bits: q = min(2^21 - 1, floor((x - xmin) * (2^21/side)))  */
/* and the three 21-bit integers are interleaved with x as the most          */
/* significant bit of every triplet, then y, then z.  side == 0 (one         */
/* particle, or all coincident) gives every particle the key 0.              */
/* box out: xmin, ymin, zmin, side, 2^21/side.                               */
/* ------------------------------------------------------------------------- */
static uint64_t interleave3(uint64_t qx, uint64_t qy, uint64_t qz) {
    uint64_t key = 0;
    for (int b = 0; b < KEY_LEVELS; b++) {
        key |= ((qx >> b) & 1u) << (3 * b + 2);
        key |= ((qy >> b) & 1u) << (3 * b + 1);
        key |= ((qz >> b) & 1u) << (3 * b + 0);
    }
    return key;
}

void or_keys_curve(int64_t n, const float *p4, uint64_t *key, double *box, int curve);

/* Peano-Hilbert index (Sec. 2.1, Appendix A: the paper's key curve), by Skilling's  */
/* transpose method (Skilling 2004): the three 21-bit integers are turned into the   */
/* "transposed" Hilbert index -- undo the rotations and reflections from the top bit */
/* down, then a Gray code across the axes -- whose bits, interleaved with axis 0 as  */
/* the most significant of every triplet, are the index.  As for Morton keys, the    */
/* first 3l bits name the level-l cube, so cells are contiguous key ranges.          */
static void hilbert_transpose(uint32_t x[3], int bits) {
    const uint32_t top = 1u << (bits - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        const uint32_t p = q - 1;
        for (int i = 0; i < 3; i++) {
            if (x[i] & q) {
                x[0] ^= p;                          /* reflect */
            } else {
                const uint32_t t = (x[0] ^ x[i]) & p; /* swap the low bits of axes 0 and i */
                x[0] ^= t;
                x[i] ^= t;
            }
        }
    }
    x[1] ^= x[0];
    x[2] ^= x[1];
    uint32_t t = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (x[2] & q) t ^= q - 1;
    for (int i = 0; i < 3; i++) x[i] ^= t;
}

void or_keys(int64_t n, const float *p4, uint64_t *key, double *box) {
    or_keys_curve(n, p4, key, box, 0);
}

uint64_t or_hilbert3(uint64_t qx, uint64_t qy, uint64_t qz) {
    uint32_t x[3] = {(uint32_t)qx, (uint32_t)qy, (uint32_t)qz};
    hilbert_transpose(x, KEY_LEVELS);
    return interleave3(x[0], x[1], x[2]);
}

void or_keys_curve(int64_t n, const float *p4, uint64_t *key, double *box, int curve) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) {
            const float v = p4[4 * i + a];
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    double side = 0.0;
    for (int a = 0; a < 3; a++) {
        if (n == 0) break;
        const double ext = (double)mx[a] - (double)mn[a];
        if (ext > side) side = ext;
    }
    const double qmax = (double)((1u << KEY_LEVELS) - 1u);
    const double scale = side > 0.0 ? (double)(1u << KEY_LEVELS) / side : 0.0;
    if (box) {
        box[0] = n ? mn[0] : 0.0;
        box[1] = n ? mn[1] : 0.0;
        box[2] = n ? mn[2] : 0.0;
        box[3] = side;
        box[4] = scale;
    }
#pragma omp parallel for
    for (int64_t i = 0; i < n; i++) {
        uint64_t q[3] = {0, 0, 0};
        if (side > 0.0)
            for (int a = 0; a < 3; a++) {
                double t = floor(((double)p4[4 * i + a] - (double)mn[a]) * scale);
                if (t > qmax) t = qmax;
                q[a] = (uint64_t)t;
            }
        if (curve == 1) {
            uint32_t x[3] = {(uint32_t)q[0], (uint32_t)q[1], (uint32_t)q[2]};
            hilbert_transpose(x, KEY_LEVELS);
            key[i] = interleave3(x[0], x[1], x[2]);
        } else {
            key[i] = interleave3(q[0], q[1], q[2]);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* A2. Sort of (key, particle index) pairs by key, ties by original index   */
/* (a stable sort, as the library radix sort the paper uses is; Sec. 2.1).   */
/* order[s] = original index of the particle at sorted position s.          */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t key; uint32_t idx; } kv_t;

static int kv_cmp(const void *a, const void *b) {
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

int or_sort(int64_t n, const uint64_t *key, uint32_t *order, uint64_t *skey) {
    kv_t *a = (kv_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(kv_t));
    if (!a) return -1;
    for (int64_t i = 0; i < n; i++) { a[i].key = key[i]; a[i].idx = (uint32_t)i; }
    qsort(a, (size_t)n, sizeof(kv_t), kv_cmp);
    for (int64_t i = 0; i < n; i++) { order[i] = a[i].idx; if (skey) skey[i] = a[i].key; }
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* A4. Breadth-first octree over sorted keys (Sec. 2.1: dividing a cube into */
/* eight sub-cubes is finding seven partitions of its key range; cells are   */
/* numbered serially level by level).                                        */
/*   root: level 0, particles [0, n).                                        */
/*   a cell at level l with count > leaf_max and l < 21 splits by the digit  */
/*   (key >> 3 (20 - l)) & 7; only non-empty children are kept, in ascending */
/*   digit order.  Nodes are numbered level by level, and within a level in  */
/*   the order of their first particle.  A leaf has child = -1.              */
/* Returns the node count, or -1 if it would exceed cap.                     */
/* ------------------------------------------------------------------------- */
int64_t or_build(int64_t n, const uint64_t *skey, int leaf_max, int64_t cap,
                 uint32_t *first, uint32_t *count, int32_t *child, uint8_t *nchild,
                 uint8_t *level, int32_t *parent, int64_t *level_start /* 23 entries */) {
    if (n == 0) {
        if (level_start) for (int l = 0; l <= KEY_LEVELS + 1; l++) level_start[l] = 0;
        return 0;
    }
    if (cap < 1) return -1;
    int64_t nn = 1;
    first[0] = 0; count[0] = (uint32_t)n; level[0] = 0; parent[0] = -1;
    int64_t lo = 0, hi = 1; /* nodes of the current level: [lo, hi) */
    for (int l = 0; l <= KEY_LEVELS; l++) {
        if (level_start) level_start[l] = lo;
        for (int64_t c = lo; c < hi; c++) {
            child[c] = -1; nchild[c] = 0;
            if (!(count[c] > (uint32_t)leaf_max && l < KEY_LEVELS)) continue;
            const int shift = 3 * (KEY_LEVELS - 1 - l);
            uint32_t s = first[c];
            const uint32_t e = first[c] + count[c];
            child[c] = (int32_t)nn;
            while (s < e) {
                const uint64_t dig = (skey[s] >> shift) & 7u;
                uint32_t t = s;
                while (t < e && ((skey[t] >> shift) & 7u) == dig) t++;
                if (nn >= cap) return -1;
                first[nn] = s; count[nn] = t - s; level[nn] = (uint8_t)(l + 1);
                parent[nn] = (int32_t)c;
                nn++; nchild[c]++;
                s = t;
            }
        }
        lo = hi; hi = nn;
        if (lo == hi) {
            if (level_start) for (int k = l + 1; k <= KEY_LEVELS + 1; k++) level_start[k] = nn;
            return nn;
        }
    }
    if (level_start) level_start[KEY_LEVELS + 1] = nn;
    return nn;
}

/* ------------------------------------------------------------------------- */
/* A5. Pseudo j-particles (Sec. 2.1, Fig. 1): m_J = sum m, r_J = sum m r /   */
/* m_J, and b_J the radius of a sphere about r_J that holds every particle   */
/* of the cell.  The sums are FP64: a leaf adds its particles in sorted      */
/* order, a cell adds its children's sums in child order.  m_J = (float)M;   */
/* r_J is the FP32 quotient (float)S / (float)M (the paper keeps r_J in      */
/* single precision, Sec. 2); a cell of one particle is that particle.       */
/* b_J (FP32): a leaf's largest |r - r_J|, a cell's largest |r_c - r_J| + b_c */
/* over its children, times (1 + 2^-20).  B_2 (the multipole MAC's second   */
/* moment, Sec. 2.2), FP32: a leaf adds m |r - r_J|^2 over its particles, a  */
/* cell adds B_2,c + m_c |r_c - r_J|^2 over its children (parallel axes), in */
/* the same orders.  Children have larger node numbers than parents, so a    */
/* reverse sweep is bottom-up.                                               */
/* jpos out: nn x (x, y, z, m) FP32; bj out: nn FP32; b2 out: nn FP32 or NULL*/
/* ------------------------------------------------------------------------- */
int or_pseudo_j(int64_t nn, const uint32_t *first, const uint32_t *count, const int32_t *child,
                const uint8_t *nchild, const float *sp4, float *jpos, float *bj, float *b2) {
    double *sum = (double *)malloc((size_t)(nn > 0 ? nn : 1) * 4 * sizeof(double));
    if (!sum) return -1;
    for (int64_t c = nn - 1; c >= 0; c--) {
        double m = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        if (child[c] < 0) {
            for (uint32_t i = first[c]; i < first[c] + count[c]; i++) {
                const double mi = sp4[4 * i + 3];
                m += mi;
                sx += mi * (double)sp4[4 * i + 0];
                sy += mi * (double)sp4[4 * i + 1];
                sz += mi * (double)sp4[4 * i + 2];
            }
        } else {
            for (int k = 0; k < nchild[c]; k++) {
                const int64_t ch = child[c] + k;
                m += sum[4 * ch + 0];
                sx += sum[4 * ch + 1];
                sy += sum[4 * ch + 2];
                sz += sum[4 * ch + 3];
            }
        }
        sum[4 * c + 0] = m; sum[4 * c + 1] = sx; sum[4 * c + 2] = sy; sum[4 * c + 3] = sz;
        float jx, jy, jz;
        if (count[c] == 1) {
            const uint32_t i = first[c];
            jx = sp4[4 * i + 0]; jy = sp4[4 * i + 1]; jz = sp4[4 * i + 2];
        } else {
            const float mf = (float)m;
            jx = (float)sx / mf; jy = (float)sy / mf; jz = (float)sz / mf;
        }
        jpos[4 * c + 0] = jx; jpos[4 * c + 1] = jy; jpos[4 * c + 2] = jz; jpos[4 * c + 3] = (float)m;
        float b = 0.0f, q = 0.0f;  /* q: B2 */
        if (child[c] < 0) {
            float d2max = 0.0f;
            for (uint32_t i = first[c]; i < first[c] + count[c]; i++) {
                const float dx = sp4[4 * i + 0] - jx, dy = sp4[4 * i + 1] - jy, dz = sp4[4 * i + 2] - jz;
                const float d2 = (dx * dx + dy * dy) + dz * dz;
                if (d2 > d2max) d2max = d2;
                q = q + sp4[4 * i + 3] * d2;
            }
            b = sqrtf(d2max);
        } else {
            for (int k = 0; k < nchild[c]; k++) {
                const int64_t ch = child[c] + k;
                const float dx = jpos[4 * ch + 0] - jx, dy = jpos[4 * ch + 1] - jy, dz = jpos[4 * ch + 2] - jz;
                const float d2 = (dx * dx + dy * dy) + dz * dz;
                const float e = sqrtf(d2) + bj[ch];
                if (e > b) b = e;
                if (b2) q = q + (b2[ch] + jpos[4 * ch + 3] * d2);
            }
        }
        bj[c] = b * RADIUS_MARGIN;
        if (b2) b2[c] = q;
    }
    free(sum);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* A6a. Active prefix: P[i] = number of active particles (sorted indices,    */
/* strictly increasing in `active`) below sorted index i, for i = 0..n.      */
/* ------------------------------------------------------------------------- */
void or_active_prefix(int64_t n, int64_t n_active, const uint32_t *active, uint32_t *P) {
    int64_t k = 0;
    for (int64_t i = 0; i <= n; i++) {
        while (k < n_active && (int64_t)active[k] < i) k++;
        P[i] = (uint32_t)k;
    }
}

/* ------------------------------------------------------------------------- */
/* A6b. Groups of i-particles (Sec. 2.3; Sec. 2.4: i-particles far apart are  */
/* not unified into one group).  A group never straddles two tree cells.  A  */
/* cell "qualifies" when it holds at most gmax actives and is a leaf or has  */
/* an enclosing radius b_J <= r_crit (the critical separation of Sec. 2.4;   */
/* r_crit <= 0 means no such limit).  Both counts and radii only shrink from  */
/* a cell to its children, so along every root-to-leaf path the qualifying   */
/* cells are a tail: the group cells are the qualifying cells whose parent   */
/* does not qualify (or the root), plus the leaves on paths where nothing    */
/* qualifies.  Each group cell with at least one active contributes its      */
/* actives in key order, cut into runs of gmax.  Returns the number of       */
/* groups; the first active position of every group, ascending, goes to      */
/* starts (room for n_active + 1 entries); starts[ng] = P[n] is appended.    */
/* ------------------------------------------------------------------------- */
static int cmp_u32(const void *a, const void *b) {
    const uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static int qualifies(int64_t c, const uint32_t *first, const uint32_t *count, const int32_t *child,
                     const uint32_t *P, int gmax, const float *bj, float r_crit) {
    const uint32_t A = P[first[c] + count[c]] - P[first[c]];
    if (A > (uint32_t)gmax) return 0;
    if (child[c] < 0 || r_crit <= 0.0f || !bj) return 1;
    return bj[c] <= r_crit;
}

int64_t or_group_starts(int64_t nn, const uint32_t *first, const uint32_t *count, const int32_t *child,
                        const int32_t *parent, const uint32_t *P, int gmax, const float *bj, float r_crit,
                        uint32_t *starts) {
    int64_t ng = 0;
    for (int64_t c = 0; c < nn; c++) {
        const uint32_t a0 = P[first[c]], A = P[first[c] + count[c]] - a0;
        if (A == 0) continue;
        if (parent[c] >= 0 && qualifies(parent[c], first, count, child, P, gmax, bj, r_crit))
            continue;                                                                  /* inside a group cell */
        if (!qualifies(c, first, count, child, P, gmax, bj, r_crit) && child[c] >= 0) continue;  /* split */
        for (uint32_t s = a0; s < a0 + A; s += (uint32_t)gmax) starts[ng++] = s;
    }
    qsort(starts, (size_t)ng, sizeof(uint32_t), cmp_u32);
    starts[ng] = nn > 0 ? P[first[0] + count[0]] : 0;
    return ng;
}

/* ------------------------------------------------------------------------- */
/* A6c. Pseudo i-particles (Sec. 2.3, Fig. 2): the sphere about the centre   */
/* of the members' bounding box (Appendix B, "GEO").  Group g holds          */
/* active[starts[g] .. starts[g+1]).                                          */
/*   r_I = 0.5f (min + max) per axis (FP32);                                  */
/*   b_I = the largest FP32 |r_i - r_I|, times (1 + 2^-20);                   */
/*   amin = min |a_old| over the group (the acceleration MAC needs one |a_old| */
/*   per group; the smallest is the conservative choice).                    */
/* sphere 0: GEO as above; sphere 1: the centre of Ritter's efficient        */
/* bounding sphere (below), the radius taken the same way.                   */
/* gI out: ng x (x, y, z, b_I); gamin out: ng.                               */
/* ------------------------------------------------------------------------- */
/* The efficient bounding sphere of Ritter (1990), the pseudo i-particle the paper uses  */
/* on its newest GPU (Appendix B): a first diameter between the extreme points of the     */
/* axis whose pair is farthest apart, then the sphere is grown towards the first member    */
/* outside it (half the way from its far side to the point) until every member is inside */
/* (at most one growth per member).  FP32, every operation in this order; only the centre */
/* is kept, the radius is the largest member distance as for GEO.  m: member positions.   */
static void ebs_centre(int64_t cnt, const float (*m)[3], float c[3]) {
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int64_t k = 1; k < cnt; k++)
        for (int a = 0; a < 3; a++) {
            if (m[k][a] < m[lo[a]][a]) lo[a] = k;
            if (m[k][a] > m[hi[a]][a]) hi[a] = k;
        }
    int best = 0;
    float bd2 = -1.0f;
    for (int a = 0; a < 3; a++) {
        const float dx = m[hi[a]][0] - m[lo[a]][0], dy = m[hi[a]][1] - m[lo[a]][1], dz = m[hi[a]][2] - m[lo[a]][2];
        const float d2 = (dx * dx + dy * dy) + dz * dz;
        if (d2 > bd2) { bd2 = d2; best = a; }
    }
    for (int a = 0; a < 3; a++) c[a] = 0.5f * (m[lo[best]][a] + m[hi[best]][a]);
    float r = 0.5f * sqrtf(bd2);
    for (int64_t it = 0; it < cnt; it++) {
        int64_t out = -1;
        float od2 = 0.0f;
        for (int64_t k = 0; k < cnt && out < 0; k++) {
            const float dx = m[k][0] - c[0], dy = m[k][1] - c[1], dz = m[k][2] - c[2];
            const float d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 > r * r) { out = k; od2 = d2; }
        }
        if (out < 0) break;
        const float d = sqrtf(od2);
        const float rn = 0.5f * (r + d);
        const float f = (d - rn) / d;
        for (int a = 0; a < 3; a++) c[a] = c[a] + f * (m[out][a] - c[a]);
        r = rn;
    }
}

void or_groups(int64_t ng, const uint32_t *starts, const uint32_t *active, const float *sp4,
               const float *aold, int sphere, float *gI, float *gamin) {
#pragma omp parallel for
    for (int64_t g = 0; g < ng; g++) {
        const int64_t a0 = starts[g], a1 = starts[g + 1];
        float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        float am = INFINITY;
        for (int64_t k = a0; k < a1; k++) {
            const uint32_t i = active[k];
            for (int a = 0; a < 3; a++) {
                const float v = sp4[4 * i + a];
                if (v < mn[a]) mn[a] = v;
                if (v > mx[a]) mx[a] = v;
            }
            const float ao = aold ? aold[i] : 0.0f;
            if (ao < am) am = ao;
        }
        float c[3];
        if (sphere == 1 && a1 > a0) {
            float (*m)[3] = malloc((size_t)(a1 - a0) * sizeof *m);
            for (int64_t k = a0; k < a1; k++)
                for (int a = 0; a < 3; a++) m[k - a0][a] = sp4[4 * active[k] + a];
            ebs_centre(a1 - a0, (const float (*)[3])m, c);
            free(m);
        } else {
            for (int a = 0; a < 3; a++) c[a] = 0.5f * (mn[a] + mx[a]);
        }
        float d2max = 0.0f;
        for (int64_t k = a0; k < a1; k++) {
            const uint32_t i = active[k];
            const float dx = sp4[4 * i + 0] - c[0], dy = sp4[4 * i + 1] - c[1], dz = sp4[4 * i + 2] - c[2];
            const float d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 > d2max) d2max = d2;
        }
        gI[4 * g + 0] = c[0]; gI[4 * g + 1] = c[1]; gI[4 * g + 2] = c[2];
        gI[4 * g + 3] = sqrtf(d2max) * RADIUS_MARGIN;
        gamin[g] = am;
    }
}

/* ------------------------------------------------------------------------- */
/* Multipole acceptance criterion, in FP32 with a fixed operation order.     */
/* Distance (Eqs. 6-7): r = |r_J - r_I|, d = lambda r = r - b_I if b_I < r,  */
/* else 0.                                                                   */
/*   mac 0, opening angle (Eq. 2):   accept iff b_J <= theta d.              */
/*   mac 1, acceleration (Eq. 5):    d >= (G m_J b_J^2 / (D_acc |a_old|))^1/4 */
/*          evaluated as  d^4 (D_acc |a_old|) >= (G m_J) (b_J b_J),          */
/*          with d^4 = (d d)(d d) and D_acc |a_old| precomputed per group.   */
/*   mac 2, multipole (Warren & Salmon, Sec. 2.2):                           */
/*          d >= b_J/2 + sqrt(b_J^2/4 + sqrt(3 B_2 / D_mul)), B_2 = sum over   */
/*          the cell of m |r - r_J|^2; D_mul is passed in delta_acc.         */
/* Equality accepts, as the printed inequalities do.                         */
/* ------------------------------------------------------------------------- */
static int mac_accept(int mac, float theta, float dacc_amin, float delta, float G, const float *gI,
                      float jx, float jy, float jz, float mJ, float bJ, float B2) {
    const float dx = jx - gI[0];
    const float dy = jy - gI[1];
    const float dz = jz - gI[2];
    const float r2 = (dx * dx + dy * dy) + dz * dz;
    const float r = sqrtf(r2);
    const float bI = gI[3];
    const float d = (bI < r) ? (r - bI) : 0.0f;
    if (mac == 0) return bJ <= theta * d;
    if (mac == 2) return d >= 0.5f * bJ + sqrtf((0.25f * bJ) * bJ + sqrtf((3.0f * B2) / delta));
    const float d2 = d * d;
    const float lhs = (d2 * d2) * dacc_amin;
    const float rhs = (G * mJ) * (bJ * bJ);
    return lhs >= rhs;
}

/* ------------------------------------------------------------------------- */
/* A7. Tree walk for groups (Sec. 2.3): a breadth-first queue starting at    */
/* the root; each queued cell is tested against the group's pseudo          */
/* i-particle; an accepted cell joins the interaction list as one pseudo     */
/* j-particle, a rejected cell queues its children, a rejected leaf puts its */
/* particles on the list one by one.  Every group member then sums Eq. (1)   */
/* over the list (FP64 sums of the FP32 inputs), the potential included.     */
/* The member's own contribution to the potential (-G m_i/eps, present when  */
/* it appears on its own list) is removed so that phi matches Eq. (1)'s      */
/* j != i (the acceleration term of j = i is exactly zero).                  */
/* Group g holds active[starts[g] .. starts[g+1]); groups: the ids to       */
/* evaluate (all ng groups if NULL).                                         */
/* acc out: n_active x 4 doubles (ax, ay, az, phi) at the active positions   */
/* of the evaluated groups; inter out: per active particle, list length;     */
/* ntest out: per evaluated group, MAC tests made.                           */
/* Returns 0, or -1 on allocation failure.                                   */
/* ------------------------------------------------------------------------- */
int or_walk(int64_t nn, const float *jpos, const float *bj, const uint32_t *first,
            const uint32_t *count, const int32_t *child, const uint8_t *nchild,
            const float *sp4, int64_t n_active, const uint32_t *active, const uint32_t *starts,
            const float *gI, const float *gamin, int mac, float theta, float delta_acc,
            float eps, float G, int64_t n_eval, const int64_t *groups, const float *b2,
            double *acc, int64_t *inter, int64_t *ntest) {
    if (nn == 0 || n_active == 0) return 0;
    int fail = 0;
#pragma omp parallel
    {
        int64_t qcap = 1024, lcap = 1024;
        int32_t *q = (int32_t *)malloc((size_t)qcap * sizeof(int32_t));
        float *list = (float *)malloc((size_t)lcap * 4 * sizeof(float));
        if (!q || !list) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t e = 0; e < n_eval; e++) {
            if (fail) continue;
            const int64_t g = groups ? groups[e] : e;
            const float *gi = gI + 4 * g;
            const float dacc_amin = delta_acc * gamin[g];
            int64_t head = 0, tail = 0, nl = 0, tests = 0;
            q[tail++] = 0;
            while (head < tail) {
                const int32_t c = q[head++];
                tests++;
                if (mac_accept(mac, theta, dacc_amin, delta_acc, G, gi, jpos[4 * c + 0], jpos[4 * c + 1],
                               jpos[4 * c + 2], jpos[4 * c + 3], bj[c], b2 ? b2[c] : 0.0f)) {
                    if (nl + 1 > lcap) {
                        lcap *= 2;
                        list = (float *)realloc(list, (size_t)lcap * 4 * sizeof(float));
                    }
                    memcpy(list + 4 * nl, jpos + 4 * c, 4 * sizeof(float));
                    nl++;
                } else if (child[c] < 0) {
                    while (nl + count[c] > lcap) {
                        lcap *= 2;
                        list = (float *)realloc(list, (size_t)lcap * 4 * sizeof(float));
                    }
                    memcpy(list + 4 * nl, sp4 + 4 * (int64_t)first[c], (size_t)count[c] * 4 * sizeof(float));
                    nl += count[c];
                } else {
                    if (tail + nchild[c] > qcap) {
                        /* compact the consumed head, then grow */
                        memmove(q, q + head, (size_t)(tail - head) * sizeof(int32_t));
                        tail -= head; head = 0;
                        while (tail + nchild[c] > qcap) {
                            qcap *= 2;
                            q = (int32_t *)realloc(q, (size_t)qcap * sizeof(int32_t));
                        }
                    }
                    for (int k = 0; k < nchild[c]; k++) q[tail++] = child[c] + k;
                }
            }
            if (ntest) ntest[e] = tests;
            const int64_t a0 = starts[g], a1 = starts[g + 1];
            const double eps2 = (double)eps * (double)eps;
            for (int64_t k = a0; k < a1; k++) {
                const uint32_t i = active[k];
                const double xi = sp4[4 * i + 0], yi = sp4[4 * i + 1], zi = sp4[4 * i + 2];
                double ax = 0.0, ay = 0.0, az = 0.0, phi = 0.0;
                for (int64_t j = 0; j < nl; j++) {
                    const double dx = (double)list[4 * j + 0] - xi;
                    const double dy = (double)list[4 * j + 1] - yi;
                    const double dz = (double)list[4 * j + 2] - zi;
                    const double r2 = dx * dx + dy * dy + dz * dz + eps2;
                    const double rinv = 1.0 / sqrt(r2);
                    const double mr = (double)list[4 * j + 3] * rinv;
                    const double mr3 = mr * rinv * rinv;
                    ax += mr3 * dx;
                    ay += mr3 * dy;
                    az += mr3 * dz;
                    phi -= mr;
                }
                phi += (double)sp4[4 * i + 3] / (double)eps;
                acc[4 * k + 0] = (double)G * ax;
                acc[4 * k + 1] = (double)G * ay;
                acc[4 * k + 2] = (double)G * az;
                acc[4 * k + 3] = (double)G * phi;
                if (inter) inter[k] = nl;
            }
        }
        free(q);
        free(list);
    }
    return fail ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Block time step (Sec. 1; Sec. 2.7, Eqs. 15-17).                          */
/* Levels k = 0 .. L-1 have steps dt_k = dt_max 2^-k, dt_max = 2^M.  Time is */
/* an integer count of the finest step dt_{L-1}; level k spans               */
/* ticks(k) = 2^(L-1-k) ticks.  Step criterion (the paper fixes none; the    */
/* acceleration form of Springel 2005, whose MAC the paper adopts):          */
/*   dt_i = sqrt(c / |a_i|),  c = 2 eta eps.                                  */
/* The level is the smallest k with dt_k <= dt_i, clamped to [0, L-1].  Both */
/* sides are positive, so this is dt_k^4 |a|^2 <= c^2, i.e.                  */
/*   2^(4(M-k)) A2 <= c2,  A2 = (ax^2 + ay^2) + az^2,  c2 = c c  (FP64),      */
/* decided exactly from the exponents and fractions (frexp) of A2 and c2.    */
/* |a_old| = sqrtf((float)A2).                                               */
/* ------------------------------------------------------------------------- */
static int64_t floordiv4(int64_t d) { return d >= 0 ? d / 4 : -((-d + 3) / 4); }

static int level_from_a2(double a2, double c2, int M, int L) {
    if (!(a2 > 0.0) || !isfinite(a2)) return 0;
    int ea, ec;
    const double fa = frexp(a2, &ea), fc = frexp(c2, &ec);
    /* level k qualifies iff 4k > D, or 4k == D and fa <= fc, with D = ea + 4M - ec */
    const int64_t D = (int64_t)ea + 4 * (int64_t)M - ec;
    const int64_t q = floordiv4(D);
    int64_t k = (4 * q == D && fa <= fc) ? q : q + 1;
    if (k < 0) k = 0;
    if (k > L - 1) k = L - 1;
    return (int)k;
}

static double c2_of(double eta, double eps) {
    const double c = (2.0 * eta) * eps;
    return c * c;
}

static double a2_of(const float *a) {
    const double ax = a[0], ay = a[1], az = a[2];
    return (ax * ax + ay * ay) + az * az;
}

void or_a2(int64_t n, const float *acc4, double *out) {
    for (int64_t i = 0; i < n; i++) out[i] = a2_of(acc4 + 4 * i);
}

/* log2 dt_max at the start: the largest M with 2^M <= max_i dt_i, i.e. the   */
/* largest M with 2^(4M) A2min <= c2 (A2min the smallest positive A2).        */
int or_dtmax_exponent(int64_t n, const float *acc4, double eta, double eps) {
    double a2min = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        const double a2 = a2_of(acc4 + 4 * i);
        if (a2 > 0.0 && a2 < a2min) a2min = a2;
    }
    if (!isfinite(a2min)) return 0;
    int ea, ec;
    const double fa = frexp(a2min, &ea), fc = frexp(c2_of(eta, eps), &ec);
    /* M qualifies iff 4M < D, or 4M == D and fa <= fc, with D = ec - ea */
    const int64_t D = (int64_t)ec - ea;
    const int64_t q = floordiv4(D);
    if (4 * q == D) return (int)(fa <= fc ? q : q - 1);
    return (int)q;
}

/* Initial levels and first half kick (t = 0): v^{1/2} = v + (dt_k/2) a     */
/* (Eq. 15 at n = 0), as one fused multiply-add.  acc4: n x 4 FP32.         */
void or_init_levels(int64_t n, const float *acc4, const double *vel, double eta, double eps,
                    int M, int L, double dt_max, uint8_t *level, int64_t *t0, double *vh,
                    float *aold) {
    const double c2 = c2_of(eta, eps);
    for (int64_t i = 0; i < n; i++) {
        const double a2 = a2_of(acc4 + 4 * i);
        const int k = level_from_a2(a2, c2, M, L);
        const double hdt = 0.5 * ldexp(dt_max, -k);
        for (int a = 0; a < 3; a++) vh[3 * i + a] = fma(hdt, (double)acc4[4 * i + a], vel[3 * i + a]);
        level[i] = (uint8_t)k;
        t0[i] = 0;
        aold[i] = sqrtf((float)a2);
    }
}

/* A8. Prediction of all j-particles to tick T (Eq. 16 with the elapsed time */
/* T - t0 in place of dt_j; the stored v^{1/2} already holds the half kick). */
/*   r(T) = fma((T - t0) dt_min, v^{1/2}, r0) in FP64, then rounded to FP32. */
void or_predict(int64_t n, const double *r0, const double *vh, const int64_t *t0,
                const float *mass, int64_t T, double dt_min, float *p4) {
#pragma omp parallel for
    for (int64_t i = 0; i < n; i++) {
        const double dt = (double)(T - t0[i]) * dt_min;
        for (int a = 0; a < 3; a++) p4[4 * i + a] = (float)fma(dt, vh[3 * i + a], r0[3 * i + a]);
        p4[4 * i + 3] = mass[i];
    }
}

/* A9. Correction of the active particles (Eq. 17), new level, and the next  */
/* half kick.  For active particle i (sorted index active[k]) at tick T:     */
/*   v     = fma(dt_old/2, a, v^{1/2})          (Eq. 17)                     */
/*   k_new = from A2; a shorter step is always taken; a longer one only by   */
/*           one level and only when T is a multiple of the longer step      */
/*   v^{1/2} <- fma(dt_new/2, a, v);  r0 <- r(T) (the predicted position);   */
/*   t0 <- T;  |a_old| <- sqrtf((float)A2).                                   */
void or_correct(int64_t n_active, const uint32_t *active, const float *acc4, int64_t T,
                double dt_max, int M, int L, double eta, double eps, double *r0, double *vh,
                int64_t *t0, uint8_t *level, float *aold, float *acc_store) {
    const double dt_min = ldexp(dt_max, -(L - 1));
    const double c2 = c2_of(eta, eps);
    for (int64_t k = 0; k < n_active; k++) {
        const uint32_t i = active[k];
        const float *a = acc4 + 4 * k;
        const int kold = level[i];
        const double hold = 0.5 * ldexp(dt_max, -kold);
        const double dtp = (double)(T - t0[i]) * dt_min;
        double v[3];
        for (int c = 0; c < 3; c++) {
            r0[3 * i + c] = fma(dtp, vh[3 * i + c], r0[3 * i + c]);
            v[c] = fma(hold, (double)a[c], vh[3 * i + c]);
        }
        const double a2 = a2_of(a);
        const int kc = level_from_a2(a2, c2, M, L);
        int knew = kold;
        if (kc > kold) {
            knew = kc;
        } else if (kc < kold) {
            const int64_t span = (int64_t)1 << (L - 1 - (kold - 1));
            if (T % span == 0) knew = kold - 1;
        }
        const double hdt = 0.5 * ldexp(dt_max, -knew);
        for (int c = 0; c < 3; c++) vh[3 * i + c] = fma(hdt, (double)a[c], v[c]);
        level[i] = (uint8_t)knew;
        t0[i] = T;
        aold[i] = sqrtf((float)a2);
        if (acc_store) memcpy(acc_store + 4 * (int64_t)i, a, 4 * sizeof(float));
    }
}

/* ---------------- small exports used by the oracle's own pin tests ---------------- */
uint64_t or_morton3(uint64_t qx, uint64_t qy, uint64_t qz) { return interleave3(qx, qy, qz); }

int or_mac_accept(int mac, float theta, float delta_acc, float amin, float G, const float *gI,
                  const float *jp, float bJ, float B2) {
    return mac_accept(mac, theta, delta_acc * amin, delta_acc, G, gI, jp[0], jp[1], jp[2], jp[3], bJ, B2);
}

int or_level_from_a2(double a2, double eta, double eps, int M, int L) {
    return level_from_a2(a2, c2_of(eta, eps), M, L);
}

/* |a_old| from FP32 accelerations: sqrtf((float)A2). */
void or_aold(int64_t n, const float *acc4, float *out) {
    for (int64_t i = 0; i < n; i++) out[i] = sqrtf((float)a2_of(acc4 + 4 * i));
}
