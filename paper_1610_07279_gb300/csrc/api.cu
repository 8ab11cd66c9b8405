// C ABI of libgothic: system lifetime, workspace layout and the entry points that
// string the kernels together (see include/gothic.h for the contract).
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <new>
#include <vector>

#include <utility>

#include "gt_system.cuh"

static std::atomic<long long> g_launches{0};

void gt_note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// The look-back of tile 1 over a tile 0 that never publishes: the wait on tile 0's
// status word runs out after the control block's spin bound, latches GT_ETIMEOUT and
// returns.  The epoch is one no build or compaction reaches, and tile 0's word is
// cleared first, so neither the wait nor its result depends on earlier contents.
namespace {
constexpr unsigned int PROBE_EPOCH = 0x3fffffffu;
__global__ void k_wait_probe(unsigned long long *status, DevCtl *ctl) {
    if (threadIdx.x == 0) status[0] = 0ull;
    __syncwarp();
    (void)lookback_warp(status, 1u, 1u, PROBE_EPOCH, ctl, GTK_PROBE);
}
}  // namespace

void gt_launch_wait_probe(unsigned long long *status, DevCtl *ctl, cudaStream_t st) {
    { k_wait_probe<<<1, 32, 0, st>>>(status, ctl); gt_note_launches(1); }
}

namespace {

constexpr size_t ALIGN = GT_WS_ALIGN;

struct Layout {
    size_t off = 0;
    template <class T>
    T *take(char *base, size_t count) {
        off = (off + ALIGN - 1) / ALIGN * ALIGN;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int check_params(const gt_params *p) {
    if (!p) return GT_EINVAL;
    if (p->mac != GT_MAC_OPENING_ANGLE && p->mac != GT_MAC_ACCELERATION && p->mac != GT_MAC_MULTIPOLE)
        return GT_EINVAL;
    if (p->mac == GT_MAC_MULTIPOLE && !(p->delta_acc > 0.0f)) return GT_EINVAL;  // Delta_mul
    if (p->leaf_max < 1) return GT_EINVAL;
    if (p->ij_share != 0 && (!pow2(p->ij_share) || p->ij_share > 32)) return GT_EINVAL;
    // up to 32 members with ij_share lanes each, or up to 64 with one lane per two members
    if (p->group_max < 1 || p->group_max > (p->ij_share > 1 ? 32 / p->ij_share : 64)) return GT_EINVAL;
    const int gm = p->group_mode & 0xff;
    if ((p->group_mode & ~(0xff | GT_SPHERE_EBS)) != 0) return GT_EINVAL;
    if (gm != GT_GROUP_RUNS && gm != GT_GROUP_CELLS && gm != GT_GROUP_CELLS_TUNED) return GT_EINVAL;
    if (p->levels < 1 || p->levels > 30) return GT_EINVAL;
    if (p->rebuild_every < 0 || p->node_factor < 1 || p->node_factor > 64) return GT_EINVAL;
    if (!pow2(p->walk_queue) || p->walk_queue < 64) return GT_EINVAL;
    if (!(p->eps > 0.0f) || !(p->theta >= 0.0f) || !(p->delta_acc >= 0.0f)) return GT_EINVAL;
    if (!(p->eta > 0.0)) return GT_EINVAL;
    if (p->dt_max > 0.0) {
        int e;
        if (frexp(p->dt_max, &e) != 0.5) return GT_EINVAL;  // must be a power of two
    }
    if (!std::isfinite(p->r_crit)) return GT_EINVAL;
    if (p->key_curve != GT_KEY_MORTON && p->key_curve != GT_KEY_HILBERT) return GT_EINVAL;
    return GT_OK;
}

bool cell_groups(const gt_params &p) { return (p.group_mode & 0xff) != GT_GROUP_RUNS; }
bool tuned_groups(const gt_params &p) { return (p.group_mode & 0xff) == GT_GROUP_CELLS_TUNED; }

// r_crit of the groupings when it is not tuned on line: the given value, or the start
// of the search for a negative one
float fixed_rcrit(const gt_params &p) { return p.r_crit > 0.0f ? p.r_crit : (p.r_crit < 0.0f ? -p.r_crit : 0.0f); }

int device_sms(int *dev, int *nsm) {
    if (cudaGetDevice(dev) != cudaSuccess) return GT_ECUDA;
    if (cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, *dev) != cudaSuccess) return GT_ECUDA;
    return GT_OK;
}


int64_t node_capacity(int64_t n, const gt_params *p) { return (int64_t)p->node_factor * n + 2048; }

// Carve every buffer out of base (or only measure when base == nullptr).
size_t carve(gt_system *s, char *base, int64_t n, const gt_params *p, int nsm, int walk_blocks,
             bool own_queue = true) {
    Layout L;
    const size_t N = (size_t)(n > 0 ? n : 1);
    s->ctl = L.take<DevCtl>(base, 1);
    for (int b = 0; b < 2; b++) {
        State &t = s->st[b];
        double *r = L.take<double>(base, 3 * N);
        double *v = L.take<double>(base, 3 * N);
        t.rx = r; t.ry = r ? r + N : nullptr; t.rz = r ? r + 2 * N : nullptr;
        t.vx = v; t.vy = v ? v + N : nullptr; t.vz = v ? v + 2 * N : nullptr;
        t.t0 = L.take<long long>(base, N);
        t.level = L.take<uint8_t>(base, N);
        t.aold = L.take<float>(base, N);
        t.acc = L.take<float4>(base, N);
        t.id = L.take<uint32_t>(base, N);
        t.mass = L.take<float>(base, N);
    }
    s->posm = L.take<float4>(base, N);
    s->posm_tmp = L.take<float4>(base, N);
    for (int b = 0; b < 2; b++) {
        s->sb.key[b] = L.take<uint64_t>(base, N);
        s->sb.val[b] = L.take<uint32_t>(base, N);
    }
    s->sb.status = (uint32_t *)L.take<char>(base, gt_sort_scratch_bytes(n));
    s->sb.hist = L.take<uint32_t>(base, 8 * 256);
    s->sb.digit_base = L.take<uint32_t>(base, 8 * 256);
    const int64_t cap = node_capacity(n, p);
    s->cap = cap;
    s->nd.first = L.take<uint32_t>(base, cap);
    s->nd.count = L.take<uint32_t>(base, cap);
    s->nd.child = L.take<int32_t>(base, cap);
    s->nd.nchild = L.take<uint32_t>(base, cap);
    s->nd.parent = L.take<int32_t>(base, cap);
    s->nd.jpos = L.take<float4>(base, cap);
    s->nd.walk = L.take<float4>(base, cap);
    s->nd.sum = L.take<DSum4>(base, cap);
    s->nd.cells = L.take<uint32_t>(base, cap);
    const int64_t st_tiles = (cap + 511) / 512 + (n + 4095) / 4096 + 64;
    s->status = L.take<unsigned long long>(base, st_tiles);
    s->active = L.take<uint32_t>(base, N);
    s->prefix = L.take<uint32_t>(base, N + 1);
    s->flags = L.take<uint8_t>(base, N);
    s->marks = L.take<uint8_t>(base, N);
    s->gstart = L.take<uint32_t>(base, N);
    s->acc_out = L.take<float4>(base, N);
    s->aold_tmp = L.take<float>(base, N);
    s->scratch3 = L.take<double>(base, 3 * N + 8);  // also stages 13 B per particle on resume
    s->bscratch = L.take<uint8_t>(base, gt_build_scratch_bytes(n));
    s->bbox_blocks = nsm * 4;
    s->bbox_partial = L.take<float>(base, 6 * (size_t)s->bbox_blocks);
    s->walk_blocks = walk_blocks;
    s->walk_warps = walk_blocks * gt_walk_warps_per_block();
    s->queue_entries = own_queue ? (int64_t)s->walk_warps * p->walk_queue : 0;
    s->queue = own_queue ? L.take<uint32_t>(base, (size_t)s->queue_entries) : nullptr;
    return (L.off + ALIGN - 1) / ALIGN * ALIGN;
}

int last_cuda() { return cudaGetLastError() == cudaSuccess ? GT_OK : GT_ECUDA; }

enum { PH_PREDICT = 0, PH_SORT, PH_PERMUTE, PH_BUILD, PH_PSEUDO, PH_ACTIVE, PH_WALK, PH_CORRECT };

bool timing(const gt_system *s) { return s->prof.on || (s->prof.created && s->prm.rebuild_every == 0); }

void ph_begin(gt_system *s, int p, cudaStream_t st) {
    if (timing(s)) cudaEventRecord(s->prof.b[p], st);
}

void ph_end(gt_system *s, int p, cudaStream_t st) {
    if (timing(s)) {
        cudaEventRecord(s->prof.e[p], st);
        s->prof.ran[p] = true;
    }
}

void ph_add(gt_system *s, int p, cudaEvent_t b, cudaEvent_t e, bool total = true) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b, e) == cudaSuccess) {
        if (total) {
            s->prof.ms[p] += ms;
            s->prof.cnt[p] += 1;
        }
        s->prof.last_ms[p] = ms;
    }
}

// Fold the finished phases' times in: every phase recorded since the last call, and
// the predictions enqueued ahead of their step -- both of them (ahead_slot < 0: the
// stream has been synchronised) or only the one of parity ahead_slot (the other may
// still be running).
void ph_collect(gt_system *s, int ahead_slot = -1) {
    if (!timing(s)) return;
    for (int p = 0; p < GT_NPHASES; p++) {
        if (!s->prof.ran[p]) continue;
        ph_add(s, p, s->prof.b[p], s->prof.e[p], !s->prof.before[p]);
        s->prof.ran[p] = false;
        s->prof.before[p] = false;
    }
    for (int q = 0; q < 2; q++) {
        if (!s->prof.aran[q] || (ahead_slot >= 0 && q != ahead_slot)) continue;
        ph_add(s, PH_PREDICT, s->prof.ab[q], s->prof.ae[q]);
        s->prof.aran[q] = false;
    }
}

int ensure_events(gt_system *s) {
    if (s->prof.created) return GT_OK;
    for (int p = 0; p < GT_NPHASES; p++)
        if (cudaEventCreate(&s->prof.b[p]) || cudaEventCreate(&s->prof.e[p])) return GT_ECUDA;
    for (int q = 0; q < 2; q++)
        if (cudaEventCreate(&s->prof.ab[q]) || cudaEventCreate(&s->prof.ae[q])) return GT_ECUDA;
    s->prof.created = true;
    return GT_OK;
}

// The look-ahead's mapped host words and events, made on first use; false if they
// cannot be had (the block step then reads the control words after a stream sync).
bool ahead_ready(gt_system *s) {
    if (s->mirror) return true;
    if (s->mirror_tried) return false;
    s->mirror_tried = true;
    void *h = nullptr, *d = nullptr;
    if (cudaHostAlloc(&h, sizeof(StepMirror), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ahead_mirror, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ahead_done, cudaEventDisableTiming) != cudaSuccess) {
        if (s->ahead_mirror) cudaEventDestroy(s->ahead_mirror);
        if (s->ahead_done) cudaEventDestroy(s->ahead_done);
        s->ahead_mirror = s->ahead_done = nullptr;
        cudaFreeHost(h);
        cudaGetLastError();
        return false;
    }
    s->mirror = (StepMirror *)h;
    s->mirror_dev = (StepMirror *)d;
    return true;
}

// Forget the prediction enqueued ahead (the state or the tree is about to change, or
// the next step runs on another stream); work on another stream is ordered after it,
// since it still writes posm_tmp.
void drop_ahead(gt_system *s, cudaStream_t st) {
    if (!s->ahead) return;
    if (st != s->ahead_st) cudaStreamWaitEvent(st, s->ahead_done, 0);
    s->ahead = false;
}

// After a synchronised block step: feed its walk time (and, after a rebuild, the
// rebuild's time) to the interval model.
void tune_after_step(gt_system *s, bool rebuilt, unsigned n_active) {
    RebuildTuner &t = s->tune;
    if (rebuilt) {
        t.y.clear();
        t.t_make = s->prof.last_ms[PH_SORT] + s->prof.last_ms[PH_PERMUTE] + s->prof.last_ms[PH_BUILD];
        t.since = 0;
        t.n_opt = 1e6;
    }
    t.since++;
    if (n_active == 0) return;
    t.nact_sum += n_active;
    t.nact_cnt++;
    const double mean = t.nact_sum / (double)t.nact_cnt;
    t.y.push_back(s->prof.last_ms[PH_WALK] * mean / (double)n_active);
    if (t.y.size() >= 3) {
        int model = -1;
        double nopt = 1e6;
        if (gt_rebuild_interval(t.y.data(), (int)t.y.size(), t.t_make, &model, &nopt, nullptr) == GT_OK) {
            t.model = model;
            t.n_opt = nopt;
        }
    }
}

// class of the block step at T: the coarsest level active then (levels k with
// T mod 2^(L-1-k) == 0 are active)
int step_class(const gt_system *s, unsigned long long T) {
    const int L = s->prm.levels;
    const int tz = T == 0ull ? 63 : __builtin_ctzll(T);
    return L - 1 - (tz < L - 1 ? tz : L - 1);
}

int gsize_candidate(const gt_system *s, int c) {
    const int g = s->prm.group_max >> (GroupTuner::NCAND - 1 - c);  // group_max / 4, / 2, / 1
    return g >= 1 ? g : 1;
}

void gsize_after_step(gt_system *s, unsigned n_active) {
    GroupTuner &t = s->gtune;
    if (t.pending_class >= 0 && n_active > 0 && s->prof.last_ms[PH_WALK] > 0.0) {
        t.sum[t.pending_class][t.pending_cand] += s->prof.last_ms[PH_WALK] / (double)n_active;
        t.cnt[t.pending_class][t.pending_cand] += 1;
    }
    t.pending_class = -1;
}

void gsize_before_step(gt_system *s, unsigned long long T) {
    GroupTuner &t = s->gtune;
    const int k0 = step_class(s, T);
    if (k0 < 0 || k0 >= GroupTuner::NCLASS) return;
    if (++t.seen[k0] % 64 == 0)
        for (int c = 0; c < GroupTuner::NCAND; c++) t.sum[k0][c] = 0.0, t.cnt[k0][c] = 0;
    int pick = -1;
    for (int c = GroupTuner::NCAND - 1; c >= 0 && pick < 0; c--)  // the largest size first
        if (t.cnt[k0][c] < 1) pick = c;
    if (pick < 0) {
        pick = GroupTuner::NCAND - 1;
        for (int c = 0; c < GroupTuner::NCAND; c++)
            if (t.sum[k0][c] / t.cnt[k0][c] < t.sum[k0][pick] / t.cnt[k0][pick]) pick = c;
    }
    s->gmax_now = gsize_candidate(s, pick);
    t.pending_class = k0;
    t.pending_cand = pick;
}

// Sec. 2.4 on line: the walk time per active particle of the step just finished goes
// to the search of its class; the step at block time T gets the next r_crit of its
// class (the coarsest level active at T).
void rcrit_after_step(gt_system *s, unsigned n_active) {
    RcritTuner &t = s->rtune;
    if (t.pending >= 0 && n_active > 0 && s->prof.last_ms[PH_WALK] > 0.0) {
        BrentSearch &b = t.search[t.pending];
        if (gt_brent_done(&b)) t.held[t.pending]++;
        else gt_brent_report(&b, s->prof.last_ms[PH_WALK] / (double)n_active);
    }
    t.pending = -1;
}

void rcrit_before_step(gt_system *s, unsigned long long T) {
    const int k0 = step_class(s, T);
    RcritTuner &t = s->rtune;
    if (k0 < 0 || k0 >= RcritTuner::NCLASS) return;
    BrentSearch &b = t.search[k0];
    const double x0 = std::log((double)fixed_rcrit(s->prm));
    if (!t.started[k0]) {
        gt_brent_start(&b, x0 - std::log(16.0), x0 + std::log(16.0), 0.0, 0.05);
        t.started[k0] = true;
    } else if (gt_brent_done(&b) && t.held[k0] >= 8) {  // perturb: search again around the best
        const double xb = b.x;
        gt_brent_start(&b, xb - std::log(2.0), xb + std::log(2.0), 0.0, 0.05);
        t.held[k0] = 0;
    }
    s->rcrit_now = (float)std::exp(gt_brent_next(&b));
    t.pending = k0;
}

void ph_sync_collect(gt_system *s, cudaStream_t st) {
    if (!s->prof.on) return;
    cudaStreamSynchronize(st);
    ph_collect(s);
}

cudaStream_t S(gt_stream s) { return (cudaStream_t)s; }

// A1-A5 on FP32 positions posm_src (s->posm or the predicted s->posm_tmp): keys, sort,
// then every particle array gathered into key order.  Buffer roles never change
// (state 0 and posm always hold the current data), so the launches can be captured
// in a CUDA graph and replayed.
void build_tree(gt_system *s, cudaStream_t st, const float4 *posm_src) {
    const int64_t n = s->n;
    gt_launch_prepare(s->ctl, 0, st);
    ph_begin(s, PH_SORT, st);
    gt_launch_bbox(posm_src, n, s->bbox_partial, s->bbox_blocks, s->ctl, st);
    gt_launch_keys(posm_src, n, s->ctl, s->prm.key_curve, s->sb.key[0], s->sb.val[0], st);
    gt_launch_sort(s->sb, n, s->ctl, st);
    ph_end(s, PH_SORT, st);
    ph_begin(s, PH_PERMUTE, st);
    if (!s->fixed_buffers) {
        // the gathered copy becomes the state: the two buffers swap roles
        float4 *dst = posm_src == s->posm_tmp ? s->posm : s->posm_tmp;
        gt_launch_permute(s->st[0], s->st[1], posm_src, dst, s->sb.val[0], n, st);
        std::swap(s->st[0], s->st[1]);
        if (dst != s->posm) std::swap(s->posm, s->posm_tmp);
    } else if (posm_src == s->posm_tmp) {
        gt_launch_permute(s->st[0], s->st[1], posm_src, s->posm, s->sb.val[0], n, st);
        gt_launch_copy_state(s->st[1], s->st[0], nullptr, nullptr, n, st);
    } else {
        gt_launch_permute(s->st[0], s->st[1], posm_src, s->posm_tmp, s->sb.val[0], n, st);
        gt_launch_copy_state(s->st[1], s->st[0], s->posm_tmp, s->posm, n, st);
    }
    ph_end(s, PH_PERMUTE, st);
    ph_begin(s, PH_BUILD, st);
    gt_launch_build(s->sb.key[0], n, s->prm.leaf_max, s->nd, s->cap, s->status, s->bscratch, s->ctl, s->nsm, st);
    gt_launch_cell_lists(s->nd, s->cap, s->ctl, s->nsm, st);
    ph_end(s, PH_BUILD, st);
    ph_begin(s, PH_PSEUDO, st);
    gt_launch_pseudo(s->nd, s->cap, s->posm, s->ctl, s->nsm, true, st);
    ph_end(s, PH_PSEUDO, st);
    s->have_tree = true;
    s->rebuilds++;
}

double c2_of(const gt_params &p) {
    const double c = (2.0 * p.eta) * (double)p.eps;
    return c * c;
}

// A6 groups + A7 walk over the active list already in s->active / ctl->n_active
// (cell grouping needs the prefix s->prefix of that list), or over a caller's list.
void walk(gt_system *s, const uint32_t *active, const float *aold, float4 *acc, int mac, cudaStream_t st) {
    if (cell_groups(s->prm))
        gt_launch_groups(s->nd, s->cap, s->prefix, s->gmax_now, s->rcrit_now, s->n, s->marks, s->ctl, s->gstart,
                         s->status, s->nsm, st);
    const WalkArgs a = gt_sys_walk_args(s, active, aold, acc, mac);
    ph_begin(s, PH_WALK, st);
    gt_launch_walk(a, s->walk_blocks, st);
    ph_end(s, PH_WALK, st);
}

// every particle active (start-up passes, gt_accel_active with no list)
void walk_all(gt_system *s, const float *aold, float4 *acc, int mac, cudaStream_t st) {
    gt_launch_prepare(s->ctl, 0, st);
    gt_launch_active(s->st[0], s->n, s->prm.levels, 1, s->ctl, s->active, s->prefix, s->status, s->nsm, st);
    walk(s, nullptr, aold, acc, mac, st);
}

}  // namespace

// ---- helpers shared with the batch and the server ------------------------------
int gt_sys_check_params(const gt_params *p) { return check_params(p); }

int gt_sys_device_sms(int *dev, int *nsm) { return device_sms(dev, nsm); }

size_t gt_sys_carve(gt_system *s, char *base, int64_t n, const gt_params *p, int nsm, int walk_blocks,
                    bool own_queue) {
    return carve(s, base, n, p, nsm, walk_blocks, own_queue);
}

int gt_sys_init(gt_system *s, int64_t n, const gt_params *p, void *ws, size_t ws_bytes, bool own_queue,
                cudaStream_t st) {
    int rc = device_sms(&s->dev, &s->nsm);
    if (rc) return rc;
    gt_sort_init();
    const int wb = gt_walk_blocks(s->nsm);
    const size_t need = carve(s, nullptr, n, p, s->nsm, wb, own_queue);
    if (ws_bytes < need) return GT_ENOMEM;
    carve(s, (char *)ws, n, p, s->nsm, wb, own_queue);
    s->n = n;
    s->fixed_buffers = !own_queue;
    gt_sys_apply_params(s, *p);
    // zero the control block and the look-back status words (on st, then wait for it;
    // without a stream, on the default stream and wait for the device)
    const size_t st_bytes = (size_t)((s->cap + 511) / 512 + (n + 4095) / 4096 + 64) * 8;
    if (cudaMemsetAsync(s->ctl, 0, sizeof(DevCtl), st) != cudaSuccess ||
        cudaMemsetAsync(s->status, 0, st_bytes, st) != cudaSuccess ||
        cudaMemsetAsync(s->sb.status, 0, gt_sort_scratch_bytes(n), st) != cudaSuccess ||
        (st ? cudaStreamSynchronize(st) : cudaDeviceSynchronize()) != cudaSuccess)
        return GT_ECUDA;
    return GT_OK;
}

void gt_sys_apply_params(gt_system *s, const gt_params &p) {
    s->prm = p;
    s->rcrit_now = fixed_rcrit(p);
    s->rtune = RcritTuner();
    s->gmax_now = p.group_max;
    s->gtune = GroupTuner();
}

void gt_sys_build_tree(gt_system *s, cudaStream_t st, const float4 *posm_src) { build_tree(s, st, posm_src); }

void gt_sys_groups_all(gt_system *s, cudaStream_t st) {
    gt_launch_prepare(s->ctl, 0, st);
    gt_launch_active(s->st[0], s->n, s->prm.levels, 1, s->ctl, s->active, s->prefix, s->status, s->nsm, st);
    if (cell_groups(s->prm))
        gt_launch_groups(s->nd, s->cap, s->prefix, s->gmax_now, s->rcrit_now, s->n, s->marks, s->ctl, s->gstart,
                         s->status, s->nsm, st);
}

WalkArgs gt_sys_walk_args(const gt_system *s, const uint32_t *active, const float *aold, float4 *acc, int mac) {
    WalkArgs a;
    a.gstart = cell_groups(s->prm) ? s->gstart : nullptr;
    a.jpos = s->nd.jpos;
    a.walk = s->nd.walk;
    a.posm = s->posm;
    a.active = active;
    a.aold = aold;
    a.acc = acc;
    a.queue = s->queue;
    a.ctl = s->ctl;
    a.n = (uint32_t)s->n;
    a.gmax = s->gmax_now;
    a.qcap = s->prm.walk_queue;
    a.mac = mac;
    a.ij_share = s->prm.ij_share;
    a.sphere = (s->prm.group_mode & GT_SPHERE_EBS) ? 1 : 0;
    a.theta = s->prm.theta;
    a.delta_acc = s->prm.delta_acc;
    a.eps2 = s->prm.eps * s->prm.eps;
    a.G = s->prm.G;
    a.inv_eps = 1.0f / s->prm.eps;
    return a;
}

void gt_sys_aold_from_acc(gt_system *s, cudaStream_t st) { gt_launch_aold(s->acc_out, s->n, s->st[0].aold, st); }

void gt_sys_step_pre(gt_system *s, cudaStream_t st, bool rebuild, bool predicted) {
    const int64_t n = s->n;
    gt_launch_prepare(s->ctl, 1, st);
    if (!predicted) {
        ph_begin(s, PH_PREDICT, st);
        gt_launch_predict(s->st[0], n, s->ctl, rebuild ? s->posm_tmp : s->posm, st);
        ph_end(s, PH_PREDICT, st);
    } else if (!rebuild) {
        std::swap(s->posm, s->posm_tmp);  // the prediction enqueued ahead went to posm_tmp
    }
    if (rebuild) {
        build_tree(s, st, s->posm_tmp);
    } else {
        ph_begin(s, PH_PSEUDO, st);
        gt_launch_pseudo(s->nd, s->cap, s->posm, s->ctl, s->nsm, false, st);  // masses as at the build
        ph_end(s, PH_PSEUDO, st);
    }
    ph_begin(s, PH_ACTIVE, st);
    gt_launch_active(s->st[0], n, s->prm.levels, 0, s->ctl, s->active, s->prefix, s->status, s->nsm, st);
    ph_end(s, PH_ACTIVE, st);
}

void gt_sys_step_groups(gt_system *s, cudaStream_t st) {
    if (cell_groups(s->prm))
        gt_launch_groups(s->nd, s->cap, s->prefix, s->gmax_now, s->rcrit_now, s->n, s->marks, s->ctl, s->gstart,
                         s->status, s->nsm, st);
}

void gt_sys_step_post(gt_system *s, cudaStream_t st) {
    ph_begin(s, PH_CORRECT, st);
    gt_launch_correct(s->st[0], s->active, s->acc_out, s->ctl, s->n, s->prm.levels, c2_of(s->prm), s->nsm, st);
    ph_end(s, PH_CORRECT, st);
    s->steps++;
}

void gt_sys_start_levels(gt_system *s, cudaStream_t st) {
    int M = 0, have_M = 0;
    if (s->prm.dt_max > 0.0) {
        int e;
        frexp(s->prm.dt_max, &e);
        M = e - 1;
        have_M = 1;
    }
    gt_launch_init_levels(s->st[0], s->acc_out, s->n, s->prm.levels, c2_of(s->prm), M, have_M, s->ctl, s->nsm, st);
    s->started = true;
    s->steps = 0;
    s->tune = RebuildTuner();
}

extern "C" {

const char *gt_strerror(int status) {
    switch (status) {
        case GT_OK: return "ok";
        case GT_EINVAL: return "invalid argument";
        case GT_ENOMEM: return "workspace too small";
        case GT_EOVERFLOW: return "device buffer overflow (tree nodes or walk queue)";
        case GT_ETIMEOUT: return "bounded device wait ran out";
        case GT_ECUDA: return "CUDA runtime error";
        case GT_EAGAIN: return "no slot or memory free; retry";
        case GT_EPENDING: return "request not finished";
        case GT_ENOTIMPL: return "not implemented";
        case GT_ESTATE: return "call out of order";
        default: return "unknown status";
    }
}

int gt_default_params(gt_params *p) {
    if (!p) return GT_EINVAL;
    memset(p, 0, sizeof(*p));
    p->mac = GT_MAC_ACCELERATION;
    p->theta = 0.5f;
    p->delta_acc = 0.0078125f;  // 2^-7
    p->eps = 0.015625f;         // 1/64
    p->G = 1.0f;
    p->leaf_max = 16;
    p->group_max = 64;
    p->ij_share = 0;
    p->group_mode = GT_GROUP_CELLS_TUNED;
    p->levels = 8;
    p->rebuild_every = 0;
    p->walk_queue = 16384;
    p->node_factor = 2;
    p->eta = 0.025;
    p->dt_max = 0.0;
    return GT_OK;
}

int gt_workspace_bytes(int64_t n, const gt_params *prm, size_t *bytes) {
    if (!bytes || n < 0 || n >= (int64_t)1 << 30) return GT_EINVAL;
    int rc = check_params(prm);
    if (rc) return rc;
    int dev, nsm;
    if ((rc = device_sms(&dev, &nsm))) return rc;
    gt_system tmp;
    *bytes = carve(&tmp, nullptr, n, prm, nsm, gt_walk_blocks(nsm));
    return GT_OK;
}

int gt_system_create(gt_system **out, int64_t n, const gt_params *prm, void *d_ws, size_t ws_bytes) {
    if (!out || n < 0 || n >= (int64_t)1 << 30 || !d_ws) return GT_EINVAL;
    if (((uintptr_t)d_ws) % ALIGN) return GT_EINVAL;
    int rc = check_params(prm);
    if (rc) return rc;
    gt_system *s = new (std::nothrow) gt_system();
    if (!s) return GT_ENOMEM;
    if ((rc = gt_sys_init(s, n, prm, d_ws, ws_bytes, true, nullptr))) {
        delete s;
        return rc;
    }
    *out = s;
    return GT_OK;
}

int gt_system_destroy(gt_system *s) {
    if (s && s->ahead) cudaEventSynchronize(s->ahead_done);  // it writes the mapped words and the workspace
    if (s && s->prof.created) {
        for (int p = 0; p < GT_NPHASES; p++) {
            cudaEventDestroy(s->prof.b[p]);
            cudaEventDestroy(s->prof.e[p]);
        }
        for (int q = 0; q < 2; q++) {
            cudaEventDestroy(s->prof.ab[q]);
            cudaEventDestroy(s->prof.ae[q]);
        }
    }
    if (s && s->mirror) {
        cudaEventDestroy(s->ahead_mirror);
        cudaEventDestroy(s->ahead_done);
        cudaFreeHost(s->mirror);
    }
    delete s;
    return GT_OK;
}

int gt_set_params(gt_system *s, const gt_params *prm) {
    if (!s) return GT_EINVAL;
    int rc = check_params(prm);
    if (rc) return rc;
    // the queue and node regions are fixed at create
    if (prm->walk_queue > s->prm.walk_queue || prm->node_factor != s->prm.node_factor) return GT_EINVAL;
    if (s->started && (prm->levels != s->prm.levels || prm->dt_max != s->prm.dt_max)) return GT_ESTATE;
    const int qcap_region = s->prm.walk_queue;
    gt_sys_apply_params(s, *prm);
    s->prm.walk_queue = prm->walk_queue;
    (void)qcap_region;
    return GT_OK;
}

int gt_set_state(gt_system *s, const double *p_pos, const double *p_vel, const float *p_mass,
                 gt_stream stream) {
    if (!s || (s->n > 0 && (!p_pos || !p_vel || !p_mass))) return GT_EINVAL;
    cudaStream_t st = S(stream);
    drop_ahead(s, st);
    const int64_t n = s->n;
    State &t = s->st[0];
    if (n > 0) {
        if (cudaMemcpyAsync(s->scratch3, p_pos, (size_t)n * 24, cudaMemcpyDefault, st) != cudaSuccess) return GT_ECUDA;
        gt_launch_deinterleave3(s->scratch3, n, t.rx, t.ry, t.rz, st);
        if (cudaMemcpyAsync(s->scratch3, p_vel, (size_t)n * 24, cudaMemcpyDefault, st) != cudaSuccess) return GT_ECUDA;
        gt_launch_deinterleave3(s->scratch3, n, t.vx, t.vy, t.vz, st);
        if (cudaMemcpyAsync(t.mass, p_mass, (size_t)n * 4, cudaMemcpyDefault, st) != cudaSuccess) return GT_ECUDA;
        gt_launch_load(t, s->posm, n, st);
    }
    s->started = false;
    s->have_tree = false;
    s->steps = 0;
    return last_cuda();
}

int gt_build_tree(gt_system *s, gt_stream stream) {
    if (!s) return GT_EINVAL;
    drop_ahead(s, S(stream));
    build_tree(s, S(stream), s->posm);
    return last_cuda();
}

int gt_accel_active(gt_system *s, const uint32_t *d_active, int64_t n_active, const float *d_aold,
                    float *d_acc, gt_stream stream) {
    if (!s || !d_acc || n_active < 0 || n_active > s->n) return GT_EINVAL;
    if (!d_active && n_active != s->n) return GT_EINVAL;
    if (!s->have_tree) return GT_ESTATE;
    cudaStream_t st = S(stream);
    drop_ahead(s, st);
    const float *aold = d_aold ? d_aold : s->st[0].aold;
    if (!d_active) {
        walk_all(s, aold, (float4 *)d_acc, s->prm.mac, st);
    } else if (cell_groups(s->prm)) {
        gt_launch_prepare(s->ctl, 0, st);
        gt_launch_active_from_list(d_active, n_active, s->n, s->flags, s->ctl, s->active, s->prefix, s->status,
                                   s->nsm, st);
        walk(s, s->active, aold, (float4 *)d_acc, s->prm.mac, st);
    } else {
        gt_launch_prepare(s->ctl, 0, st);
        gt_launch_set_nactive(s->ctl, (unsigned)n_active, st);
        walk(s, d_active, aold, (float4 *)d_acc, s->prm.mac, st);
    }
    return last_cuda();
}

int gt_start(gt_system *s, const float *p_aold_boot, gt_stream stream) {
    if (!s) return GT_EINVAL;
    cudaStream_t st = S(stream);
    drop_ahead(s, st);
    const int64_t n = s->n;
    build_tree(s, st, s->posm);
    State &t = s->st[0];
    if (p_aold_boot) {
        if (n > 0 && cudaMemcpyAsync(s->aold_tmp, p_aold_boot, (size_t)n * 4, cudaMemcpyDefault, st) != cudaSuccess)
            return GT_ECUDA;
        gt_launch_gather_f(s->aold_tmp, t.id, n, t.aold, st);
    } else {
        walk_all(s, nullptr, s->acc_out, GT_MAC_OPENING_ANGLE, st);
        gt_launch_aold(s->acc_out, n, t.aold, st);
        ph_sync_collect(s, st);
    }
    walk_all(s, t.aold, s->acc_out, s->prm.mac, st);
    gt_sys_start_levels(s, st);
    return last_cuda();
}

int gt_block_step(gt_system *s, gt_stream stream) {
    if (!s) return GT_EINVAL;
    if (!s->started) return GT_ESTATE;
    cudaStream_t st = S(stream);
    const int64_t n = s->n;
    if (n == 0) return GT_OK;
    if (s->ahead && st != s->ahead_st) drop_ahead(s, st);
    const bool predicted = s->ahead;  // this step's prediction is already enqueued
    s->ahead = false;
    bool rebuild;
    if (s->prm.rebuild_every == 0) {  // automatic interval (Sec. 2.6)
        if (ensure_events(s)) return GT_ECUDA;
        unsigned na = 0;
        unsigned long long tn = 0;
        if (predicted) {  // the previous step has finished once its mirror is written
            if (cudaEventSynchronize(s->ahead_mirror) != cudaSuccess) return GT_ECUDA;
            const volatile StepMirror *m = s->mirror;
            na = m->n_active;
            tn = m->tnext_acc;
        } else if (cudaMemcpyAsync(&na, &s->ctl->n_active, 4, cudaMemcpyDeviceToHost, st) ||
                   cudaMemcpyAsync(&tn, &s->ctl->tnext_acc, 8, cudaMemcpyDeviceToHost, st) ||
                   cudaStreamSynchronize(st)) {
            return GT_ECUDA;
        }
        if (s->steps > 0) {
            const bool was_rebuild = s->last_rebuilt;
            // this step's own prediction (parity steps & 1) may still be running
            ph_collect(s, predicted ? (int)((s->steps - 1) & 1) : -1);
            tune_after_step(s, was_rebuild, na);
            if (s->prm.r_crit < 0.0f) rcrit_after_step(s, na);
        }
        if (tuned_groups(s->prm)) {
            if (s->steps > 0) gsize_after_step(s, na);
            gsize_before_step(s, tn);
        }
        if (s->prm.r_crit < 0.0f && cell_groups(s->prm)) rcrit_before_step(s, tn);
        const double cap = 256.0;
        const double n_opt = s->tune.n_opt < cap ? s->tune.n_opt : cap;
        rebuild = s->steps == 0 || (double)s->tune.since >= std::ceil(n_opt);
    } else {
        if (s->prof.on) {  // profiling: the previous step's phase times, before their events are reused
            if (cudaStreamSynchronize(st) != cudaSuccess) return GT_ECUDA;
            ph_collect(s);
        }
        rebuild = s->steps % s->prm.rebuild_every == 0;
    }
    s->last_rebuilt = rebuild;
    gt_sys_step_pre(s, st, rebuild, predicted);
    State &t = s->st[0];
    walk(s, s->active, t.aold, s->acc_out, s->prm.mac, st);
    gt_sys_step_post(s, st);
    // Look-ahead (automatic interval; the tuners wait for every step): the control
    // words the next call reads, then the prediction of every particle to the next
    // block time (A8 does not depend on the tuners), which then runs while the host
    // tunes and enqueues the rest of that step.
    if (s->prm.rebuild_every == 0 && !s->fixed_buffers && ahead_ready(s)) {
        gt_launch_mirror(s->ctl, s->mirror_dev, st);
        cudaEventRecord(s->ahead_mirror, st);
        const int q = (int)(s->steps & 1);  // parity of the step it belongs to
        if (timing(s)) cudaEventRecord(s->prof.ab[q], st);
        gt_launch_predict(t, n, s->ctl, s->posm_tmp, st, true);
        if (timing(s)) {
            cudaEventRecord(s->prof.ae[q], st);
            s->prof.aran[q] = true;
        }
        cudaEventRecord(s->ahead_done, st);
        s->ahead = true;
        s->ahead_st = st;
    }
    return last_cuda();
}

int gt_set_integrator_state(gt_system *s, const uint8_t *p_level, const int64_t *p_t0, const float *p_aold,
                            const float *p_acc, double dt_max, int64_t T, gt_stream stream) {
    if (!s || !(dt_max > 0.0) || T < 0) return GT_EINVAL;
    if (s->n > 0 && (!p_level || !p_t0 || !p_aold)) return GT_EINVAL;
    int e;
    if (frexp(dt_max, &e) != 0.5) return GT_EINVAL;
    cudaStream_t st = S(stream);
    drop_ahead(s, st);
    const int64_t n = s->n;
    const int L = s->prm.levels;
    State &t = s->st[0];
    if (n > 0) {
        // stage the caller-order arrays in scratch (24 B per particle is enough for 1+8+4 B)
        char *base = (char *)s->scratch3;
        uint8_t *lv = (uint8_t *)base;
        long long *t0 = (long long *)(base + ((n + 15) / 16) * 16);
        float *ao = (float *)(t0 + n);
        if (cudaMemcpyAsync(lv, p_level, (size_t)n, cudaMemcpyDefault, st) ||
            cudaMemcpyAsync(t0, p_t0, (size_t)n * 8, cudaMemcpyDefault, st) ||
            cudaMemcpyAsync(ao, p_aold, (size_t)n * 4, cudaMemcpyDefault, st))
            return GT_ECUDA;
        if (p_acc && cudaMemcpyAsync(s->acc_out, p_acc, (size_t)n * 16, cudaMemcpyDefault, st)) return GT_ECUDA;
        gt_launch_gather_resume(lv, t0, ao, p_acc ? s->acc_out : nullptr, t, n, st);
    }
    gt_launch_set_clock(s->ctl, e - 1, L, T, st);
    gt_launch_tnext_all(t, n, L, s->ctl, s->nsm, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return GT_ECUDA;  // the staged scratch is reused
    s->started = true;
    s->steps = 0;
    return last_cuda();
}

int gt_predict(gt_system *s, int64_t T, float *d_posm, gt_stream stream) {
    if (!s || !d_posm || T < 0) return GT_EINVAL;
    if (!s->started) return GT_ESTATE;
    cudaStream_t st = S(stream);
    drop_ahead(s, st);
    gt_launch_set_tnext(s->ctl, T, st);
    gt_launch_predict(s->st[0], s->n, s->ctl, (float4 *)d_posm, st);
    return last_cuda();
}

int gt_correct(gt_system *s, const uint32_t *d_active, int64_t n_active, const float *d_acc, int64_t T,
               gt_stream stream) {
    if (!s || n_active < 0 || n_active > s->n || (n_active > 0 && (!d_active || !d_acc)) || T < 0)
        return GT_EINVAL;
    if (!s->started) return GT_ESTATE;
    cudaStream_t st = S(stream);
    drop_ahead(s, st);
    State &t = s->st[0];
    gt_launch_set_tnext(s->ctl, T, st);
    gt_launch_set_nactive(s->ctl, (unsigned)n_active, st);
    gt_launch_correct(t, d_active, (const float4 *)d_acc, s->ctl, s->n, s->prm.levels, c2_of(s->prm), s->nsm, st);
    // the next block time over every particle
    gt_launch_prepare(s->ctl, 1, st);
    gt_launch_tnext_all(t, s->n, s->prm.levels, s->ctl, s->nsm, st);
    gt_launch_set_tnext(s->ctl, T, st);
    return last_cuda();
}

int gt_advance(gt_system *s, int64_t T_end, int64_t *steps, gt_stream stream) {
    if (!s) return GT_EINVAL;
    if (!s->started) return GT_ESTATE;
    cudaStream_t st = S(stream);
    int64_t k = 0;
    for (;;) {
        unsigned long long tn = 0;
        int err = 0;
        if (s->ahead && s->ahead_st == st) {  // the words mirrored after the last step
            if (cudaEventSynchronize(s->ahead_mirror) != cudaSuccess) return GT_ECUDA;
            const volatile StepMirror *m = s->mirror;
            tn = m->tnext_acc;
            err = m->err;
        } else {
            if (cudaMemcpyAsync(&tn, &s->ctl->tnext_acc, 8, cudaMemcpyDeviceToHost, st) ||
                cudaMemcpyAsync(&err, &s->ctl->err, 4, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
                return GT_ECUDA;
            ph_collect(s);
        }
        if (err) return err;
        if (s->n == 0 || tn == ~0ull || (long long)tn > T_end) break;
        const int rc = gt_block_step(s, stream);
        if (rc) return rc;
        k++;
    }
    if (steps) *steps = k;
    return GT_OK;
}

int gt_profile(gt_system *s, int enable) {
    if (!s) return GT_EINVAL;
    if (enable && ensure_events(s)) return GT_ECUDA;
    s->prof.on = enable != 0;
    for (int p = 0; p < GT_NPHASES; p++) {
        s->prof.ms[p] = 0.0;
        s->prof.cnt[p] = 0;
        // a phase still to be read keeps feeding the on-line tuners, outside the new totals
        s->prof.before[p] = s->prof.ran[p];
    }
    s->prof.aran[0] = s->prof.aran[1] = false;
    return GT_OK;
}

int gt_get_timers(gt_system *s, double *ms_out, int64_t *launches_out, gt_stream stream) {
    if (!s) return GT_EINVAL;
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return GT_ECUDA;
    ph_collect(s);
    for (int p = 0; p < GT_NPHASES; p++) {
        if (ms_out) ms_out[p] = s->prof.ms[p];
        if (launches_out) launches_out[p] = s->prof.cnt[p];
    }
    return GT_OK;
}

int gt_kernel_launches(int64_t *count) {
    if (!count) return GT_EINVAL;
    *count = g_launches.load();
    return GT_OK;
}

int gt_get_state(gt_system *s, double *p_pos, double *p_vel, float *p_mass, float *p_acc, float *p_aold,
                 uint8_t *p_level, int64_t *p_t0, uint32_t *p_id, gt_stream stream) {
    if (!s) return GT_EINVAL;
    cudaStream_t st = S(stream);
    const int64_t n = s->n;
    if (n == 0) return GT_OK;
    const State &t = s->st[0];
    if (p_pos) {
        gt_launch_interleave3(t.rx, t.ry, t.rz, n, s->scratch3, st);
        if (cudaMemcpyAsync(p_pos, s->scratch3, (size_t)n * 24, cudaMemcpyDefault, st)) return GT_ECUDA;
    }
    if (p_vel) {
        gt_launch_interleave3(t.vx, t.vy, t.vz, n, s->scratch3, st);
        if (cudaMemcpyAsync(p_vel, s->scratch3, (size_t)n * 24, cudaMemcpyDefault, st)) return GT_ECUDA;
    }
    if (p_mass && cudaMemcpyAsync(p_mass, t.mass, (size_t)n * 4, cudaMemcpyDefault, st)) return GT_ECUDA;
    if (p_acc && cudaMemcpyAsync(p_acc, t.acc, (size_t)n * 16, cudaMemcpyDefault, st)) return GT_ECUDA;
    if (p_aold && cudaMemcpyAsync(p_aold, t.aold, (size_t)n * 4, cudaMemcpyDefault, st)) return GT_ECUDA;
    if (p_level && cudaMemcpyAsync(p_level, t.level, (size_t)n, cudaMemcpyDefault, st)) return GT_ECUDA;
    if (p_t0 && cudaMemcpyAsync(p_t0, t.t0, (size_t)n * 8, cudaMemcpyDefault, st)) return GT_ECUDA;
    if (p_id && cudaMemcpyAsync(p_id, t.id, (size_t)n * 4, cudaMemcpyDefault, st)) return GT_ECUDA;
    if (p_pos || p_vel) {
        // scratch3 is reused by the next call: finish these copies first
        if (cudaStreamSynchronize(st) != cudaSuccess) return GT_ECUDA;
    }
    return last_cuda();
}

int gt_get_tree(gt_system *s, uint64_t *p_keys, uint32_t *p_order, uint32_t *p_nodes, float *p_jpos,
                float *p_bj, int64_t *n_nodes_inout, gt_stream stream) {
    if (!s || !n_nodes_inout) return GT_EINVAL;
    cudaStream_t st = S(stream);
    const int64_t n = s->n;
    uint32_t ls[GT_TREE_LEVELS + 2];
    if (cudaMemcpyAsync(ls, s->ctl->level_start, sizeof(ls), cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st))
        return GT_ECUDA;
    int64_t nn = s->have_tree ? (int64_t)ls[GT_TREE_LEVELS] : 0;
    if (nn > s->cap) nn = s->cap;
    const int64_t capacity = *n_nodes_inout;
    *n_nodes_inout = nn;
    if (n > 0 && p_keys && cudaMemcpyAsync(p_keys, s->sb.key[0], (size_t)n * 8, cudaMemcpyDefault, st)) return GT_ECUDA;
    if (n > 0 && p_order && cudaMemcpyAsync(p_order, s->st[0].id, (size_t)n * 4, cudaMemcpyDefault, st))
        return GT_ECUDA;
    if (nn > capacity && (p_nodes || p_jpos || p_bj)) return GT_EOVERFLOW;
    if (nn > 0) {
        if (p_nodes) {
            const void *cols[4] = {s->nd.first, s->nd.count, s->nd.child, s->nd.nchild};
            for (int c = 0; c < 4; c++)
                if (cudaMemcpy2DAsync(p_nodes + c, 16, cols[c], 4, 4, (size_t)nn, cudaMemcpyDefault, st))
                    return GT_ECUDA;
        }
        if (p_jpos && cudaMemcpyAsync(p_jpos, s->nd.jpos, (size_t)nn * 16, cudaMemcpyDefault, st)) return GT_ECUDA;
        if (p_bj && cudaMemcpy2DAsync(p_bj, 4, s->nd.walk, 16, 4, (size_t)nn, cudaMemcpyDefault, st)) return GT_ECUDA;
    }
    if (cudaStreamSynchronize(st)) return GT_ECUDA;
    return GT_OK;
}

int gt_get_active(gt_system *s, uint32_t *p_active, int64_t *n_inout, gt_stream stream) {
    if (!s || !n_inout) return GT_EINVAL;
    cudaStream_t st = S(stream);
    unsigned na = 0;
    if (cudaMemcpyAsync(&na, &s->ctl->n_active, 4, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
        return GT_ECUDA;
    const int64_t cap = *n_inout;
    *n_inout = na;
    if (!p_active) return GT_OK;
    if ((int64_t)na > cap) return GT_EOVERFLOW;
    if (na && cudaMemcpyAsync(p_active, s->active, (size_t)na * 4, cudaMemcpyDefault, st)) return GT_ECUDA;
    return cudaStreamSynchronize(st) ? GT_ECUDA : GT_OK;
}

int gt_sync_status(gt_system *s, gt_stream stream) {
    if (!s) return GT_EINVAL;
    cudaStream_t st = S(stream);
    int err[2] = {0, 0};
    if (cudaStreamSynchronize(st) != cudaSuccess) return GT_ECUDA;
    if (cudaMemcpy(err, &s->ctl->err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) return GT_ECUDA;
    if (err[0]) {
        const int zero[2] = {0, 0};
        if (cudaMemcpy(&s->ctl->err, zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess) return GT_ECUDA;
    }
    return err[0];
}

int gt_set_wait_limit(gt_system *s, uint32_t iterations, gt_stream stream) {
    if (!s) return GT_EINVAL;
    gt_launch_set_u32(&s->ctl->spin_limit, iterations, S(stream));
    return last_cuda();
}

int gt_probe_bounded_wait(gt_system *s, uint32_t iterations, gt_stream stream) {
    if (!s) return GT_EINVAL;
    cudaStream_t st = S(stream);
    // the probe's bound replaces the system's for the probe only: read the old one back
    unsigned int old = 0;
    if (cudaMemcpyAsync(&old, &s->ctl->spin_limit, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GT_ECUDA;
    gt_launch_set_u32(&s->ctl->spin_limit, iterations, st);
    gt_launch_wait_probe(s->status, s->ctl, st);
    gt_launch_set_u32(&s->ctl->spin_limit, old, st);
    if (cudaGetLastError() != cudaSuccess) return GT_ECUDA;
    return gt_sync_status(s, stream);
}

int gt_get_stats(gt_system *s, gt_stats *o, gt_stream stream) {
    if (!s || !o) return GT_EINVAL;
    cudaStream_t st = S(stream);
    DevCtl c;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GT_ECUDA;
    if (cudaMemcpy(&c, s->ctl, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return GT_ECUDA;
    memset(o, 0, sizeof(*o));
    o->n = s->n;
    o->T = s->started ? (int64_t)c.tnext : 0;
    o->n_active = c.n_active;
    o->n_groups = cell_groups(s->prm) ? (int64_t)c.n_groups
                                      : ((int64_t)c.n_active + s->gmax_now - 1) / s->gmax_now;
    o->n_nodes = s->have_tree ? (int64_t)c.level_start[GT_TREE_LEVELS] : 0;
    int depth = 0;
    for (int l = 0; l < GT_TREE_LEVELS; l++)
        if (c.level_start[l + 1] > c.level_start[l]) depth = l + 1;
    o->depth = s->have_tree ? depth : 0;
    o->interactions = (int64_t)c.interactions;
    o->mac_tests = (int64_t)c.mac_tests;
    o->block_steps = s->steps;
    o->rebuilds = s->rebuilds;
    o->dt_max = s->started ? c.dt_max : s->prm.dt_max;
    o->err = c.err;
    o->err_where = c.err_where;
    return GT_OK;
}

}  // extern "C"
