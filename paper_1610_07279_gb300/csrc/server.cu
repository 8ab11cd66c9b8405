// Serving: continuous (iteration-level) batching of block-step requests.
//
// Every tick advances each resident request by one unit of work -- the start-up for a
// new request (tree, opening-angle pass, a_old, first force with the request's MAC,
// levels), one block step for a running one -- with the per-request parts on forked
// streams and the tree walks of all requests of the tick in one persistent launch over
// their groups (the walk-argument table of a tick is gathered on the device from a
// list passed by value, so no host buffer has to outlive a launch).  Requests join and
// leave between ticks; the host never waits for the device except to admit a request
// (its inputs are copied in before gt_submit returns) and to hand a result out.
#include <string.h>

#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "gt_system.cuh"

static_assert(sizeof(gt_request) == 120 && sizeof(gt_server_stats) == 64, "serving structs of the ABI");

namespace {

constexpr int MAX_STREAMS = 32;
constexpr int MAX_INFLIGHT = 2;  // ticks enqueued ahead of the device
enum { V_STEP = 0, V_BOOT = 1, V_FIRST = 2, NVARIANT = 3 };  // walk-argument variants per slot
enum { PH_START = 0, PH_RUN = 1, PH_FINISHING = 2, PH_DONE = 3 };

struct TickList {
    int n;
    uint16_t slot[GT_SERVER_MAX_SLOTS];
    uint8_t variant[GT_SERVER_MAX_SLOTS];
};

__global__ void k_select_args(TickList L, const WalkArgs *__restrict__ pool, DevCtl *const *__restrict__ ctl_pool,
                              WalkArgs *__restrict__ out, DevCtl **__restrict__ ctls) {
    for (int k = threadIdx.x; k < L.n; k += blockDim.x) {
        out[k] = pool[(int)L.slot[k] * NVARIANT + (int)L.variant[k]];
        ctls[k] = ctl_pool[L.slot[k]];
    }
}

struct Slot {
    bool used = false;
    uint64_t ticket = 0;
    gt_system *sys = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int phase = PH_START;
    int nsteps = 0, steps_enq = 0, rebuild_every = 4;
    long long done_tick = -1;
};

struct TickRec {
    cudaEvent_t ev;
    long long id;
};

size_t align_up(size_t v) { return (v + GT_WS_ALIGN - 1) / GT_WS_ALIGN * GT_WS_ALIGN; }

}  // namespace

struct gt_server {
    size_t hbm_cap = 0, hbm_used = 0;
    int max_slots = 0, qcap = 0;
    gt_alloc_fn alloc_fn = nullptr;
    gt_free_fn free_fn = nullptr;
    void *ctx = nullptr;
    int dev = 0, nsm = 0, walk_blocks = 0;
    void *region = nullptr;
    size_t region_bytes = 0;
    WalkArgs *d_pool = nullptr;
    DevCtl **d_ctl_pool = nullptr;
    WalkArgs *d_tick_args = nullptr;
    DevCtl **d_tick_ctls = nullptr;
    uint32_t *d_gprefix = nullptr;
    unsigned int *d_next = nullptr;
    uint32_t *queue = nullptr;
    std::vector<Slot> slots;
    std::unordered_map<uint64_t, int> by_ticket;
    uint64_t next_ticket = 1;
    cudaStream_t main = nullptr, admit = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    std::deque<TickRec> inflight;
    std::vector<cudaEvent_t> spare_events;
    long long ticks = 0, admitted = 0, completed = 0, walk_launches = 0;
};

namespace {

cudaStream_t slot_stream(gt_server *v, int slot) { return v->streams[slot % (int)v->streams.size()]; }

// fork the streams of the given slots off the main stream / join them back
void fork(gt_server *v, const std::vector<int> &use) {
    cudaEventRecord(v->ev_fork, v->main);
    for (int j : use) cudaStreamWaitEvent(v->streams[j], v->ev_fork, 0);
}

void join(gt_server *v, const std::vector<int> &use) {
    for (int j : use) {
        cudaEventRecord(v->ev_join[j], v->streams[j]);
        cudaStreamWaitEvent(v->main, v->ev_join[j], 0);
    }
}

std::vector<int> streams_of(const gt_server *v, const std::vector<int> &a, const std::vector<int> &b) {
    std::vector<char> on(v->streams.size(), 0);
    for (int k : a) on[k % (int)v->streams.size()] = 1;
    for (int k : b) on[k % (int)v->streams.size()] = 1;
    std::vector<int> use;
    for (int j = 0; j < (int)on.size(); j++)
        if (on[j]) use.push_back(j);
    return use;
}

void batched_walk(gt_server *v, const TickList &L) {
    if (L.n == 0) return;
    { k_select_args<<<1, 128, 0, v->main>>>(L, v->d_pool, v->d_ctl_pool, v->d_tick_args, v->d_tick_ctls);
      gt_note_launches(1); }
    gt_launch_walk_batch(v->d_tick_ctls, v->d_tick_args, L.n, v->d_gprefix, v->d_next, v->queue, v->qcap, -1,
                         v->walk_blocks, v->main);
    v->walk_launches++;
}

// One tick; false when no resident request has work left to enqueue.
bool enqueue_tick(gt_server *v) {
    std::vector<int> starts, runs;
    for (int k = 0; k < v->max_slots; k++) {
        const Slot &s = v->slots[k];
        if (!s.used) continue;
        if (s.phase == PH_START) starts.push_back(k);
        else if (s.phase == PH_RUN) runs.push_back(k);
    }
    if (starts.empty() && runs.empty()) return false;
    const long long id = ++v->ticks;
    const std::vector<int> all = streams_of(v, starts, runs), boot = streams_of(v, starts, {});
    fork(v, all);
    for (int k : starts) {
        gt_system *s = v->slots[k].sys;
        gt_sys_build_tree(s, slot_stream(v, k), s->posm);
        gt_sys_groups_all(s, slot_stream(v, k));
    }
    for (int k : runs) {
        Slot &sl = v->slots[k];
        const bool rebuild = sl.sys->steps % sl.rebuild_every == 0;
        gt_sys_step_pre(sl.sys, slot_stream(v, k), rebuild);
        gt_sys_step_groups(sl.sys, slot_stream(v, k));
    }
    join(v, all);
    TickList L;
    L.n = 0;
    for (int k : starts) { L.slot[L.n] = (uint16_t)k; L.variant[L.n++] = V_BOOT; }
    for (int k : runs) { L.slot[L.n] = (uint16_t)k; L.variant[L.n++] = V_STEP; }
    batched_walk(v, L);
    if (!starts.empty()) {
        fork(v, boot);
        for (int k : starts) gt_sys_aold_from_acc(v->slots[k].sys, slot_stream(v, k));
        join(v, boot);
        L.n = 0;
        for (int k : starts) { L.slot[L.n] = (uint16_t)k; L.variant[L.n++] = V_FIRST; }
        batched_walk(v, L);
    }
    fork(v, all);
    for (int k : starts) {
        Slot &sl = v->slots[k];
        gt_sys_start_levels(sl.sys, slot_stream(v, k));
        sl.phase = sl.nsteps > 0 ? PH_RUN : PH_FINISHING;
        if (sl.phase == PH_FINISHING) sl.done_tick = id;
    }
    for (int k : runs) {
        Slot &sl = v->slots[k];
        gt_sys_step_post(sl.sys, slot_stream(v, k));
        if (++sl.steps_enq == sl.nsteps) {
            sl.phase = PH_FINISHING;
            sl.done_tick = id;
        }
    }
    join(v, all);
    cudaEvent_t ev = nullptr;
    if (!v->spare_events.empty()) {
        ev = v->spare_events.back();
        v->spare_events.pop_back();
    } else {
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    }
    cudaEventRecord(ev, v->main);
    v->inflight.push_back(TickRec{ev, id});
    return true;
}

// Retire the finished ticks; their requests' results are ready.
int reap(gt_server *v) {
    while (!v->inflight.empty()) {
        const cudaError_t e = cudaEventQuery(v->inflight.front().ev);
        if (e == cudaErrorNotReady) {
            cudaGetLastError();
            break;
        }
        if (e != cudaSuccess) return GT_ECUDA;
        const long long id = v->inflight.front().id;
        for (Slot &s : v->slots)
            if (s.used && s.phase == PH_FINISHING && s.done_tick <= id) s.phase = PH_DONE;
        v->spare_events.push_back(v->inflight.front().ev);
        v->inflight.pop_front();
    }
    return GT_OK;
}

int pump(gt_server *v) {
    int rc = reap(v);
    if (rc) return rc;
    while ((int)v->inflight.size() < MAX_INFLIGHT && enqueue_tick(v)) {
    }
    return cudaGetLastError() == cudaSuccess ? GT_OK : GT_ECUDA;
}

void release(gt_server *v, int k) {
    Slot &s = v->slots[k];
    if (s.sys) gt_system_destroy(s.sys);
    if (s.ws) v->free_fn(s.ws, v->ctx);
    v->hbm_used -= s.ws_bytes;
    v->by_ticket.erase(s.ticket);
    s = Slot();
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// positions or velocities of slot k in the caller's order into out (host or device)
int copy_out(gt_server *v, gt_system *s, double *out, bool vel) {
    if (!out || s->n == 0) return GT_OK;
    const bool dev = is_device_pointer(out);
    double *dst = dev ? out : s->scratch3;  // scratch3 holds 3n + 8 doubles
    gt_launch_state_out(s->st[0], s->n, vel ? nullptr : dst, vel ? dst : nullptr, v->admit);
    if (!dev && cudaMemcpyAsync(out, dst, (size_t)s->n * 24, cudaMemcpyDeviceToHost, v->admit) != cudaSuccess)
        return GT_ECUDA;
    return cudaStreamSynchronize(v->admit) == cudaSuccess ? GT_OK : GT_ECUDA;
}

}  // namespace

extern "C" {

int gt_server_create(gt_server **out, size_t hbm_cap, int max_slots, int walk_queue, gt_alloc_fn alloc_fn,
                     gt_free_fn free_fn, void *ctx) {
    if (!out || !alloc_fn || !free_fn || max_slots < 1 || max_slots > GT_SERVER_MAX_SLOTS) return GT_EINVAL;
    if (walk_queue < 64 || (walk_queue & (walk_queue - 1))) return GT_EINVAL;
    gt_server *v = new (std::nothrow) gt_server();
    if (!v) return GT_ENOMEM;
    v->hbm_cap = hbm_cap;
    v->max_slots = max_slots;
    v->qcap = walk_queue;
    v->alloc_fn = alloc_fn;
    v->free_fn = free_fn;
    v->ctx = ctx;
    int rc = gt_sys_device_sms(&v->dev, &v->nsm);
    if (rc) { delete v; return rc; }
    gt_sort_init();
    v->walk_blocks = gt_walk_blocks(v->nsm);
    const size_t warps = (size_t)v->walk_blocks * (size_t)gt_walk_warps_per_block();
    size_t off = 0;
    const size_t o_pool = off; off = align_up(off + (size_t)max_slots * NVARIANT * sizeof(WalkArgs));
    const size_t o_ctlp = off; off = align_up(off + (size_t)max_slots * sizeof(DevCtl *));
    const size_t o_targ = off; off = align_up(off + (size_t)max_slots * sizeof(WalkArgs));
    const size_t o_tctl = off; off = align_up(off + (size_t)max_slots * sizeof(DevCtl *));
    const size_t o_gpre = off; off = align_up(off + (size_t)(max_slots + 1) * sizeof(uint32_t));
    const size_t o_next = off; off = align_up(off + sizeof(unsigned int));
    const size_t o_queue = off; off = align_up(off + warps * (size_t)walk_queue * sizeof(uint32_t));
    if (off > hbm_cap) { delete v; return GT_ENOMEM; }
    v->region = alloc_fn(off, ctx);
    if (!v->region || ((uintptr_t)v->region) % GT_WS_ALIGN) {
        if (v->region) free_fn(v->region, ctx);
        delete v;
        return GT_ENOMEM;
    }
    v->region_bytes = off;
    v->hbm_used = off;
    char *b = (char *)v->region;
    v->d_pool = (WalkArgs *)(b + o_pool);
    v->d_ctl_pool = (DevCtl **)(b + o_ctlp);
    v->d_tick_args = (WalkArgs *)(b + o_targ);
    v->d_tick_ctls = (DevCtl **)(b + o_tctl);
    v->d_gprefix = (uint32_t *)(b + o_gpre);
    v->d_next = (unsigned int *)(b + o_next);
    v->queue = (uint32_t *)(b + o_queue);
    v->slots.assign(max_slots, Slot());
    const int ns = max_slots < MAX_STREAMS ? max_slots : MAX_STREAMS;
    v->streams.assign(ns, nullptr);
    v->ev_join.assign(ns, nullptr);
    bool ok = cudaStreamCreateWithFlags(&v->main, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&v->admit, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&v->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int j = 0; ok && j < ns; j++)
        ok = cudaStreamCreateWithFlags(&v->streams[j], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&v->ev_join[j], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        gt_server_destroy(v);
        return GT_ECUDA;
    }
    *out = v;
    return GT_OK;
}

int gt_server_destroy(gt_server *v) {
    if (!v) return GT_OK;
    if (v->main) cudaStreamSynchronize(v->main);
    for (cudaStream_t s : v->streams)
        if (s) cudaStreamSynchronize(s);
    if (v->admit) cudaStreamSynchronize(v->admit);
    for (int k = 0; k < (int)v->slots.size(); k++)
        if (v->slots[k].used) release(v, k);
    for (TickRec &t : v->inflight) cudaEventDestroy(t.ev);
    for (cudaEvent_t e : v->spare_events) cudaEventDestroy(e);
    for (size_t j = 0; j < v->streams.size(); j++) {
        if (v->streams[j]) cudaStreamDestroy(v->streams[j]);
        if (v->ev_join[j]) cudaEventDestroy(v->ev_join[j]);
    }
    if (v->ev_fork) cudaEventDestroy(v->ev_fork);
    if (v->main) cudaStreamDestroy(v->main);
    if (v->admit) cudaStreamDestroy(v->admit);
    if (v->region) v->free_fn(v->region, v->ctx);
    delete v;
    return GT_OK;
}

int gt_submit(gt_server *v, const gt_request *req, uint64_t *ticket) {
    if (!v || !req || !ticket || req->n < 1 || req->n >= (int64_t)1 << 30 || req->nsteps < 0) return GT_EINVAL;
    if (!req->p_pos || !req->p_vel || !req->p_mass) return GT_EINVAL;
    gt_params prm = req->params;
    if (prm.walk_queue > v->qcap) prm.walk_queue = v->qcap;
    int rc = gt_sys_check_params(&prm);
    if (rc) return rc;
    int k = -1;
    for (int j = 0; j < v->max_slots; j++)
        if (!v->slots[j].used) { k = j; break; }
    if (k < 0) return GT_EAGAIN;
    gt_system probe;
    const size_t bytes = gt_sys_carve(&probe, nullptr, req->n, &prm, v->nsm, v->walk_blocks, false);
    if (v->hbm_used + bytes > v->hbm_cap) return GT_EAGAIN;
    void *ws = v->alloc_fn(bytes, v->ctx);
    if (!ws) return GT_ENOMEM;
    if (((uintptr_t)ws) % GT_WS_ALIGN) { v->free_fn(ws, v->ctx); return GT_EINVAL; }
    gt_system *s = new (std::nothrow) gt_system();
    if (!s) { v->free_fn(ws, v->ctx); return GT_ENOMEM; }
    Slot &sl = v->slots[k];
    sl.used = true;
    sl.sys = s;
    sl.ws = ws;
    sl.ws_bytes = bytes;
    v->hbm_used += bytes;
    sl.ticket = v->next_ticket++;
    v->by_ticket[sl.ticket] = k;
    if ((rc = gt_sys_init(s, req->n, &prm, ws, bytes, false, v->admit))) { release(v, k); return rc; }
    s->queue = v->queue;
    s->queue_entries = (int64_t)v->walk_blocks * gt_walk_warps_per_block() * v->qcap;
    sl.phase = PH_START;
    sl.nsteps = req->nsteps;
    sl.steps_enq = 0;
    sl.rebuild_every = prm.rebuild_every > 0 ? prm.rebuild_every : 4;
    if ((rc = gt_set_state(s, req->p_pos, req->p_vel, req->p_mass, (gt_stream)v->admit)) ||
        cudaStreamSynchronize(v->admit) != cudaSuccess) {
        release(v, k);
        return rc ? rc : GT_ECUDA;
    }
    // the three walk-argument variants of this slot
    WalkArgs a[NVARIANT];
    a[V_STEP] = gt_sys_walk_args(s, s->active, s->st[0].aold, s->acc_out, prm.mac);
    a[V_BOOT] = gt_sys_walk_args(s, nullptr, s->st[0].aold, s->acc_out, GT_MAC_OPENING_ANGLE);
    a[V_FIRST] = gt_sys_walk_args(s, nullptr, s->st[0].aold, s->acc_out, prm.mac);
    DevCtl *ctl = s->ctl;
    if (cudaMemcpyAsync(v->d_pool + (size_t)k * NVARIANT, a, sizeof(a), cudaMemcpyHostToDevice, v->admit) ||
        cudaMemcpyAsync(v->d_ctl_pool + k, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, v->admit) ||
        cudaStreamSynchronize(v->admit)) {
        release(v, k);
        return GT_ECUDA;
    }
    v->admitted++;
    *ticket = sl.ticket;
    return pump(v);
}

int gt_server_progress(gt_server *v, int *running) {
    if (!v) return GT_EINVAL;
    const int rc = pump(v);
    if (running) {
        int r = 0;
        for (const Slot &s : v->slots) r += s.used ? 1 : 0;
        *running = r;
    }
    return rc;
}

int gt_poll(gt_server *v, uint64_t ticket, int *state, double *p_pos_out, double *p_vel_out) {
    if (!v || !state) return GT_EINVAL;
    int rc = pump(v);
    if (rc) return rc;
    auto it = v->by_ticket.find(ticket);
    if (it == v->by_ticket.end()) {
        *state = GT_REQ_UNKNOWN;
        return GT_EINVAL;
    }
    const int k = it->second;
    Slot &sl = v->slots[k];
    if (sl.phase != PH_DONE) {
        *state = GT_REQ_RUNNING;
        return GT_EPENDING;
    }
    gt_system *s = sl.sys;
    int err[2] = {0, 0};
    if (cudaMemcpy(err, &s->ctl->err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) return GT_ECUDA;
    if ((rc = copy_out(v, s, p_pos_out, false)) || (rc = copy_out(v, s, p_vel_out, true))) return rc;
    release(v, k);
    v->completed++;
    *state = GT_REQ_DONE;
    rc = pump(v);  // the freed slot may admit more work at the next submit; keep the device busy
    return err[0] ? err[0] : rc;
}

int gt_server_get_stats(gt_server *v, gt_server_stats *o) {
    if (!v || !o) return GT_EINVAL;
    memset(o, 0, sizeof(*o));
    o->ticks = v->ticks;
    o->admitted = v->admitted;
    o->completed = v->completed;
    int r = 0;
    for (const Slot &s : v->slots) r += s.used ? 1 : 0;
    o->slots_used = r;
    o->hbm_used = (int64_t)v->hbm_used;
    o->hbm_cap = (int64_t)v->hbm_cap;
    o->walk_launches = v->walk_launches;
    return GT_OK;
}

}  // extern "C"
