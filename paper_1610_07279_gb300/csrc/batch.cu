// Batches of independent systems (Sec. 2.3, 2.5 applied across systems): the members'
// tree builds and group setup run on forked streams, so that the many small kernels of
// small systems overlap; then one persistent walk launch covers the groups of every
// member.  The whole evaluation can be captured into a CUDA graph and replayed, and an
// autotuner picks the walk's leaf size, group size and queue depth by timing replays.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "gt_system.cuh"

struct gt_batch {
    int nsys = 0;
    int dev = 0, nsm = 0, walk_blocks = 0;
    int qcap = 0;  // queue entries per warp (the largest walk_queue at create)
    std::vector<gt_system *> sys;
    std::vector<WalkArgs> h_args;
    WalkArgs *d_args = nullptr;
    DevCtl **d_ctls = nullptr;
    uint32_t *d_gprefix = nullptr;
    unsigned int *d_next = nullptr;
    uint32_t *queue = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;  // kernel launches in the captured graph
    bool args_dirty = true;
};

static_assert(sizeof(gt_tune_space) == 96 && sizeof(gt_tune_result) == 2072, "tuning structs of the ABI");

namespace {

constexpr int MAX_STREAMS = 32;

size_t align_up(size_t v) { return (v + GT_WS_ALIGN - 1) / GT_WS_ALIGN * GT_WS_ALIGN; }

const gt_params &prm_of(const gt_params *prm, int n_prm, int k) { return prm[n_prm == 1 ? 0 : k]; }

// Bytes of the batch's own region (argument tables, group prefix, shared queue) and of
// every member; returns the total.
size_t plan(int nsys, const int64_t *n, const gt_params *prm, int n_prm, int nsm, int walk_blocks,
            int *qcap_out, std::vector<size_t> *member_bytes) {
    int qcap = 0;
    for (int k = 0; k < nsys; k++) {
        const int q = prm_of(prm, n_prm, k).walk_queue;
        if (q > qcap) qcap = q;
    }
    const size_t warps = (size_t)walk_blocks * (size_t)gt_walk_warps_per_block();
    size_t off = 0;
    off = align_up(off + (size_t)nsys * sizeof(WalkArgs));
    off = align_up(off + (size_t)nsys * sizeof(DevCtl *));
    off = align_up(off + (size_t)(nsys + 1) * sizeof(uint32_t));
    off = align_up(off + sizeof(unsigned int));
    off = align_up(off + warps * (size_t)qcap * sizeof(uint32_t));
    if (member_bytes) member_bytes->clear();
    for (int k = 0; k < nsys; k++) {
        gt_system tmp;
        const size_t b = gt_sys_carve(&tmp, nullptr, n[k], &prm_of(prm, n_prm, k), nsm, walk_blocks, false);
        if (member_bytes) member_bytes->push_back(b);
        off = align_up(off + b);
    }
    *qcap_out = qcap;
    return off;
}

int check_members(int nsys, const int64_t *n, const gt_params *prm, int n_prm) {
    if (nsys < 1 || !n || !prm || (n_prm != 1 && n_prm != nsys)) return GT_EINVAL;
    for (int k = 0; k < nsys; k++) {
        if (n[k] < 0 || n[k] >= (int64_t)1 << 30) return GT_EINVAL;
        const int rc = gt_sys_check_params(&prm_of(prm, n_prm, k));
        if (rc) return rc;
    }
    return GT_OK;
}

void drop_graph(gt_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_kernels = 0;
}

// Every member's walk arguments: all particles active (identity list), a_old and the
// force buffer of the member, the batch's queue depth.
int upload_args(gt_batch *b) {
    if (!b->args_dirty) return GT_OK;
    for (int k = 0; k < b->nsys; k++) {
        gt_system *s = b->sys[k];
        b->h_args[k] = gt_sys_walk_args(s, nullptr, s->st[0].aold, s->acc_out, s->prm.mac);
        b->h_args[k].queue = b->queue;
    }
    if (cudaMemcpy(b->d_args, b->h_args.data(), (size_t)b->nsys * sizeof(WalkArgs), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return GT_ECUDA;
    b->args_dirty = false;
    return GT_OK;
}

int nstreams(const gt_batch *b) { return (int)b->streams.size(); }

void fork(gt_batch *b, cudaStream_t st) {
    cudaEventRecord(b->ev_fork, st);
    for (int j = 0; j < nstreams(b); j++) cudaStreamWaitEvent(b->streams[j], b->ev_fork, 0);
}

void join(gt_batch *b, cudaStream_t st) {
    for (int j = 0; j < nstreams(b); j++) {
        cudaEventRecord(b->ev_join[j], b->streams[j]);
        cudaStreamWaitEvent(st, b->ev_join[j], 0);
    }
}

// The evaluation itself (enqueued or captured): builds and groups on the forked
// streams, then the batch walk(s) on st.
void enqueue(gt_batch *b, int bootstrap, cudaStream_t st) {
    fork(b, st);
    for (int k = 0; k < b->nsys; k++) {
        gt_system *s = b->sys[k];
        cudaStream_t sk = b->streams[k % nstreams(b)];
        if (s->n == 0) continue;
        gt_sys_build_tree(s, sk, s->posm);
        gt_sys_groups_all(s, sk);
    }
    join(b, st);
    if (bootstrap) {
        gt_launch_walk_batch(b->d_ctls, b->d_args, b->nsys, b->d_gprefix, b->d_next, b->queue, b->qcap,
                             GT_MAC_OPENING_ANGLE, b->walk_blocks, st);
        fork(b, st);
        for (int k = 0; k < b->nsys; k++)
            if (b->sys[k]->n > 0) gt_sys_aold_from_acc(b->sys[k], b->streams[k % nstreams(b)]);
        join(b, st);
    }
    gt_launch_walk_batch(b->d_ctls, b->d_args, b->nsys, b->d_gprefix, b->d_next, b->queue, b->qcap, -1,
                         b->walk_blocks, st);
}

long long launches_now() {
    int64_t c = 0;
    gt_kernel_launches(&c);
    return (long long)c;
}

}  // namespace

extern "C" {

int gt_batch_workspace_bytes(int nsys, const int64_t *n, const gt_params *prm, int n_prm, size_t *bytes) {
    if (!bytes) return GT_EINVAL;
    int rc = check_members(nsys, n, prm, n_prm);
    if (rc) return rc;
    int dev, nsm;
    if ((rc = gt_sys_device_sms(&dev, &nsm))) return rc;
    int qcap = 0;
    *bytes = plan(nsys, n, prm, n_prm, nsm, gt_walk_blocks(nsm), &qcap, nullptr);
    return GT_OK;
}

int gt_batch_create(gt_batch **out, int nsys, const int64_t *n, const gt_params *prm, int n_prm, void *d_ws,
                    size_t ws_bytes) {
    if (!out || !d_ws || ((uintptr_t)d_ws) % GT_WS_ALIGN) return GT_EINVAL;
    int rc = check_members(nsys, n, prm, n_prm);
    if (rc) return rc;
    gt_batch *b = new (std::nothrow) gt_batch();
    if (!b) return GT_ENOMEM;
    if ((rc = gt_sys_device_sms(&b->dev, &b->nsm))) { delete b; return rc; }
    gt_sort_init();
    b->walk_blocks = gt_walk_blocks(b->nsm);
    std::vector<size_t> mb;
    const size_t need = plan(nsys, n, prm, n_prm, b->nsm, b->walk_blocks, &b->qcap, &mb);
    if (ws_bytes < need) { delete b; return GT_ENOMEM; }
    b->nsys = nsys;
    char *base = (char *)d_ws;
    size_t off = 0;
    b->d_args = (WalkArgs *)(base + off);
    off = align_up(off + (size_t)nsys * sizeof(WalkArgs));
    b->d_ctls = (DevCtl **)(base + off);
    off = align_up(off + (size_t)nsys * sizeof(DevCtl *));
    b->d_gprefix = (uint32_t *)(base + off);
    off = align_up(off + (size_t)(nsys + 1) * sizeof(uint32_t));
    b->d_next = (unsigned int *)(base + off);
    off = align_up(off + sizeof(unsigned int));
    const size_t warps = (size_t)b->walk_blocks * (size_t)gt_walk_warps_per_block();
    b->queue = (uint32_t *)(base + off);
    off = align_up(off + warps * (size_t)b->qcap * sizeof(uint32_t));
    std::vector<DevCtl *> ctls(nsys);
    b->sys.assign(nsys, nullptr);
    b->h_args.resize(nsys);
    for (int k = 0; k < nsys; k++) {
        gt_system *s = new (std::nothrow) gt_system();
        if (!s) { gt_batch_destroy(b); return GT_ENOMEM; }
        b->sys[k] = s;
        if ((rc = gt_sys_init(s, n[k], &prm_of(prm, n_prm, k), base + off, mb[k], false, nullptr))) {
            gt_batch_destroy(b);
            return rc;
        }
        s->queue = b->queue;  // the batch's queue serves the member's own walks too
        s->queue_entries = (int64_t)(warps * (size_t)b->qcap);
        ctls[k] = s->ctl;
        off = align_up(off + mb[k]);
    }
    if (cudaMemcpy(b->d_ctls, ctls.data(), (size_t)nsys * sizeof(DevCtl *), cudaMemcpyHostToDevice) != cudaSuccess) {
        gt_batch_destroy(b);
        return GT_ECUDA;
    }
    const int ns = nsys < MAX_STREAMS ? nsys : MAX_STREAMS;
    b->streams.assign(ns, nullptr);
    b->ev_join.assign(ns, nullptr);
    for (int j = 0; j < ns; j++) {
        if (cudaStreamCreateWithFlags(&b->streams[j], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[j], cudaEventDisableTiming) != cudaSuccess) {
            gt_batch_destroy(b);
            return GT_ECUDA;
        }
    }
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
        gt_batch_destroy(b);
        return GT_ECUDA;
    }
    *out = b;
    return GT_OK;
}

int gt_batch_destroy(gt_batch *b) {
    if (!b) return GT_OK;
    cudaDeviceSynchronize();
    drop_graph(b);
    for (gt_system *s : b->sys) gt_system_destroy(s);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev_join)
        if (e) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
    return GT_OK;
}

int gt_batch_system(gt_batch *b, int k, gt_system **out) {
    if (!b || !out || k < 0 || k >= b->nsys) return GT_EINVAL;
    *out = b->sys[k];
    return GT_OK;
}

int gt_batch_set_knobs(gt_batch *b, int leaf_max, int group_max, int walk_queue) {
    if (!b) return GT_EINVAL;
    if (walk_queue > b->qcap) return GT_EINVAL;
    std::vector<gt_params> next(b->nsys);
    for (int k = 0; k < b->nsys; k++) {
        gt_params p = b->sys[k]->prm;
        if (leaf_max > 0) p.leaf_max = leaf_max;
        if (group_max > 0) p.group_max = group_max;
        if (walk_queue > 0) p.walk_queue = walk_queue;
        const int rc = gt_sys_check_params(&p);
        if (rc) return rc;
        next[k] = p;
    }
    for (int k = 0; k < b->nsys; k++) gt_sys_apply_params(b->sys[k], next[k]);
    b->args_dirty = true;
    drop_graph(b);
    return GT_OK;
}

int gt_batch_accel(gt_batch *b, int bootstrap, gt_stream stream) {
    if (!b) return GT_EINVAL;
    int rc = upload_args(b);
    if (rc) return rc;
    enqueue(b, bootstrap, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? GT_OK : GT_ECUDA;
}

int gt_batch_capture(gt_batch *b, int bootstrap, gt_stream stream) {
    if (!b) return GT_EINVAL;
    int rc = upload_args(b);
    if (rc) return rc;
    drop_graph(b);
    cudaStream_t st = (cudaStream_t)stream;
    const long long before = launches_now();
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GT_ECUDA;
    enqueue(b, bootstrap, st);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(st, &g) != cudaSuccess || !g) {
        cudaGetLastError();
        return GT_ECUDA;
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        drop_graph(b);
        return GT_ECUDA;
    }
    // the launches noted while capturing happen on every replay instead
    b->graph_kernels = launches_now() - before;
    gt_note_launches(-(int)b->graph_kernels);
    return GT_OK;
}

int gt_batch_launch(gt_batch *b, gt_stream stream) {
    if (!b) return GT_EINVAL;
    if (!b->exec) return GT_ESTATE;
    if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) return GT_ECUDA;
    gt_note_launches((int)b->graph_kernels);
    return GT_OK;
}

int gt_batch_get_acc(gt_batch *b, int k, float *p_acc, uint32_t *p_id, gt_stream stream) {
    if (!b || k < 0 || k >= b->nsys) return GT_EINVAL;
    gt_system *s = b->sys[k];
    cudaStream_t st = (cudaStream_t)stream;
    if (s->n > 0) {
        if (p_acc && cudaMemcpyAsync(p_acc, s->acc_out, (size_t)s->n * 16, cudaMemcpyDefault, st)) return GT_ECUDA;
        if (p_id && cudaMemcpyAsync(p_id, s->st[0].id, (size_t)s->n * 4, cudaMemcpyDefault, st)) return GT_ECUDA;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? GT_OK : GT_ECUDA;
}

int gt_batch_sync_status(gt_batch *b, int64_t *interactions_out, gt_stream stream) {
    if (!b) return GT_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GT_ECUDA;
    int first = GT_OK;
    for (int k = 0; k < b->nsys; k++) {
        const int rc = gt_sync_status(b->sys[k], stream);
        if (rc && first == GT_OK) first = rc;
        if (interactions_out) {
            unsigned long long c = 0;
            if (cudaMemcpy(&c, &b->sys[k]->ctl->interactions, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                return GT_ECUDA;
            interactions_out[k] = (int64_t)c;
        }
    }
    return first;
}

int gt_batch_autotune(gt_batch *b, const gt_tune_space *sp, gt_tune_result *res, gt_stream stream) {
    if (!b || !sp || !res || sp->reps < 1) return GT_EINVAL;
    if (sp->n_leaf < 0 || sp->n_leaf > 8 || sp->n_group < 0 || sp->n_group > 8 || sp->n_queue < 0 ||
        sp->n_queue > 4)
        return GT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int cur_leaf = b->sys[0]->prm.leaf_max, cur_group = b->sys[0]->prm.group_max,
              cur_queue = b->sys[0]->prm.walk_queue;
    const int nl = sp->n_leaf ? sp->n_leaf : 1, ng = sp->n_group ? sp->n_group : 1,
              nq = sp->n_queue ? sp->n_queue : 1;
    memset(res, 0, sizeof(*res));
    res->best_ms = INFINITY;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GT_ECUDA;
    int rc_all = GT_OK;
    int idx = 0;
    for (int il = 0; il < nl; il++)
        for (int ig = 0; ig < ng; ig++)
            for (int iq = 0; iq < nq; iq++, idx++) {
                const int leaf = sp->n_leaf ? sp->leaf_max[il] : cur_leaf;
                const int group = sp->n_group ? sp->group_max[ig] : cur_group;
                const int queue = sp->n_queue ? sp->walk_queue[iq] : cur_queue;
                double ms = INFINITY;
                if (gt_batch_set_knobs(b, leaf, group, queue) == GT_OK && gt_batch_capture(b, 0, stream) == GT_OK &&
                    gt_batch_launch(b, stream) == GT_OK) {
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < sp->reps; r++) gt_batch_launch(b, stream);
                    cudaEventRecord(e1, st);
                    float t = 0.f;
                    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
                        gt_batch_sync_status(b, nullptr, stream) == GT_OK)
                        ms = (double)t / sp->reps;  // a candidate that raised an error is never kept
                }
                if (idx < 256) res->ms[idx] = ms;
                if (ms < res->best_ms) {
                    res->best_ms = ms;
                    res->leaf_max = leaf;
                    res->group_max = group;
                    res->walk_queue = queue;
                }
            }
    res->n_tried = idx;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!isfinite(res->best_ms)) {
        gt_batch_set_knobs(b, cur_leaf, cur_group, cur_queue);
        return GT_EINVAL;
    }
    rc_all = gt_batch_set_knobs(b, res->leaf_max, res->group_max, res->walk_queue);
    return rc_all;
}

}  // extern "C"
