// Host-side definition of gt_system and the helpers that string its kernels
// together; shared by the single-system entry points, the batch and the server.
#pragma once

#include <vector>

#include "gt_internal.cuh"

// Per-phase event timers of one system.
struct PhaseTimers {
    bool on = false, created = false;
    cudaEvent_t b[GT_NPHASES]{}, e[GT_NPHASES]{};
    bool ran[GT_NPHASES]{};
    bool before[GT_NPHASES]{};  // recorded before the timers were last zeroed: feeds last_ms only
    // the predictions enqueued ahead of their block step, by the step's parity: one is
    // still running while the other's times are read
    cudaEvent_t ab[2]{}, ae[2]{};
    bool aran[2]{};
    double ms[GT_NPHASES]{};
    double last_ms[GT_NPHASES]{};  // the most recent execution of each phase
    long long cnt[GT_NPHASES]{};
};

// Automatic tree-rebuild interval (Sec. 2.6): walk times since the last rebuild,
// normalised to the mean number of i-particles per block step (block steps vary
// N_i by orders of magnitude; the fit is meant to see the tree ageing, not that).
struct RebuildTuner {
    std::vector<double> y;
    double t_make = 0.0;
    double nact_sum = 0.0;
    long long nact_cnt = 0;
    double n_opt = 1e6;
    int model = -1;
    long long since = 0;  // block steps on the current tree
};

// On-line tuning of the critical separation of groups (Sec. 2.4): one Brent search per
// class of block step (the coarsest active level), over log r_crit, minimising the
// walk time per active particle; after convergence the best value is held for a few
// steps of its class, then searched again in a narrower bracket around it (the
// optimum drifts as the system evolves).
struct RcritTuner {
    static constexpr int NCLASS = 30;
    BrentSearch search[NCLASS];
    bool started[NCLASS] = {};
    int held[NCLASS] = {};
    int pending = -1;  // class of the step whose walk time is awaited
};

// On-line choice of the group size (GT_GROUP_CELLS_TUNED): per class of block step, the
// mean walk time per active particle of group_max / 4, / 2 and group_max; each is tried
// once (largest first), then the fastest is used, and every 64 steps of a class the
// trials start over.
struct GroupTuner {
    static constexpr int NCLASS = 30, NCAND = 3;
    double sum[NCLASS][NCAND] = {};
    int cnt[NCLASS][NCAND] = {};
    int seen[NCLASS] = {};
    int pending_class = -1, pending_cand = -1;
};

struct gt_system {
    int64_t n = 0;
    PhaseTimers prof;
    RebuildTuner tune;
    RcritTuner rtune;
    GroupTuner gtune;
    int gmax_now = 32;       // group size of the next grouping
    float rcrit_now = 0.0f;  // r_crit of the next grouping (0: no radius limit)
    gt_params prm{};
    int dev = 0, nsm = 0;
    int walk_blocks = 0, walk_warps = 0;
    bool started = false, have_tree = false, last_rebuilt = false;
    // members of a batch or a server keep their state in buffer 0 (captured graphs and
    // kernel arguments hold those addresses); a standalone system swaps its buffers instead
    bool fixed_buffers = false;
    long long steps = 0, rebuilds = 0;
    int64_t cap = 0;        // node capacity
    State st[2]{};
    float4 *posm = nullptr, *posm_tmp = nullptr;
    SortBufs sb{};
    Nodes nd{};
    unsigned long long *status = nullptr;
    uint32_t *active = nullptr;
    uint32_t *prefix = nullptr;   // P[i] = actives below internal index i (n + 1 entries)
    uint8_t *flags = nullptr;     // a caller's active list as flags
    uint8_t *marks = nullptr;     // first active position of every group
    uint32_t *gstart = nullptr;   // group starts (cell grouping)
    float4 *acc_out = nullptr;
    float *aold_tmp = nullptr;
    double *scratch3 = nullptr;
    uint8_t *bscratch = nullptr;  // tree build marks and counts
    float *bbox_partial = nullptr;
    int bbox_blocks = 0;
    uint32_t *queue = nullptr;    // the walk queue (a batch's shared queue for batch members)
    int64_t queue_entries = 0;
    DevCtl *ctl = nullptr;
    // Look-ahead of gt_block_step (automatic rebuild interval, standalone systems): after
    // a step the device copies the control words the next step's tuners read into
    // mapped host memory (event ahead_mirror) and predicts every particle to the next
    // block time into posm_tmp (event ahead_done); the next call waits only for the
    // mirror, so the prediction runs while the host tunes and enqueues the rest.
    StepMirror *mirror = nullptr, *mirror_dev = nullptr;  // pinned, mapped; 16 B
    bool mirror_tried = false;
    cudaEvent_t ahead_mirror = nullptr, ahead_done = nullptr;
    bool ahead = false;            // posm_tmp holds the prediction for the next step
    cudaStream_t ahead_st = nullptr;
};

constexpr size_t GT_WS_ALIGN = 256;

int gt_sys_check_params(const gt_params *p);
int gt_sys_device_sms(int *dev, int *nsm);
// Carve every buffer of a system out of base (or only measure when base == nullptr);
// own_queue == false leaves the walk queue to the caller (a batch).
size_t gt_sys_carve(gt_system *s, char *base, int64_t n, const gt_params *p, int nsm, int walk_blocks,
                    bool own_queue);
// Carve a system into ws (ws_bytes from gt_sys_carve) and zero its control words; waits
// for stream st (or, with st == nullptr, for the device).
int gt_sys_init(gt_system *s, int64_t n, const gt_params *p, void *ws, size_t ws_bytes, bool own_queue,
                cudaStream_t st);
// Take new parameters and reset what derives from them (group size and r_crit in use,
// their on-line tuners).
void gt_sys_apply_params(gt_system *s, const gt_params &p);
// A1-A5 on FP32 positions posm_src
void gt_sys_build_tree(gt_system *s, cudaStream_t st, const float4 *posm_src);
// A6 with every particle active: the active list and, for cell grouping, the groups
void gt_sys_groups_all(gt_system *s, cudaStream_t st);
// arguments of one walk over the current active list / groups
WalkArgs gt_sys_walk_args(const gt_system *s, const uint32_t *active, const float *aold, float4 *acc, int mac);
// |a| of the last walk over every particle -> a_old (start-up pass)
void gt_sys_aold_from_acc(gt_system *s, cudaStream_t st);
// after the start-up walks: levels and block time of every particle (the system is started)
void gt_sys_start_levels(gt_system *s, cudaStream_t st);
// One block step in three parts around the walk: predict, rebuild or pseudo j, active set
// (pre); the groups of the active set (groups); correct, levels, next block time (post).
// predicted: the prediction for this step is already in posm_tmp (enqueued ahead)
void gt_sys_step_pre(gt_system *s, cudaStream_t st, bool rebuild, bool predicted = false);
void gt_sys_step_groups(gt_system *s, cudaStream_t st);
void gt_sys_step_post(gt_system *s, cudaStream_t st);
