// FP32 instruction throughputs of the device: the denominators of the walk's roofline
// and of the paper's flop convention (Sec. 4: the rsqrt counts as the ratio of the
// add/multiply throughput to the reciprocal-square-root throughput).
//
// Every thread runs eight independent dependent chains of one instruction form (enough
// to cover the pipe latency at full occupancy); the chains are folded into one value
// that is stored under a condition the compiler cannot prove false, so no chain is
// removed.  Forms: scalar FMA, packed FMA on float2 (f32x2, two FMAs per lane and
// instruction), scalar add, scalar multiply, the SFU reciprocal square root, and the FP64
// FMA (the pipe of the centre-of-mass sums and the integration).
#include "gt_internal.cuh"

namespace {

constexpr int PT = 256;
constexpr int UNROLL = 16;
constexpr int CHAINS = 8;

enum { OP_FMA = 0, OP_FMA2, OP_ADD, OP_MUL, OP_RSQRT, OP_DFMA, NOPS };

__device__ __forceinline__ float rsqrt_sfu(float x) {
    float r;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int OP>
__global__ __launch_bounds__(PT) void k_chains(float *out, int iters, float seed) {
    float a[CHAINS];
    float2 p[CHAINS];
    double da[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        a[c] = seed + (float)(threadIdx.x & 7) + (float)c;
        p[c] = make_float2(a[c], a[c] + 0.5f);
        da[c] = (double)a[c];
    }
    const float b = 0.999999f, cc = 1e-6f;
    const float2 b2 = make_float2(b, b), c2 = make_float2(cc, cc);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < UNROLL; k++) {
#pragma unroll
            for (int c = 0; c < CHAINS; c++) {
                if (OP == OP_FMA) a[c] = fmaf(a[c], b, cc);
                if (OP == OP_FMA2) p[c] = __ffma2_rn(p[c], b2, c2);
                if (OP == OP_ADD) a[c] = __fadd_rn(a[c], cc);
                if (OP == OP_MUL) a[c] = __fmul_rn(a[c], b);
                if (OP == OP_RSQRT) a[c] = rsqrt_sfu(a[c]);  // x -> x^(-1/2): stays near 1
                if (OP == OP_DFMA) da[c] = __fma_rn(da[c], 0.999999, 1e-6);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += a[c] + p[c].x + p[c].y + (float)da[c];
    if (s == -1.0f) out[blockIdx.x] = s;
}

template <int OP>
int time_op(cudaStream_t st, int nsm, double *ops_per_s) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chains<OP>, PT, 0);
    if (per < 1) per = 1;
    const int blocks = nsm * per;
    const int iters = (OP == OP_RSQRT || OP == OP_DFMA) ? 64 : 4096;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return GT_ECUDA;
    { k_chains<OP><<<blocks, PT, 0, st>>>(nullptr, 64, 1.0f); gt_note_launches(1); }  // warm-up
    cudaEventRecord(e0, st);
    { k_chains<OP><<<blocks, PT, 0, st>>>(nullptr, iters, 1.0f); gt_note_launches(1); }
    cudaEventRecord(e1, st);
    float ms = 0.f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || ms <= 0.f) return GT_ECUDA;
    // operations per lane and instruction: two for the packed form
    const double lane_ops = OP == OP_FMA2 ? 2.0 : 1.0;
    *ops_per_s = (double)blocks * PT * (double)iters * UNROLL * CHAINS * lane_ops / (ms * 1e-3);
    return GT_OK;
}

int device_nsm(int *nsm) {
    int dev;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev)) return GT_ECUDA;
    return GT_OK;
}

}  // namespace

extern "C" int gt_measure_fp32_rates(gt_fp32_rates *out, gt_stream stream) {
    if (!out) return GT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int nsm = 0, rc;
    if ((rc = device_nsm(&nsm))) return rc;
    double r[NOPS] = {};
    if ((rc = time_op<OP_FMA>(st, nsm, &r[OP_FMA])) || (rc = time_op<OP_FMA2>(st, nsm, &r[OP_FMA2])) ||
        (rc = time_op<OP_ADD>(st, nsm, &r[OP_ADD])) || (rc = time_op<OP_MUL>(st, nsm, &r[OP_MUL])) ||
        (rc = time_op<OP_RSQRT>(st, nsm, &r[OP_RSQRT])) || (rc = time_op<OP_DFMA>(st, nsm, &r[OP_DFMA])))
        return rc;
    out->fp64_fma_per_s = r[OP_DFMA];
    out->fma_per_s = r[OP_FMA];
    out->fma2_per_s = r[OP_FMA2];
    out->add_per_s = r[OP_ADD];
    out->mul_per_s = r[OP_MUL];
    out->rsqrt_per_s = r[OP_RSQRT];
    out->peak_flops = 2.0 * (r[OP_FMA] > r[OP_FMA2] ? r[OP_FMA] : r[OP_FMA2]);
    const double addmul = r[OP_ADD] > r[OP_MUL] ? r[OP_ADD] : r[OP_MUL];
    out->rsqrt_flops = addmul / r[OP_RSQRT];
    return GT_OK;
}

extern "C" int gt_measure_fp32_peak(double *flops, gt_stream stream) {
    if (!flops) return GT_EINVAL;
    int nsm = 0, rc;
    if ((rc = device_nsm(&nsm))) return rc;
    double fma = 0.0;
    if ((rc = time_op<OP_FMA>((cudaStream_t)stream, nsm, &fma))) return rc;
    *flops = 2.0 * fma;
    return GT_OK;
}
