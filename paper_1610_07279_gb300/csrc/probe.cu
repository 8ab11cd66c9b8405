// FP32 FMA throughput of the device: the denominator of the walk's roofline.
// Every thread runs eight independent dependent-FMA chains (enough to cover the FMA
// latency at full occupancy); the result is stored under a condition the compiler
// cannot prove false, so no chain is removed.
#include "gt_internal.cuh"

namespace {

constexpr int PT = 256;
constexpr int UNROLL = 16;

__global__ __launch_bounds__(PT) void k_ffma_chains(float *out, int iters, float seed) {
    float a0 = seed + threadIdx.x, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
    float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
    const float b = 0.999999f, c = 1e-6f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < UNROLL; k++) {
            a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
            a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
        }
    }
    const float s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == -1.0f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" int gt_measure_fp32_peak(double *flops, gt_stream stream) {
    if (!flops) return GT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev, nsm, per = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) return GT_ECUDA;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ffma_chains, PT, 0);
    if (per < 1) per = 1;
    const int blocks = nsm * per;
    const int iters = 4096;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return GT_ECUDA;
    { k_ffma_chains<<<blocks, PT, 0, st>>>(nullptr, 64, 1.0f); gt_note_launches(1); }  // warm-up
    cudaEventRecord(e0, st);
    { k_ffma_chains<<<blocks, PT, 0, st>>>(nullptr, iters, 1.0f); gt_note_launches(1); }
    cudaEventRecord(e1, st);
    float ms = 0.f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || ms <= 0.f) return GT_ECUDA;
    const double fma = (double)blocks * PT * iters * UNROLL * 8.0;
    *flops = 2.0 * fma / (ms * 1e-3);
    return GT_OK;
}
