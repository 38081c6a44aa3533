// FP64 fused multiply-add throughput of the current device, measured by
// launching independent DFMA chains on every SM.  Not part of the paper's
// method: the plain-FP64 fine step on this GPU is bound by its FP64 pipe
// (the part's FP64 rate is a small fraction of its FP32 rate), so its
// roofline needs this measured denominator rather than a data-sheet figure.
#include <cuda_runtime.h>

#include <cmath>

#include "pr.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent accumulators per thread (hides the DFMA latency)
constexpr int PROBE_ITERS = 4096;  // loop trips per launch

// Each thread runs PROBE_CHAINS independent chains x <- x * m + c; m and c
// come from the arguments so the compiler cannot fold them.  The result is
// written only if it matches an impossible value, which keeps the chains live
// without memory traffic.
__global__ void __launch_bounds__(PROBE_THREADS) k_dfma(double m, double c, int iters, double* sink)
{
    double x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == -1.2345e300) sink[0] = s;
}

}  // namespace

extern "C" int pr_probe_fp64_peak(double* tflops)
{
    if (!tflops) return PR_EINVAL;
    *tflops = 0.0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma, PROBE_THREADS, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return PR_ECUDA;
    }
    const int grid = sms * per_sm;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* sink = nullptr;
    int rc = PR_ECUDA;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess && cudaMalloc(&sink, sizeof(double)) == cudaSuccess) {
        // warm-up launch (clocks ramp, module load), then the best of five
        k_dfma<<<grid, PROBE_THREADS, 0, s>>>(0.999999, 1e-7, PROBE_ITERS, sink);
        float best = 0.f;
        bool ok = cudaStreamSynchronize(s) == cudaSuccess;
        for (int rep = 0; rep < 5 && ok; ++rep) {
            ok = cudaEventRecord(e0, s) == cudaSuccess;
            k_dfma<<<grid, PROBE_THREADS, 0, s>>>(0.999999, 1e-7, PROBE_ITERS, sink);
            ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.f;
            ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            if (ok && (best == 0.f || ms < best)) best = ms;
        }
        if (ok && best > 0.f) {
            const double flops = 2.0 * PROBE_CHAINS * (double)PROBE_ITERS * PROBE_THREADS * grid;
            *tflops = flops / (best * 1e-3) / 1e12;
            rc = PR_OK;
        }
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    return rc;
}
