// FP64 fused multiply-add throughput probe.
//
// The roofline of the FP64 condensation product and factorization is the rate
// of the SM's FP64 FMA pipe.  This kernel measures that rate on the GPU at
// hand: every thread runs eight independent FMA chains (enough independent
// work per warp scheduler to hide the pipe's latency), so the time of the
// launch is the time the FP64 pipe takes for blocks x 256 x iters x 8 FMAs.
// The result of each chain is written out so that no work can be removed.
#include "internal.cuh"

namespace mdsip {

namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma_probe(int64_t iters, double *sink) {
    const double a = 1.0 + 1e-9 * threadIdx.x, b = 1e-7;
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 1e-3 * (k + 1) + 1e-6 * blockIdx.x;
    // eight chain steps per loop trip: the loop's own instructions take a
    // negligible share of the issue slots
    int64_t i = 0;
    for (; i + 8 <= iters; i += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
    }
    for (; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

void launch_fp64_fma_probe(cudaStream_t s, int blocks, int64_t iters, double *sink) {
    k_fp64_fma_probe<<<blocks, kProbeThreads, 0, s>>>(iters, sink);
    MDSIP_LAUNCHED();
}

}  // namespace mdsip
