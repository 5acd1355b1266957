// FP32 peak probe: the FMA throughput the ALU-bound kernels are measured
// against.  Every thread runs CHAINS independent fused multiply-add chains
// (enough independent work per scheduler to cover the FMA latency), so the
// kernel issues FMAs back to back on every SM; flops = 2 per FMA.
#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

constexpr int PROBE_CHAINS = 8, PROBE_BLOCK = 256;

__global__ void __launch_bounds__(PROBE_BLOCK) k_fma_chains(float* out, unsigned iters, float a, float b) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (unsigned i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    if (threadIdx.x == 0) out[blockIdx.x] = s;   // keeps the chains live
}

unsigned long long fma_probe_launch(float* out, unsigned iters, unsigned blocks, cudaStream_t s) {
    // a < 1 and small b keep every chain bounded and finite
    k_fma_chains<<<blocks, PROBE_BLOCK, 0, s>>>(out, iters, 0.999999f, 1e-6f);
    return 2ull * 4 * PROBE_CHAINS * iters * (unsigned long long)blocks * PROBE_BLOCK;
}

}  // namespace crsh
