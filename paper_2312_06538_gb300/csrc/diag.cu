// Diagnostics (include/crsh_diag.h), not steps of the method.
//
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

// Look-back self-test: one warp resolves one tile against status words the
// caller prepared, with the spin limit given, so a predecessor that never
// publishes makes the wait run out (CRSH_ERR_TIMEOUT) and the kernel return.
__global__ void k_lookback_selftest(unsigned long long* s64, unsigned* s32, int wide, unsigned tile,
                                    unsigned aggregate, unsigned spin_limit, unsigned long long* out,
                                    crsh_counters* ctr) {
    if (wide) {
        const unsigned long long e = lookback_warp(s64, tile, aggregate, ctr, spin_limit);
        if (threadIdx.x == 0) *out = e;
    } else if (threadIdx.x == 0) {
        lookback32_publish(s32, tile, 1, aggregate);
        *out = lookback32_resolve(s32, tile, 1, aggregate, ctr, spin_limit);
    }
}

void lookback_selftest_launch(unsigned long long* s64, unsigned* s32, int wide, unsigned tile, unsigned aggregate,
                              unsigned spin_limit, unsigned long long* out, crsh_counters* ctr, cudaStream_t s) {
    k_lookback_selftest<<<1, 32, 0, s>>>(s64, s32, wide, tile, aggregate, spin_limit, out, ctr);
}

}  // namespace crsh
