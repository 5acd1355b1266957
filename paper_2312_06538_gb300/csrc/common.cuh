// Shared device helpers of the CRSH library: status reporting, decoupled
// look-back prefix sums (single-pass scans with bounded waits), warp scans,
// small vector math.
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <stdint.h>

#include "crsh.h"

namespace crsh {

constexpr unsigned FULL = 0xffffffffu;

// ---- device status -------------------------------------------------------

// First error wins: later errors never overwrite an earlier one.
__device__ __forceinline__ void set_status(crsh_counters* c, unsigned code) {
    if (c) atomicCAS(&c->status, 0u, code);
}

// ---- vector helpers ------------------------------------------------------

struct f3 { float x, y, z; };
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float len(f3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ f3 unit(f3 a) { return a * rsqrtf(dot(a, a)); }
// angle between two directions; accurate near 0 and pi
__device__ __forceinline__ float angle(f3 a, f3 b) { return atan2f(len(cross(a, b)), dot(a, b)); }

constexpr float PI_F = 3.14159265358979323846f;

// ---- relaxed global loads/stores for look-back status words --------------

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed32(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---- warp reductions / scans ---------------------------------------------

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// inclusive scan of 32-bit values over the warp
__device__ __forceinline__ unsigned warp_incl_scan(unsigned v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned n = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---- programmatic dependent launch ----------------------------------------
// A kernel launched with launch_pdl may start while the kernel before it in
// the stream is still finishing; it must call pdl_wait() before touching
// anything that kernel writes (pdl_wait returns once it has completed and its
// memory is visible).  Launch latency and block scheduling then overlap the
// previous kernel's tail.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---- asynchronous global -> shared copies (16-byte aligned both sides) ----
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 4-byte copy (L1-allocating); both addresses 4-byte aligned
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// waits for every copy this thread issued
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// waits for every committed group but the newest one
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---- decoupled look-back (single-pass prefix across tiles) ---------------
//
// Tiles are handed out in increasing order (atomic counter), so every tile a
// block waits for has already been taken by a running block, which publishes
// its own total before it waits on anyone.  Status word: bits 63:62 flag
// (0 = not ready, 1 = tile total, 2 = inclusive prefix), bits 61:0 value.
// Waits are bounded: after kSpinLimit polls (or the spin_limit a caller
// passes) the tile records CRSH_ERR_TIMEOUT and continues with what it has.

constexpr unsigned long long LB_AGG = 1ull << 62;
constexpr unsigned long long LB_INC = 2ull << 62;
constexpr unsigned long long LB_VAL = (1ull << 62) - 1;
constexpr unsigned kSpinLimit = 1u << 22;

// Called by all 32 lanes of ONE warp; returns the exclusive prefix of `tile`
// (the same in every lane) and publishes the tile's inclusive prefix.
__device__ __forceinline__ unsigned long long lookback_warp(unsigned long long* status, unsigned tile,
                                                           unsigned long long aggregate,
                                                           crsh_counters* ctr, unsigned spin_limit = kSpinLimit) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_relaxed(&status[0], LB_INC | aggregate);
        return 0;
    }
    if (lane == 0) st_relaxed(&status[tile], LB_AGG | aggregate);
    unsigned long long excl = 0;
    long long k = (long long)tile - 1;
    unsigned spins = 0;
    while (true) {
        long long idx = k - lane;
        unsigned long long s = (idx >= 0) ? ld_relaxed(&status[idx]) : LB_INC;
        while (__any_sync(FULL, (s >> 62) == 0)) {
            if (++spins > spin_limit) {
                if (lane == 0) set_status(ctr, CRSH_ERR_TIMEOUT);
                if ((s >> 62) == 0) s = LB_INC;
                break;
            }
            __nanosleep(32);
            if ((s >> 62) == 0) s = ld_relaxed(&status[idx]);
        }
        unsigned inc = __ballot_sync(FULL, (s >> 62) == 2);
        unsigned long long v = s & LB_VAL;
        if (inc) {
            int first = __ffs(inc) - 1;
            excl += warp_sum64(lane <= first ? v : 0ull);
            break;
        }
        excl += warp_sum64(v);
        k -= 32;
    }
    if (lane == 0) st_relaxed(&status[tile], LB_INC | (excl + aggregate));
    return excl;
}

// 32-bit status word variant for one thread (used per radix digit):
// bits 31:30 flag, 29:0 value (counts below 2^30).
constexpr unsigned LB32_AGG = 1u << 30;
constexpr unsigned LB32_INC = 2u << 30;
constexpr unsigned LB32_VAL = (1u << 30) - 1;

// The predecessors' words are read LB32_WIN at a time (independent loads in
// flight), so a walk over many tiles that all hold only their own totals costs
// one memory latency per LB32_WIN tiles.
constexpr int LB32_WIN = 8;

// Publishes a tile's own total (tile 0: already its inclusive prefix), so
// successors can sum past it before it knows its own prefix.
__device__ __forceinline__ void lookback32_publish(unsigned* status, unsigned tile, unsigned stride,
                                                   unsigned aggregate) {
    st_relaxed32(&status[(size_t)tile * stride], (tile == 0 ? LB32_INC : LB32_AGG) | aggregate);
}

// After lookback32_publish: the tile's exclusive prefix; publishes its
// inclusive prefix.
__device__ __forceinline__ unsigned lookback32_resolve(unsigned* status, unsigned tile, unsigned stride,
                                                       unsigned aggregate, crsh_counters* ctr,
                                                       unsigned spin_limit = kSpinLimit) {
    if (tile == 0) return 0;
    unsigned excl = 0;
    unsigned spins = 0;
    long long k = (long long)tile - 1;   // next predecessor to consume
    while (k >= 0) {
        unsigned s[LB32_WIN];
#pragma unroll
        for (int i = 0; i < LB32_WIN; ++i)
            s[i] = (k - i >= 0) ? ld_relaxed32(&status[(size_t)(k - i) * stride]) : LB32_INC;
        bool done = false;
        int used = 0;
#pragma unroll
        for (int i = 0; i < LB32_WIN; ++i) {
            if ((s[i] >> 30) == 0) break;          // not published yet: poll again from here
            excl += s[i] & LB32_VAL;
            used = i + 1;
            if ((s[i] >> 30) == 2) {
                done = true;
                break;
            }
        }
        if (done) break;
        k -= used;
        if (used == 0) {
            if (++spins > spin_limit) {
                set_status(ctr, CRSH_ERR_TIMEOUT);
                break;
            }
            if (spins > 64) __nanosleep(32);   // short waits are polled, long ones back off
        }
    }
    st_relaxed32(&status[(size_t)tile * stride], LB32_INC | (excl + aggregate));
    return excl;
}

__device__ __forceinline__ unsigned lookback_thread32(unsigned* status, unsigned tile, unsigned stride,
                                                      unsigned aggregate, crsh_counters* ctr) {
    lookback32_publish(status, tile, stride, aggregate);
    return lookback32_resolve(status, tile, stride, aggregate, ctr);
}

// Hands out tiles in increasing order; returns the tile in every thread.
__device__ __forceinline__ unsigned next_tile(unsigned* counter, unsigned* smem_slot) {
    __syncthreads();
    if (threadIdx.x == 0) *smem_slot = atomicAdd(counter, 1u);
    __syncthreads();
    return *smem_slot;
}

}  // namespace crsh
