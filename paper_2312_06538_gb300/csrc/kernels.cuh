// Internal launch interface between the C-ABI entry points (api.cu) and the
// translation units that hold the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "crsh.h"

namespace crsh {

// Words per final-test work item of the word form of level 1 (crsh_pair_words):
// an item is one child's run of up to WORD_SEG consecutive chunk ballots, so a
// node with a long row is split over several items.
constexpr unsigned WORD_SEG = 32;

struct DeviceInfo {
    int device = -1;
    int sms = 0;
};

// Up to three byte ranges zeroed by one kernel (hash_sort.cu) instead of memset
// nodes, so that the zeroing chains with the launches around it by
// programmatic dependent launch.  Each range starts on a 4-byte boundary and
// spans a multiple of 4 bytes; a null range is skipped.
struct ZeroSpans {
    void* p[3];
    size_t bytes[3];
};
void zero_launch(const ZeroSpans& z, cudaStream_t s, const DeviceInfo& dev);

// Up to four bin threshold tables to fill (hash_sort.cu): entry k of table i
// is cos(k pi / n[i]) or, when is_tan[i], tan(k (pi/4) / n[i]), in FP32.
struct TableSpec {
    float* dst[4];
    unsigned n[4];
    int is_tan[4];
};
void tables_launch(const TableSpec& t, cudaStream_t s, const DeviceInfo& dev);

// Primary visibility, first-hit buffers, mesh update (primary.cu).
crsh_status primary_launch(const crsh_camera* cam, crsh_rays* out, uint32_t* n_out, cudaStream_t s,
                           const DeviceInfo& dev);
crsh_status gbuffer_from_hits_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_hits* hits,
                                     const crsh_scene* sc, const uint32_t* tri_material, crsh_gbuffer_out* out,
                                     cudaStream_t s, const DeviceInfo& dev);
crsh_status transform_launch(const crsh_scene* in, const float* xf, crsh_scene_out* out, cudaStream_t s,
                             const DeviceInfo& dev);

// Shading accumulation (shade.cu).
crsh_status shade_launch(const crsh_gbuffer* gb, const float* lights, uint32_t n_lights, const crsh_rays* rays,
                         const uint32_t* n_rays, const crsh_hits* hits, const uint32_t* tri_material, float* cells,
                         float* color, cudaStream_t s, const DeviceInfo& dev);

// Diagnostics (diag.cu): the FP32 FMA throughput probe (returns the flops
// launched) and the bounded-wait self-test of the look-back.
unsigned long long fma_probe_launch(float* out, unsigned iters, unsigned blocks, cudaStream_t s);
void lookback_selftest_launch(unsigned long long* s64, unsigned* s32, int wide, unsigned tile, unsigned aggregate,
                              unsigned spin_limit, unsigned long long* out, crsh_counters* ctr, cudaStream_t s);

// One-sweep LSD radix sort of 32-bit (key, value) pairs (hash_sort.cu).
struct RadixWs {
    unsigned* hist;      // 4 x 256, zeroed
    unsigned* offs;      // 4 x 256
    unsigned* plan;      // 5; plan[4] = buffer holding the result (0: A, 1: B)
    unsigned* tile_ctr;  // 4, zeroed
    unsigned* status;    // radix_status_words(cap), zeroed
};
size_t radix_status_words(uint32_t cap);
// counted: rw.hist already holds the digit counts of the keys (their producer made them).
// identity: the values are the element indices 0 .. n-1; vA is not read (the first pass that
// runs makes them, and one pass always runs).
void radix_sort_launch(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, const unsigned* cnt_ptr, uint32_t cap,
                       const RadixWs& rw, crsh_counters* ctr, cudaStream_t s, const DeviceInfo& dev,
                       bool counted = false, bool identity = false);

size_t hash_sort_workspace(uint32_t capacity, uint32_t max_pixels);
crsh_status hash_sort_launch(const crsh_gbuffer* gb, const crsh_rays_in* in, const float* lights, uint32_t n_lights,
                             const crsh_hash_params* hp, crsh_rays* out, uint32_t* keys_out, uint32_t* n_out,
                             crsh_counters* ctr, void* ws, size_t ws_bytes, cudaStream_t s, const DeviceInfo& dev);

crsh_status prepare_scene_launch(const crsh_scene* sc, cudaStream_t s, const DeviceInfo& dev);

crsh_status build_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_build_params* bp,
                         crsh_hierarchy* h, cudaStream_t s, const DeviceInfo& dev);

size_t traverse_workspace(const crsh_hierarchy* h, uint32_t n_tris, uint32_t n_meshes, uint64_t pair_capacity);
crsh_status traverse_launch(const crsh_hierarchy* h, const crsh_scene* sc, const crsh_traverse_params* tp,
                            crsh_pairs* out, crsh_counters* ctr, void* ws, size_t ws_bytes, cudaStream_t s,
                            const DeviceInfo& dev);

size_t closest_hit_workspace(uint32_t ray_capacity);
// ev_begin / ev_end (optional): events recorded on s around the final-test kernel (measurement).
crsh_status closest_hit_launch(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                               const crsh_scene* sc, const crsh_pairs* pairs, crsh_hits* out, crsh_counters* ctr,
                               void* ws, size_t ws_bytes, cudaStream_t s, const DeviceInfo& dev,
                               cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr);
crsh_status closest_hit_noalloc_launch(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                                       const crsh_scene* sc, const crsh_pairs* pairs, crsh_hits* out,
                                       crsh_counters* ctr, cudaStream_t s, const DeviceInfo& dev);
size_t backward_workspace(uint32_t ray_capacity);
crsh_status backward_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_scene* sc, const crsh_hits* hits,
                            const float* g_t, const float* g_u, const float* g_v, float* g_verts, float* g_orig,
                            float* g_dir, crsh_counters* ctr, void* ws, size_t ws_bytes, cudaStream_t s,
                            const DeviceInfo& dev);
crsh_status bruteforce_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_scene* sc, crsh_hits* out,
                              void* ws, size_t ws_bytes, cudaStream_t s, const DeviceInfo& dev);

}  // namespace crsh
