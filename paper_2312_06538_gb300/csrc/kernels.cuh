// Internal launch interface between the C-ABI entry points (api.cu) and the
// translation units that hold the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "crsh.h"

namespace crsh {

struct DeviceInfo {
    int device = -1;
    int sms = 0;
};

// A slice of a host-built FP32 table passed to a kernel by value.
struct TableChunk {
    static constexpr unsigned kMax = 4096;
    unsigned offset, count;
    float v[kMax];
};

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
crsh_status closest_hit_launch(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                               const crsh_scene* sc, const crsh_pairs* pairs, crsh_hits* out, crsh_counters* ctr,
                               void* ws, size_t ws_bytes, cudaStream_t s, const DeviceInfo& dev);
crsh_status closest_hit_noalloc_launch(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                                       const crsh_scene* sc, const crsh_pairs* pairs, crsh_hits* out,
                                       crsh_counters* ctr, cudaStream_t s, const DeviceInfo& dev);
crsh_status bruteforce_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_scene* sc, crsh_hits* out,
                              void* ws, size_t ws_bytes, cudaStream_t s, const DeviceInfo& dev);

}  // namespace crsh
