// C-ABI entry points of include/crsh.h and include/crsh_diag.h: argument
// checks (synchronous), device lookup, then the launches in the kernel
// translation units.
#include <cuda_runtime.h>

#include <mutex>

#include "crsh.h"
#include "crsh_diag.h"
#include "kernels.cuh"

namespace crsh {
namespace {

std::mutex g_dev_mu;
DeviceInfo g_dev[64];

bool current_device(DeviceInfo& out) {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return false;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (g_dev[d].device != d) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || sms <= 0) return false;
        g_dev[d].device = d;
        g_dev[d].sms = sms;
    }
    out = g_dev[d];
    return true;
}

bool pow2_in(unsigned v, unsigned lo, unsigned hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

bool rays_ok(const crsh_rays* r) {
    return r && r->ox && r->oy && r->oz && r->dx && r->dy && r->dz && r->tmax && r->type && r->ray_id && r->pixel &&
           r->capacity <= (1u << 30);
}

bool hier_ok(const crsh_hierarchy* h) {
    if (!h || !h->count || !pow2_in(h->bundle, 2, 64) || h->levels < 1 || h->levels > CRSH_MAX_LEVELS) return false;
    for (unsigned l = 0; l < h->levels; ++l)
        if (!h->sphere[l] || !h->cone[l] || !h->trig[l]) return false;
    return true;
}

// the word form is either absent (valid = 0) or complete
static bool words_ok(const crsh_pair_words& w, const crsh_hierarchy* h) {
    if (!w.valid) return true;
    if (w.valid != 1 || h->levels < 2) return false;
    return w.words && w.tri && w.items && w.n_items;
}

bool scene_ok(const crsh_scene* s, bool need_prepared) {
    if (!s || !s->v0x || !s->v0y || !s->v0z || !s->v1x || !s->v1y || !s->v1z || !s->v2x || !s->v2y || !s->v2z)
        return false;
    if (!s->mesh_first_tri || !s->mesh_sphere || s->n_meshes == 0) return false;
    if (need_prepared && (!s->tri_sphere || !s->tri_mt)) return false;
    return true;
}

}  // namespace
}  // namespace crsh

using namespace crsh;

extern "C" {

int crsh_version(void) { return 100; }

const char* crsh_status_string(crsh_status s) {
    switch (s) {
        case CRSH_OK: return "ok";
        case CRSH_ERR_INVALID_ARG: return "invalid argument";
        case CRSH_ERR_CAPACITY: return "capacity exceeded";
        case CRSH_ERR_CUDA: return "CUDA error";
        case CRSH_ERR_TIMEOUT: return "device wait timed out";
        case CRSH_ERR_NOT_IMPLEMENTED: return "not implemented";
        case CRSH_ERR_BAD_INPUT: return "bad input data";
        default: return "unknown status";
    }
}

crsh_status crsh_prepare_scene(const crsh_scene* scene, void* stream) {
    if (!scene_ok(scene, true)) return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return prepare_scene_launch(scene, static_cast<cudaStream_t>(stream), dev);
}

crsh_status crsh_primary_rays(const crsh_camera* cam, crsh_rays* out, uint32_t* n_out, void* stream) {
    if (!cam || !rays_ok(out) || !n_out || cam->width == 0 || cam->height == 0) return CRSH_ERR_INVALID_ARG;
    if ((uint64_t)cam->width * cam->height > out->capacity) return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return primary_launch(cam, out, n_out, static_cast<cudaStream_t>(stream), dev);
}

crsh_status crsh_gbuffer_from_hits(const crsh_rays* rays, const uint32_t* n_rays, const crsh_hits* hits,
                                   const crsh_scene* scene, const uint32_t* tri_material, crsh_gbuffer_out* out,
                                   void* stream) {
    if (!rays_ok(rays) || !n_rays || !hits || !hits->tri || !hits->t || !scene_ok(scene, false) || !tri_material ||
        !out)
        return CRSH_ERR_INVALID_ARG;
    if (!out->px || !out->py || !out->pz || !out->nx || !out->ny || !out->nz || !out->ix || !out->iy || !out->iz ||
        !out->material || !out->hit)
        return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return gbuffer_from_hits_launch(rays, n_rays, hits, scene, tri_material, out, static_cast<cudaStream_t>(stream),
                                    dev);
}

crsh_status crsh_transform_meshes(const crsh_scene* in, const float* xf, crsh_scene_out* out, void* stream) {
    if (!scene_ok(in, false) || !xf || !out || !out->v0x || !out->v0y || !out->v0z || !out->v1x || !out->v1y ||
        !out->v1z || !out->v2x || !out->v2y || !out->v2z || !out->mesh_sphere)
        return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return transform_launch(in, xf, out, static_cast<cudaStream_t>(stream), dev);
}

crsh_status crsh_shade(const crsh_gbuffer* gb, const float* lights, uint32_t n_lights, const crsh_rays* rays,
                       const uint32_t* n_rays, const crsh_hits* hits, const uint32_t* tri_material, float* cells,
                       float* color, void* stream) {
    if (!gb || !gb->nx || !gb->ny || !gb->nz || !gb->material || !gb->hit || !rays_ok(rays) || !n_rays || !hits ||
        !hits->tri || !tri_material || !cells || !color || (n_lights > 0 && !lights) || n_lights > 255)
        return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return shade_launch(gb, lights, n_lights, rays, n_rays, hits, tri_material, cells, color,
                        static_cast<cudaStream_t>(stream), dev);
}

crsh_status crsh_fma_probe(float* out, uint32_t iters, uint32_t blocks, unsigned long long* flops, void* stream) {
    if (!out || !flops || iters < 1 || blocks < 1 || blocks > (1u << 20)) return CRSH_ERR_INVALID_ARG;
    *flops = fma_probe_launch(out, iters, blocks, static_cast<cudaStream_t>(stream));
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

crsh_status crsh_lookback_selftest(unsigned long long* status64, uint32_t* status32, uint32_t wide, uint32_t tile,
                                   uint32_t aggregate, uint32_t spin_limit, unsigned long long* prefix_out,
                                   crsh_counters* counters, void* stream) {
    if (!prefix_out || !counters || tile < 1 || spin_limit < 1 || spin_limit > (1u << 22)) return CRSH_ERR_INVALID_ARG;
    if (wide ? !status64 : (!status32 || aggregate >= (1u << 30))) return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    lookback_selftest_launch(status64, status32, wide ? 1 : 0, tile, aggregate, spin_limit, prefix_out, counters,
                             static_cast<cudaStream_t>(stream));
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

crsh_status crsh_hash_tables(uint32_t theta_bits, uint32_t phi_bits, float* cos_out, float* tan_out, void* stream) {
    if (theta_bits < 1 || theta_bits > 13 || phi_bits < 3 || phi_bits > 13 || !cos_out || !tan_out)
        return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    tables_launch(TableSpec{{cos_out, tan_out, nullptr, nullptr}, {1u << theta_bits, (1u << phi_bits) / 8, 0, 0},
                            {0, 1, 0, 0}},
                  static_cast<cudaStream_t>(stream), dev);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

size_t crsh_hash_sort_workspace(uint32_t capacity, uint32_t max_pixels) {
    return hash_sort_workspace(capacity, max_pixels);
}

// Workspaces are carved into 256-byte-aligned arrays that kernels read with
// 16-byte vector accesses, so the base must be 256-byte aligned.
static bool ws_ok(const void* w) { return w != nullptr && (reinterpret_cast<uintptr_t>(w) & 255u) == 0; }

crsh_status crsh_hash_sort(const crsh_gbuffer* gbuffer, const crsh_rays_in* rays_in, const float* lights,
                           uint32_t n_lights, const crsh_hash_params* p, crsh_rays* out, uint32_t* keys_out,
                           uint32_t* n_out, crsh_counters* counters, void* workspace, size_t workspace_bytes,
                           void* stream) {
    if ((gbuffer == nullptr) == (rays_in == nullptr)) return CRSH_ERR_INVALID_ARG;
    if (!p || !rays_ok(out) || !keys_out || !n_out || !counters || !ws_ok(workspace)) return CRSH_ERR_INVALID_ARG;
    if (p->shadow_theta_bits < 1 || p->shadow_theta_bits > 13 || p->shadow_phi_bits < 3 || p->shadow_phi_bits > 13 ||
        p->shadow_theta_bits + p->shadow_phi_bits > 30)
        return CRSH_ERR_INVALID_ARG;
    if (p->sec_theta_bits < 1 || p->sec_theta_bits > 13 || p->sec_phi_bits < 3 || p->sec_phi_bits > 13 ||
        p->sec_cell_bits > 10 || 3 * p->sec_cell_bits + p->sec_theta_bits + p->sec_phi_bits > 30)
        return CRSH_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(p->hi[a] > p->lo[a])) return CRSH_ERR_INVALID_ARG;
    if (gbuffer) {
        const crsh_gbuffer* g = gbuffer;
        if (!g->px || !g->py || !g->pz || !g->nx || !g->ny || !g->nz || !g->ix || !g->iy || !g->iz || !g->material ||
            !g->hit)
            return CRSH_ERR_INVALID_ARG;
        if (n_lights > 0 && !lights) return CRSH_ERR_INVALID_ARG;
        if (n_lights > (1u << (30 - p->shadow_theta_bits - p->shadow_phi_bits)) || n_lights > 255)
            return CRSH_ERR_INVALID_ARG;
    } else {
        const crsh_rays_in* r = rays_in;
        if (r->n > 0 && (!r->ox || !r->oy || !r->oz || !r->dx || !r->dy || !r->dz || !r->tmax || !r->type))
            return CRSH_ERR_INVALID_ARG;
    }
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return hash_sort_launch(gbuffer, rays_in, lights, n_lights, p, out, keys_out, n_out, counters, workspace,
                            workspace_bytes, static_cast<cudaStream_t>(stream), dev);
}

crsh_status crsh_build(const crsh_rays* rays, const uint32_t* n_rays, const crsh_build_params* p,
                       crsh_hierarchy* out, void* stream) {
    if (!rays_ok(rays) || !n_rays || !p || !out || !out->count) return CRSH_ERR_INVALID_ARG;
    if (!pow2_in(p->bundle, 2, 64) || p->levels < 1 || p->levels > CRSH_MAX_LEVELS) return CRSH_ERR_INVALID_ARG;
    if (!(p->sphere_pad_rel >= 0) || !(p->sphere_pad_abs >= 0) || !(p->cone_pad_rel >= 0) || !(p->cone_pad_abs >= 0))
        return CRSH_ERR_INVALID_ARG;
    uint64_t need = rays->capacity;
    for (unsigned l = 0; l < p->levels; ++l) {
        need = (need + p->bundle - 1) / p->bundle;
        if (!out->sphere[l] || !out->cone[l] || !out->trig[l] || out->capacity[l] < need) return CRSH_ERR_INVALID_ARG;
    }
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return build_launch(rays, n_rays, p, out, static_cast<cudaStream_t>(stream), dev);
}

size_t crsh_traverse_workspace(const crsh_hierarchy* h, uint32_t n_tris, uint32_t n_meshes, uint64_t pair_capacity) {
    if (!h || h->levels < 1 || h->levels > CRSH_MAX_LEVELS || !pow2_in(h->bundle, 2, 64)) return 0;
    return traverse_workspace(h, n_tris, n_meshes, pair_capacity);
}

crsh_status crsh_traverse(const crsh_hierarchy* h, const crsh_scene* scene, const crsh_traverse_params* p,
                          crsh_pairs* out, crsh_counters* counters, void* workspace, size_t workspace_bytes,
                          void* stream) {
    if (!hier_ok(h) || !scene_ok(scene, true) || !p || !out || !counters || !ws_ok(workspace)) return CRSH_ERR_INVALID_ARG;
    if (p->block_threads != 0 && p->block_threads != 128 && p->block_threads != 256 && p->block_threads != 512)
        return CRSH_ERR_INVALID_ARG;
    if (p->level1_words > 1) return CRSH_ERR_INVALID_ARG;
    if (!out->node || !out->tri || !out->node_offsets || !out->count || out->capacity == 0 ||
        out->capacity > (1ull << 31))
        return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return traverse_launch(h, scene, p, out, counters, workspace, workspace_bytes, static_cast<cudaStream_t>(stream),
                           dev);
}

size_t crsh_closest_hit_workspace(uint32_t ray_capacity) { return closest_hit_workspace(ray_capacity); }

crsh_status crsh_closest_hit(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                             const crsh_scene* scene, const crsh_pairs* pairs, crsh_hits* out,
                             crsh_counters* counters, void* workspace, size_t workspace_bytes, void* stream) {
    if (!hier_ok(h) || !rays_ok(rays) || !n_rays || !scene_ok(scene, true) || !pairs || !pairs->node ||
        !pairs->tri || !pairs->count || !out || !out->tri || !out->t || !out->u || !out->v || !counters || !ws_ok(workspace))
        return CRSH_ERR_INVALID_ARG;
    if (!words_ok(pairs->words, h)) return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return closest_hit_launch(h, rays, n_rays, scene, pairs, out, counters, workspace, workspace_bytes,
                              static_cast<cudaStream_t>(stream), dev);
}

crsh_status crsh_closest_hit_timed(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                                   const crsh_scene* scene, const crsh_pairs* pairs, crsh_hits* out,
                                   crsh_counters* counters, void* workspace, size_t workspace_bytes,
                                   float* kernel_ms, void* stream) {
    if (!hier_ok(h) || !rays_ok(rays) || !n_rays || !scene_ok(scene, true) || !pairs || !pairs->node ||
        !pairs->tri || !pairs->count || !out || !out->tri || !out->t || !out->u || !out->v || !counters ||
        !ws_ok(workspace) || !kernel_ms)
        return CRSH_ERR_INVALID_ARG;
    if (!words_ok(pairs->words, h)) return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return CRSH_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CRSH_ERR_CUDA;
    }
    crsh_status st = closest_hit_launch(h, rays, n_rays, scene, pairs, out, counters, workspace, workspace_bytes, s,
                                        dev, e0, e1);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = CRSH_ERR_CUDA;
    if (st == CRSH_OK && cudaEventElapsedTime(kernel_ms, e0, e1) != cudaSuccess) st = CRSH_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

crsh_status crsh_closest_hit_noalloc(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                                     const crsh_scene* scene, const crsh_pairs* pairs, crsh_hits* out,
                                     crsh_counters* counters, void* stream) {
    if (!hier_ok(h) || !rays_ok(rays) || !n_rays || !scene_ok(scene, true) || !pairs || !pairs->node ||
        !pairs->tri || !pairs->count || !out || !out->tri || !out->t || !out->u || !out->v || !counters)
        return CRSH_ERR_INVALID_ARG;
    if (!words_ok(pairs->words, h)) return CRSH_ERR_INVALID_ARG;
    if (rays->capacity > CRSH_NOALLOC_MAX_RAYS) return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return closest_hit_noalloc_launch(h, rays, n_rays, scene, pairs, out, counters,
                                      static_cast<cudaStream_t>(stream), dev);
}

size_t crsh_closest_hit_backward_workspace(uint32_t ray_capacity) { return backward_workspace(ray_capacity); }

crsh_status crsh_closest_hit_backward(const crsh_rays* rays, const uint32_t* n_rays, const crsh_scene* scene,
                                      const crsh_hits* hits, const float* g_t, const float* g_u, const float* g_v,
                                      float* g_verts, float* g_orig, float* g_dir, crsh_counters* counters,
                                      void* workspace, size_t workspace_bytes, void* stream) {
    if (!rays_ok(rays) || !n_rays || !scene_ok(scene, false) || !hits || !hits->tri || !hits->t || !hits->u ||
        !hits->v || !g_t || !g_u || !g_v || !g_verts || !g_orig || !g_dir || !ws_ok(workspace))
        return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return backward_launch(rays, n_rays, scene, hits, g_t, g_u, g_v, g_verts, g_orig, g_dir, counters, workspace,
                           workspace_bytes, static_cast<cudaStream_t>(stream), dev);
}

crsh_status crsh_bruteforce_closest_hit(const crsh_rays* rays, const uint32_t* n_rays, const crsh_scene* scene,
                                        crsh_hits* out, void* workspace, size_t workspace_bytes, void* stream) {
    if (!rays_ok(rays) || !n_rays || !scene_ok(scene, true) || !out || !out->tri || !out->t || !out->u || !out->v ||
        !ws_ok(workspace))
        return CRSH_ERR_INVALID_ARG;
    DeviceInfo dev;
    if (!current_device(dev)) return CRSH_ERR_CUDA;
    return bruteforce_launch(rays, n_rays, scene, out, workspace, workspace_bytes, static_cast<cudaStream_t>(stream),
                             dev);
}

}  // extern "C"
