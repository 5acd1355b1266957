// Shading accumulation (NEXT row f4; Section 3.3.8: after the final tests the
// closest hits are turned into shading).  The paper names no shading model;
// this one is the reading stated in include/crsh.h: grey-level Lambert with
// hard shadows from the shadow rays, plus one mirror/glass bounce from the
// reflection and refraction rays.  Deterministic: every secondary ray writes
// its own term into a (pixel, slot) cell, and each pixel sums its cells in a
// fixed order.
#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

struct ShadeConst {
    float albedo[3], refl[3], trans[3];   // by material: diffuse, mirror, glass
    float ambient, sky, bounce_light;
};

__device__ __forceinline__ ShadeConst shade_const() {
    return ShadeConst{{0.8f, 0.2f, 0.1f}, {0.0f, 0.8f, 0.1f}, {0.0f, 0.0f, 0.8f}, 0.1f, 0.6f, 0.5f};
}

__device__ __forceinline__ unsigned mat_ix(unsigned m) { return m <= CRSH_MAT_GLASS ? m : 0u; }

// Term of secondary ray i in cell (pixel, slot): slot k < n_lights for the
// shadow ray of light k (the light whose position is the ray's origin),
// n_lights for reflection, n_lights + 1 for refraction.
__global__ void k_shade_rays(crsh_gbuffer gb, const float* lights, unsigned n_lights, crsh_rays rays,
                             const unsigned* n_ptr, crsh_hits hits, const uint32_t* tri_material, float* cells) {
    const ShadeConst K = shade_const();
    const unsigned n = *n_ptr, S = n_lights + 2;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned g = rays.ray_id[i], p = rays.pixel[i];
        if (p >= gb.n_pixels) continue;
        const int tri = hits.tri[g];
        const unsigned type = rays.type[i];
        const float dx = rays.dx[i], dy = rays.dy[i], dz = rays.dz[i];
        if (type == CRSH_RAY_SHADOW) {
            const float ox = rays.ox[i], oy = rays.oy[i], oz = rays.oz[i];
            unsigned k = 0;
            while (k < n_lights && !(lights[3 * k] == ox && lights[3 * k + 1] == oy && lights[3 * k + 2] == oz)) ++k;
            if (k == n_lights) continue;
            float v = 0.0f;
            if (tri < 0) {   // unoccluded: Lambert term n . l with l = -d
                float c = __fmul_rn(gb.nx[p], -dx);
                c = __fadd_rn(c, __fmul_rn(gb.ny[p], -dy));
                c = __fadd_rn(c, __fmul_rn(gb.nz[p], -dz));
                v = fmaxf(c, 0.0f);
            }
            cells[(size_t)p * S + k] = v;
        } else if (type == CRSH_RAY_REFLECTION || type == CRSH_RAY_REFRACTION) {
            const float v = tri < 0 ? K.sky
                                    : __fmul_rn(K.albedo[mat_ix(tri_material[tri])], __fadd_rn(K.ambient, K.bounce_light));
            cells[(size_t)p * S + n_lights + (type == CRSH_RAY_REFRACTION ? 1u : 0u)] = v;
        }
    }
}

__global__ void k_shade_pixels(crsh_gbuffer gb, unsigned n_lights, const float* cells, float* color) {
    const ShadeConst K = shade_const();
    const unsigned S = n_lights + 2;
    for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < gb.n_pixels; p += gridDim.x * blockDim.x) {
        if (!gb.hit[p]) {
            color[p] = K.sky;
            continue;
        }
        const unsigned m = mat_ix(gb.material[p]);
        const float* c = cells + (size_t)p * S;
        float s = K.ambient;
        for (unsigned k = 0; k < n_lights; ++k) s = __fadd_rn(s, c[k]);
        float col = __fmul_rn(K.albedo[m], s);
        col = __fadd_rn(col, __fmul_rn(K.refl[m], c[n_lights]));
        col = __fadd_rn(col, __fmul_rn(K.trans[m], c[n_lights + 1]));
        color[p] = col;
    }
}

crsh_status shade_launch(const crsh_gbuffer* gb, const float* lights, uint32_t n_lights, const crsh_rays* rays,
                         const uint32_t* n_rays, const crsh_hits* hits, const uint32_t* tri_material, float* cells,
                         float* color, cudaStream_t s, const DeviceInfo& dev) {
    const size_t S = (size_t)n_lights + 2;
    if (cudaMemsetAsync(cells, 0, (size_t)gb->n_pixels * S * sizeof(float), s) != cudaSuccess) return CRSH_ERR_CUDA;
    {
        const unsigned blocks = (rays->capacity + 255) / 256;
        const unsigned grid = blocks < (unsigned)dev.sms * 8 ? (blocks ? blocks : 1) : dev.sms * 8;
        k_shade_rays<<<grid, 256, 0, s>>>(*gb, lights, n_lights, *rays, n_rays, *hits, tri_material, cells);
    }
    const unsigned blocks = (gb->n_pixels + 255) / 256;
    const unsigned grid = blocks < (unsigned)dev.sms * 8 ? (blocks ? blocks : 1) : dev.sms * 8;
    k_shade_pixels<<<grid, 256, 0, s>>>(*gb, n_lights, cells, color);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

}  // namespace crsh
