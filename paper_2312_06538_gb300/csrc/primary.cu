// Primary visibility, next-bounce hit points and the per-frame mesh update
// (NEXT row f3).  Primary rays go through the same hierarchy path as
// secondary ones: a pinhole camera's rays are coherent in tile order, so they
// are generated directly in an order whose aligned runs of B rays cover
// compact pixel tiles, and need no hashing or sorting.  First-hit buffers are
// written from closest hits in FP32 with a fixed operation order; feeding one
// to crsh_hash_sort emits the next bounce (Section 3.3.8).
#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }

// Z-order index inside an 8 x 8 block: x bit b at 2b, y bit b at 2b + 1
__device__ __forceinline__ unsigned z8(unsigned x, unsigned y) {
    unsigned z = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) z |= ((x >> b) & 1u) << (2 * b) | ((y >> b) & 1u) << (2 * b + 1);
    return z;
}

// Position of pixel (x, y) in tile order (see crsh_primary_rays).
__device__ __forceinline__ unsigned tile_rank(unsigned x, unsigned y, unsigned W, unsigned H) {
    const unsigned bx = x >> 3, by = y >> 3, lx = x & 7u, ly = y & 7u;
    const unsigned bw = min(8u, W - 8 * bx), bh = min(8u, H - 8 * by);
    const unsigned before = by * 8u * W + bx * 8u * bh;
    const unsigned z = z8(lx, ly);
    if (bw == 8 && bh == 8) return before + z;
    unsigned r = 0;   // edge block: in-image pixels with a smaller Z index
    for (unsigned q = 0; q < z; ++q) {
        unsigned qx = 0, qy = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            qx |= ((q >> (2 * b)) & 1u) << b;
            qy |= ((q >> (2 * b + 1)) & 1u) << b;
        }
        r += (qx < bw && qy < bh) ? 1u : 0u;
    }
    return before + r;
}

__global__ void k_primary(crsh_camera cam, crsh_rays out, unsigned* n_out) {
    const unsigned W = cam.width, H = cam.height, n = W * H;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = n;
    const float inf = __int_as_float(0x7f800000);
    for (unsigned p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const unsigned x = p % W, y = p / W;
        // sx = (2 (x + 0.5) / W - 1) tan_x, sy = (1 - 2 (y + 0.5) / H) tan_y
        const float sx = rn_mul(rn_sub(rn_div(rn_mul(2.0f, rn_add((float)x, 0.5f)), (float)W), 1.0f), cam.tan_x);
        const float sy = rn_mul(rn_sub(1.0f, rn_div(rn_mul(2.0f, rn_add((float)y, 0.5f)), (float)H)), cam.tan_y);
        const float d0 = rn_add(rn_add(cam.fwd[0], rn_mul(sx, cam.right[0])), rn_mul(sy, cam.up[0]));
        const float d1 = rn_add(rn_add(cam.fwd[1], rn_mul(sx, cam.right[1])), rn_mul(sy, cam.up[1]));
        const float d2 = rn_add(rn_add(cam.fwd[2], rn_mul(sx, cam.right[2])), rn_mul(sy, cam.up[2]));
        const float len = __fsqrt_rn(rn_add(rn_add(rn_mul(d0, d0), rn_mul(d1, d1)), rn_mul(d2, d2)));
        const unsigned i = tile_rank(x, y, W, H);
        out.ox[i] = cam.eye[0];
        out.oy[i] = cam.eye[1];
        out.oz[i] = cam.eye[2];
        out.dx[i] = rn_div(d0, len);
        out.dy[i] = rn_div(d1, len);
        out.dz[i] = rn_div(d2, len);
        out.tmax[i] = inf;
        out.type[i] = CRSH_RAY_PRIMARY;
        out.ray_id[i] = p;
        out.pixel[i] = p;
    }
}

crsh_status primary_launch(const crsh_camera* cam, crsh_rays* out, uint32_t* n_out, cudaStream_t s,
                           const DeviceInfo& dev) {
    const unsigned n = cam->width * cam->height;
    const unsigned blocks = (n + 255) / 256;
    const unsigned grid = blocks < (unsigned)dev.sms * 8 ? (blocks ? blocks : 1) : dev.sms * 8;
    k_primary<<<grid, 256, 0, s>>>(*cam, *out, n_out);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

__global__ void k_gbuffer(crsh_rays rays, const unsigned* n_ptr, crsh_hits hits, crsh_scene sc,
                          const uint32_t* tri_material, crsh_gbuffer_out out) {
    const unsigned n = *n_ptr;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned g = rays.ray_id[i];
        if (g >= out.n) continue;
        const float dx = rays.dx[i], dy = rays.dy[i], dz = rays.dz[i];
        out.ix[g] = dx;
        out.iy[g] = dy;
        out.iz[g] = dz;
        const int tri = hits.tri[g];
        if (tri < 0) {
            out.px[g] = out.py[g] = out.pz[g] = 0.0f;
            out.nx[g] = out.ny[g] = out.nz[g] = 0.0f;
            out.material[g] = 0;
            out.hit[g] = 0;
            continue;
        }
        const float t = hits.t[g];
        out.px[g] = rn_add(rays.ox[i], rn_mul(t, dx));
        out.py[g] = rn_add(rays.oy[i], rn_mul(t, dy));
        out.pz[g] = rn_add(rays.oz[i], rn_mul(t, dz));
        const float ax = sc.v0x[tri], ay = sc.v0y[tri], az = sc.v0z[tri];
        const float e1x = rn_sub(sc.v1x[tri], ax), e1y = rn_sub(sc.v1y[tri], ay), e1z = rn_sub(sc.v1z[tri], az);
        const float e2x = rn_sub(sc.v2x[tri], ax), e2y = rn_sub(sc.v2y[tri], ay), e2z = rn_sub(sc.v2z[tri], az);
        float nx = rn_sub(rn_mul(e1y, e2z), rn_mul(e1z, e2y));
        float ny = rn_sub(rn_mul(e1z, e2x), rn_mul(e1x, e2z));
        float nz = rn_sub(rn_mul(e1x, e2y), rn_mul(e1y, e2x));
        const float len = __fsqrt_rn(rn_add(rn_add(rn_mul(nx, nx), rn_mul(ny, ny)), rn_mul(nz, nz)));
        nx = rn_div(nx, len);
        ny = rn_div(ny, len);
        nz = rn_div(nz, len);
        if (rn_add(rn_add(rn_mul(nx, dx), rn_mul(ny, dy)), rn_mul(nz, dz)) > 0.0f) {
            nx = -nx;
            ny = -ny;
            nz = -nz;
        }
        out.nx[g] = nx;
        out.ny[g] = ny;
        out.nz[g] = nz;
        out.material[g] = tri_material[tri];
        out.hit[g] = 1;
    }
}

crsh_status gbuffer_from_hits_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_hits* hits,
                                     const crsh_scene* sc, const uint32_t* tri_material, crsh_gbuffer_out* out,
                                     cudaStream_t s, const DeviceInfo& dev) {
    const unsigned blocks = (rays->capacity + 255) / 256;
    const unsigned grid = blocks < (unsigned)dev.sms * 8 ? (blocks ? blocks : 1) : dev.sms * 8;
    k_gbuffer<<<grid, 256, 0, s>>>(*rays, n_rays, *hits, *sc, tri_material, *out);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

// Mesh of triangle t: the last m with first[m] <= t.
__device__ __forceinline__ unsigned mesh_of(const uint32_t* first, unsigned n_meshes, unsigned t) {
    unsigned lo = 0, hi = n_meshes - 1;
    while (lo < hi) {
        const unsigned mid = (lo + hi + 1) >> 1;
        if (first[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void affine(const float* A, float x, float y, float z, float& ox, float& oy, float& oz) {
    ox = fmaf(A[0], x, fmaf(A[1], y, fmaf(A[2], z, A[3])));
    oy = fmaf(A[4], x, fmaf(A[5], y, fmaf(A[6], z, A[7])));
    oz = fmaf(A[8], x, fmaf(A[9], y, fmaf(A[10], z, A[11])));
}

__global__ void k_transform(crsh_scene in, const float* xf, crsh_scene_out out) {
    const unsigned stride = gridDim.x * blockDim.x;
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned t = tid; t < in.n_tris; t += stride) {
        const float* A = xf + 12 * (size_t)mesh_of(in.mesh_first_tri, in.n_meshes, t);
        float x, y, z;
        affine(A, in.v0x[t], in.v0y[t], in.v0z[t], x, y, z);
        out.v0x[t] = x; out.v0y[t] = y; out.v0z[t] = z;
        affine(A, in.v1x[t], in.v1y[t], in.v1z[t], x, y, z);
        out.v1x[t] = x; out.v1y[t] = y; out.v1z[t] = z;
        affine(A, in.v2x[t], in.v2y[t], in.v2z[t], x, y, z);
        out.v2x[t] = x; out.v2y[t] = y; out.v2z[t] = z;
    }
    for (unsigned m = tid; m < in.n_meshes; m += stride) {
        const float* A = xf + 12 * (size_t)m;
        const float4 sp = reinterpret_cast<const float4*>(in.mesh_sphere)[m];
        float x, y, z;
        affine(A, sp.x, sp.y, sp.z, x, y, z);
        float f2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 12; ++k)
            if ((k & 3) != 3) f2 = fmaf(A[k], A[k], f2);
        // Frobenius norm >= the largest stretch; a few ulps up for the rounding
        // of the norm, the product and the moved centre
        const float r = sp.w * sqrtf(f2) * (1.0f + 4.8e-7f) +
                        3.9e-6f * (fabsf(x) + fabsf(y) + fabsf(z));
        reinterpret_cast<float4*>(out.mesh_sphere)[m] = make_float4(x, y, z, r);
    }
}

crsh_status transform_launch(const crsh_scene* in, const float* xf, crsh_scene_out* out, cudaStream_t s,
                             const DeviceInfo& dev) {
    const unsigned n = in->n_tris > in->n_meshes ? in->n_tris : in->n_meshes;
    const unsigned blocks = (n + 255) / 256;
    const unsigned grid = blocks < (unsigned)dev.sms * 8 ? (blocks ? blocks : 1) : dev.sms * 8;
    k_transform<<<grid, 256, 0, s>>>(*in, xf, *out);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

}  // namespace crsh
