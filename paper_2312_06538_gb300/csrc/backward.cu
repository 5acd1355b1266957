// Gradients of the closest hit (not a step of the paper: the adjoint of the
// final test of Section 3.3.8 with the hit assignment held fixed).
//
// With A = [-d | e1 | e2] and an upstream gradient g = dL/d(t, u, v), the
// implicit-function theorem on o + t d = V0 + u e1 + v e2 gives
//   lambda = A^-T g = (g_t n - g_u (e2 x d) - g_v (d x e1)) / D,
//   n = e1 x e2, D = -(d . n),
//   dL/do = lambda, dL/dd = t lambda,
//   dL/dV0 = -(1 - u - v) lambda, dL/dV1 = -u lambda, dL/dV2 = -v lambda.
//
// GB300 design, deterministic and atomics-free: hit rays are compacted in
// sorted-ray order into (triangle, ray) pairs and radix-sorted by triangle
// (stable); then one warp per tile of 1,024 sorted pairs computes lambda and
// the per-ray gradients, and reduces each triangle's contributions with a
// segmented warp scan in a fixed order.  Triangles inside a tile are written
// directly; a triangle whose run crosses tiles is finished by a second pass
// that adds the per-tile partial sums in tile order.  Identical inputs give
// identical bits.
#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

constexpr int BW_TILE = 1024;
constexpr unsigned KEY_END = 0xffffffffu;

// ---- 1. hit rays -> (triangle, sorted ray index), stable ------------------
constexpr int HC_BLOCK = 256, HC_ITEMS = 4, HC_TILE = HC_BLOCK * HC_ITEMS;
static_assert(HC_ITEMS * (HC_BLOCK / 32) == 32, "one warp scans the per-warp counts");

__global__ void __launch_bounds__(HC_BLOCK) k_bw_collect(const uint32_t* ray_id, const int32_t* hit_tri,
                                                         const unsigned* n_ptr, uint32_t* keys, uint32_t* vals,
                                                         unsigned* h_out, unsigned long long* status,
                                                         unsigned* tile_ctr, crsh_counters* ctr) {
    __shared__ unsigned s_tile;
    __shared__ unsigned s_cnt[HC_ITEMS][HC_BLOCK / 32];
    __shared__ unsigned long long s_prefix;
    const unsigned n = *n_ptr;
    const unsigned n_tiles = (n + HC_TILE - 1) / HC_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        const unsigned tile = next_tile(tile_ctr, &s_tile);
        if (tile >= n_tiles) break;
        bool f[HC_ITEMS];
        unsigned bal[HC_ITEMS], k[HC_ITEMS];
#pragma unroll
        for (int i = 0; i < HC_ITEMS; ++i) {
            const unsigned e = tile * HC_TILE + i * HC_BLOCK + threadIdx.x;
            f[i] = false;
            k[i] = 0;
            if (e < n) {
                const int t = hit_tri[ray_id[e]];
                f[i] = t >= 0;
                k[i] = (unsigned)t;
            }
            bal[i] = __ballot_sync(FULL, f[i]);
            if (lane == 0) s_cnt[i][warp] = __popc(bal[i]);
        }
        __syncthreads();
        if (warp == 0) {
            const unsigned v = s_cnt[lane / (HC_BLOCK / 32)][lane % (HC_BLOCK / 32)];
            const unsigned inc = warp_incl_scan(v);
            s_cnt[lane / (HC_BLOCK / 32)][lane % (HC_BLOCK / 32)] = inc - v;
            const unsigned total = __shfl_sync(FULL, inc, 31);
            const unsigned long long pre = lookback_warp(status, tile, total, ctr);
            if (lane == 0) {
                s_prefix = pre;
                if (tile == n_tiles - 1) *h_out = (unsigned)(pre + total);
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < HC_ITEMS; ++i) {
            if (f[i]) {
                const unsigned pos = (unsigned)s_prefix + s_cnt[i][warp] + __popc(bal[i] & lanemask_lt());
                keys[pos] = k[i];
                vals[pos] = tile * HC_TILE + i * HC_BLOCK + threadIdx.x;
            }
        }
    }
}

// ---- 2/3. per-ray gradients and per-triangle segmented sums ---------------
struct BwIn {
    const float *ox, *oy, *oz, *dx, *dy, *dz;   // sorted rays
    const uint32_t* ray_id;
    const int32_t* hit_tri;                       // generation order
    const float *t, *u, *v;
    const float *g_t, *g_u, *g_v;
    const float *v0x, *v0y, *v0z, *v1x, *v1y, *v1z, *v2x, *v2y, *v2z;
};

struct Owner {
    unsigned key, tile;
    float part[9];
};

struct BwOut {
    float* g_verts;   // 9 per triangle
    float* g_orig;    // 3 per ray, generation order
    float* g_dir;
    float* tail;      // 9 per tile: partial of the run that continues into the next tile
    Owner* owners;
    unsigned* n_owners;
};

// lambda and the three corner contributions of sorted ray i hitting triangle tri;
// also writes the ray's own gradients
__device__ __forceinline__ void ray_contrib(const BwIn& in, const BwOut& out, unsigned i, unsigned tri, float c[9]) {
    const unsigned gen = in.ray_id[i];
    const float dx = in.dx[i], dy = in.dy[i], dz = in.dz[i];
    const float ax = in.v0x[tri], ay = in.v0y[tri], az = in.v0z[tri];
    const float e1x = in.v1x[tri] - ax, e1y = in.v1y[tri] - ay, e1z = in.v1z[tri] - az;
    const float e2x = in.v2x[tri] - ax, e2y = in.v2y[tri] - ay, e2z = in.v2z[tri] - az;
    const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const float D = -(dx * nx + dy * ny + dz * nz);
    const float gt = in.g_t[gen], gu = in.g_u[gen], gv = in.g_v[gen];
    // e2 x d and d x e1
    const float ax2 = e2y * dz - e2z * dy, ay2 = e2z * dx - e2x * dz, az2 = e2x * dy - e2y * dx;
    const float bx = dy * e1z - dz * e1y, by = dz * e1x - dx * e1z, bz = dx * e1y - dy * e1x;
    const float inv = D != 0.0f ? 1.0f / D : 0.0f;
    const float lx = (gt * nx - gu * ax2 - gv * bx) * inv;
    const float ly = (gt * ny - gu * ay2 - gv * by) * inv;
    const float lz = (gt * nz - gu * az2 - gv * bz) * inv;
    const float t = in.t[gen], u = in.u[gen], v = in.v[gen];
    out.g_orig[3 * (size_t)gen + 0] = lx;
    out.g_orig[3 * (size_t)gen + 1] = ly;
    out.g_orig[3 * (size_t)gen + 2] = lz;
    out.g_dir[3 * (size_t)gen + 0] = t * lx;
    out.g_dir[3 * (size_t)gen + 1] = t * ly;
    out.g_dir[3 * (size_t)gen + 2] = t * lz;
    const float w0 = -(1.0f - u - v), w1 = -u, w2 = -v;
    c[0] = w0 * lx; c[1] = w0 * ly; c[2] = w0 * lz;
    c[3] = w1 * lx; c[4] = w1 * ly; c[5] = w1 * lz;
    c[6] = w2 * lx; c[7] = w2 * ly; c[8] = w2 * lz;
}

__device__ __forceinline__ unsigned lanemask_le_u(int lane) { return lane == 31 ? FULL : ((1u << (lane + 1)) - 1u); }

// One warp per tile of BW_TILE sorted pairs, 32 rounds of 32: segmented
// inclusive scan per round (fixed order), carried across rounds.
__global__ void __launch_bounds__(256) k_bw_tiles(BwIn in, const uint32_t* kA, const uint32_t* vA, const uint32_t* kB,
                                                  const uint32_t* vB, const unsigned* plan, const unsigned* h_ptr,
                                                  BwOut out) {
    const uint32_t* keys = plan[4] ? kB : kA;
    const uint32_t* vals = plan[4] ? vB : vA;
    const unsigned H = *h_ptr;
    const unsigned n_tiles = (H + BW_TILE - 1) / BW_TILE;
    const int lane = threadIdx.x & 31;
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (unsigned tile = gw; tile < n_tiles; tile += nw) {
        const unsigned base = tile * BW_TILE, end = min(base + BW_TILE, H);
        unsigned carry_key = base > 0 ? keys[base - 1] : KEY_END;
        bool carry_from_prev = true;   // the carried run began in an earlier tile
        float carry[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) carry[k] = 0.0f;
        for (unsigned r0 = base; r0 < end; r0 += 32) {
            const unsigned idx = r0 + lane;
            const bool valid = idx < end;
            const unsigned key = valid ? keys[idx] : KEY_END;
            const unsigned nkey = (valid && idx + 1 < H) ? keys[idx + 1] : KEY_END;
            float c[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) c[k] = 0.0f;
            if (valid) ray_contrib(in, out, vals[idx], key, c);
            unsigned prev = __shfl_up_sync(FULL, key, 1);
            if (lane == 0) prev = carry_key;
            const bool head = valid && key != prev;
            const unsigned hm = __ballot_sync(FULL, head);
            const unsigned le = hm & lanemask_le_u(lane);
            const int my_head = le ? 31 - __clz(le) : -1;
            const int lo = my_head < 0 ? 0 : my_head;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float x = __shfl_up_sync(FULL, c[k], off);
                    if (lane - off >= lo) c[k] += x;
                }
            }
            if (my_head < 0) {
#pragma unroll
                for (int k = 0; k < 9; ++k) c[k] += carry[k];
            }
            const bool before = my_head < 0 && carry_from_prev;
            if (valid && (nkey != key || idx + 1 == end)) {   // last pair of its run inside this tile
                if (nkey == key) {                              // the run goes on in the next tile
#pragma unroll
                    for (int k = 0; k < 9; ++k) out.tail[9 * (size_t)tile + k] = c[k];
                } else if (before) {                            // run began in an earlier tile
                    const unsigned o = atomicAdd(out.n_owners, 1u);
                    out.owners[o].key = key;
                    out.owners[o].tile = tile;
#pragma unroll
                    for (int k = 0; k < 9; ++k) out.owners[o].part[k] = c[k];
                } else {                                        // whole run inside this tile
#pragma unroll
                    for (int k = 0; k < 9; ++k) out.g_verts[9 * (size_t)key + k] = c[k];
                }
            }
            const int last = (int)min(31u, end - 1 - r0);
            carry_key = __shfl_sync(FULL, key, last);
#pragma unroll
            for (int k = 0; k < 9; ++k) carry[k] = __shfl_sync(FULL, c[k], last);
            if (hm & lanemask_le_u(last)) carry_from_prev = false;
        }
    }
}

// Runs that cross tiles: partial of every earlier tile (in tile order, strided
// over lanes then a fixed butterfly) plus the closing piece.
__global__ void k_bw_owners(const Owner* owners, const unsigned* n_owners, const uint32_t* kA, const uint32_t* kB,
                            const unsigned* plan, const unsigned* h_ptr, const float* tail, float* g_verts) {
    const uint32_t* keys = plan[4] ? kB : kA;
    const unsigned H = *h_ptr, n = *n_owners;
    const int lane = threadIdx.x & 31;
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (unsigned o = gw; o < n; o += nw) {
        const unsigned key = owners[o].key, tb = owners[o].tile;
        unsigned lo = 0, hi = H;   // first pair of this triangle
        while (lo < hi) {
            const unsigned mid = (lo + hi) >> 1;
            if (keys[mid] < key) lo = mid + 1; else hi = mid;
        }
        const unsigned ta = lo / BW_TILE;
        float s[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) s[k] = 0.0f;
        for (unsigned t = ta + lane; t < tb; t += 32)
#pragma unroll
            for (int k = 0; k < 9; ++k) s[k] += tail[9 * (size_t)t + k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < 9; ++k) s[k] += __shfl_xor_sync(FULL, s[k], off);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 9; ++k) g_verts[9 * (size_t)key + k] = s[k] + owners[o].part[k];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
struct Carve {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

struct BwWs {
    uint32_t *kA, *vA, *kB, *vB;
    float* tail;
    Owner* owners;
    char* ctl;
    size_t ctl_bytes;
    unsigned* h;           // hit rays
    unsigned* n_owners;
    unsigned* tile_ctr;    // [0] collect, [1..4] radix passes
    unsigned* hist;
    unsigned* offs;
    unsigned* plan;
    unsigned long long* st_collect;
    unsigned* st_radix;
    size_t total;
};

BwWs carve_bw(void* ws, uint32_t cap) {
    Carve c{reinterpret_cast<char*>(ws)};
    BwWs w{};
    const size_t tiles = ((size_t)cap + BW_TILE - 1) / BW_TILE + 1;
    w.kA = c.take<uint32_t>(cap);
    w.vA = c.take<uint32_t>(cap);
    w.kB = c.take<uint32_t>(cap);
    w.vB = c.take<uint32_t>(cap);
    w.tail = c.take<float>(9 * tiles);
    w.owners = c.take<Owner>(tiles);
    w.offs = c.take<unsigned>(1024);
    w.plan = c.take<unsigned>(8);
    c.off = (c.off + 255) & ~size_t(255);
    const size_t ctl0 = c.off;
    w.h = c.take<unsigned>(1);
    w.n_owners = c.take<unsigned>(1);
    w.tile_ctr = c.take<unsigned>(8);
    w.hist = c.take<unsigned>(1024);
    w.st_collect = c.take<unsigned long long>(((size_t)cap + HC_TILE - 1) / HC_TILE + 1);
    w.st_radix = c.take<unsigned>(radix_status_words(cap));
    w.ctl = ws ? reinterpret_cast<char*>(ws) + ctl0 : nullptr;
    w.ctl_bytes = c.off - ctl0;
    w.total = c.off + 256;
    return w;
}
}  // namespace

size_t backward_workspace(uint32_t cap) { return carve_bw(nullptr, cap).total; }

crsh_status backward_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_scene* sc, const crsh_hits* hits,
                            const float* g_t, const float* g_u, const float* g_v, float* g_verts, float* g_orig,
                            float* g_dir, crsh_counters* ctr, void* ws, size_t ws_bytes, cudaStream_t s,
                            const DeviceInfo& dev) {
    const uint32_t cap = rays->capacity;
    if (ws_bytes < backward_workspace(cap)) return CRSH_ERR_INVALID_ARG;
    BwWs w = carve_bw(ws, cap);
    if (cudaMemsetAsync(w.ctl, 0, w.ctl_bytes, s) != cudaSuccess) return CRSH_ERR_CUDA;
    if (cudaMemsetAsync(g_verts, 0, sizeof(float) * 9 * (size_t)sc->n_tris, s) != cudaSuccess) return CRSH_ERR_CUDA;
    if (cudaMemsetAsync(g_orig, 0, sizeof(float) * 3 * (size_t)cap, s) != cudaSuccess) return CRSH_ERR_CUDA;
    if (cudaMemsetAsync(g_dir, 0, sizeof(float) * 3 * (size_t)cap, s) != cudaSuccess) return CRSH_ERR_CUDA;
    const unsigned persist = dev.sms * 8;
    {
        const unsigned tiles = (cap + HC_TILE - 1) / HC_TILE;
        const unsigned grid = tiles < persist ? (tiles ? tiles : 1) : persist;
        k_bw_collect<<<grid, HC_BLOCK, 0, s>>>(rays->ray_id, hits->tri, n_rays, w.kA, w.vA, w.h, w.st_collect,
                                               &w.tile_ctr[0], ctr);
    }
    RadixWs rw{w.hist, w.offs, w.plan, &w.tile_ctr[1], w.st_radix};
    radix_sort_launch(w.kA, w.vA, w.kB, w.vB, w.h, cap, rw, ctr, s, dev);
    BwIn in{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz, rays->ray_id, hits->tri, hits->t, hits->u,
            hits->v, g_t, g_u, g_v, sc->v0x, sc->v0y, sc->v0z, sc->v1x, sc->v1y, sc->v1z, sc->v2x, sc->v2y, sc->v2z};
    BwOut out{g_verts, g_orig, g_dir, w.tail, w.owners, w.n_owners};
    k_bw_tiles<<<dev.sms * 8, 256, 0, s>>>(in, w.kA, w.vA, w.kB, w.vB, w.plan, w.h, out);
    k_bw_owners<<<dev.sms * 2, 256, 0, s>>>(w.owners, w.n_owners, w.kA, w.kB, w.plan, w.h, w.tail, g_verts);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

}  // namespace crsh
