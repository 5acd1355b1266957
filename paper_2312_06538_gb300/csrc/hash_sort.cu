// Section 3.3.2-3.3.5: secondary ray generation, per-type hashing, trimming,
// compression into chunks, radix sort of the chunks, decompression.
//
// GB300 design: one kernel over the G-buffer generates, hashes and trims
// (each tile counts its pixels' rays, then writes them at the scanned
// position: stable compaction by decoupled look-back); compression is one
// more compaction over the keys; the sort is a one-sweep LSD radix sort
// (8-bit digits, one kernel per digit, digits that are the same for every key
// skipped on the device) with stable per-warp multisplit ranking, whose first
// pass makes the sort values (generation or chunk indices) instead of reading
// them; decompression and the gather of the sorted rays are one kernel.
// Sizes stay on the device: every kernel runs a persistent grid and reads the
// count it works on; each is launched with programmatic dependent launch and
// waits on its predecessor before its first access.
#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

// ---------------------------------------------------------------------------
// FP32 ray generation with a fixed operation order (no contraction): the keys
// derived from these rays are integers, decided in the paper's 32-bit
// precision, and must not depend on how a compiler fuses operations.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float len3_rn(float x, float y, float z) {
    return __fsqrt_rn(fa(fa(fm(x, x), fm(y, y)), fm(z, z)));
}

struct GenRay {
    float o[3], d[3], tmax;
    uint8_t type, light;
};

// Tables: theta thresholds cos(k pi / 2^tb) and phi thresholds
// tan(j (pi/4) / M), M = 2^pb / 8, rounded to FP32 (k_tables).
struct HashDev {
    const float* cosS;  // 2^stb entries
    const float* tanS;  // 2^spb / 8 entries
    const float* cosR;
    const float* tanR;
    float lo[3], scale[3];   // origin-cell box and 2^cb / (hi - lo) per axis
    unsigned stb, spb, cb, tb, pb;
};

// #{k in [1, B-1] : dz < T[k]}, T non-increasing: the largest such k (or 0).
// Start from an approximate bin and move until the exact table condition holds.
__device__ __forceinline__ unsigned theta_bin(float dz, const float* T, unsigned bits) {
    const unsigned B = 1u << bits;
    int b;
    if (!(dz < 1.0f)) b = 0;
    else if (!(dz > -1.0f)) b = (int)B - 1;
    else b = (int)(acosf(dz) * ((float)B / PI_F));
    b = min(max(b, 0), (int)B - 1);
    while (b < (int)B - 1 && dz < __ldg(&T[b + 1])) ++b;
    while (b > 0 && !(dz < __ldg(&T[b]))) --b;
    return (unsigned)b;
}

// #{j in [1, M-1] : r >= T[j]} (strict = false) or r > T[j] (strict = true);
// T increasing.
__device__ __forceinline__ unsigned tan_count(float r, const float* T, unsigned M, bool strict) {
    int j = (int)(atanf(r) * ((float)(4 * M) / PI_F));
    j = min(max(j, 0), (int)M - 1);
    auto ok = [&](int k) { float t = __ldg(&T[k]); return strict ? (r > t) : (r >= t); };
    while (j < (int)M - 1 && ok(j + 1)) ++j;
    while (j > 0 && !ok(j)) --j;
    return (unsigned)j;
}

__device__ __forceinline__ unsigned phi_bin(float x, float y, const float* T, unsigned bits) {
    const unsigned Bp = 1u << bits, M = Bp / 8, Q = Bp / 4;
    unsigned q;
    float a, b;
    if (x > 0.0f && y >= 0.0f) { q = 0; a = x; b = y; }
    else if (x <= 0.0f && y > 0.0f) { q = 1; a = y; b = -x; }
    else if (x < 0.0f && y <= 0.0f) { q = 2; a = -x; b = -y; }
    else if (x >= 0.0f && y < 0.0f) { q = 3; a = -y; b = x; }
    else return 0;
    unsigned psi;
    if (b < a) psi = tan_count(fd(b, a), T, M, false);
    else psi = 2 * M - 1 - tan_count(fd(a, b), T, M, true);
    return q * Q + psi;
}

// bit b of x -> bit 2b (x < 2^16)
__device__ __forceinline__ unsigned spread2(unsigned x) {
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// bit b of x -> bit 3b (x < 2^10)
__device__ __forceinline__ unsigned spread3(unsigned x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// Z-order code of the (theta, phi) bins: the low min(tb, pb) bits of both
// interleaved (phi bit b at 2b, theta bit b at 2b + 1), the longer bin's
// remaining bits above them.
__device__ __forceinline__ unsigned interleave2(unsigned th, unsigned tb, unsigned ph, unsigned pb) {
    const unsigned common = min(tb, pb), m = (1u << common) - 1u;
    return spread2(ph & m) | (spread2(th & m) << 1) | ((ph >> common) << (2 * common)) |
           ((th >> common) << (2 * common));
}

// scale = fl(2^bits / fl(hi - lo)), computed once per call on the host (IEEE
// single precision there too, so the same bits)
__device__ __forceinline__ unsigned cell_coord(float o, float lo, float scale, unsigned bits) {
    const float cells = (float)(1u << bits);
    float q = floorf(fm(fs(o, lo), scale));
    if (!(q >= 0.0f)) return 0;
    if (q > cells - 1.0f) return (1u << bits) - 1;
    return (unsigned)q;
}

// Morton code of a cell (coordinates below 2^bits, bits <= 10)
__device__ __forceinline__ unsigned morton3(unsigned x, unsigned y, unsigned z, unsigned) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

__device__ __forceinline__ unsigned ray_key(const GenRay& r, const HashDev& h) {
    if (r.type == CRSH_RAY_SHADOW) {
        unsigned th = theta_bin(r.d[2], h.cosS, h.stb);
        unsigned ph = phi_bin(r.d[0], r.d[1], h.tanS, h.spb);
        return ((unsigned)r.light << (h.stb + h.spb)) | interleave2(th, h.stb, ph, h.spb);
    }
    unsigned th = theta_bin(r.d[2], h.cosR, h.tb);
    unsigned ph = phi_bin(r.d[0], r.d[1], h.tanR, h.pb);
    unsigned cell = morton3(cell_coord(r.o[0], h.lo[0], h.scale[0], h.cb), cell_coord(r.o[1], h.lo[1], h.scale[1], h.cb),
                            cell_coord(r.o[2], h.lo[2], h.scale[2], h.cb), h.cb);
    return ((unsigned)r.type << 30) | (cell << (h.tb + h.pb)) | interleave2(th, h.tb, ph, h.pb);
}

// Generates the rays of one pixel in slot order; calls emit(ray) for each
// existing ray.  Returns the count.  Mirrors the paper's ray types
// (Section 3.3.2) with the origin of shadow rays inverted to the light.
template <class Emit>
__device__ __forceinline__ unsigned pixel_rays(const crsh_gbuffer& g, unsigned p, const float* lights,
                                               unsigned n_lights, bool cull, Emit emit) {
    if (!g.hit[p]) return 0;
    const float P0 = g.px[p], P1 = g.py[p], P2 = g.pz[p];
    const float N0 = g.nx[p], N1 = g.ny[p], N2 = g.nz[p];
    const float I0 = g.ix[p], I1 = g.iy[p], I2 = g.iz[p];
    unsigned cnt = 0;
    for (unsigned k = 0; k < n_lights; ++k) {
        const float L0 = __ldg(&lights[3 * k]), L1 = __ldg(&lights[3 * k + 1]), L2 = __ldg(&lights[3 * k + 2]);
        const float v0 = fs(P0, L0), v1 = fs(P1, L1), v2 = fs(P2, L2);
        float facing = fa(fa(fm(N0, v0), fm(N1, v1)), fm(N2, v2));
        if (cull && !(facing < 0.0f)) continue;
        float len = len3_rn(v0, v1, v2);
        if (!(len > 0.0f)) continue;
        GenRay r;
        r.o[0] = L0; r.o[1] = L1; r.o[2] = L2;
        r.d[0] = fd(v0, len); r.d[1] = fd(v1, len); r.d[2] = fd(v2, len);
        r.tmax = fm(len, 0.9999f);
        r.type = CRSH_RAY_SHADOW;
        r.light = (uint8_t)k;
        emit(r);
        ++cnt;
    }
    const unsigned m = g.material[p];
    if (m != CRSH_MAT_MIRROR && m != CRSH_MAT_GLASS) return cnt;
    const float c = fa(fa(fm(I0, N0), fm(I1, N1)), fm(I2, N2));
    const float off = (c > 0.0f) ? -1e-4f : 1e-4f;
    {
        const float two_c = fm(2.0f, c);
        const float r0 = fs(I0, fm(two_c, N0)), r1 = fs(I1, fm(two_c, N1)), r2 = fs(I2, fm(two_c, N2));
        const float rl = len3_rn(r0, r1, r2);
        GenRay r;
        r.o[0] = fa(P0, fm(off, N0)); r.o[1] = fa(P1, fm(off, N1)); r.o[2] = fa(P2, fm(off, N2));
        r.d[0] = fd(r0, rl); r.d[1] = fd(r1, rl); r.d[2] = fd(r2, rl);
        r.tmax = __int_as_float(0x7f800000);
        r.type = CRSH_RAY_REFLECTION;
        r.light = 0;
        emit(r);
        ++cnt;
    }
    if (m == CRSH_MAT_GLASS) {
        const float ior = 1.5f;
        float eta, cosi, M0, M1, M2;
        if (c < 0.0f) { eta = fd(1.0f, ior); cosi = -c; M0 = N0; M1 = N1; M2 = N2; }
        else { eta = ior; cosi = c; M0 = -N0; M1 = -N1; M2 = -N2; }
        const float sin2 = fs(1.0f, fm(cosi, cosi));
        const float k = fs(1.0f, fm(fm(eta, eta), sin2));
        if (!(k < 0.0f)) {
            const float coef = fs(fm(eta, cosi), __fsqrt_rn(k));
            const float t0 = fa(fm(eta, I0), fm(coef, M0));
            const float t1 = fa(fm(eta, I1), fm(coef, M1));
            const float t2 = fa(fm(eta, I2), fm(coef, M2));
            const float tl = len3_rn(t0, t1, t2);
            GenRay r;
            r.o[0] = fs(P0, fm(off, N0)); r.o[1] = fs(P1, fm(off, N1)); r.o[2] = fs(P2, fm(off, N2));
            r.d[0] = fd(t0, tl); r.d[1] = fd(t1, tl); r.d[2] = fd(t2, tl);
            r.tmax = __int_as_float(0x7f800000);
            r.type = CRSH_RAY_REFRACTION;
            r.light = 0;
            emit(r);
            ++cnt;
        }
    }
    return cnt;
}

// Rays in generation order: one 32-byte record per ray, (ox, oy, oz, dx) and
// (dy, dz, t_max, pixel bits), so the gather after the sort reads each ray as
// one aligned 32-byte sector.  The type is not stored: it is the key's top
// two bits (Section 3.3.2 layout).
struct GenOut {
    float4* rec;     // 2 per ray
    uint32_t* key;   // generation-order keys
    uint32_t* val;   // sort values: written by the radix passes only (the generation index is implicit)
    uint32_t capacity;
};

__device__ __forceinline__ void store_ray(const GenOut& o, unsigned pos, const GenRay& r, unsigned key,
                                          unsigned pixel) {
    o.rec[2 * (size_t)pos] = make_float4(r.o[0], r.o[1], r.o[2], r.d[0]);
    o.rec[2 * (size_t)pos + 1] = make_float4(r.d[1], r.d[2], r.tmax, __uint_as_float(pixel));
    o.key[pos] = key;
}

constexpr int GEN_BLOCK = 256;

// GEN_SUB striped sub-tiles of GEN_BLOCK pixels per look-back tile (one pixel
// per thread and sub-tile, so the G-buffer loads stay coalesced; a blocked
// layout of several consecutive pixels per thread measured slower, and so did
// four sub-tiles, at 77 registers); stable trimming of empty slots by a block
// scan of the per-thread ray counts plus decoupled look-back across tiles.
constexpr int GEN_SUB = 2, GEN_TILE = GEN_BLOCK * GEN_SUB;
constexpr int GEN_NC = GEN_SUB * (GEN_BLOCK / 32);   // (sub-tile, warp) counts, scanned by one warp
constexpr int GEN_PER = (GEN_NC + 31) / 32;           // per lane

__global__ void __launch_bounds__(GEN_BLOCK) k_gen_gbuffer(crsh_gbuffer g, const float* lights, unsigned n_lights,
                                                           int cull, HashDev h, GenOut out, unsigned* n_out,
                                                           unsigned long long* status, unsigned* tile_ctr,
                                                           crsh_counters* ctr) {
    pdl_wait();
    __shared__ unsigned s_tile;
    __shared__ unsigned s_cnt[GEN_SUB][GEN_BLOCK / 32];
    __shared__ unsigned long long s_prefix;
    const unsigned n_tiles = (g.n_pixels + GEN_TILE - 1) / GEN_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        const unsigned tile = next_tile(tile_ctr, &s_tile);
        if (tile >= n_tiles) break;
        const unsigned p0 = tile * GEN_TILE + threadIdx.x;
        unsigned cnt[GEN_SUB], inc[GEN_SUB];
#pragma unroll
        for (int j = 0; j < GEN_SUB; ++j) {
            const unsigned p = p0 + j * GEN_BLOCK;
            cnt[j] = p < g.n_pixels ? pixel_rays(g, p, lights, n_lights, cull != 0, [](const GenRay&) {}) : 0u;
            inc[j] = warp_incl_scan(cnt[j]);
            if (lane == 31) s_cnt[j][warp] = inc[j];
        }
        __syncthreads();
        if (warp == 0) {
            // scan the (sub-tile, warp) totals in pixel order, GEN_PER per lane
            unsigned* flat = &s_cnt[0][0];
            unsigned v[GEN_PER], sum = 0;
#pragma unroll
            for (int j = 0; j < GEN_PER; ++j) {
                v[j] = (lane * GEN_PER + j < GEN_NC) ? flat[lane * GEN_PER + j] : 0u;
                sum += v[j];
            }
            const unsigned wi = warp_incl_scan(sum);
            unsigned run = wi - sum;
#pragma unroll
            for (int j = 0; j < GEN_PER; ++j) {
                if (lane * GEN_PER + j < GEN_NC) flat[lane * GEN_PER + j] = run;
                run += v[j];
            }
            const unsigned total = __shfl_sync(FULL, wi, 31);
            const unsigned long long pre = lookback_warp(status, tile, total, ctr);
            if (lane == 0) {
                s_prefix = pre;
                if (tile == n_tiles - 1) {
                    const unsigned long long all = pre + total;
                    ctr->rays = all;
                    *n_out = (unsigned)min(all, (unsigned long long)out.capacity);
                    if (all > out.capacity) set_status(ctr, CRSH_ERR_CAPACITY);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < GEN_SUB; ++j) {
            if (!cnt[j]) continue;
            const unsigned p = p0 + j * GEN_BLOCK;
            unsigned long long pos = s_prefix + s_cnt[j][warp] + inc[j] - cnt[j];
            pixel_rays(g, p, lights, n_lights, cull != 0, [&](const GenRay& r) {
                if (pos < out.capacity) store_ray(out, (unsigned)pos, r, ray_key(r, h), p);
                ++pos;
            });
        }
    }
}

// Prebuilt rays: hash and copy (every input is a ray, order kept).
__global__ void k_gen_rays(crsh_rays_in in, HashDev h, GenOut out, unsigned* n_out, crsh_counters* ctr) {
    pdl_wait();
    const unsigned n = min(in.n, out.capacity);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->rays = in.n;
        *n_out = n;
        if (in.n > out.capacity) set_status(ctr, CRSH_ERR_CAPACITY);
    }
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        GenRay r;
        r.o[0] = in.ox[i]; r.o[1] = in.oy[i]; r.o[2] = in.oz[i];
        r.d[0] = in.dx[i]; r.d[1] = in.dy[i]; r.d[2] = in.dz[i];
        r.tmax = in.tmax[i];
        r.type = in.type[i];
        r.light = in.light ? in.light[i] : 0;
        if (r.type > CRSH_RAY_REFRACTION ||
            (r.type == CRSH_RAY_SHADOW && (unsigned)r.light >= (1u << (30 - h.stb - h.spb)))) {
            set_status(ctr, CRSH_ERR_BAD_INPUT);
            r.type = CRSH_RAY_REFLECTION;
        }
        store_ray(out, i, r, ray_key(r, h), i);
    }
}

// Zeroing of the ranges of a ZeroSpans: 16-byte stores over each range's
// aligned middle, 4-byte stores at its ends.
__global__ void k_zero(ZeroSpans z) {
    pdl_wait();
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        char* p = static_cast<char*>(z.p[r]);
        const size_t n = p ? z.bytes[r] : 0;
        const size_t head = min(n, (size_t)((16u - ((uintptr_t)p & 15u)) & 15u));
        const size_t n16 = (n - head) / 16, tail = head + 16 * n16;
        for (size_t i = tid; i < head / 4; i += nt) reinterpret_cast<unsigned*>(p)[i] = 0u;
        for (size_t i = tid; i < n16; i += nt) reinterpret_cast<uint4*>(p + head)[i] = make_uint4(0u, 0u, 0u, 0u);
        for (size_t i = tid; i < (n - tail) / 4; i += nt) reinterpret_cast<unsigned*>(p + tail)[i] = 0u;
    }
}

void zero_launch(const ZeroSpans& z, cudaStream_t s, const DeviceInfo& dev) {
    launch_pdl(k_zero, dev.sms * 4, 256, 0, s, z);
}

// Threshold tables of the bins: cos(k pi / B) for k < B and tan(j (pi/4) / M)
// for j < M, each evaluated in FP64 from the same FP64 argument expression as
// the definition and rounded to FP32; one thread per entry.
__global__ void k_tables(TableSpec t) {
    pdl_wait();
    const double pi = 3.14159265358979323846;
    unsigned total = 0;
    for (int i = 0; i < 4; ++i) total += t.n[i];
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        unsigned i = 0, k = e;
        while (k >= t.n[i]) k -= t.n[i++];
        t.dst[i][k] = t.is_tan[i] ? (float)tan((double)k * (pi / 4.0) / (double)t.n[i])
                                  : (float)cos((double)k * pi / (double)t.n[i]);
    }
}

void tables_launch(const TableSpec& t, cudaStream_t s, const DeviceInfo& dev) {
    const unsigned total = t.n[0] + t.n[1] + t.n[2] + t.n[3];
    const unsigned blocks = (total + 255) / 256;
    const unsigned grid = blocks < (unsigned)dev.sms ? (blocks ? blocks : 1) : dev.sms;
    launch_pdl(k_tables, grid, 256, 0, s, t);
}

// ---------------------------------------------------------------------------
// Section 3.3.3: compression.  Head flag where the key differs from the
// previous one; a stable compaction of the heads gives chunk key and base.
// The same pass counts the chunk keys' digits for the radix sort (hist: 4 x
// 256, zeroed); the top byte, which holds the ray type and few distinct
// values, is aggregated per warp before its atomic.
// ---------------------------------------------------------------------------
// 16 striped items per thread: 4096 keys per look-back tile (18 % faster than
// 1024-key tiles at 12.8 M keys)
constexpr int CMP_BLOCK = 256, CMP_ITEMS = 16, CMP_TILE = CMP_BLOCK * CMP_ITEMS;
constexpr int CMP_PER = CMP_ITEMS * (CMP_BLOCK / 32) / 32;   // (item, warp) counts per lane of the scan

__device__ __forceinline__ void count_digits(unsigned (*s_h)[256], unsigned k, bool valid) {
    if (valid) {
        atomicAdd(&s_h[0][k & 255u], 1u);
        atomicAdd(&s_h[1][(k >> 8) & 255u], 1u);
        atomicAdd(&s_h[2][(k >> 16) & 255u], 1u);
    }
    const unsigned d3 = valid ? (k >> 24) : 256u;
    const unsigned peers = __match_any_sync(FULL, d3);
    if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&s_h[3][d3], (unsigned)__popc(peers));
}

__global__ void __launch_bounds__(CMP_BLOCK) k_chunk(const uint32_t* key, const unsigned* n_ptr, uint32_t* ckey,
                                                     uint32_t* cbase, unsigned* c_out,
                                                     unsigned* hist, unsigned long long* status, unsigned* tile_ctr,
                                                     crsh_counters* ctr) {
    pdl_wait();
    __shared__ unsigned s_tile;
    __shared__ unsigned s_cnt[CMP_ITEMS][CMP_BLOCK / 32];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned s_h[4][256];
    for (int i = threadIdx.x; i < 1024; i += CMP_BLOCK) (&s_h[0][0])[i] = 0;
    const unsigned n = *n_ptr;
    const unsigned n_tiles = (n + CMP_TILE - 1) / CMP_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        *c_out = 0;
        cbase[0] = 0;
        ctr->chunks = 0;
    }
    for (;;) {
        const unsigned tile = next_tile(tile_ctr, &s_tile);
        if (tile >= n_tiles) break;
        bool f[CMP_ITEMS];
        unsigned bal[CMP_ITEMS];
        unsigned k[CMP_ITEMS];
#pragma unroll
        for (int i = 0; i < CMP_ITEMS; ++i) {
            unsigned e = tile * CMP_TILE + i * CMP_BLOCK + threadIdx.x;
            f[i] = false;
            if (e < n) {
                k[i] = key[e];
                f[i] = (e == 0) || (key[e - 1] != k[i]);
            }
            bal[i] = __ballot_sync(FULL, f[i]);
            if (lane == 0) s_cnt[i][warp] = __popc(bal[i]);
        }
        __syncthreads();
        if (warp == 0) {
            // scan the (item, warp) counts in element order, CMP_PER per lane
            unsigned* flat = &s_cnt[0][0];
            unsigned v[CMP_PER], sum = 0;
#pragma unroll
            for (int j = 0; j < CMP_PER; ++j) {
                v[j] = flat[lane * CMP_PER + j];
                sum += v[j];
            }
            const unsigned inc = warp_incl_scan(sum);
            unsigned run = inc - sum;
#pragma unroll
            for (int j = 0; j < CMP_PER; ++j) {
                flat[lane * CMP_PER + j] = run;
                run += v[j];
            }
            unsigned total = __shfl_sync(FULL, inc, 31);
            unsigned long long pre = lookback_warp(status, tile, total, ctr);
            if (lane == 0) {
                s_prefix = pre;
                if (tile == n_tiles - 1) {
                    unsigned all = (unsigned)(pre + total);
                    *c_out = all;
                    cbase[all] = n;
                    ctr->chunks = all;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < CMP_ITEMS; ++i) {
            if (f[i]) {
                unsigned pos = (unsigned)s_prefix + s_cnt[i][warp] + __popc(bal[i] & lanemask_lt());
                unsigned e = tile * CMP_TILE + i * CMP_BLOCK + threadIdx.x;
                ckey[pos] = k[i];
                cbase[pos] = e;
            }
            count_digits(s_h, f[i] ? k[i] : 0u, f[i]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += CMP_BLOCK) {
        const unsigned v = (&s_h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}
static_assert(CMP_PER * 32 == CMP_ITEMS * (CMP_BLOCK / 32), "one warp scans the per-warp counts");

// ---------------------------------------------------------------------------
// Section 3.3.4: radix sort (LSD, 8-bit digits, one sweep per digit).
// ---------------------------------------------------------------------------
constexpr int RS_BLOCK = 256, RS_WARPS = RS_BLOCK / 32, RS_KPT = 16, RS_TILE = RS_BLOCK * RS_KPT;

__global__ void k_radix_hist(const uint32_t* key, const unsigned* n_ptr, unsigned* hist /* 4 x 256 */) {
    pdl_wait();
    __shared__ unsigned s_h[4][256];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const unsigned n = *n_ptr;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned k = key[i];
        atomicAdd(&s_h[0][k & 255], 1u);
        atomicAdd(&s_h[1][(k >> 8) & 255], 1u);
        atomicAdd(&s_h[2][(k >> 16) & 255], 1u);
        atomicAdd(&s_h[3][k >> 24], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        unsigned v = (&s_h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// plan[p]: 0 = pass skipped (one digit holds every key), else 1 + source
// buffer (0 = A, 1 = B); plan[4] = buffer holding the sorted result.
// offs[p][d] = keys with a smaller digit d at pass p.
__global__ void k_radix_plan(const unsigned* hist, const unsigned* n_ptr, unsigned* offs, unsigned* plan,
                             int sort_enabled, int identity) {
    pdl_wait();
    __shared__ unsigned s_triv[4];
    const unsigned n = *n_ptr;
    const int d = threadIdx.x;   // 256 threads
    if (d < 4) s_triv[d] = 0;
    __syncthreads();
    for (int p = 0; p < 4; ++p) {
        unsigned v = hist[p * 256 + d];
        if (v == n) s_triv[p] = 1;   // includes n == 0
        // exclusive scan over 256 digits
        __shared__ unsigned s_w[8];
        unsigned inc = warp_incl_scan(v);
        if ((d & 31) == 31) s_w[d >> 5] = inc;
        __syncthreads();
        unsigned wpre = 0;
        for (int w = 0; w < (d >> 5); ++w) wpre += s_w[w];
        offs[p * 256 + d] = wpre + inc - v;
        __syncthreads();
    }
    if (d == 0) {
        unsigned cur = 0;
        for (int p = 0; p < 4; ++p) {
            if (!sort_enabled || s_triv[p]) plan[p] = 0;
            else { plan[p] = 1 + cur; cur ^= 1u; }
        }
        // identity values exist only inside the first pass: keep one
        if (sort_enabled && identity && cur == 0 && plan[0] == 0 && plan[1] == 0 && plan[2] == 0 && plan[3] == 0) {
            plan[0] = 1;
            cur = 1;
        }
        plan[4] = cur;
    }
}

// One LSD pass (8-bit digit) over tiles of RS_TILE keys taken in order from a
// counter.  A tile is ranked in registers (per-warp match of equal digits,
// counts in the warp's shared histogram, element order kept), its digit
// totals are published at once (decoupled look-back), then it is sorted by
// digit in shared memory while predecessors publish, and finally written out
// in that local order: consecutive threads write consecutive positions of one
// digit's run, so the stores are coalesced.
__device__ __forceinline__ void radix_pass_body(int pass, uint32_t* kA, uint32_t* vA, uint32_t* kB,
                                                uint32_t* vB, const unsigned* n_ptr, const unsigned* offs,
                                                const unsigned* plan, unsigned* status, unsigned* tile_ctr,
                                                crsh_counters* ctr, int identity) {
    pdl_wait();
    const unsigned pl = plan[pass];
    if (pl == 0) return;
    // identity values (element index) are made, not read, by the first pass that runs
    bool first = identity != 0;
    for (int q = 0; q < pass; ++q) first = first && plan[q] == 0;
    const uint32_t* sk = (pl == 1) ? kA : kB;
    const uint32_t* sv = (pl == 1) ? vA : vB;
    uint32_t* dk = (pl == 1) ? kB : kA;
    uint32_t* dv = (pl == 1) ? vB : vA;
    const unsigned shift = 8 * pass;
    __shared__ unsigned s_tile;
    __shared__ unsigned s_wh[RS_WARPS][256];   // per-warp digit counts, then their exclusive prefix over warps
    __shared__ unsigned s_loc[256];            // tile-local start of each digit
    __shared__ unsigned s_glob[256];           // global start of each digit minus its local start
    __shared__ unsigned s_wsum[RS_WARPS];
    __shared__ uint32_t s_key[RS_TILE];
    __shared__ uint32_t s_val[RS_TILE];
    const unsigned n = *n_ptr;
    const unsigned n_tiles = (n + RS_TILE - 1) / RS_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    for (;;) {
        const unsigned tile = next_tile(tile_ctr, &s_tile);
        if (tile >= n_tiles) break;
        for (int i = lane; i < 256; i += 32) s_wh[warp][i] = 0;
        __syncwarp();
        unsigned key[RS_KPT], val[RS_KPT], rank[RS_KPT];
        const unsigned t0 = tile * RS_TILE;
        const unsigned cnt = min((unsigned)RS_TILE, n - t0);
        const unsigned wbase = warp * (32 * RS_KPT);   // this warp's elements: wbase + r * 32 + lane
#pragma unroll
        for (int r = 0; r < RS_KPT; ++r) {
            const unsigned e = wbase + r * 32 + lane;
            const bool valid = e < cnt;
            key[r] = valid ? sk[t0 + e] : 0u;
            val[r] = valid ? (first ? t0 + e : sv[t0 + e]) : 0u;
        }
#pragma unroll
        for (int r = 0; r < RS_KPT; ++r) {
            const bool valid = wbase + r * 32 + lane < cnt;
            const unsigned d = valid ? ((key[r] >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(FULL, d);
            const unsigned pre = valid ? s_wh[warp][d] : 0u;
            rank[r] = pre + __popc(peers & lt);
            __syncwarp();
            if (valid && (peers & lt) == 0) s_wh[warp][d] = pre + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // thread = digit: prefix over warps, tile total published at once, then
        // the exclusive scan over digits gives each digit's local start
        const unsigned d = threadIdx.x;
        unsigned tot = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const unsigned c = s_wh[w][d];
            s_wh[w][d] = tot;
            tot += c;
        }
        lookback32_publish(status + d, tile, 256, tot);
        const unsigned inc = warp_incl_scan(tot);
        if (lane == 31) s_wsum[warp] = inc;
        __syncthreads();
        unsigned wpre = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) wpre += (w < warp) ? s_wsum[w] : 0u;
        const unsigned loc = wpre + inc - tot;
        s_loc[d] = loc;
        __syncthreads();
        // local sort by digit
#pragma unroll
        for (int r = 0; r < RS_KPT; ++r) {
            if (wbase + r * 32 + lane < cnt) {
                const unsigned dd = (key[r] >> shift) & 255u;
                const unsigned lp = s_loc[dd] + s_wh[warp][dd] + rank[r];
                s_key[lp] = key[r];
                s_val[lp] = val[r];
            }
        }
        // global starts (predecessors have had the ranking time to publish)
        const unsigned excl = lookback32_resolve(status + d, tile, 256, tot, ctr);
        s_glob[d] = offs[pass * 256 + d] + excl - loc;
        __syncthreads();
        for (unsigned i = threadIdx.x; i < cnt; i += RS_BLOCK) {
            const uint32_t k = s_key[i];
            const unsigned pos = s_glob[(k >> shift) & 255u] + i;
            dk[pos] = k;
            dv[pos] = s_val[i];
        }
    }
}
// Two entry points of the same pass: the unconstrained one (its register
// allocation measured best on small sorts, one block per SM) and one capped
// at three resident blocks per SM (80 registers, a few values spilled) for
// sorts of 16 M keys of capacity and more, 2 % faster at 51 M keys.
__global__ void __launch_bounds__(RS_BLOCK) k_radix_pass(int pass, uint32_t* kA, uint32_t* vA, uint32_t* kB,
                                                         uint32_t* vB, const unsigned* n_ptr, const unsigned* offs,
                                                         const unsigned* plan, unsigned* status,
                                                         unsigned* tile_ctr, crsh_counters* ctr, int identity) {
    radix_pass_body(pass, kA, vA, kB, vB, n_ptr, offs, plan, status, tile_ctr, ctr, identity);
}
__global__ void __launch_bounds__(RS_BLOCK, 3) k_radix_pass_3(int pass, uint32_t* kA, uint32_t* vA, uint32_t* kB,
                                                              uint32_t* vB, const unsigned* n_ptr,
                                                              const unsigned* offs, const unsigned* plan,
                                                              unsigned* status, unsigned* tile_ctr,
                                                              crsh_counters* ctr, int identity) {
    radix_pass_body(pass, kA, vA, kB, vB, n_ptr, offs, plan, status, tile_ctr, ctr, identity);
}
static_assert(RS_BLOCK == 256, "one thread per digit");

size_t radix_status_words(uint32_t cap) {
    const size_t rs_tiles = ((size_t)cap + RS_TILE - 1) / RS_TILE + 1;
    return 4 * rs_tiles * 256;
}

// Stable LSD sort of (kA, vA)[0 .. *cnt) by key, kB/vB as the other buffer.
// rw.hist, rw.tile_ctr (4) and rw.status must be zero; rw.plan[4] tells which
// buffer holds the result (0: A, 1: B).
void radix_sort_launch(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, const unsigned* cnt_ptr, uint32_t cap,
                       const RadixWs& rw, crsh_counters* ctr, cudaStream_t s, const DeviceInfo& dev, bool counted,
                       bool identity) {
    const unsigned cap_tiles = (cap + RS_TILE - 1) / RS_TILE;
    if (!counted) launch_pdl(k_radix_hist, dev.sms * 2, 256, 0, s, kA, cnt_ptr, rw.hist);
    launch_pdl(k_radix_plan, 1, 256, 0, s, rw.hist, cnt_ptr, rw.offs, rw.plan, 1, identity ? 1 : 0);
    const unsigned grid = cap_tiles < (unsigned)(dev.sms * 4) ? (cap_tiles ? cap_tiles : 1) : dev.sms * 4;
    const size_t rs_tiles = (size_t)cap_tiles + 1;
    const bool big = cap >= (1u << 24);
    for (int p = 0; p < 4; ++p) {
        unsigned* st = rw.status + (size_t)p * rs_tiles * 256;
        if (big)
            launch_pdl(k_radix_pass_3, grid, RS_BLOCK, 0, s, p, kA, vA, kB, vB, cnt_ptr, rw.offs, rw.plan, st,
                                                     &rw.tile_ctr[p], ctr, identity ? 1 : 0);
        else
            launch_pdl(k_radix_pass, grid, RS_BLOCK, 0, s, p, kA, vA, kB, vB, cnt_ptr, rw.offs, rw.plan, st,
                                                   &rw.tile_ctr[p], ctr, identity ? 1 : 0);
    }
}

struct SortedOut {
    float *ox, *oy, *oz, *dx, *dy, *dz, *tmax;
    uint8_t* type;
    uint32_t *ray_id, *pixel, *keys;
};

__device__ __forceinline__ void copy_ray(const GenOut& gen, unsigned src, const SortedOut& out, unsigned i,
                                         unsigned key) {
    const float4 a = gen.rec[2 * (size_t)src], b = gen.rec[2 * (size_t)src + 1];
    out.ox[i] = a.x; out.oy[i] = a.y; out.oz[i] = a.z;
    out.dx[i] = a.w; out.dy[i] = b.x; out.dz[i] = b.y;
    out.tmax[i] = b.z;
    out.type[i] = (uint8_t)(key >> 30);
    out.pixel[i] = __float_as_uint(b.w);
    out.ray_id[i] = src;
    out.keys[i] = key;
}

// ---------------------------------------------------------------------------
// Section 3.3.5: decompression.  Chunk sizes in sorted order, exclusive scan
// (the skeleton: the sorted position of each chunk's first ray), then every
// sorted position finds its chunk (k_gather).
// ---------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 256, SCAN_ITEMS = 16, SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_BLOCK) k_chunk_pos(const uint32_t* kA, const uint32_t* vA, const uint32_t* kB,
                                                          const uint32_t* vB, const unsigned* plan,
                                                          const uint32_t* cbase, const unsigned* c_ptr,
                                                          uint32_t* cpos, uint32_t* sbase,
                                                          unsigned long long* status, unsigned* tile_ctr,
                                                          crsh_counters* ctr) {
    pdl_wait();
    __shared__ unsigned s_tile;
    __shared__ unsigned s_warp[SCAN_BLOCK / 32];
    __shared__ unsigned long long s_prefix;
    const uint32_t* sv = plan[4] ? vB : vA;
    const unsigned C = *c_ptr;
    const unsigned n_tiles = (C + SCAN_TILE - 1) / SCAN_TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        const unsigned tile = next_tile(tile_ctr, &s_tile);
        if (tile >= n_tiles) break;
        // blocked: thread handles SCAN_ITEMS consecutive chunks (16-byte
        // loads and stores when all of them exist)
        const unsigned e0 = tile * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
        const bool full = e0 + SCAN_ITEMS <= C;
        unsigned sz[SCAN_ITEMS], cb[SCAN_ITEMS], cv[SCAN_ITEMS], sum = 0;
        if (full) {
#pragma unroll
            for (int i = 0; i < SCAN_ITEMS; i += 4) {
                const uint4 q = *reinterpret_cast<const uint4*>(sv + e0 + i);
                cv[i] = q.x; cv[i + 1] = q.y; cv[i + 2] = q.z; cv[i + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < SCAN_ITEMS; ++i) cv[i] = (e0 + i < C) ? sv[e0 + i] : 0xffffffffu;
        }
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            sz[i] = 0;
            cb[i] = 0;
            if (cv[i] != 0xffffffffu) {
                cb[i] = cbase[cv[i]];
                sz[i] = cbase[cv[i] + 1] - cb[i];
            }
            sum += sz[i];
        }
        unsigned inc = warp_incl_scan(sum);
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            unsigned w = lane < SCAN_BLOCK / 32 ? s_warp[lane] : 0;
            unsigned wi = warp_incl_scan(w);
            if (lane < SCAN_BLOCK / 32) s_warp[lane] = wi - w;
            unsigned total = __shfl_sync(FULL, wi, SCAN_BLOCK / 32 - 1);
            unsigned long long pre = lookback_warp(status, tile, total, ctr);
            if (lane == 0) s_prefix = pre;
        }
        __syncthreads();
        unsigned run = (unsigned)s_prefix + s_warp[warp] + inc - sum;
        unsigned rp[SCAN_ITEMS];
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            rp[i] = run;
            run += sz[i];
        }
        // sbase: generation index of the chunk's first ray, in sorted order
        if (full) {
#pragma unroll
            for (int i = 0; i < SCAN_ITEMS; i += 4) {
                *reinterpret_cast<uint4*>(cpos + e0 + i) = make_uint4(rp[i], rp[i + 1], rp[i + 2], rp[i + 3]);
                *reinterpret_cast<uint4*>(sbase + e0 + i) = make_uint4(cb[i], cb[i + 1], cb[i + 2], cb[i + 3]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < SCAN_ITEMS; ++i) {
                if (e0 + i < C) {
                    cpos[e0 + i] = rp[i];
                    sbase[e0 + i] = cb[i];
                }
            }
        }
    }
}

// mode 0: generation order; 1: sorted (value = ray index); 2: sorted chunks.
// Warps walk contiguous runs of 32-ray groups; in mode 2 the 32 rays of a
// group lie in at most 32 consecutive chunks from the chunk of its first ray
// (every chunk holds a ray), so lane l holds that window's start position l,
// each ray finds its chunk by a binary search over the lanes, and the next
// group starts from its first ray's chunk (the last ray's or the one after).
__global__ void k_gather(int mode, GenOut gen, const uint32_t* kA, const uint32_t* vA, const uint32_t* kB,
                         const uint32_t* vB, const unsigned* plan, const uint32_t* sbase, const uint32_t* cpos,
                         const unsigned* c_ptr, const unsigned* n_ptr, SortedOut out) {
    pdl_wait();
    const unsigned n = *n_ptr;
    const uint32_t* sv = (mode != 0 && plan[4]) ? vB : vA;
    const uint32_t* sk = (mode != 0 && plan[4]) ? kB : kA;
    if (mode != 2) {
        for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const unsigned src = mode == 0 ? i : sv[i];
            const unsigned key = mode == 0 ? gen.key[i] : sk[i];
            copy_ray(gen, src, out, i, key);
        }
        return;
    }
    const unsigned C = *c_ptr;
    const int lane = threadIdx.x & 31;
    const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const unsigned groups = (n + 31) / 32, per = (groups + nw - 1) / nw;
    const unsigned g0 = min(groups, gw * per), g1 = min(groups, g0 + per);
    if (g0 >= g1 || C == 0) return;
    unsigned lo = 0, hi = C - 1;   // last chunk starting at or before the first ray
    while (lo < hi) {
        const unsigned mid = lo + (hi - lo + 1) / 2;
        if (cpos[mid] <= g0 * 32) lo = mid; else hi = mid - 1;
    }
    for (unsigned g = g0; g < g1; ++g) {
        const unsigned i = g * 32 + lane;
        const unsigned cl = (lo + lane < C) ? cpos[lo + lane] : 0xffffffffu;
        unsigned l = 0;
#pragma unroll
        for (unsigned step = 16; step > 0; step >>= 1) {
            const unsigned v = __shfl_sync(FULL, cl, l + step);
            if (v <= i) l += step;
        }
        const unsigned start = __shfl_sync(FULL, cl, l);
        const unsigned chunk = lo + l;
        if (i < n) copy_ray(gen, sbase[chunk] + (i - start), out, i, sk[chunk]);
        // chunk of the next group's first ray: the last ray's chunk or the one after it
        const unsigned l31 = __shfl_sync(FULL, l, 31);
        const unsigned after = __shfl_sync(FULL, cl, min(l31 + 1, 31u));
        const unsigned nxt = l31 < 31 ? after : (lo + 32 < C ? cpos[lo + 32] : 0xffffffffu);
        lo = lo + l31 + (nxt <= (g + 1) * 32 ? 1u : 0u);
        lo = min(lo, C - 1);
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
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

struct HashWs {
    GenOut gen;
    uint32_t *chK, *chV, *chBase, *chPos, *chSB, *altK, *altV;
    float* tables;
    // control region (zeroed per call)
    char* ctl_begin;
    size_t ctl_bytes;
    size_t total;
    unsigned* tile_ctr;      // 8 counters
    unsigned* counts;        // [0] chunk count
    unsigned* hist;          // 4 x 256
    unsigned* offs;          // 4 x 256
    unsigned* plan;          // 5
    unsigned long long* st_gen;
    unsigned long long* st_chunk;
    unsigned long long* st_pos;
    unsigned* st_radix;      // 4 passes x tiles x 256
};

size_t table_floats() { return (1u << 13) * 2 + (1u << 13) / 8 * 2; }

HashWs carve_hash(void* ws, uint32_t cap, uint32_t max_pixels) {
    Carve c{reinterpret_cast<char*>(ws)};
    HashWs w{};
    w.gen.rec = c.take<float4>(2 * (size_t)cap);
    w.gen.key = c.take<uint32_t>(cap);
    w.gen.val = c.take<uint32_t>(cap);
    w.gen.capacity = cap;
    w.chK = c.take<uint32_t>(cap);
    w.chV = c.take<uint32_t>(cap);
    w.chBase = c.take<uint32_t>((size_t)cap + 1);
    w.chPos = c.take<uint32_t>(cap);
    w.chSB = c.take<uint32_t>(cap);
    w.altK = c.take<uint32_t>(cap);
    w.altV = c.take<uint32_t>(cap);
    w.tables = c.take<float>(table_floats());
    c.off = (c.off + 255) & ~size_t(255);
    size_t ctl0 = c.off;
    w.tile_ctr = c.take<unsigned>(16);
    w.counts = c.take<unsigned>(4);
    w.hist = c.take<unsigned>(1024);
    w.offs = c.take<unsigned>(1024);
    w.plan = c.take<unsigned>(8);
    const size_t gen_tiles = ((size_t)max_pixels + GEN_TILE - 1) / GEN_TILE + 1;
    const size_t cmp_tiles = ((size_t)cap + CMP_TILE - 1) / CMP_TILE + 1;
    const size_t sc_tiles = ((size_t)cap + SCAN_TILE - 1) / SCAN_TILE + 1;
    w.st_gen = c.take<unsigned long long>(gen_tiles);
    w.st_chunk = c.take<unsigned long long>(cmp_tiles);
    w.st_pos = c.take<unsigned long long>(sc_tiles);
    w.st_radix = c.take<unsigned>(radix_status_words(cap));
    w.ctl_begin = ws ? reinterpret_cast<char*>(ws) + ctl0 : nullptr;
    w.ctl_bytes = c.off - ctl0;
    w.total = c.off + 256;
    return w;
}
}  // namespace

size_t hash_sort_workspace(uint32_t cap, uint32_t max_pixels) {
    return carve_hash(nullptr, cap, max_pixels).total;
}

crsh_status hash_sort_launch(const crsh_gbuffer* gb, const crsh_rays_in* in, const float* lights, uint32_t n_lights,
                             const crsh_hash_params* hp, crsh_rays* out, uint32_t* keys_out, uint32_t* n_out,
                             crsh_counters* ctr, void* ws, size_t ws_bytes, cudaStream_t s, const DeviceInfo& dev) {
    const uint32_t cap = out->capacity;
    const uint32_t max_pixels = gb ? gb->n_pixels : 0;
    if (ws_bytes < hash_sort_workspace(cap, max_pixels)) return CRSH_ERR_INVALID_ARG;
    HashWs w = carve_hash(ws, cap, max_pixels);

    // threshold tables, FP32-rounded from double libm values
    const unsigned BS = 1u << hp->shadow_theta_bits, MS = (1u << hp->shadow_phi_bits) / 8;
    const unsigned BR = 1u << hp->sec_theta_bits, MR = (1u << hp->sec_phi_bits) / 8;
    float* tcosS = w.tables;
    float* ttanS = tcosS + BS;
    float* tcosR = ttanS + MS;
    float* ttanR = tcosR + BR;
    tables_launch(TableSpec{{tcosS, ttanS, tcosR, ttanR}, {BS, MS, BR, MR}, {0, 1, 0, 1}}, s, dev);
    HashDev h;
    h.cosS = tcosS; h.tanS = ttanS; h.cosR = tcosR; h.tanR = ttanR;
    for (int a = 0; a < 3; ++a) {
        // IEEE single-precision subtraction and division, rounded to nearest as on the device
        volatile float ext = hp->hi[a] - hp->lo[a];
        volatile float sc = (float)(1u << hp->sec_cell_bits) / ext;
        h.lo[a] = hp->lo[a];
        h.scale[a] = sc;
    }
    h.stb = hp->shadow_theta_bits; h.spb = hp->shadow_phi_bits;
    h.cb = hp->sec_cell_bits; h.tb = hp->sec_theta_bits; h.pb = hp->sec_phi_bits;

    zero_launch(ZeroSpans{{w.ctl_begin, ctr, n_out}, {w.ctl_bytes, sizeof(crsh_counters), sizeof(uint32_t)}}, s, dev);

    const int persist = dev.sms * 8;
    if (gb) {
        const unsigned tiles = (gb->n_pixels + GEN_TILE - 1) / GEN_TILE;
        const unsigned grid = tiles < (unsigned)persist ? (tiles ? tiles : 1) : (unsigned)persist;
        launch_pdl(k_gen_gbuffer, grid, GEN_BLOCK, 0, s, *gb, lights, n_lights, (int)hp->shadow_cull, h, w.gen, n_out,
                                                 w.st_gen, &w.tile_ctr[0], ctr);
    } else {
        unsigned blocks = (in->n + 255) / 256;
        if (blocks > (unsigned)persist) blocks = persist;
        if (blocks == 0) blocks = 1;
        launch_pdl(k_gen_rays, blocks, 256, 0, s, *in, h, w.gen, n_out, ctr);
    }

    const bool sort = hp->sort != 0;
    const bool compress = sort && hp->compress != 0;
    uint32_t *kA = w.gen.key, *vA = w.gen.val;
    const unsigned* cnt_ptr = n_out;
    if (compress) {
        unsigned tiles = (cap + CMP_TILE - 1) / CMP_TILE;
        unsigned grid = tiles < (unsigned)persist ? (tiles ? tiles : 1) : (unsigned)persist;
        launch_pdl(k_chunk, grid, CMP_BLOCK, 0, s, w.gen.key, n_out, w.chK, w.chBase, &w.counts[0], w.hist, w.st_chunk,
                                           &w.tile_ctr[1], ctr);
        kA = w.chK;
        vA = w.chV;
        cnt_ptr = &w.counts[0];
    }
    if (sort) {
        RadixWs rw{w.hist, w.offs, w.plan, &w.tile_ctr[2], w.st_radix};
        radix_sort_launch(kA, vA, w.altK, w.altV, cnt_ptr, cap, rw, ctr, s, dev, compress, true);
    } else {
        launch_pdl(k_radix_plan, 1, 256, 0, s, w.hist, cnt_ptr, w.offs, w.plan, 0, 0);
    }
    if (compress) {
        unsigned tiles = (cap + SCAN_TILE - 1) / SCAN_TILE;
        unsigned grid = tiles < (unsigned)persist ? (tiles ? tiles : 1) : (unsigned)persist;
        launch_pdl(k_chunk_pos, grid, SCAN_BLOCK, 0, s, kA, vA, w.altK, w.altV, w.plan, w.chBase, cnt_ptr, w.chPos, w.chSB,
                                                 w.st_pos, &w.tile_ctr[6], ctr);
    }
    SortedOut so{out->ox, out->oy, out->oz, out->dx, out->dy, out->dz, out->tmax, out->type,
                 out->ray_id, out->pixel, keys_out};
    {
        unsigned blocks = (cap + 255) / 256;
        if (blocks > (unsigned)dev.sms * 4) blocks = dev.sms * 4;
        if (blocks == 0) blocks = 1;
        const int mode = !sort ? 0 : (compress ? 2 : 1);
        launch_pdl(k_gather, blocks, 256, 0, s, mode, w.gen, kA, vA, w.altK, w.altV, w.plan, w.chSB, w.chPos, cnt_ptr,
                                        n_out, so);
    }
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

}  // namespace crsh
