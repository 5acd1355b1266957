// Section 3.3.6: bottom-up hierarchy of sphere-cones, and the per-triangle
// data the traversal and final tests read (triangle bounding spheres,
// Moller-Trumbore edge layout).
//
// GB300 design: a warp builds 32 level-1 nodes.  Their rays' directions are
// staged in shared memory with all loads in flight and lane k folds node k's
// cone (eqs. 1-4); then the origins go through the same rows and lane k builds
// the sphere tree (eqs. 7-8) in place.  The warp then merges its 32 nodes into
// level 2 in B-lane groups; higher levels merge their B children the same way
// in a kernel per level, as balanced trees of shuffle-downs (eqs. 5-8).  Every
// node is padded outward after its merge so the FP32 hierarchy contains its
// rays, and stores tan(spread), 1/cos(spread) for the eq. 9 tests of the
// traversal.
#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

struct SC {
    f3 c;
    float r;
    f3 x;
    float phi;
};

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Square root and quotient to a few ulps (special-function unit); the
// padding applied after each merge covers their error.
__device__ __forceinline__ float sqrt_fast(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ float div_fast(float a, float b) { return __fdividef(a, b); }

// eqs. 7-8: sphere union, centre at the midpoint.
__device__ __forceinline__ void sphere_union(SC& a, const SC& b) {
    f3 c = (a.c + b.c) * 0.5f;
    const f3 dc = b.c - a.c;
    float r = 0.5f * sqrt_fast(dot(dc, dc)) + fmaxf(a.r, b.r);
    a.c = c;
    a.r = r;
}

// eqs. 5-6: cone union about the normalised axis sum; spread = half the axis
// angle + the larger child spread; opposite axes give the whole sphere.
__device__ __forceinline__ void cone_union(SC& a, const SC& b) {
    f3 s = a.x + b.x;
    float ls = len(s);
    if (a.phi >= PI_F || b.phi >= PI_F || !(ls > 1e-6f)) {
        a.phi = PI_F;
        return;
    }
    float th = angle(a.x, b.x);
    a.x = s * (1.0f / ls);
    a.phi = fminf(PI_F, 0.5f * th + fmaxf(a.phi, b.phi));
}

// eqs. 1-4: widen the cone (x, phi) to hold direction r.  When r lies outside
// (theta = angle(x, r) > phi), the far edge e of the cone in the plane of x
// and r (eqs. 1-2) and r span the new cone: axis the bisector of e and r
// (eq. 3), spread the angle from the axis to r (eq. 4).  In closed form the
// new spread is (phi + theta) / 2 and the axis turns toward r by
// (theta - phi) / 2; the fold is carried as (axis, cos phi, sin phi), and the
// sine and cosine of every angle a step needs follow from products of these
// and of cos theta = x.r, sin theta = |x x r|, with tangent half-angle
// formulas for the halved angles.  Only multiplies, adds, a few reciprocals
// and square roots, and stable at small angles (sines are never taken from
// cosines).  A result whose half-angle would reach pi/2 (theta + phi >=
// pi - 1e-6) is the whole sphere, which eq. 9 accepts everywhere anyway.
struct ConeFold {
    f3 x;
    float cp, sp;   // cos, sin of the spread
    bool full;
    __device__ __forceinline__ void start(f3 d) {
        x = d;
        cp = 1.0f;
        sp = 0.0f;
        full = false;
    }
    __device__ __forceinline__ void add(f3 r) {
        if (full) return;
        const float c = dot(x, r);
        const f3 w = cross(x, r);
        const float s = sqrt_fast(dot(w, w));
        // inside iff theta <= phi: sin(phi - theta) >= 0, excluding phi - theta = -pi
        const float sd = sp * c - cp * s, cd = cp * c + sp * s;   // sin, cos of (phi - theta)
        if (sd > 0.0f || (sd == 0.0f && cd > 0.0f)) return;
        const float ss = sp * c + cp * s, cs = cp * c - sp * s;   // sin, cos of (phi + theta)
        if (ss < 0.0f || (ss <= 1e-6f && cs < 0.0f)) {            // theta + phi >= pi - 1e-6
            full = true;
            return;
        }
        // turn the axis toward r by delta = (theta - phi) / 2: tan(delta) = sin(2 delta) / (1 + cos(2 delta))
        // = (1 - cos(2 delta)) / sin(2 delta), whichever side has no cancellation
        const float td = cd >= 0.0f ? div_fast(-sd, 1.0f + cd) : div_fast(1.0f - cd, -sd);
        const float cdl = rsqrtf(1.0f + td * td), sdl = td * cdl;
        const float is = div_fast(1.0f, s);
        const f3 u = (r - x * c) * is;                              // unit normal to x toward r
        x = unit(x * cdl + u * sdl);
        // new spread (phi + theta) / 2: tan = sin(phi + theta) / (1 + cos(phi + theta)), or its other form
        const float tp = cs >= 0.0f ? div_fast(ss, 1.0f + cs) : div_fast(1.0f - cs, ss);
        cp = rsqrtf(1.0f + tp * tp);
        sp = tp * cp;
    }
    __device__ __forceinline__ float phi() const { return full ? PI_F : atan2f(sp, cp); }
};

struct Pads {
    float sr, sa, cr, ca;
};

// Caller's padding, plus a margin of a few FP32 ulps of the centre's
// coordinates that covers the rounding of the eq. 9 test near this node.
__device__ __forceinline__ void pad_node(SC& n, const Pads& p) {
    n.r = n.r * (1.0f + p.sr) + p.sa + 3.9e-6f * (fabsf(n.c.x) + fabsf(n.c.y) + fabsf(n.c.z));
    n.phi = fminf(PI_F, n.phi * (1.0f + p.cr) + p.ca);
}

// Balanced binary tree of merges in item order: at steps s = 1, 2, 4, ...,
// item i (a multiple of 2s) absorbs item i + s when it exists.  A node's items
// sit in B consecutive lanes (B a power of two <= 32), so each step is one
// shuffle-down within the lane group.  (B = 64 spans two warps: each warp
// runs the steps below 32 and the last step, item 0 absorbing item 32, goes
// through shared memory in k_build_up.)
__device__ __forceinline__ SC shfl_down_sc(const SC& v, unsigned s, int width) {
    SC o;
    o.c.x = __shfl_down_sync(FULL, v.c.x, s, width);
    o.c.y = __shfl_down_sync(FULL, v.c.y, s, width);
    o.c.z = __shfl_down_sync(FULL, v.c.z, s, width);
    o.r = __shfl_down_sync(FULL, v.r, s, width);
    o.x.x = __shfl_down_sync(FULL, v.x.x, s, width);
    o.x.y = __shfl_down_sync(FULL, v.x.y, s, width);
    o.x.z = __shfl_down_sync(FULL, v.x.z, s, width);
    o.phi = __shfl_down_sync(FULL, v.phi, s, width);
    return o;
}

template <bool CONES>
__device__ __forceinline__ void group_tree_merge(SC& item, unsigned r, unsigned m, unsigned B) {
    const unsigned W = B < 32u ? B : 32u;   // steps below the warp width
    for (unsigned s = 1; s < W; s <<= 1) {
        const SC other = shfl_down_sc(item, s, (int)W);
        if ((r & (2 * s - 1)) == 0 && r + s < m) {
            sphere_union(item, other);
            if (CONES) cone_union(item, other);
        }
    }
}

struct LevelOut {
    float4* sphere;
    float4* cone;
    float2* trig;
    unsigned cap;
};

__device__ __forceinline__ void store_node(const LevelOut& o, unsigned j, const SC& n) {
    o.sphere[j] = make_float4(n.c.x, n.c.y, n.c.z, n.r);
    o.cone[j] = make_float4(n.x.x, n.x.y, n.x.z, n.phi);
    float t, s;
    if (n.phi >= 0.5f * PI_F - 1e-6f) {
        t = s = __int_as_float(0x7f800000);   // accept everything (eq. 9 reading)
    } else {
        float sp, cp;
        sincosf(n.phi, &sp, &cp);
        t = sp / cp;
        s = 1.0f / cp;
        // round both up by the rounding margin of the FP32 eq. 9 evaluation
        // (a few ulps for tan/sec themselves, 2^-20 for the test's own sums
        // and products), so the test in the traversal stays conservative
        t = t * (1.0f + 1.5e-6f);
        s = s * (1.0f + 1.5e-6f);
    }
    o.trig[j] = make_float2(t, s);
}

struct RaysIn {
    const float *ox, *oy, *oz, *dx, *dy, *dz;
};

struct Caps {
    unsigned v[CRSH_MAX_LEVELS];
};

// A warp builds 32 consecutive level-1 nodes (one block = one warp).  It
// first copies the 32 B rays' origins and directions into shared memory with
// every load in flight at once (coalesced, node-major rows of B + 1 floats),
// then lane k builds node k alone: the sphere as the balanced pairwise tree of
// eqs. 7-8 merged in place, the cone by the fold of eqs. 1-4.  The odd row
// stride puts the 32 lanes' reads in 32 distinct banks.
template <int B>
__global__ void __launch_bounds__(32) k_build_l1(RaysIn rays, const unsigned* n_ptr, unsigned L, Pads pads,
                                                 LevelOut out, LevelOut out2, unsigned* counts, Caps caps) {
    pdl_wait();
    constexpr unsigned S = B + 1, W = 32 * S;
    // 4 x W floats: three staged components (directions for the cone, then
    // origins for the sphere) and the sphere radii; staging the two halves in
    // turn halves the shared memory of a warp, so twice as many warps are
    // resident to hide the loads and the FP32 dependency chains
    extern __shared__ float s_rows[];
    float* s0 = s_rows;
    float* s1 = s_rows + W;
    float* s2 = s_rows + 2 * W;
    float* srad = s_rows + 3 * W;
    const unsigned n = *n_ptr;
    const unsigned cnt = (n + B - 1) / B;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned c = n;
        for (unsigned l = 0; l < CRSH_MAX_LEVELS; ++l) {
            if (l < L) {
                c = (c + B - 1) / B;
                c = min(c, caps.v[l]);   // capacities are checked on the host
                counts[l] = c;
            } else {
                counts[l] = 0;
            }
        }
    }
    const unsigned lim = min(cnt, out.cap);
    const unsigned cnt2 = min((lim + B - 1) / B, caps.v[1]);   // level-2 nodes (when L >= 2)
    const unsigned lane = threadIdx.x;
    // 16-byte loads need every array 16-byte aligned (B >= 4 keeps a float4 in one node)
    const bool vec = B >= 4 && ((reinterpret_cast<uintptr_t>(rays.ox) | reinterpret_cast<uintptr_t>(rays.oy) |
                                 reinterpret_cast<uintptr_t>(rays.oz) | reinterpret_cast<uintptr_t>(rays.dx) |
                                 reinterpret_cast<uintptr_t>(rays.dy) | reinterpret_cast<uintptr_t>(rays.dz)) &
                                15u) == 0;
    // the 32 nodes' rays of three arrays into s0..s2 (coalesced: lane = ray,
    // or lane = 4 rays when the whole block exists)
    auto stage = [&](unsigned j0, const float* ax, const float* ay, const float* az) {
        if (vec && j0 + 32 <= lim && (size_t)(j0 + 32) * B <= n) {
            const float4* vx = reinterpret_cast<const float4*>(ax + (size_t)j0 * B);
            const float4* vy = reinterpret_cast<const float4*>(ay + (size_t)j0 * B);
            const float4* vz = reinterpret_cast<const float4*>(az + (size_t)j0 * B);
#pragma unroll
            for (int t = 0; t < B / 4; ++t) {
                const unsigned q = t * 32u + lane;       // float4 within the block
                const unsigned e = 4 * q, a = (e / B) * S + e % B;
                const float4 X = vx[q], Y = vy[q], Z = vz[q];
                s0[a] = X.x; s0[a + 1] = X.y; s0[a + 2] = X.z; s0[a + 3] = X.w;
                s1[a] = Y.x; s1[a + 1] = Y.y; s1[a + 2] = Y.z; s1[a + 3] = Y.w;
                s2[a] = Z.x; s2[a + 1] = Z.y; s2[a + 2] = Z.z; s2[a + 3] = Z.w;
            }
        } else {
#pragma unroll
            for (unsigned t = 0; t < B; ++t) {
                const unsigned idx = t * 32 + lane;      // ray within this block of 32 nodes
                const unsigned k = idx / B, r = idx % B;
                const size_t i = (size_t)j0 * B + idx;   // sorted ray
                if (j0 + k < lim && i < n) {
                    const unsigned a = k * S + r;
                    s0[a] = ax[i];
                    s1[a] = ay[i];
                    s2[a] = az[i];
                }
            }
        }
        __syncwarp();
    };
    // warm L2 with three arrays' spans of the block of 32 nodes at j0 (one
    // 128-byte line per lane and array: 32 nodes x B rays x 4 bytes = B lines)
    auto warm = [&](unsigned j0, const float* ax, const float* ay, const float* az) {
        if (j0 >= lim) return;
        const size_t i0 = (size_t)j0 * B;
        for (unsigned l = lane; l < B; l += 32) {
            const size_t i = i0 + 32 * l;
            if (i < n) {
                prefetch_l2(ax + i);
                prefetch_l2(ay + i);
                prefetch_l2(az + i);
            }
        }
    };
    const bool unroll = lim >= 4u * 32u * gridDim.x;
    for (unsigned j0 = blockIdx.x * 32; j0 < lim; j0 += gridDim.x * 32) {
        const unsigned j = j0 + lane;
        const unsigned m = j < lim ? min((unsigned)B, n - j * B) : 0u;
        const unsigned b = lane * S;
        // this block's origins and the next block's directions load into L2
        // while the cone and the sphere of this block are built
        warm(j0, rays.ox, rays.oy, rays.oz);
        warm(j0 + gridDim.x * 32, rays.dx, rays.dy, rays.dz);
        // cone: the rays in sorted order (eqs. 1-4)
        stage(j0, rays.dx, rays.dy, rays.dz);
        // a full node (every node but perhaps the last) takes the unrolled
        // loops: static shared-memory offsets, no loop or address arithmetic;
        // only when each warp builds at least four blocks of nodes, so the
        // longer code is fetched once for many nodes (on a 500 K-ray frame,
        // one block per warp, the rolled loops measured faster)
        ConeFold f;
        if (unroll && m == B) {
            f.start(unit(mk3(s0[b], s1[b], s2[b])));
#pragma unroll
            for (unsigned i = 1; i < B; ++i) f.add(unit(mk3(s0[b + i], s1[b + i], s2[b + i])));
        } else if (m) {
            f.start(unit(mk3(s0[b], s1[b], s2[b])));
            for (unsigned i = 1; i < m; ++i) f.add(unit(mk3(s0[b + i], s1[b + i], s2[b + i])));
        }
        __syncwarp();
        // sphere: radius-0 leaves, balanced pairwise tree in ray order (eqs. 7-8)
        stage(j0, rays.ox, rays.oy, rays.oz);
        auto merge = [&](unsigned i, unsigned st) {
            SC x, y;
            x.c = mk3(s0[b + i], s1[b + i], s2[b + i]);
            x.r = srad[b + i];
            y.c = mk3(s0[b + i + st], s1[b + i + st], s2[b + i + st]);
            y.r = srad[b + i + st];
            sphere_union(x, y);
            s0[b + i] = x.c.x;
            s1[b + i] = x.c.y;
            s2[b + i] = x.c.z;
            srad[b + i] = x.r;
        };
        if (unroll && m == B) {
#pragma unroll
            for (unsigned i = 0; i < B; ++i) srad[b + i] = 0.0f;
#pragma unroll
            for (unsigned st = 1; st < B; st <<= 1) {
#pragma unroll
                for (unsigned i = 0; i + st < B; i += 2 * st) merge(i, st);
            }
        } else if (m) {
            for (unsigned i = 0; i < m; ++i) srad[b + i] = 0.0f;
            for (unsigned st = 1; st < m; st <<= 1) {
                for (unsigned i = 0; i + st < m; i += 2 * st) merge(i, st);
            }
        }
        SC node;
        node.c = mk3(0.f, 0.f, 0.f);
        node.r = 0.0f;
        node.x = mk3(1.f, 0.f, 0.f);
        node.phi = 0.0f;
        if (m) {
            node.c = mk3(s0[b], s1[b], s2[b]);
            node.r = srad[b];
            node.x = f.x;
            node.phi = f.phi();
            pad_node(node, pads);
            store_node(out, j, node);
        }
        // level 2 (eqs. 5-8): the block's 32 nodes are 32 / B whole groups,
        // merged here as the level-2 pass would merge them after reading the
        // stored nodes back (the same values, in the same order); with B = 64
        // a group spans two blocks and level 2 is built by k_build_up
        if (B <= 32 && L >= 2) {
            const unsigned g = j / B, r2 = lane & (B - 1);
            const unsigned m2 = g < cnt2 ? min((unsigned)B, lim - g * B) : 0u;
            group_tree_merge<true>(node, r2, m2, B);
            if (r2 == 0 && g < cnt2) {
                pad_node(node, pads);
                store_node(out2, g, node);
            }
        }
        __syncwarp();
    }
}

template <int B>
static void launch_build_l1(const RaysIn& ri, const uint32_t* n_rays, unsigned L, const Pads& pads,
                            const LevelOut& o1, const LevelOut& o2, unsigned* counts, const Caps& caps,
                            unsigned cap0, cudaStream_t s, const DeviceInfo& dev) {
    const size_t smem = 4 * 32 * (B + 1) * sizeof(float);
    const unsigned blocks = (cap0 + 31) / 32;
    const unsigned grid = blocks < (unsigned)dev.sms * 32 ? (blocks ? blocks : 1) : dev.sms * 32;
    launch_pdl(k_build_l1<B>, grid, 32, smem, s, ri, n_rays, L, pads, o1, o2, counts, caps);
}

__global__ void k_build_up(const float4* csph, const float4* ccone, const unsigned* counts, unsigned level_idx,
                           unsigned B, Pads pads, LevelOut out) {
    pdl_wait();
    __shared__ SC s_half[4];   // B = 64: each group's second-half result (128-thread blocks: 2 groups)
    const unsigned below = counts[level_idx - 1];
    const unsigned cnt = counts[level_idx];
    const unsigned r = threadIdx.x & (B - 1);   // child slot in the group (groups of B <= 64 threads)
    const unsigned groups_per_block = blockDim.x / B;
    const unsigned gstart = blockIdx.x * groups_per_block + threadIdx.x / B;
    const unsigned gstride = gridDim.x * groups_per_block;
    const unsigned iters = (cnt + gstride - 1) / gstride;
    for (unsigned it = 0; it < iters; ++it) {
        const unsigned j = gstart + it * gstride;
        const bool node_ok = j < cnt;
        const unsigned first = j * B;
        const unsigned m = node_ok ? min(B, below - first) : 0u;
        SC ch;
        ch.c = mk3(0.f, 0.f, 0.f);
        ch.r = 0.0f;
        ch.x = mk3(1.f, 0.f, 0.f);
        ch.phi = 0.0f;
        if (r < m) {
            const float4 sp = csph[first + r], co = ccone[first + r];
            ch.c = mk3(sp.x, sp.y, sp.z);
            ch.r = sp.w;
            ch.x = mk3(co.x, co.y, co.z);
            ch.phi = co.w;
        }
        group_tree_merge<true>(ch, r, m, B);   // eqs. 5-8 in child order
        if (B > 32) {   // the last step: child 0's subtree absorbs child 32's (block-uniform branch)
            const unsigned gl = threadIdx.x / B;
            if (r == 32) s_half[gl] = ch;
            __syncthreads();
            if (r == 0 && 32 < m) {
                const SC other = s_half[gl];
                sphere_union(ch, other);
                cone_union(ch, other);
            }
            __syncthreads();
        }
        if (r == 0 && node_ok) {
            pad_node(ch, pads);
            store_node(out, j, ch);
        }
    }
}

crsh_status build_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_build_params* bp,
                         crsh_hierarchy* h, cudaStream_t s, const DeviceInfo& dev) {
    const unsigned B = bp->bundle, L = bp->levels;
    Pads pads{bp->sphere_pad_rel, bp->sphere_pad_abs, bp->cone_pad_rel, bp->cone_pad_abs};
    h->levels = L;
    h->bundle = B;
    Caps caps{};
    for (unsigned l = 0; l < L; ++l) caps.v[l] = h->capacity[l];
    RaysIn ri{rays->ox, rays->oy, rays->oz, rays->dx, rays->dy, rays->dz};
    LevelOut o1{reinterpret_cast<float4*>(h->sphere[0]), reinterpret_cast<float4*>(h->cone[0]),
                reinterpret_cast<float2*>(h->trig[0]), h->capacity[0]};
    LevelOut o2{nullptr, nullptr, nullptr, 0};
    if (L >= 2)
        o2 = LevelOut{reinterpret_cast<float4*>(h->sphere[1]), reinterpret_cast<float4*>(h->cone[1]),
                      reinterpret_cast<float2*>(h->trig[1]), h->capacity[1]};
    // a warp per 32 level-1 nodes, which also merges them into level 2
    switch (B) {
        case 2: launch_build_l1<2>(ri, n_rays, L, pads, o1, o2, h->count, caps, h->capacity[0], s, dev); break;
        case 4: launch_build_l1<4>(ri, n_rays, L, pads, o1, o2, h->count, caps, h->capacity[0], s, dev); break;
        case 8: launch_build_l1<8>(ri, n_rays, L, pads, o1, o2, h->count, caps, h->capacity[0], s, dev); break;
        case 16: launch_build_l1<16>(ri, n_rays, L, pads, o1, o2, h->count, caps, h->capacity[0], s, dev); break;
        case 32: launch_build_l1<32>(ri, n_rays, L, pads, o1, o2, h->count, caps, h->capacity[0], s, dev); break;
        case 64: launch_build_l1<64>(ri, n_rays, L, pads, o1, o2, h->count, caps, h->capacity[0], s, dev); break;
        default: return CRSH_ERR_INVALID_ARG;
    }
    // levels 3 and up (2 and up when B = 64): B-lane groups over the stored nodes below
    for (unsigned l = (B > 32 ? 1u : 2u); l < L; ++l) {
        LevelOut o{reinterpret_cast<float4*>(h->sphere[l]), reinterpret_cast<float4*>(h->cone[l]),
                   reinterpret_cast<float2*>(h->trig[l]), h->capacity[l]};
        const unsigned blocks = (unsigned)(((size_t)h->capacity[l] * B + 127) / 128);
        const unsigned grid = blocks < (unsigned)dev.sms * 16 ? (blocks ? blocks : 1) : dev.sms * 16;
        launch_pdl(k_build_up, grid, 128, 0, s, reinterpret_cast<const float4*>(h->sphere[l - 1]),
                                        reinterpret_cast<const float4*>(h->cone[l - 1]), h->count, l, B, pads, o);
    }
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Scene preparation: triangle spheres (centroid, largest vertex distance,
// padded outward by a few FP32 ulps of the coordinates) and the record read
// by the final tests: v0, e1 = v1 - v0, e2 = v2 - v0, n = e1 x e2, and the
// sphere with the pre-test's squared radius.
// ---------------------------------------------------------------------------
__global__ void k_prepare(crsh_scene sc) {
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < sc.n_tris; t += gridDim.x * blockDim.x) {
        f3 a = mk3(sc.v0x[t], sc.v0y[t], sc.v0z[t]);
        f3 b = mk3(sc.v1x[t], sc.v1y[t], sc.v1z[t]);
        f3 c = mk3(sc.v2x[t], sc.v2y[t], sc.v2z[t]);
        f3 m = (a + b + c) * (1.0f / 3.0f);
        float r = fmaxf(len(a - m), fmaxf(len(b - m), len(c - m)));
        float mag = fabsf(m.x) + fabsf(m.y) + fabsf(m.z) + r;
        r = r * (1.0f + 9.6e-7f) + 3.9e-6f * mag;   // covers the FP32 error of eq. 9 at this distance
        reinterpret_cast<float4*>(sc.tri_sphere)[t] = make_float4(m.x, m.y, m.z, r);
        f3 e1 = b - a, e2 = c - a;
        f3 n = cross(e1, e2);
        float4* mt = reinterpret_cast<float4*>(sc.tri_mt) + 4 * (size_t)t;
        mt[0] = make_float4(a.x, a.y, a.z, n.x);
        mt[1] = make_float4(e1.x, e1.y, e1.z, n.y);
        mt[2] = make_float4(e2.x, e2.y, e2.z, n.z);
        // the final tests' pre-test sphere: the tightest of the spheres about the
        // centroid, the three edge midpoints and the circumcentre that hold all three
        // vertices (the smallest enclosing sphere is centred at one of the last four);
        // its radius is measured from the chosen centre, so any centre is safe, and
        // padded as above.  Squared and scaled: 1.05 r^2 (with the grazing slack of
        // the test, (a + b)^2 <= 1.05 a^2 + 21 b^2)
        f3 pc = m;
        float pr = fmaxf(len(a - m), fmaxf(len(b - m), len(c - m)));
        auto consider = [&](f3 x) {
            const float rx = fmaxf(len(a - x), fmaxf(len(b - x), len(c - x)));
            if (rx < pr) { pr = rx; pc = x; }   // a NaN centre (degenerate triangle) is never taken
        };
        consider((a + b) * 0.5f);
        consider((b + c) * 0.5f);
        consider((a + c) * 0.5f);
        const float nn = dot(n, n);
        consider(a + (cross(n, e1) * dot(e2, e2) + cross(e2, n) * dot(e1, e1)) * (0.5f / nn));
        const float pmag = fabsf(pc.x) + fabsf(pc.y) + fabsf(pc.z) + pr;
        pr = pr * (1.0f + 9.6e-7f) + 3.9e-6f * pmag;
        mt[3] = make_float4(pc.x, pc.y, pc.z, 1.05f * pr * pr);
    }
}

crsh_status prepare_scene_launch(const crsh_scene* sc, cudaStream_t s, const DeviceInfo& dev) {
    const unsigned blocks = (sc->n_tris + 255) / 256;
    const unsigned grid = blocks < (unsigned)dev.sms * 8 ? (blocks ? blocks : 1) : dev.sms * 8;
    k_prepare<<<grid, 256, 0, s>>>(*sc);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

}  // namespace crsh
