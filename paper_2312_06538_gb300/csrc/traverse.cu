// Section 3.3.7, eq. 9: top-down traversal of the sphere-cone hierarchy.
//
// GB300 design.  Every stage is one persistent "expand - test - compact"
// kernel over an implicit index space whose size is read on the device:
//   mesh stage   (top node n, mesh m)           eq. 9 against the mesh sphere
//   top stage    (n, triangle of an accepted m) eq. 9 against the triangle sphere
//   level stage  (pair (p, t) of the level above, child c of p), laid out
//                child-major inside each parent's run of pairs, so the output
//                comes out grouped by child node with triangles ascending.
// Each tile of elements tests, ballots, scans across warps and takes its
// output offset by decoupled look-back, then writes its pairs: one read of
// the parent pairs, one write of the children, no flag arrays in memory.
// A CSR offset table per level (binary search over the sorted node column)
// lets the next level find a parent's run.
#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

constexpr int TV_BLOCK = 256, TV_ITEMS = 4, TV_TILE = TV_BLOCK * TV_ITEMS;
static_assert(TV_ITEMS * (TV_BLOCK / 32) == 32, "one warp scans the per-warp counts");

// eq. 9 in FP32.  C = node sphere centre (cone apex), d = node radius, x =
// unit axis, tan/sec of the spread precomputed (sec = +inf: accept all);
// (P, r) = tested sphere.  Accept iff |s| tan + (d + r) sec >= |P - H| with
// s = (P - C).x and H = C + s x, compared squared, with the left side raised
// by 2^-20 (node and triangle radii already carry the coordinate-scaled
// rounding margins).
__device__ __forceinline__ bool eq9(float4 sph, float4 cone, float2 trig, float4 P) {
    if (trig.y == __int_as_float(0x7f800000)) return true;
    const float vx = P.x - sph.x, vy = P.y - sph.y, vz = P.z - sph.z;
    const float s = vx * cone.x + vy * cone.y + vz * cone.z;
    const float wx = vx - s * cone.x, wy = vy - s * cone.y, wz = vz - s * cone.z;
    const float w2 = wx * wx + wy * wy + wz * wz;
    float lhs = fabsf(s) * trig.x + (sph.w + P.w) * trig.y;
    lhs *= 1.00000095f;
    return lhs * lhs >= w2;
}

struct Node3 {
    const float4* sphere;
    const float4* cone;
    const float2* trig;
};

struct PairOut {
    uint32_t* node;
    uint32_t* tri;
    unsigned* count;   // device: written pairs (clamped to cap)
    unsigned long long cap;
};

struct TvCtl {
    unsigned long long* status;
    unsigned* tile_ctr;
    crsh_counters* ctr;
    int level_idx;     // counters index (level - 1); -1 for the mesh stage
};

// Generic expand-test-compact.  Op provides:
//   size()                             elements (device read)
//   test(e, a, b, valid)               -> accept; payload (a, b); valid = a test was made
//   emit(pos, a, b)
//   finish(total, tests_paper_base)    stage totals, written by the last tile
template <class Op>
__global__ void __launch_bounds__(TV_BLOCK) k_compact(Op op, TvCtl ctl) {
    __shared__ unsigned s_tile;
    __shared__ unsigned s_cnt[TV_ITEMS][TV_BLOCK / 32];
    __shared__ unsigned long long s_prefix;
    const unsigned long long E = op.size();
    const unsigned n_tiles = (unsigned)((E + TV_TILE - 1) / TV_TILE);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (n_tiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) op.finish(0ull);
        return;
    }
    unsigned long long tests = 0;
    for (;;) {
        const unsigned tile = next_tile(ctl.tile_ctr, &s_tile);
        if (tile >= n_tiles) break;
        bool f[TV_ITEMS];
        unsigned bal[TV_ITEMS];
        uint32_t pa[TV_ITEMS], pb[TV_ITEMS];
#pragma unroll
        for (int i = 0; i < TV_ITEMS; ++i) {
            const unsigned long long e = (unsigned long long)tile * TV_TILE + i * TV_BLOCK + threadIdx.x;
            bool valid = false;
            f[i] = (e < E) && op.test(e, pa[i], pb[i], valid);
            tests += valid;
            bal[i] = __ballot_sync(FULL, f[i]);
            if (lane == 0) s_cnt[i][warp] = __popc(bal[i]);
        }
        __syncthreads();
        if (warp == 0) {
            unsigned v = s_cnt[lane / (TV_BLOCK / 32)][lane % (TV_BLOCK / 32)];
            unsigned inc = warp_incl_scan(v);
            s_cnt[lane / (TV_BLOCK / 32)][lane % (TV_BLOCK / 32)] = inc - v;
            unsigned total = __shfl_sync(FULL, inc, 31);
            unsigned long long pre = lookback_warp(ctl.status, tile, total, ctl.ctr);
            if (lane == 0) {
                s_prefix = pre;
                if (tile == n_tiles - 1) op.finish(pre + total);
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < TV_ITEMS; ++i) {
            if (f[i]) {
                unsigned long long pos = s_prefix + s_cnt[i][warp] + __popc(bal[i] & lanemask_lt());
                op.emit(pos, pa[i], pb[i]);
            }
        }
    }
    tests = warp_sum64(tests);
    if (lane == 0 && tests) {
        if (ctl.level_idx >= 0) atomicAdd(&ctl.ctr->tests[ctl.level_idx], tests);
        else atomicAdd(&ctl.ctr->mesh_tests, tests);
    }
}

__device__ __forceinline__ void store_pair(const PairOut& o, unsigned long long pos, uint32_t a, uint32_t b) {
    if (pos < o.cap) {
        o.node[pos] = a;
        o.tri[pos] = b;
    }
}

__device__ __forceinline__ void finish_pairs(const PairOut& o, unsigned long long total, crsh_counters* ctr,
                                             int level_idx) {
    *o.count = (unsigned)min(total, o.cap);
    if (level_idx >= 0) ctr->hits[level_idx] = total;
    atomicMax(&ctr->needed_pairs, total);
    if (total > o.cap) set_status(ctr, CRSH_ERR_CAPACITY);
}

// ---- mesh stage: (top node, mesh) ----------------------------------------
struct MeshOp {
    Node3 top;
    const unsigned* top_count;
    const float4* mesh_sphere;
    const uint32_t* mesh_first;
    unsigned n_meshes;
    int cull;
    PairOut out;   // (node, mesh)
    crsh_counters* ctr;
    __device__ unsigned long long size() const { return (unsigned long long)(*top_count) * n_meshes; }
    __device__ bool test(unsigned long long e, uint32_t& a, uint32_t& b, bool& valid) const {
        a = (uint32_t)(e / n_meshes);
        b = (uint32_t)(e % n_meshes);
        if (!cull) return true;
        valid = true;
        float4 s = mesh_sphere[b];
        // rounding margin of the FP32 test for an input sphere (triangle
        // spheres carry theirs from scene preparation)
        s.w = s.w * (1.0f + 9.6e-7f) + 3.9e-6f * (fabsf(s.x) + fabsf(s.y) + fabsf(s.z) + s.w);
        return eq9(top.sphere[a], top.cone[a], top.trig[a], s);
    }
    __device__ void emit(unsigned long long pos, uint32_t a, uint32_t b) const { store_pair(out, pos, a, b); }
    __device__ void finish(unsigned long long total) const {
        *out.count = (unsigned)min(total, out.cap);
        ctr->mesh_hits = cull ? total : 0;
        if (total > out.cap) set_status(ctr, CRSH_ERR_CAPACITY);
    }
};

// exclusive prefix of the triangle counts of the accepted (node, mesh) pairs
__global__ void k_mesh_scan(const uint32_t* mp_mesh, const unsigned* a_ptr, const uint32_t* mesh_first,
                            unsigned long long* mesh_off) {
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    const unsigned A = *a_ptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (unsigned base = 0; base < A; base += blockDim.x) {
        unsigned i = base + threadIdx.x;
        unsigned long long v = 0;
        if (i < A) {
            uint32_t m = mp_mesh[i];
            v = mesh_first[m + 1] - mesh_first[m];
        }
        unsigned long long inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long n = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += n;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        unsigned long long wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_w[w];
        if (i < A) mesh_off[i] = s_carry + wpre + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < nw; ++w) t += s_w[w];
            s_carry += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) mesh_off[A] = s_carry;
}

// ---- top stage: (top node, triangle of an accepted mesh) -----------------
struct TopOp {
    Node3 top;
    const uint32_t* mp_node;
    const uint32_t* mp_mesh;
    const unsigned* a_ptr;
    const unsigned long long* mesh_off;
    const uint32_t* mesh_first;
    const float4* tri_sphere;
    PairOut out;
    crsh_counters* ctr;
    int level_idx;
    __device__ unsigned long long size() const { return mesh_off[*a_ptr]; }
    __device__ bool test(unsigned long long e, uint32_t& a, uint32_t& b, bool& valid) const {
        const unsigned A = *a_ptr;
        unsigned lo = 0, hi = A - 1;   // last i with mesh_off[i] <= e
        while (lo < hi) {
            unsigned mid = lo + (hi - lo + 1) / 2;
            if (mesh_off[mid] <= e) lo = mid; else hi = mid - 1;
        }
        a = mp_node[lo];
        b = mesh_first[mp_mesh[lo]] + (uint32_t)(e - mesh_off[lo]);
        valid = true;
        return eq9(top.sphere[a], top.cone[a], top.trig[a], tri_sphere[b]);
    }
    __device__ void emit(unsigned long long pos, uint32_t a, uint32_t b) const { store_pair(out, pos, a, b); }
    __device__ void finish(unsigned long long total) const {
        finish_pairs(out, total, ctr, level_idx);
        ctr->tests_paper[level_idx] = mesh_off[*a_ptr];
    }
};

// ---- level stage: (pair (p, t) of level l+1, child c of p) ---------------
struct LevelOp {
    Node3 child;
    const unsigned* child_count;
    const uint32_t* pnode;     // parent pairs, grouped by parent
    const uint32_t* ptri;
    const unsigned* p_count;
    const uint32_t* poff;      // CSR of the parent level
    unsigned logB;
    const float4* tri_sphere;
    PairOut out;
    crsh_counters* ctr;
    int level_idx;
    __device__ unsigned long long size() const { return (unsigned long long)(*p_count) << logB; }
    __device__ bool test(unsigned long long e, uint32_t& a, uint32_t& b, bool& valid) const {
        const unsigned j = (unsigned)(e >> logB);
        const uint32_t p = pnode[j];
        const uint32_t s = poff[p];
        const uint32_t len = poff[p + 1] - s;
        const uint32_t o = (uint32_t)(e - ((unsigned long long)s << logB));   // < B * len
        const uint32_t c = o / len;
        const uint32_t k = o - c * len;
        a = (p << logB) + c;
        if (a >= *child_count) return false;   // padded slot of a partial last node
        b = ptri[s + k];
        valid = true;
        return eq9(child.sphere[a], child.cone[a], child.trig[a], tri_sphere[b]);
    }
    __device__ void emit(unsigned long long pos, uint32_t a, uint32_t b) const { store_pair(out, pos, a, b); }
    __device__ void finish(unsigned long long total) const {
        finish_pairs(out, total, ctr, level_idx);
        ctr->tests_paper[level_idx] = (unsigned long long)(*p_count) << logB;
    }
};

// CSR offsets over a node-sorted pair list: off[n] = first pair of node n.
__global__ void k_csr(const uint32_t* node, const unsigned* p_count, const unsigned* n_count, uint32_t* off) {
    const unsigned P = *p_count, Nn = *n_count;
    for (unsigned n = blockIdx.x * blockDim.x + threadIdx.x; n <= Nn; n += gridDim.x * blockDim.x) {
        unsigned lo = 0, hi = P;
        while (lo < hi) {
            unsigned mid = (lo + hi) >> 1;
            if (node[mid] < n) lo = mid + 1; else hi = mid;
        }
        off[n] = lo;
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

struct TvWs {
    uint32_t *bufN[2], *bufT[2];         // ping-pong pair lists of the levels above 1
    uint32_t *mpN, *mpM;                 // accepted (node, mesh)
    unsigned long long* mesh_off;
    uint32_t* off[CRSH_MAX_LEVELS];      // CSR per level >= 2
    char* ctl;
    size_t ctl_bytes;
    unsigned* counts;                    // [0] mesh pairs, [1 + l] pairs of level l+1
    unsigned* tile_ctr;                  // one per stage
    unsigned long long* st[CRSH_MAX_LEVELS + 2];
    size_t total;
};

TvWs carve_tv(void* ws, const crsh_hierarchy* h, uint32_t n_tris, uint32_t n_meshes, uint64_t cap) {
    Carve c{reinterpret_cast<char*>(ws)};
    TvWs w{};
    const unsigned L = h->levels, B = h->bundle;
    const uint64_t top_cap = h->capacity[L - 1];
    const size_t mp = (size_t)top_cap * (n_meshes ? n_meshes : 1);
    if (L > 1) {
        for (int k = 0; k < 2; ++k) {
            w.bufN[k] = c.take<uint32_t>(cap);
            w.bufT[k] = c.take<uint32_t>(cap);
        }
    }
    w.mpN = c.take<uint32_t>(mp);
    w.mpM = c.take<uint32_t>(mp);
    w.mesh_off = c.take<unsigned long long>(mp + 1);
    for (unsigned l = 1; l < L; ++l) w.off[l] = c.take<uint32_t>((size_t)h->capacity[l] + 1);
    c.off = (c.off + 255) & ~size_t(255);
    const size_t ctl0 = c.off;
    w.counts = c.take<unsigned>(CRSH_MAX_LEVELS + 2);
    w.tile_ctr = c.take<unsigned>(CRSH_MAX_LEVELS + 2);
    w.st[0] = c.take<unsigned long long>(mp / TV_TILE + 2);                                  // mesh stage
    w.st[1] = c.take<unsigned long long>((size_t)(top_cap * (uint64_t)n_tris / TV_TILE) + 2); // top stage
    for (unsigned l = 2; l < L + 1; ++l) w.st[l] = c.take<unsigned long long>((size_t)(cap * B / TV_TILE) + 2);
    w.ctl = ws ? reinterpret_cast<char*>(ws) + ctl0 : nullptr;
    w.ctl_bytes = c.off - ctl0;
    w.total = c.off + 256;
    return w;
}

unsigned log2u(unsigned v) {
    unsigned r = 0;
    while ((1u << r) < v) ++r;
    return r;
}
}  // namespace

size_t traverse_workspace(const crsh_hierarchy* h, uint32_t n_tris, uint32_t n_meshes, uint64_t cap) {
    return carve_tv(nullptr, h, n_tris, n_meshes, cap).total;
}

template <class Op>
static void launch_compact(const Op& op, TvCtl ctl, unsigned grid, cudaStream_t s) {
    k_compact<Op><<<grid, TV_BLOCK, 0, s>>>(op, ctl);
}

crsh_status traverse_launch(const crsh_hierarchy* h, const crsh_scene* sc, const crsh_traverse_params* tp,
                            crsh_pairs* out, crsh_counters* ctr, void* ws, size_t ws_bytes, cudaStream_t s,
                            const DeviceInfo& dev) {
    const unsigned L = h->levels, B = h->bundle, logB = log2u(B);
    const uint64_t cap = out->capacity;
    if (ws_bytes < traverse_workspace(h, sc->n_tris, sc->n_meshes, cap)) return CRSH_ERR_INVALID_ARG;
    TvWs w = carve_tv(ws, h, sc->n_tris, sc->n_meshes, cap);
    if (cudaMemsetAsync(w.ctl, 0, w.ctl_bytes, s) != cudaSuccess) return CRSH_ERR_CUDA;
    // reset this call's counters: mesh_tests .. needed_pairs
    {
        char* c0 = reinterpret_cast<char*>(&ctr->mesh_tests);
        char* c1 = reinterpret_cast<char*>(&ctr->final_tests);
        if (cudaMemsetAsync(c0, 0, (size_t)(c1 - c0), s) != cudaSuccess) return CRSH_ERR_CUDA;
        if (cudaMemsetAsync(&ctr->needed_pairs, 0, sizeof(unsigned long long), s) != cudaSuccess) return CRSH_ERR_CUDA;
    }
    const unsigned grid = dev.sms * 4;
    auto level_nodes = [&](unsigned l) {   // l = 1..L
        return Node3{reinterpret_cast<const float4*>(h->sphere[l - 1]), reinterpret_cast<const float4*>(h->cone[l - 1]),
                     reinterpret_cast<const float2*>(h->trig[l - 1])};
    };
    const float4* tsph = reinterpret_cast<const float4*>(sc->tri_sphere);
    // pair list of level l: level 1 -> out; others ping-pong in the workspace
    auto pairs_of = [&](unsigned l) {
        if (l == 1) return PairOut{out->node, out->tri, out->count, cap};
        return PairOut{w.bufN[l & 1], w.bufT[l & 1], &w.counts[1 + l], cap};
    };

    // mesh stage
    MeshOp mop{level_nodes(L), h->count + (L - 1), reinterpret_cast<const float4*>(sc->mesh_sphere),
               sc->mesh_first_tri, sc->n_meshes, (int)tp->mesh_cull,
               PairOut{w.mpN, w.mpM, &w.counts[0], (unsigned long long)h->capacity[L - 1] * sc->n_meshes}, ctr};
    launch_compact(mop, TvCtl{w.st[0], &w.tile_ctr[0], ctr, -1}, grid, s);
    k_mesh_scan<<<1, 1024, 0, s>>>(w.mpM, &w.counts[0], sc->mesh_first_tri, w.mesh_off);
    // top stage
    TopOp top{level_nodes(L), w.mpN, w.mpM, &w.counts[0], w.mesh_off, sc->mesh_first_tri, tsph, pairs_of(L), ctr,
              (int)L - 1};
    launch_compact(top, TvCtl{w.st[1], &w.tile_ctr[1], ctr, (int)L - 1}, grid, s);
    // lower levels
    for (unsigned l = L - 1; l >= 1; --l) {
        PairOut par = pairs_of(l + 1);
        uint32_t* poff = w.off[l];   // CSR of level l+1 (index l = level l+1 - 1)
        const unsigned csr_blocks = (h->capacity[l] + 1 + 255) / 256;
        k_csr<<<csr_blocks < (unsigned)grid ? csr_blocks : grid, 256, 0, s>>>(par.node, par.count, h->count + l, poff);
        LevelOp op{level_nodes(l), h->count + (l - 1), par.node, par.tri, par.count, poff, logB, tsph, pairs_of(l), ctr,
                   (int)l - 1};
        launch_compact(op, TvCtl{w.st[l + 1], &w.tile_ctr[l + 1], ctr, (int)l - 1}, grid, s);
        if (l == 1) break;
    }
    {
        const unsigned csr_blocks = (h->capacity[0] + 1 + 255) / 256;
        k_csr<<<csr_blocks < (unsigned)grid ? csr_blocks : grid, 256, 0, s>>>(out->node, out->count, h->count,
                                                                               out->node_offsets);
    }
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

}  // namespace crsh
