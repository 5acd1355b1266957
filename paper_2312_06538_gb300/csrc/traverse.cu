// Section 3.3.7, eq. 9: top-down traversal of the sphere-cone hierarchy.
//
// GB300 design.
//   mesh stage  (top node n, mesh m): eq. 9 against the whole-mesh sphere,
//               compacted in one pass (decoupled look-back; tiny index space).
//   triangle stages (top level, then levels L-1 .. 1): the pairs of the stage
//               above are the "parents".  A warp takes a chunk of 32 of a
//               parent's triangles, loads their spheres once and tests them
//               against every child of the parent (warp-uniform node loads),
//               storing one ballot word per (child, chunk) in output order.
//               A block-sum pass and an emit pass turn the ballots into
//               (child, triangle) pairs grouped by child, triangles ascending.
//               No per-element division, no chains of dependent loads, no
//               waits between blocks.
// The emit pass also records each child's run [start, end) of the output,
// which is how the next level finds a parent's triangles.  In word form
// (crsh_traverse_params.level1_words) the last stage stops after its count
// pass: its ballots, with one work-item descriptor per (parent, child,
// segment of WORD_SEG chunks) written by k_items, are level 1's candidates,
// read by the final tests in place.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

constexpr int TV_BLOCK = 256, TV_ITEMS = 4, TV_TILE = TV_BLOCK * TV_ITEMS;
static_assert(TV_ITEMS * (TV_BLOCK / 32) == 32, "one warp scans the per-warp counts");

// eq. 9 in FP32.  C = node sphere centre (cone apex), d = node radius, x =
// unit axis, T/S = tan/sec of the spread (precomputed, rounded up by the
// rounding margin of this evaluation; both +inf for a node that accepts
// everything); (P, r) = tested sphere.  Accept iff |s| T + (d + r) S >= |P - H|
// with s = (P - C).x and H = C + s x, compared squared and written as
// !(lhs^2 < |P - H|^2) so that a NaN (0 * inf on an accept-all node) accepts.
// Branch-free; node and triangle radii already carry the coordinate-scaled
// rounding margins.
__device__ __forceinline__ bool eq9(float4 sph, float4 cone, float2 trig, float4 P) {
    const float vx = P.x - sph.x, vy = P.y - sph.y, vz = P.z - sph.z;
    const float s = vx * cone.x + vy * cone.y + vz * cone.z;
    const float wx = vx - s * cone.x, wy = vy - s * cone.y, wz = vz - s * cone.z;
    const float w2 = wx * wx + wy * wy + wz * wz;
    const float lhs = fmaf(fabsf(s), trig.x, (sph.w + P.w) * trig.y);
    return !(lhs * lhs < w2);
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
    pdl_wait();
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

// o.node == nullptr: a list whose node column nobody reads (the levels
// between the top and level 1: the next level finds a node's triangles by
// its run), so only the triangle column is written
__device__ __forceinline__ void store_pair(const PairOut& o, unsigned long long pos, uint32_t a, uint32_t b) {
    if (pos < o.cap) {
        if (o.node) o.node[pos] = a;
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

// ---------------------------------------------------------------------------
// Triangle stages (top level and every lower level).
//
// "Parents" are the pair lists of the stage above: accepted (top node, mesh)
// pairs for the top level, the nodes of level l+1 with their triangle runs for
// level l.  A work unit is (parent, chunk of 32 of its triangles): one warp
// loads the 32 triangle spheres once, tests them against every child of the
// parent with warp-uniform node loads, and stores one 32-bit ballot per
// (child, chunk) at its place in output order (parent, child, chunk).  A
// block-sum pass and an emit pass then compact the ballots into (child,
// triangle) pairs: output grouped by child, triangles ascending.
// ---------------------------------------------------------------------------

struct LevelParents {           // parents: nodes of level l+1, pair runs [start, end)
    static constexpr bool kChunkCull = true;   // B children per parent: pre-test chunk spheres
    const uint32_t* ptri;
    const unsigned* pstart;
    const unsigned* pend;
    const unsigned* n_parent;   // nodes of level l+1
    const unsigned* n_child;    // nodes of level l
    Node3 child;
    unsigned logB;
    __device__ unsigned count() const { return *n_parent; }
    __device__ void range(unsigned p, unsigned& s, unsigned& len) const {
        s = pstart[p];
        len = pend[p] - s;
    }
    __device__ unsigned nchild(unsigned p) const {
        const unsigned first = p << logB, cc = *n_child;
        return first >= cc ? 0u : min(1u << logB, cc - first);
    }
    __device__ unsigned child_id(unsigned p, unsigned c) const { return (p << logB) + c; }
    __device__ unsigned tri(unsigned s, unsigned j) const { return ptri[s + j]; }
    // this parent's children own [first, last) of the output; no two parents share a child
    __device__ bool first_of_child(unsigned, unsigned) const { return true; }
    __device__ bool last_of_child(unsigned, unsigned) const { return true; }
};

struct TopParents {             // parents: accepted (top node, mesh) pairs, grouped by node
    static constexpr bool kChunkCull = false;  // one child per parent: nothing to share
    const uint32_t* mp_node;
    const uint32_t* mp_mesh;
    const unsigned* a_count;
    const uint32_t* mesh_first;
    Node3 child;                // the top level
    __device__ unsigned count() const { return *a_count; }
    __device__ void range(unsigned i, unsigned& s, unsigned& len) const {
        const uint32_t m = mp_mesh[i];
        s = mesh_first[m];
        len = mesh_first[m + 1] - s;
    }
    __device__ unsigned nchild(unsigned) const { return 1u; }
    __device__ unsigned child_id(unsigned i, unsigned) const { return mp_node[i]; }
    __device__ unsigned tri(unsigned s, unsigned j) const { return s + j; }
    // a top node's pairs span its accepted meshes' runs (parents are grouped by
    // node): its first mesh parent records the run's start, its last the end
    __device__ bool first_of_child(unsigned i, unsigned) const { return i == 0 || mp_node[i - 1] != mp_node[i]; }
    __device__ bool last_of_child(unsigned i, unsigned) const {
        return i + 1 == *a_count || mp_node[i + 1] != mp_node[i];
    }
};

struct StageBuf {
    unsigned* ubase;            // per parent: first unit        (n + 1 entries)
    unsigned* obase;            // per parent: first ballot word (n + 1 entries)
    unsigned* ibase;            // per parent: first final-test work item of the word form (n + 1 entries)
    unsigned* totals;           // [0] units, [1] ballot words, [2] work items
    unsigned* mask;             // ballot words in output order (parent, child, chunk)
    unsigned* pos;              // exclusive prefix of the ballot popcounts (O + 1 entries)
    unsigned* bsum;             // per scan block: accepted pairs
    unsigned* work;             // [0] count pass, [1] emit pass: claimed unit batches (zeroed per call)
};

// Pair runs of the level a stage writes: [start[n], end[n]) for node n
// (both 0 for a node without pairs).
struct RunOut {
    unsigned* start;
    unsigned* end;
};

// Single block: exclusive scans over the parents of units (chunks of 32
// triangles), ballot words (children x chunks) and the work items of the
// word form's final tests (children x segments of WORD_SEG chunks); the
// stage's test counters.
template <class Parents>
__global__ void __launch_bounds__(1024) k_unit_scan(Parents par, StageBuf sb, crsh_counters* ctr, int level_idx,
                                                    unsigned B_paper) {
    pdl_wait();
    __shared__ unsigned long long s_w[32][5];
    __shared__ unsigned long long s_tot[5];
    const unsigned n = par.count();
    const unsigned per = (n + blockDim.x - 1) / blockDim.x;
    const unsigned b0 = min(n, threadIdx.x * per), b1 = min(n, b0 + per);
    unsigned long long u = 0, o = 0, it = 0, tests = 0, paper = 0;
    for (unsigned p = b0; p < b1; ++p) {
        unsigned s, len;
        par.range(p, s, len);
        const unsigned nch = (len + 31) >> 5;
        const unsigned nc = par.nchild(p);
        u += nch;
        o += (unsigned long long)nc * nch;
        it += (unsigned long long)nc * ((nch + WORD_SEG - 1) / WORD_SEG);
        tests += (unsigned long long)nc * len;
        paper += len;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long iu = u, io = o, ii = it;
    for (int d = 1; d < 32; d <<= 1) {
        unsigned long long a = __shfl_up_sync(FULL, iu, d), b = __shfl_up_sync(FULL, io, d),
                           c = __shfl_up_sync(FULL, ii, d);
        if (lane >= d) { iu += a; io += b; ii += c; }
    }
    const unsigned long long st = warp_sum64(tests), sp = warp_sum64(paper);
    if (lane == 31) { s_w[warp][0] = iu; s_w[warp][1] = io; s_w[warp][4] = ii; }
    if (lane == 0) { s_w[warp][2] = st; s_w[warp][3] = sp; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0, c = 0, t = 0, q = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const unsigned long long x = s_w[w][0], y = s_w[w][1], z = s_w[w][4];
            t += s_w[w][2];
            q += s_w[w][3];
            s_w[w][0] = a;
            s_w[w][1] = b;
            s_w[w][4] = c;
            a += x;
            b += y;
            c += z;
        }
        s_tot[0] = a; s_tot[1] = b; s_tot[2] = t; s_tot[3] = q; s_tot[4] = c;
    }
    __syncthreads();
    unsigned long long ru = s_w[warp][0] + iu - u, ro = s_w[warp][1] + io - o, ri = s_w[warp][4] + ii - it;
    for (unsigned p = b0; p < b1; ++p) {
        unsigned s, len;
        par.range(p, s, len);
        const unsigned nch = (len + 31) >> 5;
        const unsigned nc = par.nchild(p);
        sb.ubase[p] = (unsigned)ru;
        sb.obase[p] = (unsigned)ro;
        sb.ibase[p] = (unsigned)ri;
        ru += nch;
        ro += (unsigned long long)nc * nch;
        ri += (unsigned long long)nc * ((nch + WORD_SEG - 1) / WORD_SEG);
    }
    if (threadIdx.x == 0) {
        sb.ubase[n] = (unsigned)s_tot[0];
        sb.obase[n] = (unsigned)s_tot[1];
        sb.ibase[n] = (unsigned)s_tot[4];
        sb.totals[0] = (unsigned)s_tot[0];
        sb.totals[1] = (unsigned)s_tot[1];
        sb.totals[2] = (unsigned)s_tot[4];
        ctr->tests[level_idx] = s_tot[2];
        ctr->tests_paper[level_idx] = B_paper ? (unsigned long long)B_paper * s_tot[3] : s_tot[3];
    }
}

// last p with base[p] <= u (base non-decreasing, base[0] = 0)
__device__ __forceinline__ unsigned find_parent(const unsigned* base, unsigned n, unsigned u) {
    unsigned lo = 0, hi = n - 1;
    while (lo < hi) {
        const unsigned mid = lo + (hi - lo + 1) / 2;
        if (base[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Position in the unit list: the parent p owning the current unit, its
// triangle run [s, s + len), its first unit ub and first ballot word ob.
template <class Parents>
struct UnitCursor {
    unsigned p, next, s, len, ub, ob;
    __device__ __forceinline__ void enter(const Parents& par, const StageBuf& sb) {
        next = sb.ubase[p + 1];
        ub = sb.ubase[p];
        ob = sb.obase[p];
        par.range(p, s, len);
    }
    __device__ __forceinline__ void start(const Parents& par, const StageBuf& sb, unsigned u) {
        p = find_parent(sb.ubase, par.count(), u);
        enter(par, sb);
    }
    // u must be below the unit total (parents without triangles own no units)
    __device__ __forceinline__ void seek(const Parents& par, const StageBuf& sb, unsigned u) {
        while (u >= next) {
            ++p;
            enter(par, sb);
        }
    }
    // this lane's triangle of unit u (0 when past the parent's run)
    __device__ __forceinline__ unsigned tri(const Parents& par, unsigned u, bool& valid) const {
        const unsigned j = ((u - ub) << 5) + (threadIdx.x & 31);
        valid = j < len;
        return valid ? par.tri(s, j) : 0u;
    }
    // the same with an in-range load for every lane (the run is not empty); the
    // caller masks the lanes that are not valid
    __device__ __forceinline__ unsigned tri_any(const Parents& par, unsigned u, bool& valid) const {
        const unsigned j = ((u - ub) << 5) + (threadIdx.x & 31);
        valid = j < len;
        return par.tri(s, valid ? j : 0u);
    }
};

// Work split of a count or emit pass.  With at least dyn_min units per warp
// the units are handed out in batches from an atomic counter (the cost of a
// unit depends on how many children accept it), about four batches per warp
// and at most COUNT_BATCH / EMIT_BATCH units each; a warp claims the batch after the
// current one when it starts a batch, so the claim's latency is hidden.  With
// fewer, each warp takes one contiguous range (no atomics: at a few units per
// warp the claims themselves would dominate).  The position (cursor, unit u,
// batch end e) advances one unit at a time.  All calls are warp-uniform.
constexpr unsigned COUNT_BATCH = 24;  // units per claim of the count pass (of 8, 16, 24, 32: 24 measured best on the 1024x1024 frame)
constexpr unsigned EMIT_BATCH = 16;   // units per claim of the emit pass (of 8, 16, 32: 16 measured best on the 1024x1024 frame)

struct WorkSplit {
    unsigned U, nw, per, batch;   // per = 0: claimed batches; else the static range length
    unsigned* work;
    __device__ __forceinline__ WorkSplit(unsigned U_, unsigned* work_, unsigned dyn_min, unsigned max_batch)
        : U(U_), work(work_) {
        nw = gridDim.x * (blockDim.x >> 5);
        per = (U >= dyn_min * nw) ? 0u : (U + nw - 1) / nw;
        batch = max(1u, min(max_batch, U / (4u * nw)));
    }
    // first claim: the warp's own index for a static split
    __device__ __forceinline__ unsigned first_claim() const {
        if (per) return (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        return ((threadIdx.x & 31) == 0) ? atomicAdd(work, 1u) : 0u;
    }
};

template <class Parents>
struct UnitStream {
    UnitCursor<Parents> c;
    unsigned u, e;
    __device__ __forceinline__ bool take(const Parents& par, const StageBuf& sb, const WorkSplit& ws,
                                         unsigned& claim) {
        const unsigned b = __shfl_sync(FULL, claim, 0);
        if (ws.per) {
            if (b >= ws.nw) return false;
            u = b * ws.per;
            if (u >= ws.U) return false;
            e = min(ws.U, u + ws.per);
            claim = ws.nw;   // one range per warp
        } else {
            if (b >= (ws.U + ws.batch - 1) / ws.batch) return false;
            if ((threadIdx.x & 31) == 0) claim = atomicAdd(ws.work, 1u);
            u = b * ws.batch;
            e = min(ws.U, u + ws.batch);
        }
        c.start(par, sb, u);
        return true;
    }
    __device__ __forceinline__ bool step(const Parents& par, const StageBuf& sb, const WorkSplit& ws,
                                         unsigned& claim) {
        if (u + 1 < e) {
            ++u;
            c.seek(par, sb, u);
            return true;
        }
        return take(par, sb, ws, claim);
    }
};

__device__ __forceinline__ float warp_min_f(float v) {
    float r;
    asm("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float warp_max_f(float v) {
    float r;
    asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// Bounding sphere of the chunk's triangle spheres (warp-uniform): centre the
// middle of the centres' bounding box, radius the largest |c_i - K| + r_i,
// padded outward like a triangle sphere (FP32 rounding of this radius and of
// the eq. 9 evaluation), so the exact sphere contains every triangle sphere.
__device__ __forceinline__ float4 chunk_sphere(float4 ts, bool valid) {
    const float inf = __int_as_float(0x7f800000);
    const float lx = warp_min_f(valid ? ts.x : inf), hx = warp_max_f(valid ? ts.x : -inf);
    const float ly = warp_min_f(valid ? ts.y : inf), hy = warp_max_f(valid ? ts.y : -inf);
    const float lz = warp_min_f(valid ? ts.z : inf), hz = warp_max_f(valid ? ts.z : -inf);
    const float kx = 0.5f * (lx + hx), ky = 0.5f * (ly + hy), kz = 0.5f * (lz + hz);
    const float dx = ts.x - kx, dy = ts.y - ky, dz = ts.z - kz;
    float R = warp_max_f(valid ? sqrtf(dx * dx + dy * dy + dz * dz) + ts.w : 0.f);
    const float mag = fabsf(kx) + fabsf(ky) + fabsf(kz) + R;
    R = R * (1.0f + 9.6e-7f) + 3.9e-6f * mag;
    return make_float4(kx, ky, kz, R);
}

// Count pass: one 32-bit ballot per (child, chunk): eq. 9 for 32 triangles.
// Software-pipelined over the warp's units: the triangle index of unit u+2
// and the triangle sphere of unit u+1 are in flight while unit u is tested.
// Below the top level, lane c first tests child c against the chunk's
// bounding sphere: eq. 9 is an exact sphere-against-region test, so a child
// that rejects the bounding sphere rejects every triangle sphere inside it
// (its word is 0) and only the children that accept it run the 32-lane tests.
// 1024 threads per SM (64 registers): at 1536 threads (40 registers) the
// pipeline's state spilled and the pass ran 2-3 % slower.
template <class Parents, int BLK, bool WIDE>
__global__ void __launch_bounds__(BLK, 1024 / BLK) k_count(Parents par, StageBuf sb, const float4* tri_sphere,
                                                          unsigned long long* popsum) {
    constexpr int NCH = WIDE ? 64 : 32;   // child slots per warp
    // the tested parent's children, copied when the parent changes
    __shared__ float4 s_sp[BLK / 32][NCH], s_co[BLK / 32][NCH];
    __shared__ float2 s_tg[BLK / 32][NCH];
    pdl_wait();
    const WorkSplit ws(sb.totals[0], sb.work + 0, 16u, COUNT_BATCH);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned claim = ws.first_claim();
    // one cursor leads two units ahead of the tested one; the units in flight keep only
    // their parent, first ballot word and the parent's triangle count
    UnitStream<Parents> lead;
    if (!lead.take(par, sb, ws, claim)) return;
    struct Slot {
        unsigned p, wo, len;
    };
    auto slot_of = [&]() { return Slot{lead.c.p, lead.c.ob + (lead.u - lead.c.ub), lead.c.len}; };
    // the tested unit's parent: its children (set when the parent changes)
    unsigned cur_p = 0xffffffffu, nc = 0;
    unsigned long long accepted = 0;   // pairs accepted by this warp (word form's level count)
    const float4* csp = s_sp[warp];
    const float4* cco = s_co[warp];
    const float2* ctg = s_tg[warp];
    // three units in flight in rotating slot sets A, B, C: the loop is unrolled three times so
    // that no slot is copied (STEP(X, Y, Z): test unit X, fetch unit Y's sphere, unit Z's index)
    Slot sA = slot_of(), sB = sA, sC = sA;
    bool vA = false, vB = false, vC = false, hB = false, hC = false;
    float4 tsA = zero, tsB = zero, tsC = zero;
    unsigned tB = 0, tC = 0;
    {
        const unsigned t0 = lead.c.tri_any(par, lead.u, vA);
        tsA = tri_sphere[vA ? t0 : 0u];
    }
    hB = lead.step(par, sb, ws, claim);
    if (hB) {
        sB = slot_of();
        tB = lead.c.tri_any(par, lead.u, vB);
    }
    (void)tsC; (void)tC; (void)hC; (void)vC;
#define CRSH_TEST_UNIT(S0, V0, TS0)                                                          \
    {                                                                                        \
        if (S0.p != cur_p) {                                                                 \
            cur_p = S0.p;                                                                    \
            nc = par.nchild(cur_p);                                                          \
            const unsigned a0 = par.child_id(cur_p, 0);                                      \
            __syncwarp();                                                                    \
            for (unsigned cl = lane; cl < nc; cl += 32) {                                    \
                s_sp[warp][cl] = par.child.sphere[a0 + cl];                                  \
                s_co[warp][cl] = par.child.cone[a0 + cl];                                    \
                s_tg[warp][cl] = par.child.trig[a0 + cl];                                    \
            }                                                                                \
            __syncwarp();                                                                    \
        }                                                                                    \
        const unsigned nch = (S0.len + 31) >> 5;                                             \
        unsigned* mw = sb.mask + S0.wo;                                                      \
        if (Parents::kChunkCull) {                                                           \
            const float4 K = chunk_sphere(TS0, V0);                                          \
            _Pragma("unroll") for (unsigned cb = 0; cb < (WIDE ? 64u : 32u); cb += 32) {     \
                const unsigned cl = cb + lane;                                               \
                const bool mine = cl < nc;                                                   \
                const bool acc = WIDE ? (mine && eq9(csp[cl], cco[cl], ctg[cl], K)) : (mine & eq9(csp[cl], cco[cl], ctg[cl], K));                  \
                if (mine && !acc) mw[cl * nch] = 0u;                                         \
                unsigned todo = __ballot_sync(FULL, acc);                                    \
                while (todo) {                                                               \
                    const unsigned c = cb + __ffs(todo) - 1;                                 \
                    todo &= todo - 1;                                                        \
                    const bool ok = V0 & eq9(csp[c], cco[c], ctg[c], TS0);                   \
                    const unsigned m = __ballot_sync(FULL, ok);                              \
                    mw[c * nch] = m;                                                         \
                    accepted += __popc(m);                                                   \
                }                                                                            \
            }                                                                                \
        } else {                                                                             \
            _Pragma("unroll 4") for (unsigned c = 0; c < nc; ++c) {                          \
                const bool ok = V0 & eq9(csp[c], cco[c], ctg[c], TS0);                       \
                const unsigned m = __ballot_sync(FULL, ok);                                  \
                mw[c * nch] = m;                                                             \
                accepted += __popc(m);                                                       \
            }                                                                                \
        }                                                                                    \
    }
#define CRSH_COUNT_STEP(X, Y, Z)                                                             \
    {                                                                                        \
        ts##Y = tri_sphere[v##Y ? t##Y : 0u];                                                \
        h##Z = false;                                                                        \
        v##Z = false;                                                                        \
        t##Z = 0;                                                                            \
        if (h##Y) {                                                                          \
            h##Z = lead.step(par, sb, ws, claim);                                            \
            if (h##Z) {                                                                      \
                s##Z = slot_of();                                                            \
                t##Z = lead.c.tri_any(par, lead.u, v##Z);                                        \
            }                                                                                \
        }                                                                                    \
        CRSH_TEST_UNIT(s##X, v##X, ts##X)                                                    \
        if (!h##Y) break;                                                                    \
    }
    bool hA = false;
    unsigned tA = 0;
    for (;;) {
        CRSH_COUNT_STEP(A, B, C)
        CRSH_COUNT_STEP(B, C, A)
        CRSH_COUNT_STEP(C, A, B)
    }
#undef CRSH_COUNT_STEP
#undef CRSH_TEST_UNIT
    if (popsum && lane == 0 && accepted) atomicAdd(popsum, accepted);
}

constexpr int SC_BLOCK = 256, SC_ITEMS = 8, SC_TILE = SC_BLOCK * SC_ITEMS, SC_GRID_MAX = 2048;

__device__ __forceinline__ void block_range(unsigned O, unsigned& w0, unsigned& w1) {
    const unsigned per = (((O + gridDim.x - 1) / gridDim.x) + SC_TILE - 1) / SC_TILE * SC_TILE;
    w0 = min(O, blockIdx.x * per);
    w1 = min(O, w0 + per);
}

// Accepted pairs per scan block (contiguous ranges of ballot words; ranges
// start on multiples of SC_TILE words, so 16-byte loads are aligned).
__global__ void __launch_bounds__(SC_BLOCK) k_reduce(StageBuf sb) {
    pdl_wait();
    const unsigned O = sb.totals[1];
    unsigned w0, w1;
    block_range(O, w0, w1);
    unsigned c = 0;
    const unsigned w1v = w0 + ((w1 - w0) & ~3u);
    for (unsigned w = w0 + 4 * threadIdx.x; w < w1v; w += 4 * blockDim.x) {
        const uint4 m = *reinterpret_cast<const uint4*>(sb.mask + w);
        c += __popc(m.x) + __popc(m.y) + __popc(m.z) + __popc(m.w);
    }
    for (unsigned w = w1v + threadIdx.x; w < w1; w += blockDim.x) c += __popc(sb.mask[w]);
    c = __reduce_add_sync(FULL, c);
    __shared__ unsigned s_w[SC_BLOCK / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int i = 0; i < SC_BLOCK / 32; ++i) t += s_w[i];
        sb.bsum[blockIdx.x] = t;
    }
}

// Exclusive prefix of the ballot popcounts: pos[w] = output index of the first
// pair of word w; pos[O] = total; the stage's pair count and counters.
__global__ void __launch_bounds__(SC_BLOCK) k_wordscan(StageBuf sb, PairOut out, crsh_counters* ctr,
                                                       int level_idx) {
    pdl_wait();
    __shared__ unsigned long long s_pre;
    __shared__ unsigned s_w[SC_BLOCK / 32 + 1];
    const unsigned O = sb.totals[1];
    unsigned w0, w1;
    block_range(O, w0, w1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        unsigned long long a = 0;
        for (unsigned b = threadIdx.x; b < blockIdx.x; b += blockDim.x) a += sb.bsum[b];
        a = warp_sum64(a);
        __shared__ unsigned long long s_a[SC_BLOCK / 32];
        if (lane == 0) s_a[warp] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int i = 0; i < SC_BLOCK / 32; ++i) t += s_a[i];
            s_pre = t;
        }
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        const unsigned long long total = s_pre + sb.bsum[blockIdx.x];
        sb.pos[O] = (unsigned)total;
        finish_pairs(out, total, ctr, level_idx);
    }
    unsigned long long run = s_pre;
    for (unsigned t0 = w0; t0 < w1; t0 += SC_TILE) {
        const unsigned wb = t0 + threadIdx.x * SC_ITEMS;   // blocked: consecutive words per thread
        unsigned c[SC_ITEMS], sum = 0;
        if (wb + SC_ITEMS <= w1) {   // aligned: wb is a multiple of 8 words
            const uint4 a = *reinterpret_cast<const uint4*>(sb.mask + wb);
            const uint4 b = *reinterpret_cast<const uint4*>(sb.mask + wb + 4);
            c[0] = __popc(a.x); c[1] = __popc(a.y); c[2] = __popc(a.z); c[3] = __popc(a.w);
            c[4] = __popc(b.x); c[5] = __popc(b.y); c[6] = __popc(b.z); c[7] = __popc(b.w);
        } else {
#pragma unroll
            for (int i = 0; i < SC_ITEMS; ++i) c[i] = (wb + i < w1) ? __popc(sb.mask[wb + i]) : 0u;
        }
#pragma unroll
        for (int i = 0; i < SC_ITEMS; ++i) sum += c[i];
        const unsigned inc = warp_incl_scan(sum);
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned a = 0;
            for (int i = 0; i < SC_BLOCK / 32; ++i) { const unsigned x = s_w[i]; s_w[i] = a; a += x; }
            s_w[SC_BLOCK / 32] = a;
        }
        __syncthreads();
        unsigned long long r = run + s_w[warp] + inc - sum;
        unsigned pv[SC_ITEMS];
#pragma unroll
        for (int i = 0; i < SC_ITEMS; ++i) {
            pv[i] = (unsigned)r;
            r += c[i];
        }
        if (wb + SC_ITEMS <= w1) {
            *reinterpret_cast<uint4*>(sb.pos + wb) = make_uint4(pv[0], pv[1], pv[2], pv[3]);
            *reinterpret_cast<uint4*>(sb.pos + wb + 4) = make_uint4(pv[4], pv[5], pv[6], pv[7]);
        } else {
#pragma unroll
            for (int i = 0; i < SC_ITEMS; ++i)
                if (wb + i < w1) sb.pos[wb + i] = pv[i];
        }
        run += s_w[SC_BLOCK / 32];
        __syncthreads();
    }
}

// Emit pass: the count pass's walk again; each set ballot bit becomes a
// (child, triangle) pair at pos[word] + rank.  Unit (p, 0) also records the
// children's runs [start, end).  The triangle index and the children's words
// of the next unit are loaded while the current unit is written.
template <class Parents, int G>
struct EmitLoads {
    // triangle; per group of 32 children, child `lane`'s mask and position and
    // its run end (first chunk); G = 2 groups only when B = 64
    unsigned t, mc[G], pc[G], pe[G];
    __device__ __forceinline__ void load(const Parents& par, const StageBuf& sb, const UnitStream<Parents>& q) {
        const int lane = threadIdx.x & 31;
        bool valid;
        t = q.c.tri(par, q.u, valid);
        const unsigned nch = (q.c.len + 31) >> 5, nc = par.nchild(q.c.p), ch = q.u - q.c.ub;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const unsigned cl = 32u * g + lane;
            mc[g] = pc[g] = pe[g] = 0;
            if (cl < nc) {
                const unsigned w = q.c.ob + cl * nch + ch;
                mc[g] = sb.mask[w];
                pc[g] = sb.pos[w];
                if (ch == 0) pe[g] = sb.pos[q.c.ob + (cl + 1) * nch];
            }
        }
    }
};

template <class Parents, int BLK, bool WIDE>
__global__ void __launch_bounds__(BLK) k_emit(Parents par, StageBuf sb, PairOut out, RunOut runs) {
    constexpr int G = WIDE ? 2 : 1;
    pdl_wait();
    const WorkSplit ws(sb.totals[0], sb.work + 1, 32u, EMIT_BATCH);
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    unsigned claim = ws.first_claim();
    UnitStream<Parents> p0;
    if (!p0.take(par, sb, ws, claim)) return;
    EmitLoads<Parents, G> l0, l1;
    l0.load(par, sb, p0);
    UnitStream<Parents> p1 = p0;
    bool has1 = p1.step(par, sb, ws, claim);
    for (;;) {
        if (has1) l1.load(par, sb, p1);
        UnitStream<Parents> p2 = p1;
        bool has2 = false;
        if (has1) has2 = p2.step(par, sb, ws, claim);
        const UnitCursor<Parents>& c0 = p0.c;
        const unsigned nc = par.nchild(c0.p), ch = p0.u - c0.ub;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            unsigned any = __ballot_sync(FULL, l0.mc[g] != 0);
            while (any) {
                const int c = __ffs(any) - 1;
                any &= any - 1;
                const unsigned m = __shfl_sync(FULL, l0.mc[g], c);
                const unsigned base = __shfl_sync(FULL, l0.pc[g], c);
                // predicated stores (no branch): this lane's bit, inside the list's capacity
                const unsigned long long pos = base + __popc(m & lt);
                const bool wr = ((m >> lane) & 1u) && pos < out.cap;
                if (wr) out.tri[pos] = l0.t;
                if (out.node && wr) out.node[pos] = par.child_id(c0.p, 32 * g + c);
            }
            const unsigned cl = 32u * g + lane;
            if (ch == 0 && cl < nc) {
                // runs index the written list: clamp to its capacity (a list
                // that overflowed is truncated and flagged CRSH_ERR_CAPACITY)
                const unsigned a = par.child_id(c0.p, cl);
                if (par.first_of_child(c0.p, cl)) runs.start[a] = (unsigned)min((unsigned long long)l0.pc[g], out.cap);
                if (par.last_of_child(c0.p, cl)) runs.end[a] = (unsigned)min((unsigned long long)l0.pe[g], out.cap);
            }
        }
        if (!has1) break;
        p0 = p1;
        l0 = l1;
        p1 = p2;
        has1 = has2;
    }
}

// Word form of level 1: one descriptor per final-test work item (level-2
// node p, child c, segment s of WORD_SEG chunks), written at item_base[p] +
// c * segments + s: (level-1 node, position in the parent list of the
// segment's first chunk, index of its first ballot word, word count).  One
// warp per parent.
__global__ void k_items(LevelParents par, StageBuf sb, uint4* items) {
    pdl_wait();
    const unsigned n = par.count(), cc = *par.n_child;
    const unsigned lane = threadIdx.x & 31;
    for (unsigned p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += (gridDim.x * blockDim.x) >> 5) {
        unsigned s, len;
        par.range(p, s, len);
        const unsigned nch = (len + 31) >> 5, nseg = (nch + WORD_SEG - 1) / WORD_SEG;
        const unsigned first = p << par.logB;
        const unsigned nc = first >= cc ? 0u : min(1u << par.logB, cc - first);
        const unsigned ob = sb.obase[p], ib = sb.ibase[p];
        // item j = c * nseg + g of the parent: consecutive lanes write consecutive descriptors
        for (unsigned j = lane; j < nc * nseg; j += 32) {
            const unsigned c = j / nseg, g = j - c * nseg;
            const unsigned k = g * WORD_SEG;
            items[ib + j] = make_uint4(first + c, s + 32 * k, ob + c * nch + k, min(WORD_SEG, nch - k));
        }
    }
}

// CSR offsets (n + 1) of the node-sorted level-1 list: a node's offset is the
// start of its run; a node without pairs takes the start of the next node
// with pairs (the list end if none).  A few steps forward over the runs find
// it in the common case; longer gaps fall back to a binary search of the node
// column.
__global__ void k_runs_to_csr(RunOut runs, const uint32_t* node, const unsigned* n_count, const unsigned* p_count,
                              unsigned long long cap, uint32_t* off) {
    pdl_wait();
    const unsigned n = *n_count;
    const unsigned total = (unsigned)min((unsigned long long)*p_count, cap);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x) {
        unsigned o = total;
        bool found = false;
        for (unsigned q = k; q < n && q < k + 8; ++q) {
            if (runs.end[q] > runs.start[q]) {
                o = runs.start[q];
                found = true;
                break;
            }
        }
        if (!found && k + 8 < n) {   // first pair whose node >= k
            unsigned lo = 0, hi = total;
            while (lo < hi) {
                const unsigned mid = (lo + hi) >> 1;
                if (node[mid] < k) lo = mid + 1; else hi = mid;
            }
            o = lo;
        }
        off[k] = o;
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
    uint32_t* bufT[2];                   // ping-pong pair lists (triangles) of the levels above 1
    uint4* items;                        // word form of level 1: work item descriptors
    uint32_t *mpN, *mpM;                 // accepted (node, mesh)
    RunOut runs[CRSH_MAX_LEVELS];        // pair runs per level
    StageBuf sb;
    char* ctl;                           // zeroed per call: counts, counters, runs
    size_t ctl_bytes;
    unsigned* counts;                    // [0] mesh pairs, [1 + l] pairs of level l+1
    unsigned* work;                      // 2 per stage (count, emit): claimed unit batches
    unsigned* tile_ctr;
    unsigned long long* st_mesh;
    size_t total;
};

TvWs carve_tv(void* ws, const crsh_hierarchy* h, uint32_t n_tris, uint32_t n_meshes, uint64_t cap) {
    Carve c{reinterpret_cast<char*>(ws)};
    TvWs w{};
    const unsigned L = h->levels, B = h->bundle;
    const uint64_t top_cap = h->capacity[L - 1];
    const size_t mp = (size_t)top_cap * (n_meshes ? n_meshes : 1);
    if (L > 1) {
        for (int k = 0; k < 2; ++k) w.bufT[k] = c.take<uint32_t>(cap);
    }
    w.mpN = c.take<uint32_t>(mp);
    w.mpM = c.take<uint32_t>(mp);
    size_t max_parents = mp, max_words = (size_t)(top_cap * (uint64_t)n_tris / 32) + mp;
    for (unsigned l = 1; l < L; ++l) {
        max_parents = std::max(max_parents, (size_t)h->capacity[l]);
        max_words = std::max(max_words, (size_t)B * ((size_t)(cap / 32) + h->capacity[l]));
    }
    w.sb.ubase = c.take<unsigned>(max_parents + 1);
    w.sb.obase = c.take<unsigned>(max_parents + 1);
    w.sb.ibase = c.take<unsigned>(max_parents + 1);
    // word form: an item covers at most WORD_SEG words and every (parent, child) row starts one
    w.items = c.take<uint4>(max_words / WORD_SEG + (size_t)B * max_parents + 1);
    w.sb.totals = c.take<unsigned>(4);
    w.sb.mask = c.take<unsigned>(max_words + 1);
    w.sb.pos = c.take<unsigned>(max_words + 1);
    w.sb.bsum = c.take<unsigned>(SC_GRID_MAX);
    c.off = (c.off + 255) & ~size_t(255);
    const size_t ctl0 = c.off;
    w.counts = c.take<unsigned>(CRSH_MAX_LEVELS + 2);
    w.work = c.take<unsigned>(2 * (CRSH_MAX_LEVELS + 1));
    w.tile_ctr = c.take<unsigned>(4);
    w.st_mesh = c.take<unsigned long long>(mp / TV_TILE + 2);
    for (unsigned l = 0; l < L; ++l) {
        w.runs[l].start = c.take<unsigned>((size_t)h->capacity[l] + 1);
        w.runs[l].end = c.take<unsigned>((size_t)h->capacity[l] + 1);
    }
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

// Blocks of a kernel resident on one SM (cached per kernel and device).
template <class K>
static unsigned resident_blocks(K kernel, int block, const DeviceInfo& dev) {
    static std::atomic<int> per_sm[64];
    const int d = (dev.device >= 0 && dev.device < 64) ? dev.device : 0;
    int b = per_sm[d].load(std::memory_order_relaxed);
    if (b <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, block, 0) != cudaSuccess || b <= 0) b = 1;
        per_sm[d].store(b, std::memory_order_relaxed);
    }
    return (unsigned)b;
}

// stage: 0 = top level, then 1, 2, ... for levels L-1, L-2, ...  BLK: threads
// per block of the count and emit passes (a tuning knob: the passes claim
// their work from counters, so results do not depend on it).
template <int BLK, bool WIDE, class Parents>
static void run_stage(const Parents& par, const TvWs& w, unsigned stage, const float4* tsph, PairOut out,
                      RunOut runs, crsh_counters* ctr, int level_idx, unsigned B_paper, const DeviceInfo& dev,
                      cudaStream_t s, bool words_only = false) {
    StageBuf sb = w.sb;
    sb.work = w.work + 2 * stage;
    const unsigned sg = std::min<unsigned>(SC_GRID_MAX, dev.sms * 8);
    // persistent grids: the count and emit passes claim unit batches
    const unsigned gc = dev.sms * resident_blocks(k_count<Parents, BLK, WIDE>, BLK, dev);
    const unsigned ge = dev.sms * resident_blocks(k_emit<Parents, BLK, WIDE>, BLK, dev);
    launch_pdl(k_unit_scan<Parents>, 1, 1024, 0, s, par, sb, ctr, level_idx, B_paper);
    // word form (level 1 only): the ballots are the output, their popcounts the level's count
    launch_pdl(k_count<Parents, BLK, WIDE>, gc, BLK, 0, s, par, sb, tsph,
               words_only ? &ctr->hits[level_idx] : (unsigned long long*)nullptr);
    if (words_only) {
        if constexpr (std::is_same<Parents, LevelParents>::value)
            launch_pdl(k_items, dev.sms * 8, 256, 0, s, par, sb, w.items);
        return;
    }
    launch_pdl(k_reduce, sg, SC_BLOCK, 0, s, sb);
    launch_pdl(k_wordscan, sg, SC_BLOCK, 0, s, sb, out, ctr, level_idx);
    launch_pdl(k_emit<Parents, BLK, WIDE>, ge, BLK, 0, s, par, sb, out, runs);
}

crsh_status traverse_launch(const crsh_hierarchy* h, const crsh_scene* sc, const crsh_traverse_params* tp,
                            crsh_pairs* out, crsh_counters* ctr, void* ws, size_t ws_bytes, cudaStream_t s,
                            const DeviceInfo& dev) {
    const unsigned L = h->levels, B = h->bundle, logB = log2u(B);
    const uint64_t cap = out->capacity;
    if (ws_bytes < traverse_workspace(h, sc->n_tris, sc->n_meshes, cap)) return CRSH_ERR_INVALID_ARG;
    TvWs w = carve_tv(ws, h, sc->n_tris, sc->n_meshes, cap);
    {   // the control region, and this call's counters: mesh_tests .. tests_paper, and needed_pairs
        char* c0 = reinterpret_cast<char*>(&ctr->mesh_tests);
        char* c1 = reinterpret_cast<char*>(&ctr->final_tests);
        zero_launch(ZeroSpans{{w.ctl, c0, &ctr->needed_pairs}, {w.ctl_bytes, (size_t)(c1 - c0), sizeof(unsigned long long)}},
                    s, dev);
    }
    auto level_nodes = [&](unsigned l) {   // l = 1..L
        return Node3{reinterpret_cast<const float4*>(h->sphere[l - 1]), reinterpret_cast<const float4*>(h->cone[l - 1]),
                     reinterpret_cast<const float2*>(h->trig[l - 1])};
    };
    const float4* tsph = reinterpret_cast<const float4*>(sc->tri_sphere);
    // level 1's node column is the output; the levels above keep only
    // triangles (the next level finds a node's triangles by its run)
    auto pairs_of = [&](unsigned l) {
        if (l == 1) return PairOut{out->node, out->tri, out->count, cap};
        return PairOut{nullptr, w.bufT[l & 1], &w.counts[1 + l], cap};
    };
    // mesh stage: (top node, mesh)
    MeshOp mop{level_nodes(L), h->count + (L - 1), reinterpret_cast<const float4*>(sc->mesh_sphere),
               sc->mesh_first_tri, sc->n_meshes, (int)tp->mesh_cull,
               PairOut{w.mpN, w.mpM, &w.counts[0], (unsigned long long)h->capacity[L - 1] * sc->n_meshes}, ctr};
    launch_pdl(k_compact<MeshOp>, dev.sms * 2, TV_BLOCK, 0, s, mop, TvCtl{w.st_mesh, &w.tile_ctr[0], ctr, -1});
    // top level: triangles of the accepted meshes
    TopParents top{w.mpN, w.mpM, &w.counts[0], sc->mesh_first_tri, level_nodes(L)};
    // the block shape, and for the level stages whether a parent has more
    // than 32 children (B = 64); the top stage has one child per parent
    auto stage = [&](const auto& par, unsigned st, PairOut o, RunOut rn, int li, unsigned Bp, auto wide,
                     bool words_only) {
        constexpr bool W = decltype(wide)::value;
        switch (tp->block_threads) {
            case 128: run_stage<128, W>(par, w, st, tsph, o, rn, ctr, li, Bp, dev, s, words_only); break;
            case 512: run_stage<512, W>(par, w, st, tsph, o, rn, ctr, li, Bp, dev, s, words_only); break;
            default: run_stage<256, W>(par, w, st, tsph, o, rn, ctr, li, Bp, dev, s, words_only); break;
        }
    };
    const bool words = tp->level1_words != 0 && L >= 2;
    out->words = crsh_pair_words{};
    stage(top, 0u, pairs_of(L), w.runs[L - 1], (int)L - 1, 0u, std::false_type{}, false);
    // levels L-1 .. 1: parents are the nodes of level l+1 and their pair runs
    for (unsigned l = L - 1; l >= 1; --l) {
        PairOut par = pairs_of(l + 1);
        LevelParents lp{par.tri, w.runs[l].start, w.runs[l].end, h->count + l, h->count + (l - 1), level_nodes(l), logB};
        const bool wo = words && l == 1;
        if (B > 32)
            stage(lp, L - l, pairs_of(l), w.runs[l - 1], (int)l - 1, B, std::true_type{}, wo);
        else
            stage(lp, L - l, pairs_of(l), w.runs[l - 1], (int)l - 1, B, std::false_type{}, wo);
        if (wo) {   // level 1 stays in the ballots of its count pass
            out->words = crsh_pair_words{w.sb.mask, par.tri, reinterpret_cast<const uint32_t*>(w.items),
                                         w.sb.totals + 2, 1u, 0u};
        }
        if (l == 1) break;
    }
    if (!words) {
        const unsigned blocks = (h->capacity[0] + 256) / 256;
        launch_pdl(k_runs_to_csr, std::min<unsigned>(blocks, dev.sms * 8), 256, 0, s, w.runs[0], out->node,
                   (const unsigned*)h->count, (const unsigned*)out->count, cap, out->node_offsets);
    }
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

}  // namespace crsh
