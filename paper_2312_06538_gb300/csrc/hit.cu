// Section 3.3.8: final ray-triangle tests (Moller-Trumbore [Mol97]) over the
// level-1 (node, triangle) pairs, closest hit per ray; and the N x M brute
// force of Section 1 built on the same test, for comparison.
//
// GB300 design.  Warps claim fixed chunks of the node-sorted pair list from a
// counter, so long and short triangle lists balance across the 152 SMs, and
// walk them in groups of up to 32 pairs of one node.  In a warp, lane =
// (ray slot r < B/2, stream s < 64/B): each lane holds two of the node's rays
// (slots r and r + B/2) in registers; a group's triangle records (64 bytes
// each, L2-resident) are copied into shared memory while the previous group
// is tested, and each stream walks every (64/B)-th triangle against both of
// its rays.  Every candidate first gets a ray-line vs triangle-sphere
// pre-test (paired FP32 operations, two rays per instruction); the few
// survivors run Moller-Trumbore.  The per-ray best is a packed (t bits,
// triangle id) 64-bit key, reduced across streams by shuffles and published
// with one atomicMin per ray per node run, so the result does not depend on
// scheduling.  A last pass recomputes (t, u, v) of each ray's winning
// triangle and scatters hits to the rays' generation order.  Decisions
// (which triangle is closest) are FP32; the reported (t, u, v) of the winner
// are recomputed in double-word (float + float) arithmetic from the FP32
// inputs.  With level 1 in word form (crsh_pair_words) the groups are gathered
// from the traversal's ballots instead (k_closest_words) and run the same
// group test.
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace crsh {

// Moller-Trumbore in FP32 with an explicit operation sequence (fused
// multiply-adds written out), so every kernel that calls it gets the same
// bits.  Cramer's rule for o + t d = a + u e1 + v e2 with the triangle normal
// n = e1 x e2 precomputed: D = -(d.n), t = (s.n)/D, u = (e2.q)/D,
// v = -(e1.q)/D with s = o - a and q = s x d (21 FP32 operations).  The
// numerators are compared against |D| after folding D's sign into them, so no
// reciprocal is needed; the one division t = t'/|D| happens only on a hit.
// Two-sided, inclusive edges, 0 < t <= t_max, D == 0 never hits.
// Triangle record: (a.xyz, n.x), (e1.xyz, n.y), (e2.xyz, n.z).
__device__ __forceinline__ bool mt_hit(float ox, float oy, float oz, float dx, float dy, float dz, float tmax,
                                       float4 A, float4 E1, float4 E2, float& t) {
    const float dn = __fmaf_rn(dx, A.w, __fmaf_rn(dy, E1.w, __fmul_rn(dz, E2.w)));   // d.n = -D
    const float sx = __fsub_rn(ox, A.x), sy = __fsub_rn(oy, A.y), sz = __fsub_rn(oz, A.z);
    const float qx = __fmaf_rn(sy, dz, __fmul_rn(-sz, dy));
    const float qy = __fmaf_rn(sz, dx, __fmul_rn(-sx, dz));
    const float qz = __fmaf_rn(sx, dy, __fmul_rn(-sy, dx));
    const float tn = __fmaf_rn(sx, A.w, __fmaf_rn(sy, E1.w, __fmul_rn(sz, E2.w)));     // s.n
    const float un = __fmaf_rn(E2.x, qx, __fmaf_rn(E2.y, qy, __fmul_rn(E2.z, qz)));    // e2.q
    const float wn = __fmaf_rn(E1.x, qx, __fmaf_rn(E1.y, qy, __fmul_rn(E1.z, qz)));    // e1.q = -v D
    // sign of D = -dn: fold it into t' = s.n, u' = e2.q and v' = -(e1.q)
    const unsigned sgD = (__float_as_uint(dn) & 0x80000000u) ^ 0x80000000u;
    const float u = __uint_as_float(__float_as_uint(un) ^ sgD);
    const float v = __uint_as_float(__float_as_uint(wn) ^ sgD ^ 0x80000000u);
    const float tp = __uint_as_float(__float_as_uint(tn) ^ sgD);
    const float ad = fabsf(dn);
    // (|D| = 0 cannot pass: tp > 0 and tp <= t_max |D| exclude it, 0 * inf being NaN)
    const bool hit = (u >= 0.0f) & (v >= 0.0f) & (__fadd_rn(u, v) <= ad) & (tp > 0.0f) & (tp <= __fmul_rn(tmax, ad));
    if (hit) t = __fdiv_rn(tp, ad);
    return hit && t > 0.0f && t <= tmax;
}

__device__ __forceinline__ unsigned long long hit_key(float t, unsigned tri) {
    return ((unsigned long long)__float_as_uint(t) << 32) | tri;
}

// Pre-test of a final test: a ray can only hit a triangle if its line passes
// through the triangle's bounding sphere.  With v = c - o and s = v.d, the
// squared distance from the centre to the line is |v|^2 - s^2 / |d|^2;
// accept iff |v|^2 <= q + (1 + K) s^2 / |d|^2 with q = 1.05 r^2 and K = 2e-6.
// Whenever the line passes within r + 1e-4 x the distance along the ray (a
// slack far above the FP32 error of Moller-Trumbore's hit point, even at
// grazing incidence; (a + b)^2 <= 1.05 a^2 + 21 b^2) this holds with room for
// the FP32 rounding of |v|^2 and s^2 (a few ulps of |v|^2), so every
// triangle Moller-Trumbore would hit passes.  The brute force takes the same
// pre-test, so both paths decide hits with one function.
// kid2 = (1 + K) / |d|^2; a zero direction makes s = 0 and 0 x inf a NaN, so
// the test rejects, as Moller-Trumbore would (its determinant is 0).
constexpr float PRETEST_K1 = 1.000002f;
// Operation order written out: the packed twin below computes each of its
// two lanes with exactly these FP32 operations, so both give the same bits.
__device__ __forceinline__ bool near_line(float ox, float oy, float oz, float dx, float dy, float dz, float kid2,
                                          float4 C) {
    const float vx = __fadd_rn(C.x, -ox), vy = __fadd_rn(C.y, -oy), vz = __fadd_rn(C.z, -oz);
    const float vv = __fmaf_rn(vz, vz, __fmaf_rn(vy, vy, __fmul_rn(vx, vx)));
    const float s = __fmaf_rn(vz, dz, __fmaf_rn(vy, dy, __fmul_rn(vx, dx)));
    return vv <= __fmaf_rn(__fmul_rn(s, s), kid2, C.w);
}

// The same pre-test for two rays at once (Blackwell's paired FP32 operations,
// one instruction for both lanes of a float2): rays in the .x and .y lanes of
// (-o, d, kid2), the triangle's centre and q repeated in both lanes.  Each lane
// computes the scalar test's FP32 operations in the same order and returns the
// margin rhs - vv, whose sign bit is clear exactly when vv <= rhs for finite
// operands (an exact tie gives +0; a negative difference never rounds to -0),
// so the sign bits carry the scalar test's decisions.  A missing ray (kid2
// NaN) gives a NaN whose sign is not specified: it may pass, and
// Moller-Trumbore then rejects it (its t_max is 0).
struct RayPair {
    float2 nox, noy, noz, dx, dy, dz, kid2;
};
__device__ __forceinline__ float2 near_line2_margin(const RayPair& p, float4 cxy, float4 czq) {
    const float2 vx = __fadd2_rn(make_float2(cxy.x, cxy.y), p.nox);
    const float2 vy = __fadd2_rn(make_float2(cxy.z, cxy.w), p.noy);
    const float2 vz = __fadd2_rn(make_float2(czq.x, czq.y), p.noz);
    const float2 vv = __ffma2_rn(vz, vz, __ffma2_rn(vy, vy, __fmul2_rn(vx, vx)));
    const float2 sd = __ffma2_rn(vz, p.dz, __ffma2_rn(vy, p.dy, __fmul2_rn(vx, p.dx)));
    const float2 rhs = __ffma2_rn(__fmul2_rn(sd, sd), p.kid2, make_float2(czq.z, czq.w));
    return __fadd2_rn(rhs, make_float2(-vv.x, -vv.y));
}

constexpr unsigned long long NO_HIT = ~0ull;

struct RaysDev {
    const float *ox, *oy, *oz, *dx, *dy, *dz, *tmax;
    const uint32_t* ray_id;
};

constexpr int CH_WARPS = 4, CH_BLOCK = CH_WARPS * 32;

// kid2 of a ray, with its operation order written out (every kernel that
// pre-tests a ray computes the same bits)
__device__ __forceinline__ float ray_kid2(float dx, float dy, float dz) {
    return __fdiv_rn(PRETEST_K1, __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
}

// Pairs per work chunk: a multiple of the 32-pair group, about CH_CLAIMS
// claims per warp, between CH_MIN and CH_MAX.  Larger chunks cost fewer
// claims and node changes per pair; smaller ones balance the end of the
// launch (fixed sizes: on the 512x512 frame 96 pairs measured best of 64 to
// 256, on the 1024x1024 frame 256; of 16, 32, 48, 64 and 96 claims per warp,
// 32 measured best there, 1.95 ms).
constexpr unsigned CH_MIN = 96, CH_MAX = 512, CH_CLAIMS = 32;
__device__ __forceinline__ unsigned chunk_pairs(unsigned P) {
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    return max(CH_MIN, min(CH_MAX, (P / (nw * CH_CLAIMS)) & ~31u));
}

// min over the lanes that hold the same ray (one per stream), then one
// atomicMin per ray
template <int H>
__device__ __forceinline__ void flush_best(unsigned long long bk, bool rvalid, int sidx, unsigned ray,
                                           unsigned long long* best) {
#pragma unroll
    for (int o = H; o < 32; o <<= 1) {
        const unsigned long long other = __shfl_xor_sync(FULL, bk, o);
        bk = other < bk ? other : bk;
    }
    if (rvalid && sidx == 0 && bk != NO_HIT) atomicMin(&best[ray], bk);
}

// Warps take chunks of chunk_pairs(P) consecutive pairs of the node-sorted pair
// list from an atomic counter (the cost of a chunk depends on how many nodes
// it spans) and walk them in groups: up to 32 consecutive pairs of one node.
// Each lane holds two rays of the node (slots r and r + B/2) as a RayPair;
// the 32 / (B/2) streams of the warp walk every S-th triangle of the group and
// pre-test it against both rays with one set of paired FP32 operations, then
// run Moller-Trumbore on the survivors.  Software pipeline: while group g is
// tested, the records of group g+1 are copied into the other shared buffer
// (cp.async), the pair window of group g+2 is loaded into registers and the
// chunk after the current one is already claimed, so the chain counter ->
// pair -> triangle -> record never stalls the tests.  *work must be 0 at
// launch.
template <int B>
__global__ void __launch_bounds__(CH_BLOCK, 8) k_closest(const uint32_t* pnode, const uint32_t* ptri,
                                                         const unsigned* p_count, unsigned long long p_cap,
                                                         RaysDev rays, const unsigned* n_ptr, unsigned n_cap,
                                                         const float4* tri_mt,
                                                         unsigned long long* best, unsigned* work,
                                                         crsh_counters* ctr) {
    pdl_wait();
    constexpr int H = B / 2;            // lanes per node (two rays each)
    constexpr int S = 32 / H;           // streams
    // one 64-byte record per triangle: a lane's four copies land side by side
    // (a component-major layout measured 25 % slower on the copies)
    __shared__ __align__(16) float4 s_tri[CH_WARPS][2][32][4];    // (a, n.x) (e1, n.y) (e2, n.z) (c, q)
    __shared__ unsigned s_tid[CH_WARPS][2][32];
    const unsigned P = (unsigned)min((unsigned long long)*p_count, p_cap);
    const unsigned N = min(*n_ptr, n_cap);   // rays past the capacity are never touched
    const unsigned CH_PAIRS = chunk_pairs(P);
    const unsigned n_chunks = (P + CH_PAIRS - 1) / CH_PAIRS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = lane % H, sidx = lane / H;
    unsigned long long n_tests = 0, n_hits = 0;
    // claims are issued by lane 0 and read (broadcast) one chunk later
    unsigned claim = 0;
    if (lane == 0) claim = atomicAdd(work, 1u);
    const unsigned c_first = __shfl_sync(FULL, claim, 0);
    if (c_first < n_chunks) {
        if (lane == 0) claim = atomicAdd(work, 1u);
        // pair window at q (chunk end e): lane i holds pair q + i (node ~0 past e)
        auto window = [&](unsigned q, unsigned e, unsigned& pw, unsigned& pt) {
            const bool in = q + lane < e;
            pw = in ? pnode[q + lane] : 0xffffffffu;
            pt = in ? ptri[q + lane] : 0u;
        };
        // position after a group of cnt pairs at (q, e); false when the work is done
        auto advance = [&](unsigned& q, unsigned& e, unsigned cnt) -> bool {
            q += cnt;
            if (q < e) return true;
            const unsigned c = __shfl_sync(FULL, claim, 0);
            if (c >= n_chunks) return false;
            if (lane == 0) claim = atomicAdd(work, 1u);
            q = c * CH_PAIRS;
            e = min(P, q + CH_PAIRS);
            return true;
        };
        // records of a group's triangles into buffer b (one commit per call)
        auto stage = [&](int b, unsigned cnt, unsigned pt) {
            if ((unsigned)lane < cnt) {
                const float4* m = tri_mt + 4 * (size_t)pt;
                cp_async16(&s_tri[warp][b][lane][0], m);
                cp_async16(&s_tri[warp][b][lane][1], m + 1);
                cp_async16(&s_tri[warp][b][lane][2], m + 2);
                cp_async16(&s_tri[warp][b][lane][3], m + 3);
                s_tid[warp][b][lane] = pt;
            } else {
                // past the group: a sphere no line passes through (q = -inf makes the pre-test's
                // right side -inf, so its margin is negative)
                s_tri[warp][b][lane][3] = make_float4(0.f, 0.f, 0.f, __int_as_float(0xff800000));
            }
            cp_async_commit();
        };
        // the node's two rays of this lane (a missing ray gets kid2 = NaN:
        // its pre-tests all fail)
        RayPair rp;
        float ta = 0.f, tb = 0.f;
        unsigned cur, ray0, ray1;
        bool v0, v1;
        auto enter_node = [&](unsigned node) {
            cur = node;
            ray0 = cur * B + r;
            ray1 = ray0 + H;
            v0 = ray0 < N;
            v1 = ray1 < N;
            float ax = 0, ay = 0, az = 0, adx = 0, ady = 0, adz = 0;
            float bx = 0, by = 0, bz = 0, bdx = 0, bdy = 0, bdz = 0;
            ta = tb = 0.f;
            if (v0) {
                ax = rays.ox[ray0]; ay = rays.oy[ray0]; az = rays.oz[ray0];
                adx = rays.dx[ray0]; ady = rays.dy[ray0]; adz = rays.dz[ray0]; ta = rays.tmax[ray0];
            }
            if (v1) {
                bx = rays.ox[ray1]; by = rays.oy[ray1]; bz = rays.oz[ray1];
                bdx = rays.dx[ray1]; bdy = rays.dy[ray1]; bdz = rays.dz[ray1]; tb = rays.tmax[ray1];
            }
            rp.nox = make_float2(-ax, -bx); rp.noy = make_float2(-ay, -by); rp.noz = make_float2(-az, -bz);
            rp.dx = make_float2(adx, bdx); rp.dy = make_float2(ady, bdy); rp.dz = make_float2(adz, bdz);
            rp.kid2 = make_float2(v0 ? ray_kid2(adx, ady, adz) : __int_as_float(0x7fc00000),
                                  v1 ? ray_kid2(bdx, bdy, bdz) : __int_as_float(0x7fc00000));
        };
        unsigned q1 = c_first * CH_PAIRS, e1 = min(P, q1 + CH_PAIRS);
        unsigned pw1, pt1;
        window(q1, e1, pw1, pt1);
        enter_node(__shfl_sync(FULL, pw1, 0));
        unsigned cnt = __popc(__ballot_sync(FULL, pw1 == cur));   // a prefix: pairs are node-sorted
        stage(0, cnt, pt1);
        bool has1 = advance(q1, e1, cnt);
        if (has1) window(q1, e1, pw1, pt1);
        unsigned long long k0 = NO_HIT, k1 = NO_HIT;
        int buf = 0;
        for (;;) {
            unsigned nnode = 0xffffffffu, ncnt = 0;
            unsigned pw2 = 0xffffffffu, pt2 = 0;
            bool has2 = false;
            if (has1) {   // warp-uniform
                nnode = __shfl_sync(FULL, pw1, 0);
                ncnt = __popc(__ballot_sync(FULL, pw1 == nnode));
                stage(buf ^ 1, ncnt, pt1);
                has2 = advance(q1, e1, ncnt);
                if (has2) window(q1, e1, pw2, pt2);
            } else {
                cp_async_commit();   // keeps "all but the newest group" meaning this group
            }
            cp_async_wait_prev();
            __syncwarp();
            const unsigned nrays = min((unsigned)B, N - cur * B);
            if (lane == 0) n_tests += (unsigned long long)cnt * nrays;
            // pre-test every (ray, triangle) of the lane: row k is triangle sidx + S k; the
            // margins' sign bits (miss flags) are shifted in, so after the loop bit kmax - 1 - k
            // is row k's, and the hit masks are their complements.  Rows past the group's
            // triangles are skipped; slots past it in the last row hold a sphere that fails.
            constexpr int K = 32 / S;
            const unsigned kmax = (cnt + S - 1) / S;   // warp-uniform: rows of the group that hold triangles
            unsigned x0 = 0, x1 = 0;
            auto row = [&](int k) {
                const float4 c = s_tri[warp][buf][sidx + S * k][3];
                const float2 d = near_line2_margin(rp, make_float4(c.x, c.x, c.y, c.y), make_float4(c.z, c.z, c.w, c.w));
                x0 = __funnelshift_l(__float_as_uint(d.x), x0, 1);
                x1 = __funnelshift_l(__float_as_uint(d.y), x1, 1);
            };
            if (kmax == (unsigned)K) {   // a full group: no row test
#pragma unroll
                for (int k = 0; k < K; ++k) row(k);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if ((unsigned)k >= kmax) break;
                    row(k);
                }
            }
            const unsigned rows = kmax >= 32 ? 0xffffffffu : (1u << kmax) - 1u;
            const unsigned m0 = ~x0 & rows, m1 = ~x1 & rows;
            // Moller-Trumbore on the survivors (o = -(-o) is exact)
            unsigned m = m0 | m1;
            while (m) {
                const unsigned kk = __ffs(m) - 1;
                m &= m - 1;
                const unsigned j = sidx + S * (kmax - 1 - kk);
                const float4 A = s_tri[warp][buf][j][0], E1 = s_tri[warp][buf][j][1], E2 = s_tri[warp][buf][j][2];
                float t;
                if (((m0 >> kk) & 1u) &&
                    mt_hit(-rp.nox.x, -rp.noy.x, -rp.noz.x, rp.dx.x, rp.dy.x, rp.dz.x, ta, A, E1, E2, t)) {
                    ++n_hits;
                    const unsigned long long key = hit_key(t, s_tid[warp][buf][j]);
                    k0 = key < k0 ? key : k0;
                }
                if (((m1 >> kk) & 1u) &&
                    mt_hit(-rp.nox.y, -rp.noy.y, -rp.noz.y, rp.dx.y, rp.dy.y, rp.dz.y, tb, A, E1, E2, t)) {
                    ++n_hits;
                    const unsigned long long key = hit_key(t, s_tid[warp][buf][j]);
                    k1 = key < k1 ? key : k1;
                }
            }
            __syncwarp();   // buffer buf is refilled two groups on
            if (!has1) break;
            if (nnode != cur) {
                flush_best<H>(k0, v0, sidx, ray0, best);
                flush_best<H>(k1, v1, sidx, ray1, best);
                enter_node(nnode);
                k0 = k1 = NO_HIT;
            }
            cnt = ncnt;
            buf ^= 1;
            has1 = has2;
            pw1 = pw2;
            pt1 = pt2;
        }
        flush_best<H>(k0, v0, sidx, ray0, best);
        flush_best<H>(k1, v1, sidx, ray1, best);
    }
    n_tests = warp_sum64(n_tests);
    n_hits = warp_sum64(n_hits);
    if (lane == 0) {
        if (n_tests) atomicAdd(&ctr->final_tests, n_tests);
        if (n_hits) atomicAdd(&ctr->final_hits, n_hits);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->final_tests_paper = (unsigned long long)P * B;
}

// ---------------------------------------------------------------------------
// Final tests over the word form of level 1 (crsh_pair_words): the same
// candidate set, read from the traversal's last ballots instead of a written
// pair list.  Warps claim batches of work items (one child's run of up to 32
// chunk ballots; a node's items are consecutive), load the batch's
// descriptors at once, and for each item scan its words, copy the triangle
// ids of the set bits from the parent list into a ring in shared memory
// (cp.async), and cut the ring into groups of up to 32 triangles of one node.
// Each group runs k_closest's group test; the next group is gathered and its
// records copied while the current one is tested, and each item's words are
// loaded while the item before it is gathered.
// ---------------------------------------------------------------------------
constexpr unsigned WI_BATCH = 4;   // work items per claim at most (of 2, 3, 4, 6, 8, 16: 4 measured best)

template <int B>
__global__ void __launch_bounds__(CH_BLOCK, 7) k_closest_words(crsh_pair_words pw, RaysDev rays,
                                                               const unsigned* n_ptr, unsigned n_cap,
                                                               const float4* tri_mt, unsigned long long* best,
                                                               unsigned* work, crsh_counters* ctr) {
    pdl_wait();
    constexpr int H = B / 2;            // lanes per node (two rays each)
    constexpr int S = 32 / H;           // streams
    constexpr int K = 32 / S;           // pre-test rows of a full group
    __shared__ __align__(16) float4 s_tri[CH_WARPS][2][32][4];    // (a, n.x) (e1, n.y) (e2, n.z) (c, q)
    __shared__ unsigned s_tid[CH_WARPS][2][32];
    __shared__ unsigned s_q[CH_WARPS][64];                         // ring of gathered triangle ids
    const unsigned N = min(*n_ptr, n_cap);   // rays past the capacity are never touched
    const unsigned I = *pw.n_items;
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    const uint4* items = reinterpret_cast<const uint4*>(pw.items);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int r = lane % H, sidx = lane / H;
    unsigned long long n_tests = 0, n_hits = 0;
    // ---- producer: items -> words -> triangle ids -> groups (warp-uniform but the per-lane values) ----
    // batches of items from the counter: lane 0 holds the next one (start, size), claimed one
    // batch ahead; sizes shrink toward the end (about a sixteenth of the items left per warp)
    unsigned cl_base = 0, cl_size = WI_BATCH;
    if (lane == 0) cl_base = atomicAdd(work, WI_BATCH);
    uint4 desc = make_uint4(0, 0, 0, 0);       // lane j < nb: item j of the batch
    unsigned nb = 0, ib = 0;                   // items in the batch, next item of it
    unsigned node = 0, rs = 0;                 // current item: level-1 node, run position of its first chunk
    unsigned wl = 0, any = 0;                  // its words (this lane's), nonzero words left
    unsigned wnext = 0;                        // the next item's words (this lane's), loaded ahead
    unsigned qh = 0, qn = 0, qnode = 0;        // ring head, ids queued, their node
    bool more = true;
    auto words_of = [&](unsigned j) -> unsigned {   // lane's word of batch item j (j < nb)
        const unsigned w0 = __shfl_sync(FULL, desc.z, j), c = __shfl_sync(FULL, desc.w, j);
        return (unsigned)lane < c ? pw.words[w0 + lane] : 0u;
    };
    auto claim_batch = [&]() -> bool {
        const unsigned base = __shfl_sync(FULL, cl_base, 0), size = __shfl_sync(FULL, cl_size, 0);
        if (base >= I) return false;
        if (lane == 0) {
            const unsigned done = base + size, left = done < I ? I - done : 0u;
            cl_size = max(1u, min(WI_BATCH, left / (16u * nw)));
            cl_base = atomicAdd(work, cl_size);
        }
        nb = min(size, I - base);
        if ((unsigned)lane < nb) desc = items[base + lane];
        ib = 0;
        wnext = words_of(0);
        return true;
    };
    // the next item (its words were loaded ahead); false when the warp's work is done
    auto next_item = [&]() -> bool {
        if (ib >= nb && !claim_batch()) return false;
        node = __shfl_sync(FULL, desc.x, ib);
        rs = __shfl_sync(FULL, desc.y, ib);
        wl = wnext;
        any = __ballot_sync(FULL, wl != 0);
        ++ib;
        if (ib < nb) wnext = words_of(ib);
        return true;
    };
    // Groups are made one step ahead of their use: gather() issues the copies of
    // the next group's triangle ids into the ring and records the group (its
    // size and node); emit() later waits for those copies (issued a group test
    // earlier) and starts the copies of the group's triangle records.
    unsigned pend_cnt = 0, pend_node = 0;      // the gathered group not yet emitted
    auto gather = [&]() {
        pend_cnt = 0;
        for (;;) {
            if (qn >= 32) {   // a full group (ids past it stay for the next one)
                pend_cnt = 32;
                pend_node = qnode;
                return;
            }
            if (any) {   // the triangle ids of the item's nonzero words, copied into the ring
                do {
                    const unsigned kk = __ffs(any) - 1;
                    any &= any - 1;
                    const unsigned m = __shfl_sync(FULL, wl, kk);
                    if ((m >> lane) & 1u)
                        cp_async4(&s_q[warp][(qh + qn + __popc(m & lt)) & 63], pw.tri + rs + 32 * kk + lane);
                    qn += __popc(m);
                } while (any && qn < 32);
                continue;
            }
            if (more && (qn == 0 || node == qnode)) {
                more = next_item();
                if (more && qn == 0) qnode = node;
                if (more && node == qnode) continue;
            }
            // a new node (or the end) closes the ring's group
            pend_cnt = qn;
            pend_node = qnode;
            return;
        }
    };
    // stage the gathered group's ids as triangle records into buffer b (one commit)
    auto emit = [&](int b) {
        const unsigned cnt = pend_cnt;
        cp_async_wait_all();
        __syncwarp();
        if ((unsigned)lane < cnt) {
            const unsigned t = s_q[warp][(qh + lane) & 63];
            const float4* m = tri_mt + 4 * (size_t)t;
            cp_async16(&s_tri[warp][b][lane][0], m);
            cp_async16(&s_tri[warp][b][lane][1], m + 1);
            cp_async16(&s_tri[warp][b][lane][2], m + 2);
            cp_async16(&s_tri[warp][b][lane][3], m + 3);
            s_tid[warp][b][lane] = t;
        } else {
            // past the group: a sphere no line passes through (q = -inf)
            s_tri[warp][b][lane][3] = make_float4(0.f, 0.f, 0.f, __int_as_float(0xff800000));
        }
        cp_async_commit();
        __syncwarp();   // the ring slots just read may be refilled
        qh = (qh + cnt) & 63;
        qn -= cnt;
        if (qn == 0) qnode = node;   // a closed node: the ring continues with the current item's
    };
    gather();
    unsigned cnt = pend_cnt, gnode = pend_node;
    if (cnt) {
        emit(0);
        gather();
        // the node's two rays of this lane (a missing ray gets kid2 = NaN:
        // its pre-tests all fail)
        RayPair rp;
        float ta = 0.f, tb = 0.f;
        unsigned cur, ray0, ray1;
        bool v0, v1;
        auto enter_node = [&](unsigned nd) {
            cur = nd;
            ray0 = cur * B + r;
            ray1 = ray0 + H;
            v0 = ray0 < N;
            v1 = ray1 < N;
            float ax = 0, ay = 0, az = 0, adx = 0, ady = 0, adz = 0;
            float bx = 0, by = 0, bz = 0, bdx = 0, bdy = 0, bdz = 0;
            ta = tb = 0.f;
            if (v0) {
                ax = rays.ox[ray0]; ay = rays.oy[ray0]; az = rays.oz[ray0];
                adx = rays.dx[ray0]; ady = rays.dy[ray0]; adz = rays.dz[ray0]; ta = rays.tmax[ray0];
            }
            if (v1) {
                bx = rays.ox[ray1]; by = rays.oy[ray1]; bz = rays.oz[ray1];
                bdx = rays.dx[ray1]; bdy = rays.dy[ray1]; bdz = rays.dz[ray1]; tb = rays.tmax[ray1];
            }
            rp.nox = make_float2(-ax, -bx); rp.noy = make_float2(-ay, -by); rp.noz = make_float2(-az, -bz);
            rp.dx = make_float2(adx, bdx); rp.dy = make_float2(ady, bdy); rp.dz = make_float2(adz, bdz);
            rp.kid2 = make_float2(v0 ? ray_kid2(adx, ady, adz) : __int_as_float(0x7fc00000),
                                  v1 ? ray_kid2(bdx, bdy, bdz) : __int_as_float(0x7fc00000));
        };
        enter_node(gnode);
        unsigned long long k0 = NO_HIT, k1 = NO_HIT;
        int buf = 0;
        for (;;) {
            // the next group's records into the other buffer, then the ids of the one after it
            const unsigned ncnt = pend_cnt, nnode = pend_node;
            if (ncnt) {
                emit(buf ^ 1);
                gather();
            } else {
                cp_async_commit();   // keeps "all but the newest group" meaning this group
            }
            cp_async_wait_prev();
            __syncwarp();
            const unsigned nrays = min((unsigned)B, N - cur * B);
            if (lane == 0) n_tests += (unsigned long long)cnt * nrays;
            // the group test of k_closest
            const unsigned kmax = (cnt + S - 1) / S;
            unsigned x0 = 0, x1 = 0;
            auto row = [&](int k) {
                const float4 c = s_tri[warp][buf][sidx + S * k][3];
                const float2 d = near_line2_margin(rp, make_float4(c.x, c.x, c.y, c.y), make_float4(c.z, c.z, c.w, c.w));
                x0 = __funnelshift_l(__float_as_uint(d.x), x0, 1);
                x1 = __funnelshift_l(__float_as_uint(d.y), x1, 1);
            };
            if (kmax == (unsigned)K) {
#pragma unroll
                for (int k = 0; k < K; ++k) row(k);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if ((unsigned)k >= kmax) break;
                    row(k);
                }
            }
            const unsigned rows = kmax >= 32 ? 0xffffffffu : (1u << kmax) - 1u;
            const unsigned m0 = ~x0 & rows, m1 = ~x1 & rows;
            unsigned m = m0 | m1;
            while (m) {
                const unsigned kk = __ffs(m) - 1;
                m &= m - 1;
                const unsigned j = sidx + S * (kmax - 1 - kk);
                const float4 A = s_tri[warp][buf][j][0], E1 = s_tri[warp][buf][j][1], E2 = s_tri[warp][buf][j][2];
                float t;
                if (((m0 >> kk) & 1u) &&
                    mt_hit(-rp.nox.x, -rp.noy.x, -rp.noz.x, rp.dx.x, rp.dy.x, rp.dz.x, ta, A, E1, E2, t)) {
                    ++n_hits;
                    const unsigned long long key = hit_key(t, s_tid[warp][buf][j]);
                    k0 = key < k0 ? key : k0;
                }
                if (((m1 >> kk) & 1u) &&
                    mt_hit(-rp.nox.y, -rp.noy.y, -rp.noz.y, rp.dx.y, rp.dy.y, rp.dz.y, tb, A, E1, E2, t)) {
                    ++n_hits;
                    const unsigned long long key = hit_key(t, s_tid[warp][buf][j]);
                    k1 = key < k1 ? key : k1;
                }
            }
            __syncwarp();   // buffer buf is refilled two groups on
            if (!ncnt) break;
            if (nnode != cur) {
                flush_best<H>(k0, v0, sidx, ray0, best);
                flush_best<H>(k1, v1, sidx, ray1, best);
                enter_node(nnode);
                k0 = k1 = NO_HIT;
            }
            cnt = ncnt;
            buf ^= 1;
        }
        flush_best<H>(k0, v0, sidx, ray0, best);
        flush_best<H>(k1, v1, sidx, ray1, best);
    }
    n_tests = warp_sum64(n_tests);
    n_hits = warp_sum64(n_hits);
    if (lane == 0) {
        if (n_tests) atomicAdd(&ctr->final_tests, n_tests);
        if (n_hits) atomicAdd(&ctr->final_hits, n_hits);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->final_tests_paper = ctr->hits[0] * B;
}

// n_cap: rays the scratch and the ray arrays hold; a larger device count is
// clamped to it and reported as CRSH_ERR_CAPACITY (no access past the end)
__global__ void k_fill_best(unsigned long long* best, const unsigned* n_ptr, unsigned n_cap, unsigned* work,
                            crsh_counters* ctr) {
    pdl_wait();
    const unsigned n = min(*n_ptr, n_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (work) *work = 0;
        ctr->final_tests = ctr->final_tests_paper = ctr->final_hits = 0;   // this call's counters
        if (*n_ptr > n_cap) set_status(ctr, CRSH_ERR_CAPACITY);
    }
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) best[i] = NO_HIT;
}

// ---- double-word (float + float) arithmetic --------------------------------
// A value is the unevaluated sum h + l of two FP32 numbers (about 48 bits).
// Error-free transformations: TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|),
// TwoProd with an FMA; sums and products of double-words follow Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic" (ACM TOMS 2017): the accurate sum
// (relative error <= 3u^2 + 13u^3) and the FMA product (<= 5u^2), u = 2^-24.
// Every step is an explicit _rn intrinsic, so nothing is contracted or
// reassociated.
struct DW {
    float h, l;
};
__device__ __forceinline__ DW two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DW fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DW dw_add(DW x, DW y) {
    const DW s = two_sum(x.h, y.h), t = two_sum(x.l, y.l);
    const DW v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
__device__ __forceinline__ DW dw_neg(DW x) { return {-x.h, -x.l}; }
__device__ __forceinline__ DW dw_mul(DW x, DW y) {
    const float ch = __fmul_rn(x.h, y.h);
    const float cl1 = __fmaf_rn(x.h, y.h, -ch);
    const float cl2 = __fmaf_rn(x.l, y.h, __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l)));
    return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
// a (one FP32 number) times a double-word
__device__ __forceinline__ DW dw_mul(float a, DW y) {
    const float ch = __fmul_rn(a, y.h);
    const float cl = __fmaf_rn(a, y.l, __fmaf_rn(a, y.h, -ch));
    return fast_two_sum(ch, cl);
}
// x / y rounded to FP32: an FP32 quotient corrected by the double-word
// remainder x - q y (the product q y.h is exact as a TwoProd)
__device__ __forceinline__ float dw_div_f(DW x, DW y) {
    const float q = __fdiv_rn(x.h, y.h);
    const float ph = __fmul_rn(q, y.h);
    const float pl = __fmaf_rn(q, y.h, -ph);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, ph), pl), __fmaf_rn(-q, y.l, x.l));
    return __fadd_rn(q, __fdiv_rn(r, y.h));
}

// Moller-Trumbore in double-word arithmetic on the FP32 inputs, for the one
// winning triangle of a ray: the FP32 test decides which triangle is closest,
// this pass reports its (t, u, v) to about FP32 rounding (FP32 alone loses
// digits in proportion to distance / triangle size).  Differences of the
// FP32 inputs are exact double-words; the rest carries about 2^-44 relative
// error, far below the FP32 rounding of the results.
__device__ __forceinline__ void mt_refine(float ox, float oy, float oz, float dx, float dy, float dz,
                                          const crsh_scene& sc, unsigned tri, float& t, float& u, float& v) {
    const float ax = sc.v0x[tri], ay = sc.v0y[tri], az = sc.v0z[tri];
    const DW e1x = two_sum(sc.v1x[tri], -ax), e1y = two_sum(sc.v1y[tri], -ay), e1z = two_sum(sc.v1z[tri], -az);
    const DW e2x = two_sum(sc.v2x[tri], -ax), e2y = two_sum(sc.v2y[tri], -ay), e2z = two_sum(sc.v2z[tri], -az);
    // p = d x e2
    const DW px = dw_add(dw_mul(dy, e2z), dw_neg(dw_mul(dz, e2y)));
    const DW py = dw_add(dw_mul(dz, e2x), dw_neg(dw_mul(dx, e2z)));
    const DW pz = dw_add(dw_mul(dx, e2y), dw_neg(dw_mul(dy, e2x)));
    const DW det = dw_add(dw_add(dw_mul(e1x, px), dw_mul(e1y, py)), dw_mul(e1z, pz));
    const DW sx = two_sum(ox, -ax), sy = two_sum(oy, -ay), sz = two_sum(oz, -az);
    // q = s x e1
    const DW qx = dw_add(dw_mul(sy, e1z), dw_neg(dw_mul(sz, e1y)));
    const DW qy = dw_add(dw_mul(sz, e1x), dw_neg(dw_mul(sx, e1z)));
    const DW qz = dw_add(dw_mul(sx, e1y), dw_neg(dw_mul(sy, e1x)));
    u = dw_div_f(dw_add(dw_add(dw_mul(sx, px), dw_mul(sy, py)), dw_mul(sz, pz)), det);
    v = dw_div_f(dw_add(dw_add(dw_mul(dx, qx), dw_mul(dy, qy)), dw_mul(dz, qz)), det);
    t = dw_div_f(dw_add(dw_add(dw_mul(e2x, qx), dw_mul(e2y, qy)), dw_mul(e2z, qz)), det);
}

// winner's (t, u, v) from the double-word refinement; scatter to ray_id order
__global__ void k_finalize(RaysDev rays, const unsigned* n_ptr, unsigned n_cap, crsh_scene sc,
                           const unsigned long long* best, crsh_hits out) {
    pdl_wait();
    const unsigned n = min(*n_ptr, n_cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = best[i];
        const unsigned dst = rays.ray_id[i];
        if (k == NO_HIT) {
            out.tri[dst] = -1;
            out.t[dst] = out.u[dst] = out.v[dst] = 0.0f;
            continue;
        }
        const unsigned tri = (unsigned)(k & 0xffffffffu);
        float t, u, v;
        mt_refine(rays.ox[i], rays.oy[i], rays.oz[i], rays.dx[i], rays.dy[i], rays.dz[i], sc, tri, t, u, v);
        out.tri[dst] = (int)tri;
        out.t[dst] = t;
        out.u[dst] = u;
        out.v[dst] = v;
    }
}

// N x M: one ray per thread, triangles streamed through shared memory.
constexpr int BF_BLOCK = 256;
__global__ void __launch_bounds__(BF_BLOCK) k_brute(RaysDev rays, const unsigned* n_ptr, unsigned n_cap,
                                                    const float4* tri_mt, unsigned n_tris, unsigned long long* best) {
    __shared__ float4 s_tri[BF_BLOCK][4];
    const unsigned n = min(*n_ptr, n_cap);
    for (unsigned base = blockIdx.x * BF_BLOCK; base < n; base += gridDim.x * BF_BLOCK) {
        const unsigned i = base + threadIdx.x;
        const bool valid = i < n;
        float ox = 0, oy = 0, oz = 0, dx = 0, dy = 0, dz = 0, tmax = 0;
        if (valid) {
            ox = rays.ox[i]; oy = rays.oy[i]; oz = rays.oz[i];
            dx = rays.dx[i]; dy = rays.dy[i]; dz = rays.dz[i];
            tmax = rays.tmax[i];
        }
        const float id2 = ray_kid2(dx, dy, dz);
        unsigned long long bk = NO_HIT;
        for (unsigned t0 = 0; t0 < n_tris; t0 += BF_BLOCK) {
            __syncthreads();
            if (t0 + threadIdx.x < n_tris) {
                const float4* m = tri_mt + 4 * (size_t)(t0 + threadIdx.x);
                s_tri[threadIdx.x][0] = m[0];
                s_tri[threadIdx.x][1] = m[1];
                s_tri[threadIdx.x][2] = m[2];
                s_tri[threadIdx.x][3] = m[3];
            }
            __syncthreads();
            const unsigned cnt = min((unsigned)BF_BLOCK, n_tris - t0);
            for (unsigned j = 0; j < cnt; ++j) {
                float t;
                if (near_line(ox, oy, oz, dx, dy, dz, id2, s_tri[j][3]) &&
                    mt_hit(ox, oy, oz, dx, dy, dz, tmax, s_tri[j][0], s_tri[j][1], s_tri[j][2], t)) {
                    const unsigned long long k = hit_key(t, t0 + j);
                    bk = k < bk ? k : bk;
                }
            }
        }
        if (valid) best[i] = bk;
    }
}

size_t closest_hit_workspace(uint32_t cap) { return (size_t)cap * sizeof(unsigned long long) + 256; }

static RaysDev rays_dev(const crsh_rays* r) {
    return RaysDev{r->ox, r->oy, r->oz, r->dx, r->dy, r->dz, r->tmax, r->ray_id};
}

// One wave of resident blocks: every warp owns an equal contiguous share of
// the pairs, so a second partial wave would double the time.
template <int B>
static void launch_closest(const crsh_pairs* pairs, const RaysDev& rd, const uint32_t* n_rays, unsigned n_cap,
                           const float4* mt,
                           unsigned long long* best, unsigned* work, crsh_counters* ctr, cudaStream_t s,
                           const DeviceInfo& dev) {
    static std::atomic<int> per_sm[64];   // resident blocks per SM, per device
    const int d = (dev.device >= 0 && dev.device < 64) ? dev.device : 0;
    int b = per_sm[d].load(std::memory_order_relaxed);
    if (b <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_closest<B>, CH_BLOCK, 0) != cudaSuccess || b <= 0) b = 1;
        per_sm[d].store(b, std::memory_order_relaxed);
    }
    if (pairs->words.valid) {
        static std::atomic<int> per_sm_w[64];
        int bw = per_sm_w[d].load(std::memory_order_relaxed);
        if (bw <= 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bw, k_closest_words<B>, CH_BLOCK, 0) != cudaSuccess ||
                bw <= 0)
                bw = 1;
            per_sm_w[d].store(bw, std::memory_order_relaxed);
        }
        launch_pdl(k_closest_words<B>, dev.sms * bw, CH_BLOCK, 0, s, pairs->words, rd, n_rays, n_cap, mt, best, work,
                   ctr);
        return;
    }
    launch_pdl(k_closest<B>, dev.sms * b, CH_BLOCK, 0, s, pairs->node, pairs->tri, pairs->count, pairs->capacity, rd,
               n_rays, n_cap, mt, best, work, ctr);
}

crsh_status closest_hit_launch(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                               const crsh_scene* sc, const crsh_pairs* pairs, crsh_hits* out, crsh_counters* ctr,
                               void* ws, size_t ws_bytes, cudaStream_t s, const DeviceInfo& dev,
                               cudaEvent_t ev_begin, cudaEvent_t ev_end) {
    if (ws_bytes < closest_hit_workspace(rays->capacity)) return CRSH_ERR_INVALID_ARG;
    unsigned long long* best = reinterpret_cast<unsigned long long*>(ws);
    unsigned* work = reinterpret_cast<unsigned*>(best + rays->capacity);   // in the 256 spare bytes
    const unsigned fb = dev.sms * 8;
    const unsigned cap = rays->capacity;
    launch_pdl(k_fill_best, fb, 256, 0, s, best, n_rays, cap, work, ctr);
    const RaysDev rd = rays_dev(rays);
    const float4* mt = reinterpret_cast<const float4*>(sc->tri_mt);
    if (ev_begin && cudaEventRecord(ev_begin, s) != cudaSuccess) return CRSH_ERR_CUDA;
    switch (h->bundle) {
        case 2: launch_closest<2>(pairs, rd, n_rays, cap, mt, best, work, ctr, s, dev); break;
        case 4: launch_closest<4>(pairs, rd, n_rays, cap, mt, best, work, ctr, s, dev); break;
        case 8: launch_closest<8>(pairs, rd, n_rays, cap, mt, best, work, ctr, s, dev); break;
        case 16: launch_closest<16>(pairs, rd, n_rays, cap, mt, best, work, ctr, s, dev); break;
        case 32: launch_closest<32>(pairs, rd, n_rays, cap, mt, best, work, ctr, s, dev); break;
        case 64: launch_closest<64>(pairs, rd, n_rays, cap, mt, best, work, ctr, s, dev); break;
        default: return CRSH_ERR_INVALID_ARG;
    }
    if (ev_end && cudaEventRecord(ev_end, s) != cudaSuccess) return CRSH_ERR_CUDA;
    launch_pdl(k_finalize, fb, 256, 0, s, rd, n_rays, cap, *sc, best, *out);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

crsh_status bruteforce_launch(const crsh_rays* rays, const uint32_t* n_rays, const crsh_scene* sc, crsh_hits* out,
                              void* ws, size_t ws_bytes, cudaStream_t s, const DeviceInfo& dev) {
    if (ws_bytes < closest_hit_workspace(rays->capacity)) return CRSH_ERR_INVALID_ARG;
    unsigned long long* best = reinterpret_cast<unsigned long long*>(ws);
    const RaysDev rd = rays_dev(rays);
    const float4* mt = reinterpret_cast<const float4*>(sc->tri_mt);
    const unsigned blocks = (rays->capacity + BF_BLOCK - 1) / BF_BLOCK;
    const unsigned grid = blocks < (unsigned)dev.sms * 8 ? (blocks ? blocks : 1) : dev.sms * 8;
    k_brute<<<grid, BF_BLOCK, 0, s>>>(rd, n_rays, rays->capacity, mt, sc->n_tris, best);
    launch_pdl(k_finalize, dev.sms * 8, 256, 0, s, rd, n_rays, (unsigned)rays->capacity, *sc, best, *out);
    return cudaPeekAtLastError() == cudaSuccess ? CRSH_OK : CRSH_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Allocation-free closest hit.  The per-ray scratch that crsh_closest_hit
// takes from the caller's workspace (one 64-bit key per ray) lives here in a
// fixed device array instead, so a caller that cannot allocate device memory
// passes only inputs and outputs.  Every GPU that loads the library holds the
// array until the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned long long g_noalloc_best[CRSH_NOALLOC_MAX_RAYS + 32];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64];

crsh_status closest_hit_noalloc_launch(const crsh_hierarchy* h, const crsh_rays* rays, const uint32_t* n_rays,
                                       const crsh_scene* sc, const crsh_pairs* pairs, crsh_hits* out,
                                       crsh_counters* ctr, cudaStream_t s, const DeviceInfo& dev) {
    if (rays->capacity > CRSH_NOALLOC_MAX_RAYS) return CRSH_ERR_INVALID_ARG;
    if (dev.device < 0 || dev.device >= 64) return CRSH_ERR_CUDA;
    void* scratch = nullptr;
    {
        // Host code only knows the array by its host-side stand-in: look up
        // its device address once per device, with that device current.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev.device]) {
            void* a = nullptr;
            if (cudaGetSymbolAddress(&a, g_noalloc_best) != cudaSuccess || !a) return CRSH_ERR_CUDA;
            g_noalloc_addr[dev.device] = a;
        }
        scratch = g_noalloc_addr[dev.device];
    }
    // the existing path; it re-initialises every key it reads (no-hit) first
    return closest_hit_launch(h, rays, n_rays, sc, pairs, out, ctr, scratch, sizeof(g_noalloc_best), s, dev);
}

}  // namespace crsh
