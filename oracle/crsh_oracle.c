/* CPU oracle of the Coherent Ray-Space Hierarchy (Reis, Costa, Pereira,
 * "Ray-Tracing With a Coherent Ray-Space Hierarchy", arXiv 2312.06538).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded C99 written from the
 * paper.  It shares no code, header, table or constant generator with the
 * CUDA library, and only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  The product path never calls it.
 *
 * Precision: ray generation and hashing are FP32 with a fixed operation order
 * (no FMA contraction: build with -ffp-contract=off) because their results are
 * integers (hash keys) that both sides must decide in the paper's precision
 * (the paper's G-buffer is 32-bit float, Section 3.2).  Everything else
 * (hierarchy, culling tests, Moller-Trumbore, counting) is FP64 evaluated on
 * the FP32 inputs.
 *
 * Readings of passages the paper leaves open are marked READING; every one is
 * listed in the design notes of the repository.
 *
 * Parity pins: every function below is pinned by a CPU test against values
 * fixed by the mathematics or printed by the paper (closed forms, brute
 * force, library routines, invariants, Tables 1-4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Section 3.3.2: secondary ray generation from the primary-hit buffer.      */
/* ------------------------------------------------------------------------ */

enum { RAY_SHADOW = 0, RAY_REFLECTION = 1, RAY_REFRACTION = 2 };
enum { MAT_DIFFUSE = 0, MAT_MIRROR = 1, MAT_GLASS = 2 };

/* FP32 length with a fixed summation order. */
static float len3f(float x, float y, float z) {
    float s = x * x;
    s = s + y * y;
    s = s + z * z;
    return sqrtf(s);
}

/* Rays of every hit pixel, pixel-major; within a pixel: one shadow ray per
 * light (light 0 first), then the reflection ray, then the refraction ray.
 * Slots that hold no ray are dropped, keeping order (the trimming of
 * Section 3.3.2 / Figure 4).
 *
 * Shadow ray (Section 3.3.2, origin inverted to the light): origin L, direction
 * (P - L)/|P - L|, t_max = |P - L| * 0.9999.  READING: with shadow_cull the ray
 * exists only when the light lies in front of the surface, n . (P - L) < 0.
 * Reflection ray (mirror and glass): r = i - 2 (i.n) n normalised, origin
 * P + 1e-4 s n with s = -1 if i.n > 0 else +1, t_max = +inf.
 * Refraction ray (glass, IOR 1.5, Snell): entering when i.n < 0 (eta = 1/1.5,
 * normal n), leaving otherwise (eta = 1.5, normal -n); none on total internal
 * reflection; origin P - 1e-4 s n, t_max = +inf.
 * Returns the number of rays written. */
int64_t oracle_generate_rays(uint32_t n_pixels, const float* px, const float* py, const float* pz,
                             const float* nx, const float* ny, const float* nz, const float* ix,
                             const float* iy, const float* iz, const uint32_t* material,
                             const uint8_t* hit, uint32_t n_lights, const float* lights,
                             int shadow_cull, float* ox, float* oy, float* oz, float* dx, float* dy,
                             float* dz, float* tmax, uint8_t* type, uint8_t* light, uint32_t* pixel) {
    int64_t n = 0;
    const float eps = 1e-4f;
    const float shorten = 0.9999f;
    const float ior = 1.5f;
    for (uint32_t p = 0; p < n_pixels; ++p) {
        if (!hit[p]) continue;
        float P[3] = {px[p], py[p], pz[p]};
        float N[3] = {nx[p], ny[p], nz[p]};
        float I[3] = {ix[p], iy[p], iz[p]};
        for (uint32_t k = 0; k < n_lights; ++k) {
            float L[3] = {lights[3 * k], lights[3 * k + 1], lights[3 * k + 2]};
            float v0 = P[0] - L[0], v1 = P[1] - L[1], v2 = P[2] - L[2];
            float facing = N[0] * v0;
            facing = facing + N[1] * v1;
            facing = facing + N[2] * v2;
            if (shadow_cull && !(facing < 0.0f)) continue;
            float len = len3f(v0, v1, v2);
            if (!(len > 0.0f)) continue;
            ox[n] = L[0]; oy[n] = L[1]; oz[n] = L[2];
            dx[n] = v0 / len; dy[n] = v1 / len; dz[n] = v2 / len;
            tmax[n] = len * shorten;
            type[n] = RAY_SHADOW; light[n] = (uint8_t)k; pixel[n] = p;
            ++n;
        }
        uint32_t m = material[p];
        if (m != MAT_MIRROR && m != MAT_GLASS) continue;
        float c = I[0] * N[0];
        c = c + I[1] * N[1];
        c = c + I[2] * N[2];
        float side = (c > 0.0f) ? -1.0f : 1.0f;   /* s: which side the incident ray came from */
        float off = eps * side;
        {   /* reflection */
            float two_c = 2.0f * c;
            float r0 = I[0] - two_c * N[0], r1 = I[1] - two_c * N[1], r2 = I[2] - two_c * N[2];
            float rl = len3f(r0, r1, r2);
            ox[n] = P[0] + off * N[0]; oy[n] = P[1] + off * N[1]; oz[n] = P[2] + off * N[2];
            dx[n] = r0 / rl; dy[n] = r1 / rl; dz[n] = r2 / rl;
            tmax[n] = INFINITY;
            type[n] = RAY_REFLECTION; light[n] = 0; pixel[n] = p;
            ++n;
        }
        if (m == MAT_GLASS) {   /* refraction */
            float eta, cosi, M0, M1, M2;
            if (c < 0.0f) { eta = 1.0f / ior; cosi = -c; M0 = N[0]; M1 = N[1]; M2 = N[2]; }
            else { eta = ior; cosi = c; M0 = -N[0]; M1 = -N[1]; M2 = -N[2]; }
            float sin2 = 1.0f - cosi * cosi;
            float k = 1.0f - (eta * eta) * sin2;
            if (k < 0.0f) continue;   /* total internal reflection: no ray */
            float coef = eta * cosi - sqrtf(k);
            float t0 = eta * I[0] + coef * M0, t1 = eta * I[1] + coef * M1, t2 = eta * I[2] + coef * M2;
            float tl = len3f(t0, t1, t2);
            ox[n] = P[0] - off * N[0]; oy[n] = P[1] - off * N[1]; oz[n] = P[2] - off * N[2];
            dx[n] = t0 / tl; dy[n] = t1 / tl; dz[n] = t2 / tl;
            tmax[n] = INFINITY;
            type[n] = RAY_REFRACTION; light[n] = 0; pixel[n] = p;
            ++n;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Section 3.3.2, Figures 2-3: per-ray-type hash keys.                        */
/* ------------------------------------------------------------------------ */
/* READING (figures missing): 32-bit key, ray type in bits 31:30.
 *   shadow:     [29 : tb+pb] light index | [tb+pb-1 : 0] direction code
 *   refl/refr:  [29 : tb+pb] Morton-interleaved origin cell (cb bits per axis)
 *               | [tb+pb-1 : 0] direction code
 * The direction code is the Z-order interleave of the theta and phi bins, so
 * that runs of consecutive keys cover compact patches of directions (a
 * theta-major concatenation makes runs into thin rings of constant theta).
 * No facing cull or light bits beyond the layout: the caller keeps the light
 * count within 2^(30 - tb - pb).
 * Spherical coordinates of the direction [Pae95]: theta = acos(dz) in [0, pi],
 * phi = atan2(dy, dx) in [0, 2 pi).  Bins are defined by comparisons with
 * FP32 tables so that any two implementations agree bit for bit:
 *   cosT[k] = fl32(cos(k pi / Btheta)), theta bin = #{k in [1, Btheta-1] : dz < cosT[k]}
 *   tanT[j] = fl32(tan(j (pi/4) / M)), M = Bphi / 8.  The quadrant q
 *   (phi in [q pi/2, (q+1) pi/2), chosen by the signs of dx, dy) is rotated
 *   onto the first one, giving (a, b) with a > 0, b >= 0; then
 *   psi bin = #{j in [1, M-1] : b/a >= tanT[j]}          if b < a,
 *           = 2M - 1 - #{j in [1, M-1] : a/b > tanT[j]}   otherwise,
 *   and phi bin = q Bphi/4 + psi bin.  The pole (dx = dy = 0) has phi bin 0. */

typedef struct {
    float lo[3], hi[3];
    uint32_t shadow_theta_bits, shadow_phi_bits;
    uint32_t sec_cell_bits, sec_theta_bits, sec_phi_bits;
} oracle_hash_params;

/* number of k in [1, B-1] with dz < cosT[k]; the table is non-increasing in k,
 * so the qualifying k form a prefix 1..count, found by bisection. */
static uint32_t theta_bin(float dz, const float* cosT, uint32_t B) {
    uint32_t lo = 0, hi = B - 1;   /* answer in [lo, hi] */
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo + 1) / 2;
        if (dz < cosT[mid]) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* number of j in [1, M-1] with r >= tanT[j] (tanT increasing). */
static uint32_t tan_count(float r, const float* tanT, uint32_t M) {
    uint32_t lo = 0, hi = M - 1;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo + 1) / 2;
        if (r >= tanT[mid]) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* quadrant q holds phi in [q pi/2, (q+1) pi/2); (a, b) is the direction turned
 * back into the first quadrant (a > 0, b >= 0) and psi = atan2(b, a). */
static uint32_t phi_bin(float x, float y, const float* tanT, uint32_t Bphi) {
    uint32_t M = Bphi / 8, Q = Bphi / 4, q;
    float a, b;
    if (x > 0.0f && y >= 0.0f) { q = 0; a = x; b = y; }
    else if (x <= 0.0f && y > 0.0f) { q = 1; a = y; b = -x; }
    else if (x < 0.0f && y <= 0.0f) { q = 2; a = -x; b = -y; }
    else if (x >= 0.0f && y < 0.0f) { q = 3; a = -y; b = x; }
    else return 0;   /* pole: dx = dy = 0 (or NaN) */
    uint32_t psi;
    if (b < a) {
        psi = tan_count(b / a, tanT, M);                  /* psi in [0, pi/4) */
    } else {                                              /* psi in [pi/4, pi/2) */
        float r = a / b;
        uint32_t lo = 0, hi = M - 1;                      /* #{j : r > tanT[j]} */
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo + 1) / 2;
            if (r > tanT[mid]) lo = mid; else hi = mid - 1;
        }
        psi = 2 * M - 1 - lo;
    }
    return q * Q + psi;
}

/* Z-order of the two spherical bins: from the least significant bit, phi bit
 * 0, theta bit 0, phi bit 1, theta bit 1, ...; the bits of the longer one that
 * have no partner follow in order. */
static uint32_t interleave2(uint32_t th, uint32_t tb, uint32_t ph, uint32_t pb) {
    uint32_t code = 0, pos = 0;
    uint32_t common = tb < pb ? tb : pb;
    for (uint32_t b = 0; b < common; ++b) {
        code |= ((ph >> b) & 1u) << pos++;
        code |= ((th >> b) & 1u) << pos++;
    }
    for (uint32_t b = common; b < pb; ++b) code |= ((ph >> b) & 1u) << pos++;
    for (uint32_t b = common; b < tb; ++b) code |= ((th >> b) & 1u) << pos++;
    return code;
}

static uint32_t morton3(uint32_t qx, uint32_t qy, uint32_t qz, uint32_t bits) {
    uint32_t code = 0;
    for (uint32_t b = 0; b < bits; ++b) {
        code |= ((qx >> b) & 1u) << (3 * b);
        code |= ((qy >> b) & 1u) << (3 * b + 1);
        code |= ((qz >> b) & 1u) << (3 * b + 2);
    }
    return code;
}

static uint32_t cell_coord(float o, float lo, float hi, uint32_t bits) {
    float cells = (float)(1u << bits);
    float scale = cells / (hi - lo);
    float q = floorf((o - lo) * scale);
    if (!(q >= 0.0f)) return 0;   /* also NaN */
    if (q > cells - 1.0f) return (1u << bits) - 1;
    return (uint32_t)q;
}

static float* make_cos_table(uint32_t B) {
    float* t = (float*)malloc(sizeof(float) * B);
    for (uint32_t k = 0; k < B; ++k) t[k] = (float)cos((double)k * O_PI / (double)B);
    return t;
}

static float* make_tan_table(uint32_t M) {
    float* t = (float*)malloc(sizeof(float) * M);
    for (uint32_t j = 0; j < M; ++j) t[j] = (float)tan((double)j * (O_PI / 4.0) / (double)M);
    return t;
}

/* The two threshold tables of a (theta bits, phi bits) layout, as the hash
 * above builds them: 2^theta_bits cosines and 2^phi_bits / 8 tangents. */
void oracle_tables(uint32_t theta_bits, uint32_t phi_bits, float* cos_out, float* tan_out) {
    float* c = make_cos_table(1u << theta_bits);
    float* t = make_tan_table((1u << phi_bits) / 8);
    memcpy(cos_out, c, sizeof(float) * (1u << theta_bits));
    memcpy(tan_out, t, sizeof(float) * ((1u << phi_bits) / 8));
    free(c);
    free(t);
}

/* Returns 0, or -1 for a parameter set the key layout cannot hold. */
int oracle_hash(int64_t n, const float* ox, const float* oy, const float* oz, const float* dx,
                const float* dy, const float* dz, const uint8_t* type, const uint8_t* light,
                const oracle_hash_params* hp, uint32_t* keys) {
    uint32_t stb = hp->shadow_theta_bits, spb = hp->shadow_phi_bits;
    uint32_t cb = hp->sec_cell_bits, tb = hp->sec_theta_bits, pb = hp->sec_phi_bits;
    if (stb < 1 || spb < 3 || stb + spb > 30 || tb < 1 || pb < 3 || 3 * cb + tb + pb > 30) return -1;
    float* cosS = make_cos_table(1u << stb);
    float* tanS = make_tan_table((1u << spb) / 8);
    float* cosR = make_cos_table(1u << tb);
    float* tanR = make_tan_table((1u << pb) / 8);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t key;
        if (type[i] == RAY_SHADOW) {
            uint32_t th = theta_bin(dz[i], cosS, 1u << stb);
            uint32_t ph = phi_bin(dx[i], dy[i], tanS, 1u << spb);
            key = ((uint32_t)light[i] << (stb + spb)) | interleave2(th, stb, ph, spb);
        } else {
            uint32_t th = theta_bin(dz[i], cosR, 1u << tb);
            uint32_t ph = phi_bin(dx[i], dy[i], tanR, 1u << pb);
            uint32_t cell = morton3(cell_coord(ox[i], hp->lo[0], hp->hi[0], cb),
                                    cell_coord(oy[i], hp->lo[1], hp->hi[1], cb),
                                    cell_coord(oz[i], hp->lo[2], hp->hi[2], cb), cb);
            key = ((uint32_t)type[i] << 30) | (cell << (tb + pb)) | interleave2(th, tb, ph, pb);
        }
        keys[i] = key;
    }
    free(cosS); free(tanS); free(cosR); free(tanR);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sections 3.3.3-3.3.5: compression, radix sort of chunks, decompression.   */
/* The three steps together place the rays in key order and keep equal keys */
/* in their original order (chunks keep their base order), i.e. they compute */
/* the stable sort of the ray indices by key, which is what is written here. */
/* ------------------------------------------------------------------------ */

typedef struct { uint32_t key, idx; } kv;

static int kv_cmp(const void* a, const void* b) {
    const kv* x = (const kv*)a;
    const kv* y = (const kv*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

void oracle_stable_sort(int64_t n, const uint32_t* keys, uint32_t* perm) {
    kv* a = (kv*)malloc(sizeof(kv) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { a[i].key = keys[i]; a[i].idx = (uint32_t)i; }
    qsort(a, (size_t)n, sizeof(kv), kv_cmp);
    for (int64_t i = 0; i < n; ++i) perm[i] = a[i].idx;
    free(a);
}

/* Section 3.3.3: one chunk per run of equal consecutive keys. */
int64_t oracle_chunk_count(int64_t n, const uint32_t* keys) {
    if (n == 0) return 0;
    int64_t c = 1;
    for (int64_t i = 1; i < n; ++i) c += keys[i] != keys[i - 1];
    return c;
}

/* ------------------------------------------------------------------------ */
/* Section 3.3.6: bottom-up hierarchy of sphere-cones (eqs. 1-8).            */
/* ------------------------------------------------------------------------ */
/* Node = 8 doubles: sphere centre (3), sphere radius, cone axis (3), spread.
 * READING: the spread is the cone's half-angle (eq. 4).  Level-1 node j holds
 * sorted rays [jB, min(jB+B, N)); level-l node j holds level-(l-1) nodes
 * [jB, min(jB+B, n_{l-1})).  Leaves: sphere of radius 0 at the ray origin,
 * cone of spread 0 along the ray (Section 3.3.6). */

typedef struct { double x, y, z; } d3;
static d3 D3(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static d3 dsub(d3 a, d3 b) { return D3(a.x - b.x, a.y - b.y, a.z - b.z); }
static d3 dadd(d3 a, d3 b) { return D3(a.x + b.x, a.y + b.y, a.z + b.z); }
static d3 dscl(d3 a, double s) { return D3(a.x * s, a.y * s, a.z * s); }
static double ddot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static d3 dcross(d3 a, d3 b) {
    return D3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double dlen(d3 a) { return sqrt(ddot(a, a)); }
static d3 dunit(d3 a) { return dscl(a, 1.0 / dlen(a)); }
/* angle between two directions, robust near 0 and pi */
static double dangle(d3 a, d3 b) { return atan2(dlen(dcross(a, b)), ddot(a, b)); }

typedef struct { d3 c; double r; d3 x; double phi; } node;

/* eqs. 7-8: union of two spheres (midpoint centre). */
static void sphere_union(node* a, const node* b) {
    d3 c = dscl(dadd(a->c, b->c), 0.5);
    double r = 0.5 * dlen(dsub(b->c, a->c)) + fmax(a->r, b->r);
    a->c = c;
    a->r = r;
}

/* eqs. 5-6: union of two cones.  READING of the garbled eq. 6: the new spread
 * is half the angle between the two axes plus the larger child spread, about
 * the normalised axis sum of eq. 5; axes that cancel give the whole sphere. */
static void cone_union(node* a, const node* b) {
    d3 s = dadd(a->x, b->x);
    double ls = dlen(s);
    if (a->phi >= O_PI || b->phi >= O_PI || ls <= 1e-12) {
        a->phi = O_PI;
        return;
    }
    double theta = dangle(a->x, b->x);
    a->x = dscl(s, 1.0 / ls);
    a->phi = fmin(O_PI, 0.5 * theta + fmax(a->phi, b->phi));
}

/* eqs. 1-4: widen the cone (x, phi) until it holds direction r [Sze06].
 * READING of the garbled eq. 1: q = ((r x x) x x)/|.|, the unit vector normal
 * to x, in the plane of x and r, pointing away from r; eq. 2 gives the far
 * edge e of the current cone, eq. 3 the new axis (bisector of e and r), eq. 4
 * the new spread, the angle between the new axis and r.
 * READING: eq. 3 bisects the arc from e to r through x only while that arc is
 * shorter than pi (theta + phi < pi); a wider result would reach a half-angle
 * of pi/2 or more, which eq. 9 accepts everywhere, so the cone becomes the
 * whole sphere (phi = pi). */
static void cone_add_ray(d3* x, double* phi, d3 r) {
    if (*phi >= O_PI) return;
    double theta = dangle(*x, r);
    if (theta <= *phi) return;
    if (theta + *phi >= O_PI - 1e-9) { *phi = O_PI; return; }
    d3 q = dunit(dcross(dcross(r, *x), *x));                    /* eq. 1 */
    d3 e = dadd(dscl(*x, cos(*phi)), dscl(q, sin(*phi)));      /* eq. 2 */
    *x = dunit(dadd(e, r));                                    /* eq. 3 */
    *phi = dangle(*x, r);                                      /* eq. 4 */
}

/* READING (the paper does not give the merge order for B > 2): the B items of
 * a node are merged as a balanced binary tree in item order: at step s = 1,
 * 2, 4, ..., item i (i a multiple of 2s) absorbs item i + s when it exists. */
static void tree_merge(node* items, int n, int spheres, int cones) {
    for (int s = 1; s < n; s *= 2)
        for (int i = 0; i + s < n; i += 2 * s) {
            if (spheres) sphere_union(&items[i], &items[i + s]);
            if (cones) cone_union(&items[i], &items[i + s]);
        }
}

/* READING (needed for a conservative FP32 hierarchy; the paper is silent):
 * after a node is built its radius becomes r (1 + sr) + sa and its spread
 * min(pi, phi (1 + cr) + ca). */
static void pad(node* nd, double sr, double sa, double cr, double ca) {
    nd->r = nd->r * (1.0 + sr) + sa;
    nd->phi = fmin(O_PI, nd->phi * (1.0 + cr) + ca);
}

static int64_t level_size(int64_t below, uint32_t B) { return (below + B - 1) / B; }

/* Builds levels 1..L over n sorted rays.  out: 8 doubles per node, level 1
 * first.  counts[l-1] = nodes of level l.  Returns total nodes. */
int64_t oracle_build(int64_t n, const float* ox, const float* oy, const float* oz, const float* dx,
                     const float* dy, const float* dz, uint32_t B, uint32_t L, double sr, double sa,
                     double cr, double ca, double* out, int64_t* counts) {
    int64_t total = 0;
    int64_t below = n;
    node* items = (node*)malloc(sizeof(node) * B);
    node* prev = NULL;
    for (uint32_t l = 1; l <= L; ++l) {
        int64_t cnt = level_size(below, B);
        counts[l - 1] = cnt;
        node* cur = (node*)malloc(sizeof(node) * (size_t)(cnt > 0 ? cnt : 1));
        for (int64_t j = 0; j < cnt; ++j) {
            int64_t first = j * B, last = first + B < below ? first + B : below;
            int m = (int)(last - first);
            if (l == 1) {
                /* cone: fold the rays in sorted order (eqs. 1-4) */
                d3 x = dunit(D3(dx[first], dy[first], dz[first]));
                double phi = 0.0;
                for (int64_t i = first + 1; i < last; ++i)
                    cone_add_ray(&x, &phi, dunit(D3(dx[i], dy[i], dz[i])));
                /* sphere: radius-0 leaves merged by eqs. 7-8 */
                for (int k = 0; k < m; ++k) {
                    items[k].c = D3(ox[first + k], oy[first + k], oz[first + k]);
                    items[k].r = 0.0;
                }
                tree_merge(items, m, 1, 0);
                cur[j].c = items[0].c;
                cur[j].r = items[0].r;
                cur[j].x = x;
                cur[j].phi = phi;
            } else {
                for (int k = 0; k < m; ++k) items[k] = prev[first + k];
                tree_merge(items, m, 1, 1);
                cur[j] = items[0];
            }
            pad(&cur[j], sr, sa, cr, ca);
        }
        for (int64_t j = 0; j < cnt; ++j) {
            double* o = out + 8 * (total + j);
            o[0] = cur[j].c.x; o[1] = cur[j].c.y; o[2] = cur[j].c.z; o[3] = cur[j].r;
            o[4] = cur[j].x.x; o[5] = cur[j].x.y; o[6] = cur[j].x.z; o[7] = cur[j].phi;
        }
        total += cnt;
        free(prev);
        prev = cur;
        below = cnt;
    }
    free(prev);
    free(items);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Section 3.3.7, eq. 9: sphere-cone test [Ama84, RAH07].                    */
/* ------------------------------------------------------------------------ */
/* READING of the unnamed variables: C = node sphere centre (cone apex), d =
 * node sphere radius, x = cone axis, alpha = spread, (P, r) = tested sphere,
 * H = projection of P on the axis line.  |C - H| is unsigned as printed (a
 * double cone: conservative).  alpha >= pi/2 - 1e-6 accepts everything. */
int oracle_sphere_cone(const double* nd, double Px, double Py, double Pz, double r) {
    double alpha = nd[7];
    if (alpha >= O_PI / 2 - 1e-6) return 1;
    d3 C = D3(nd[0], nd[1], nd[2]);
    d3 x = dunit(D3(nd[4], nd[5], nd[6]));
    d3 v = dsub(D3(Px, Py, Pz), C);
    double s = ddot(v, x);
    d3 PH = dsub(v, dscl(x, s));
    double lhs = fabs(s) * tan(alpha) + (nd[3] + r) / cos(alpha);
    return lhs >= dlen(PH);
}

/* READING (the paper does not say which triangle sphere): centroid centre,
 * radius the largest vertex distance. */
static void tri_sphere(const float* v, double* s) {
    d3 a = D3(v[0], v[1], v[2]), b = D3(v[3], v[4], v[5]), c = D3(v[6], v[7], v[8]);
    d3 m = dscl(dadd(dadd(a, b), c), 1.0 / 3.0);
    double r = fmax(dlen(dsub(a, m)), fmax(dlen(dsub(b, m)), dlen(dsub(c, m))));
    s[0] = m.x; s[1] = m.y; s[2] = m.z; s[3] = r;
}

void oracle_tri_spheres(int64_t n_tris, const float* verts, double* out) {
    for (int64_t t = 0; t < n_tris; ++t) tri_sphere(verts + 9 * t, out + 4 * t);
}

/* Counters in the schema of Tables 1-3 (index l-1 for level l). */
typedef struct {
    int64_t mesh_tests, mesh_hits;
    int64_t tests[8], hits[8], tests_paper[8];
    int64_t final_tests, final_tests_paper, final_hits;
} oracle_counters;

typedef struct { uint32_t* node; uint32_t* tri; int64_t n, cap; } pairlist;

static void push(pairlist* p, uint32_t nd, uint32_t t) {
    if (p->n == p->cap) {
        p->cap = p->cap ? 2 * p->cap : 1024;
        p->node = (uint32_t*)realloc(p->node, sizeof(uint32_t) * (size_t)p->cap);
        p->tri = (uint32_t*)realloc(p->tri, sizeof(uint32_t) * (size_t)p->cap);
    }
    p->node[p->n] = nd;
    p->tri[p->n] = t;
    ++p->n;
}

/* Top-down traversal (Section 3.3.7).  nodes: 8 doubles per node, level 1
 * first, counts per level.  Top level: every top node against every whole-mesh
 * sphere, then against the triangle spheres of the meshes it hits (all meshes
 * when mesh_cull == 0, the unsorted-RSH comparison mode).  Level l < L: every
 * pair (p, t) of level l+1 expands to the children of p, each tested against
 * t.  Pair lists are produced grouped by node, triangles in increasing id.
 * Returns level-1 pairs in malloc'd arrays (free with oracle_free).
 * Counting: tests = sphere-cone tests actually made; tests_paper counts B per
 * parent pair, the convention that reproduces Tables 1-4; mesh tests are kept
 * apart (the tables leave them out). */
int64_t oracle_traverse(const double* nodes, const int64_t* counts, uint32_t B, uint32_t L,
                        int64_t n_tris, const float* verts, uint32_t n_meshes,
                        const uint32_t* mesh_first_tri, const float* mesh_sphere, int mesh_cull,
                        uint32_t** out_node, uint32_t** out_tri, oracle_counters* ctr) {
    memset(ctr, 0, sizeof(*ctr));
    double* ts = (double*)malloc(sizeof(double) * 4 * (size_t)(n_tris > 0 ? n_tris : 1));
    oracle_tri_spheres(n_tris, verts, ts);
    int64_t* base = (int64_t*)malloc(sizeof(int64_t) * (L + 1));
    base[0] = 0;
    for (uint32_t l = 1; l <= L; ++l) base[l] = base[l - 1] + counts[l - 1];
    pairlist cur = {0, 0, 0, 0};
    /* top level */
    {
        uint32_t l = L;
        const double* lv = nodes + 8 * base[l - 1];
        for (int64_t nd = 0; nd < counts[l - 1]; ++nd) {
            for (uint32_t m = 0; m < n_meshes; ++m) {
                if (mesh_cull) {
                    ++ctr->mesh_tests;
                    const float* s = mesh_sphere + 4 * m;
                    if (!oracle_sphere_cone(lv + 8 * nd, s[0], s[1], s[2], s[3])) continue;
                    ++ctr->mesh_hits;
                }
                for (uint32_t t = mesh_first_tri[m]; t < mesh_first_tri[m + 1]; ++t) {
                    ++ctr->tests[l - 1];
                    ++ctr->tests_paper[l - 1];
                    const double* s = ts + 4 * t;
                    if (oracle_sphere_cone(lv + 8 * nd, s[0], s[1], s[2], s[3])) push(&cur, (uint32_t)nd, t);
                }
            }
        }
        ctr->hits[l - 1] = cur.n;
    }
    /* levels L-1 .. 1 */
    for (uint32_t l = L - 1; l >= 1; --l) {
        const double* lv = nodes + 8 * base[l - 1];
        int64_t nl = counts[l - 1];
        pairlist nxt = {0, 0, 0, 0};
        int64_t i = 0;
        while (i < cur.n) {   /* one parent node's run of pairs */
            uint32_t p = cur.node[i];
            int64_t j = i;
            while (j < cur.n && cur.node[j] == p) ++j;
            for (uint32_t c = 0; c < B; ++c) {
                int64_t child = (int64_t)p * B + c;
                for (int64_t k = i; k < j; ++k) {
                    ++ctr->tests_paper[l - 1];
                    if (child >= nl) continue;   /* padded slot of a partial last node */
                    ++ctr->tests[l - 1];
                    const double* s = ts + 4 * cur.tri[k];
                    if (oracle_sphere_cone(lv + 8 * child, s[0], s[1], s[2], s[3]))
                        push(&nxt, (uint32_t)child, cur.tri[k]);
                }
            }
            i = j;
        }
        free(cur.node);
        free(cur.tri);
        cur = nxt;
        ctr->hits[l - 1] = cur.n;
        if (l == 1) break;
    }
    free(ts);
    free(base);
    *out_node = cur.node;
    *out_tri = cur.tri;
    return cur.n;
}

void oracle_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Section 3.3.8: final ray-triangle tests, Moller-Trumbore [Mol97].          */
/* ------------------------------------------------------------------------ */
/* READING (the paper gives no tolerances): two-sided, rejected only when the
 * determinant is exactly 0, inclusive barycentric bounds (u >= 0, v >= 0,
 * u + v <= 1), and 0 < t <= t_max.  t is in units of the stored direction. */
int oracle_mt(double ox, double oy, double oz, double dx, double dy, double dz, double tmax,
              const float* v, double* t_out, double* u_out, double* v_out) {
    d3 o = D3(ox, oy, oz), d = D3(dx, dy, dz);
    d3 v0 = D3(v[0], v[1], v[2]), v1 = D3(v[3], v[4], v[5]), v2 = D3(v[6], v[7], v[8]);
    d3 e1 = dsub(v1, v0), e2 = dsub(v2, v0);
    d3 p = dcross(d, e2);
    double det = ddot(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    d3 s = dsub(o, v0);
    double u = ddot(s, p) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    d3 q = dcross(s, e1);
    double w = ddot(d, q) * inv;
    if (w < 0.0 || u + w > 1.0) return 0;
    double t = ddot(e2, q) * inv;
    if (!(t > 0.0 && t <= tmax)) return 0;
    *t_out = t;
    *u_out = u;
    *v_out = w;
    return 1;
}

/* closest hit = smallest t; READING: equal t goes to the smaller triangle id. */
static int better(double t, uint32_t tri, double bt, int32_t btri) {
    return btri < 0 || t < bt || (t == bt && (int32_t)tri < btri);
}

/* Brute force N x M (Section 1): the definition the hierarchy must reproduce. */
void oracle_bruteforce(int64_t n, const float* ox, const float* oy, const float* oz, const float* dx,
                       const float* dy, const float* dz, const float* tmax, int64_t n_tris,
                       const float* verts, int32_t* hit_tri, double* hit_t, double* hit_u,
                       double* hit_v) {
    for (int64_t i = 0; i < n; ++i) {
        int32_t bt = -1;
        double tb = 0, ub = 0, vb = 0;
        for (int64_t t = 0; t < n_tris; ++t) {
            double tt, uu, vv;
            if (oracle_mt(ox[i], oy[i], oz[i], dx[i], dy[i], dz[i], tmax[i], verts + 9 * t, &tt, &uu, &vv) &&
                better(tt, (uint32_t)t, tb, bt)) {
                bt = (int32_t)t; tb = tt; ub = uu; vb = vv;
            }
        }
        hit_tri[i] = bt; hit_t[i] = tb; hit_u[i] = ub; hit_v[i] = vb;
    }
}

/* Final tests over the level-1 pair list: every ray of node n against every
 * triangle paired with n; closest hit per ray, written at the ray's original
 * index perm[sorted position] (Section 3.3.6: rays map back to their pixels). */
void oracle_final(int64_t n_pairs, const uint32_t* pair_node, const uint32_t* pair_tri, uint32_t B,
                  int64_t n, const float* ox, const float* oy, const float* oz, const float* dx,
                  const float* dy, const float* dz, const float* tmax, const uint32_t* perm,
                  const float* verts, int32_t* hit_tri, double* hit_t, double* hit_u, double* hit_v,
                  oracle_counters* ctr) {
    for (int64_t i = 0; i < n; ++i) { hit_tri[i] = -1; hit_t[i] = hit_u[i] = hit_v[i] = 0.0; }
    ctr->final_tests = ctr->final_tests_paper = ctr->final_hits = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        int64_t first = (int64_t)pair_node[k] * B, last = first + B < n ? first + B : n;
        uint32_t t = pair_tri[k];
        ctr->final_tests_paper += B;
        for (int64_t s = first; s < last; ++s) {
            ++ctr->final_tests;
            double tt, uu, vv;
            if (!oracle_mt(ox[s], oy[s], oz[s], dx[s], dy[s], dz[s], tmax[s], verts + 9 * t, &tt, &uu, &vv))
                continue;
            ++ctr->final_hits;
            uint32_t r = perm[s];
            if (better(tt, t, hit_t[r], hit_tri[r])) {
                hit_tri[r] = (int32_t)t; hit_t[r] = tt; hit_u[r] = uu; hit_v[r] = vv;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Invariants of a hierarchy given in FP32 (e.g. produced elsewhere),        */
/* checked exactly in FP64: every level-1 sphere holds its rays' origins and  */
/* every cone their directions; every upper node holds its children.          */
/* sphere/cone: 4 floats per node, level 1 first.  Returns the violations.    */
/* ------------------------------------------------------------------------ */
int64_t oracle_check_hierarchy(int64_t n, const float* ox, const float* oy, const float* oz,
                               const float* dx, const float* dy, const float* dz, uint32_t B,
                               uint32_t L, const int64_t* counts, const float* sphere,
                               const float* cone, double* worst) {
    int64_t bad = 0, base = 0;
    double w = -INFINITY;
    for (uint32_t l = 1; l <= L; ++l) {
        int64_t below = (l == 1) ? n : counts[l - 2];
        int64_t pbase = base - (l == 1 ? 0 : counts[l - 2]);
        for (int64_t j = 0; j < counts[l - 1]; ++j) {
            const float* S = sphere + 4 * (base + j);
            const float* K = cone + 4 * (base + j);
            d3 c = D3(S[0], S[1], S[2]);
            d3 x = dunit(D3(K[0], K[1], K[2]));
            double r = S[3], phi = K[3];
            int64_t first = j * B, last = first + B < below ? first + B : below;
            for (int64_t i = first; i < last; ++i) {
                double ds, da;
                if (l == 1) {
                    ds = dlen(dsub(D3(ox[i], oy[i], oz[i]), c)) - r;
                    da = dangle(x, dunit(D3(dx[i], dy[i], dz[i]))) - phi;
                } else {
                    const float* cs = sphere + 4 * (pbase + i);
                    const float* ck = cone + 4 * (pbase + i);
                    ds = dlen(dsub(D3(cs[0], cs[1], cs[2]), c)) + cs[3] - r;
                    da = (ck[3] >= O_PI) ? (phi >= O_PI ? -1.0 : 1.0)
                                         : dangle(x, dunit(D3(ck[0], ck[1], ck[2]))) + ck[3] - phi;
                }
                if (phi >= O_PI) da = -1.0;
                if (ds > 0.0 || da > 0.0) ++bad;
                if (ds > w) w = ds;
                if (da > w) w = da;
            }
        }
        base += counts[l - 1];
    }
    if (worst) *worst = w;
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Gradients of the closest hit (not a step of the paper: the adjoint of the  */
/* final test, Section 3.3.8, with the hit assignment held fixed).            */
/* ------------------------------------------------------------------------ */
/* For a ray o + t d hitting triangle (V0, V1, V2) at barycentrics (u, v),
 * F = o + t d - V0 - u (V1 - V0) - v (V2 - V0) = 0 defines (t, u, v)
 * implicitly.  With A = [-d | e1 | e2] (columns) and an upstream gradient
 * g = dL/d(t, u, v), the implicit-function theorem gives lambda = A^-T g and
 *   dL/do = lambda, dL/dd = t lambda,
 *   dL/dV0 = -(1 - u - v) lambda, dL/dV1 = -u lambda, dL/dV2 = -v lambda.
 * A^T lambda = g is solved here by Cramer's rule with 3x3 determinants.
 * Rays with tri < 0 contribute nothing.  FP64 throughout. */
static double det3(const double m[3][3]) {
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

void oracle_adjoint(int64_t n, const float* ox, const float* oy, const float* oz, const float* dx, const float* dy,
                    const float* dz, const int32_t* tri, const double* t, const double* u, const double* v,
                    const double* g_t, const double* g_u, const double* g_v, int64_t n_tris, const float* verts,
                    double* g_verts, double* g_orig, double* g_dir) {
    (void)ox; (void)oy; (void)oz;
    for (int64_t k = 0; k < 9 * n_tris; ++k) g_verts[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) g_orig[3 * i + c] = g_dir[3 * i + c] = 0.0;
        if (tri[i] < 0) continue;
        const float* V = verts + 9 * (int64_t)tri[i];
        double e1[3], e2[3], d[3] = {dx[i], dy[i], dz[i]};
        for (int c = 0; c < 3; ++c) { e1[c] = (double)V[3 + c] - V[c]; e2[c] = (double)V[6 + c] - V[c]; }
        /* A^T: rows -d, e1, e2 */
        double M[3][3], g[3] = {g_t[i], g_u[i], g_v[i]}, lam[3];
        for (int c = 0; c < 3; ++c) { M[0][c] = -d[c]; M[1][c] = e1[c]; M[2][c] = e2[c]; }
        double D = det3(M);
        if (D == 0.0) continue;
        for (int col = 0; col < 3; ++col) {
            double Mc[3][3];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) Mc[r][c] = (c == col) ? g[r] : M[r][c];
            lam[col] = det3(Mc) / D;
        }
        double w0 = -(1.0 - u[i] - v[i]), w1 = -u[i], w2 = -v[i];
        for (int c = 0; c < 3; ++c) {
            g_orig[3 * i + c] = lam[c];
            g_dir[3 * i + c] = t[i] * lam[c];
            g_verts[9 * (int64_t)tri[i] + c] += w0 * lam[c];
            g_verts[9 * (int64_t)tri[i] + 3 + c] += w1 * lam[c];
            g_verts[9 * (int64_t)tri[i] + 6 + c] += w2 * lam[c];
        }
    }
}

/* ---- Primary visibility and first-hit buffers (NEXT row f3) ------------
 * The paper rasterises the primary hits (Section 3.2); here camera rays go
 * through the same traced path, and first-hit buffers are written from
 * closest hits: the G-buffer for primary rays, and for secondary rays the
 * hit points the next bounce is generated from (Section 3.3.8). */

/* Camera rays of a w x h pinhole camera, cam = eye[3], fwd[3], right[3],
 * up[3], tan_x, tan_y.  Pixel (x, y) looks along fwd + sx right + sy up with
 * sx = (2 (x + 0.5) / w - 1) tan_x and sy = (1 - 2 (y + 0.5) / h) tan_y,
 * normalised as d / sqrt(d.d); FP32, fixed order.  The rays are listed in
 * tile order: 8 x 8 pixel blocks in block-row-major order and, inside a
 * block, the pixels in Z order (x bit b at 2b, y bit b at 2b + 1), pixels
 * outside the image skipped.  Returns the ray count. */
int64_t oracle_primary_rays(const float* cam, uint32_t w, uint32_t h, float* ox, float* oy, float* oz, float* dx,
                            float* dy, float* dz, uint32_t* pixel) {
    int64_t n = 0;
    for (uint32_t by = 0; by * 8 < h; ++by)
        for (uint32_t bx = 0; bx * 8 < w; ++bx)
            for (uint32_t z = 0; z < 64; ++z) {
                uint32_t lx = 0, ly = 0;
                for (int b = 0; b < 3; ++b) {
                    lx |= ((z >> (2 * b)) & 1u) << b;
                    ly |= ((z >> (2 * b + 1)) & 1u) << b;
                }
                uint32_t x = 8 * bx + lx, y = 8 * by + ly;
                if (x >= w || y >= h) continue;
                float sx = (2.0f * ((float)x + 0.5f)) / (float)w;
                sx = (sx - 1.0f) * cam[12];
                float sy = (2.0f * ((float)y + 0.5f)) / (float)h;
                sy = (1.0f - sy) * cam[13];
                float d[3];
                for (int a = 0; a < 3; ++a) {
                    float v = cam[3 + a] + sx * cam[6 + a];
                    d[a] = v + sy * cam[9 + a];
                }
                float len = len3f(d[0], d[1], d[2]);
                ox[n] = cam[0]; oy[n] = cam[1]; oz[n] = cam[2];
                dx[n] = d[0] / len; dy[n] = d[1] / len; dz[n] = d[2] / len;
                pixel[n] = y * w + x;
                ++n;
            }
    return n;
}

/* First-hit buffer entry g of ray g = (o, d) with hit (tri[g], t[g]): on a
 * hit, position o + t d, normal (v1 - v0) x (v2 - v0) normalised and turned
 * to face the ray (n.d <= 0), incident d, material tri_material[tri]; on a
 * miss zeros except the incident direction.  FP32, fixed order. */
void oracle_gbuffer_from_hits(int64_t n, const float* ox, const float* oy, const float* oz, const float* dx,
                              const float* dy, const float* dz, const int32_t* tri, const float* t,
                              const float* verts, const int32_t* tri_material, float* px, float* py, float* pz,
                              float* nx, float* ny, float* nz, float* ix, float* iy, float* iz, uint32_t* material,
                              uint8_t* hit) {
    for (int64_t g = 0; g < n; ++g) {
        ix[g] = dx[g]; iy[g] = dy[g]; iz[g] = dz[g];
        if (tri[g] < 0) {
            px[g] = py[g] = pz[g] = 0.0f;
            nx[g] = ny[g] = nz[g] = 0.0f;
            material[g] = 0;
            hit[g] = 0;
            continue;
        }
        const float* v = verts + 9 * (int64_t)tri[g];
        float tt = t[g];
        float a = tt * dx[g]; px[g] = ox[g] + a;
        a = tt * dy[g]; py[g] = oy[g] + a;
        a = tt * dz[g]; pz[g] = oz[g] + a;
        float e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
        float e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
        float p, q;
        p = e1y * e2z; q = e1z * e2y; float cx = p - q;
        p = e1z * e2x; q = e1x * e2z; float cy = p - q;
        p = e1x * e2y; q = e1y * e2x; float cz = p - q;
        float len = len3f(cx, cy, cz);
        cx = cx / len; cy = cy / len; cz = cz / len;
        float f = cx * dx[g];
        f = f + cy * dy[g];
        f = f + cz * dz[g];
        if (f > 0.0f) { cx = -cx; cy = -cy; cz = -cz; }
        nx[g] = cx; ny[g] = cy; nz[g] = cz;
        material[g] = (uint32_t)tri_material[tri[g]];
        hit[g] = 1;
    }
}

/* ---- Shading accumulation (NEXT row f4; Section 3.3.8 accumulates shading
 * after the final tests; the paper names no model, so this is a reading):
 * grey level per pixel, Lambert with hard shadows plus one mirror/glass
 * bounce.  Material m: albedo a = (0.8, 0.2, 0.1), reflectance k_r =
 * (0, 0.8, 0.1), transmittance k_t = (0, 0, 0.8); ambient 0.1, sky 0.6.
 *   no primary hit: sky
 *   else a (ambient + sum_k S_k) + k_r R + k_t T, in this order, with
 *   S_k = max(0, n . (-d)) for light k's shadow ray when it has no hit (0 if
 *   it hit something or was not emitted), R / T = a(hit material) x
 *   (ambient + 0.5) when the reflection / refraction ray hit, sky when it
 *   missed, 0 when it was not emitted.  FP32, fixed order.
 * Rays in generation order with their light index; tri[g] = closest hit of
 * ray g (-1 = miss). */
void oracle_shade(uint32_t n_pixels, const float* nx, const float* ny, const float* nz, const uint32_t* material,
                  const uint8_t* hit, int64_t n_rays, const float* dx, const float* dy, const float* dz,
                  const uint8_t* type, const uint8_t* light, const uint32_t* pixel, const int32_t* tri,
                  const int32_t* tri_material, uint32_t n_lights, float* color) {
    const float albedo[3] = {0.8f, 0.2f, 0.1f}, refl[3] = {0.0f, 0.8f, 0.1f}, trans[3] = {0.0f, 0.0f, 0.8f};
    const float ambient = 0.1f, sky = 0.6f, bounce = 0.5f;
    const size_t S = (size_t)n_lights + 2;
    float* cell = (float*)calloc((size_t)n_pixels * S, sizeof(float));
    for (int64_t g = 0; g < n_rays; ++g) {
        uint32_t p = pixel[g];
        if (type[g] == RAY_SHADOW) {
            float v = 0.0f;
            if (tri[g] < 0) {
                float c = nx[p] * -dx[g];
                c = c + ny[p] * -dy[g];
                c = c + nz[p] * -dz[g];
                v = c > 0.0f ? c : 0.0f;
            }
            cell[p * S + light[g]] = v;
        } else {
            float v = sky;
            if (tri[g] >= 0) {
                uint32_t hm = (uint32_t)tri_material[tri[g]];
                v = albedo[hm <= 2 ? hm : 0] * (ambient + bounce);
            }
            cell[p * S + n_lights + (type[g] == RAY_REFRACTION ? 1 : 0)] = v;
        }
    }
    for (uint32_t p = 0; p < n_pixels; ++p) {
        if (!hit[p]) { color[p] = sky; continue; }
        uint32_t m = material[p] <= 2 ? material[p] : 0;
        float s = ambient;
        for (uint32_t k = 0; k < n_lights; ++k) s = s + cell[p * S + k];
        float col = albedo[m] * s;
        col = col + refl[m] * cell[p * S + n_lights];
        col = col + trans[m] * cell[p * S + n_lights + 1];
        color[p] = col;
    }
    free(cell);
}
