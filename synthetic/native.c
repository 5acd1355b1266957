/* Native helpers of the synthetic input generator.
 *
 *  - synth_raster_gbuffer: primary visibility.  It stands in for the
 *    rasterization pass that fills the G-buffer before any secondary ray is
 *    traced (Section 3.2): for every pixel centre the nearest triangle hit by
 *    the camera ray, found in double precision with screen-space bounding-box
 *    culling.  Output per pixel: position, viewer-facing unit geometric normal,
 *    unit incident direction, material and a hit flag.
 *  - synth_min_ball: smallest enclosing sphere of a point set (Welzl's
 *    randomised algorithm, the problem solved offline per mesh in Section 3.3.1
 *    with Gaertner's method), used as the whole-mesh bounding sphere.
 *
 * Input generation only: nothing here is a step of the traced method.
 * Plain C99, no architecture-specific code; identical results on x86-64 and
 * aarch64 (built with -ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double norm(v3 a) { return sqrt(dot(a, a)); }

/* Camera: eye, forward (unit), right (unit), up (unit), tan of half the
 * horizontal and vertical field of view. */
typedef struct { v3 eye, fwd, right, up; double tanx, tany; int w, h; } camera;

static v3 pixel_dir(const camera* c, int px, int py) {
    double sx = (2.0 * (px + 0.5) / c->w - 1.0) * c->tanx;
    double sy = (1.0 - 2.0 * (py + 0.5) / c->h) * c->tany;
    v3 d = add(c->fwd, add(scl(c->right, sx), scl(c->up, sy)));
    return scl(d, 1.0 / norm(d));
}

/* Ray-plane distance plus an inclusive inside test on the three edges. */
static int hit_tri(v3 o, v3 d, v3 a, v3 b, v3 c, double* t_out) {
    v3 e1 = sub(b, a), e2 = sub(c, a);
    v3 n = cross(e1, e2);
    double den = dot(n, d);
    if (den == 0.0) return 0;
    double t = dot(n, sub(a, o)) / den;
    if (!(t > 1e-9)) return 0;
    v3 p = add(o, scl(d, t));
    if (dot(n, cross(sub(b, a), sub(p, a))) < 0.0) return 0;
    if (dot(n, cross(sub(c, b), sub(p, b))) < 0.0) return 0;
    if (dot(n, cross(sub(a, c), sub(p, c))) < 0.0) return 0;
    *t_out = t;
    return 1;
}

/* verts: n_tri x 3 vertices x 3 floats.  cam: eye[3], fwd[3], right[3], up[3],
 * tanx, tany.  Returns the number of hit pixels. */
int synth_raster_gbuffer(int w, int h, const double* cam_in, int n_tri, const float* verts,
                         const int32_t* tri_material,
                         float* px, float* py, float* pz, float* nx, float* ny, float* nz,
                         float* ix, float* iy, float* iz, uint32_t* material, uint8_t* hit,
                         int32_t* tri_out) {
    camera c;
    c.eye = mk(cam_in[0], cam_in[1], cam_in[2]);
    c.fwd = mk(cam_in[3], cam_in[4], cam_in[5]);
    c.right = mk(cam_in[6], cam_in[7], cam_in[8]);
    c.up = mk(cam_in[9], cam_in[10], cam_in[11]);
    c.tanx = cam_in[12];
    c.tany = cam_in[13];
    c.w = w;
    c.h = h;
    size_t np = (size_t)w * h;
    double* tbuf = (double*)malloc(np * sizeof(double));
    v3* dirs = (v3*)malloc(np * sizeof(v3));
    if (!tbuf || !dirs) { free(tbuf); free(dirs); return -1; }
    for (size_t p = 0; p < np; ++p) {
        tbuf[p] = INFINITY;
        tri_out[p] = -1;
        dirs[p] = pixel_dir(&c, (int)(p % w), (int)(p / w));
    }
    for (int t = 0; t < n_tri; ++t) {
        const float* f = verts + (size_t)9 * t;
        v3 a = mk(f[0], f[1], f[2]), b = mk(f[3], f[4], f[5]), cc = mk(f[6], f[7], f[8]);
        v3 vs[3] = {a, b, cc};
        int x0 = 0, x1 = w - 1, y0 = 0, y1 = h - 1, in_front = 1, behind = 0;
        double mnx = 1e300, mxx = -1e300, mny = 1e300, mxy = -1e300;
        for (int k = 0; k < 3; ++k)
            if (!(dot(sub(vs[k], c.eye), c.fwd) > 0.0)) ++behind;
        if (behind == 3) continue; /* entirely behind the camera: never visible */
        for (int k = 0; k < 3; ++k) {
            v3 r = sub(vs[k], c.eye);
            double z = dot(r, c.fwd);
            if (!(z > 1e-6)) { in_front = 0; break; }
            double sx = dot(r, c.right) / (z * c.tanx), sy = dot(r, c.up) / (z * c.tany);
            double qx = (sx + 1.0) * 0.5 * w - 0.5, qy = (1.0 - sy) * 0.5 * h - 0.5;
            if (qx < mnx) mnx = qx;
            if (qx > mxx) mxx = qx;
            if (qy < mny) mny = qy;
            if (qy > mxy) mxy = qy;
        }
        if (in_front) {
            if (mxx < -2.0 || mnx > w + 1.0 || mxy < -2.0 || mny > h + 1.0) continue;
            x0 = (int)floor(mnx) - 1; x1 = (int)ceil(mxx) + 1;
            y0 = (int)floor(mny) - 1; y1 = (int)ceil(mxy) + 1;
            if (x0 < 0) x0 = 0;
            if (y0 < 0) y0 = 0;
            if (x1 > w - 1) x1 = w - 1;
            if (y1 > h - 1) y1 = h - 1;
        }
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                size_t p = (size_t)y * w + x;
                double tt;
                if (hit_tri(c.eye, dirs[p], a, b, cc, &tt)) {
                    if (tt < tbuf[p]) { tbuf[p] = tt; tri_out[p] = t; }
                }
            }
    }
    int n_hit = 0;
    for (size_t p = 0; p < np; ++p) {
        v3 d = dirs[p];
        ix[p] = (float)d.x; iy[p] = (float)d.y; iz[p] = (float)d.z;
        if (tri_out[p] < 0) {
            hit[p] = 0; material[p] = 0;
            px[p] = py[p] = pz[p] = 0.0f;
            nx[p] = ny[p] = nz[p] = 0.0f;
            continue;
        }
        const float* f = verts + (size_t)9 * tri_out[p];
        v3 a = mk(f[0], f[1], f[2]), b = mk(f[3], f[4], f[5]), cc = mk(f[6], f[7], f[8]);
        v3 n = cross(sub(b, a), sub(cc, a));
        n = scl(n, 1.0 / norm(n));
        if (dot(n, d) > 0.0) n = scl(n, -1.0);
        v3 pos = add(c.eye, scl(d, tbuf[p]));
        px[p] = (float)pos.x; py[p] = (float)pos.y; pz[p] = (float)pos.z;
        nx[p] = (float)n.x; ny[p] = (float)n.y; nz[p] = (float)n.z;
        material[p] = (uint32_t)tri_material[tri_out[p]];
        hit[p] = 1;
        ++n_hit;
    }
    free(tbuf);
    free(dirs);
    return n_hit;
}

/* ---- smallest enclosing ball (Welzl, randomised incremental) ---- */

typedef struct { v3 c; double r; } ball;

static ball ball_pair(v3 a, v3 b) {
    ball s;
    s.c = scl(add(a, b), 0.5);
    s.r = 0.5 * norm(sub(b, a));
    return s;
}

static ball ball_three(v3 a, v3 b, v3 c) {
    v3 ab = sub(b, a), ac = sub(c, a);
    v3 n = cross(ab, ac);
    double den = 2.0 * dot(n, n);
    double scale = dot(ab, ab) * dot(ac, ac);
    if (den <= 1e-24 * scale || den == 0.0) {
        /* collinear: the ball of the farthest pair */
        ball s1 = ball_pair(a, b), s2 = ball_pair(a, c), s3 = ball_pair(b, c);
        ball s = s1;
        if (s2.r > s.r) s = s2;
        if (s3.r > s.r) s = s3;
        return s;
    }
    v3 num = add(scl(cross(n, ab), dot(ac, ac)), scl(cross(ac, n), dot(ab, ab)));
    ball s;
    s.c = add(a, scl(num, 1.0 / den));
    s.r = norm(sub(s.c, a));
    return s;
}

static ball ball_four(v3 a, v3 b, v3 c, v3 d) {
    v3 u = sub(b, a), v = sub(c, a), w = sub(d, a);
    double det = dot(u, cross(v, w));
    double scale = norm(u) * norm(v) * norm(w);
    if (fabs(det) <= 1e-12 * scale) {
        ball s = ball_three(a, b, c);
        double e = norm(sub(d, s.c));
        if (e > s.r) s.r = e;
        return s;
    }
    double uu = dot(u, u), vv = dot(v, v), ww = dot(w, w);
    v3 num = add(add(scl(cross(v, w), uu), scl(cross(w, u), vv)), scl(cross(u, v), ww));
    ball s;
    s.c = add(a, scl(num, 1.0 / (2.0 * det)));
    s.r = norm(sub(s.c, a));
    return s;
}

static ball support_ball(const v3* r, int nr) {
    ball s;
    if (nr == 0) { s.c = mk(0, 0, 0); s.r = -1.0; return s; }
    if (nr == 1) { s.c = r[0]; s.r = 0.0; return s; }
    if (nr == 2) return ball_pair(r[0], r[1]);
    if (nr == 3) return ball_three(r[0], r[1], r[2]);
    return ball_four(r[0], r[1], r[2], r[3]);
}

static int outside(ball s, v3 p) {
    if (s.r < 0.0) return 1;
    return norm(sub(p, s.c)) > s.r * (1.0 + 1e-12) + 1e-15;
}

static ball welzl(const v3* p, int n, v3* r, int nr) {
    ball s = support_ball(r, nr);
    if (nr == 4) return s;
    for (int i = 0; i < n; ++i) {
        if (outside(s, p[i])) {
            r[nr] = p[i];
            s = welzl(p, i, r, nr + 1);
        }
    }
    return s;
}

/* pts: n x 3 floats.  Writes centre (double[3]) and the radius that encloses
 * every point about that centre.  Points are visited in a seeded random
 * order (expected linear time). */
int synth_min_ball(int n, const float* pts, uint64_t seed, double* out_c, double* out_r) {
    if (n <= 0) return -1;
    v3* p = (v3*)malloc((size_t)n * sizeof(v3));
    if (!p) return -1;
    for (int i = 0; i < n; ++i) p[i] = mk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    uint64_t s = seed;
    for (int i = n - 1; i > 0; --i) {
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        int j = (int)((s >> 33) % (uint64_t)(i + 1));
        v3 tmp = p[i]; p[i] = p[j]; p[j] = tmp;
    }
    v3 r[4];
    ball b = welzl(p, n, r, 0);
    double rr = 0.0;
    for (int i = 0; i < n; ++i) {
        double e = norm(sub(p[i], b.c));
        if (e > rr) rr = e;
    }
    out_c[0] = b.c.x; out_c[1] = b.c.y; out_c[2] = b.c.z;
    *out_r = rr;
    free(p);
    return 0;
}
