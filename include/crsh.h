/* crsh.h - C ABI of the Coherent Ray-Space Hierarchy library for NVIDIA GB300
 * (sm_103a).
 *
 * Method: Reis, Costa, Pereira, "Ray-Tracing With a Coherent Ray-Space
 * Hierarchy" (arXiv 2312.06538).  The calls follow the paper's pipeline:
 *
 *   crsh_prepare_scene   triangle bounding spheres and Moller-Trumbore layout
 *   crsh_hash_sort       Section 3.3.2-3.3.5: secondary ray generation from the
 *                        primary-hit buffer, per-type hashing, trimming,
 *                        compression, radix sort, decompression
 *   crsh_build           Section 3.3.6, eqs. 1-8: bottom-up sphere-cone levels
 *   crsh_traverse        Section 3.3.7, eq. 9: whole-mesh then triangle culling,
 *                        top-down, into compacted (node, triangle) pair lists
 *   crsh_closest_hit     Section 3.3.8: final Moller-Trumbore tests, closest hit
 *   crsh_closest_hit_backward   gradients of the closest hit (not in the paper)
 *
 * Conventions shared by every call
 *  - Pointers inside the structs are DEVICE pointers unless a field says
 *    otherwise; the structs themselves live in host memory and are read during
 *    the call only.
 *  - The caller owns every buffer (inputs, outputs, workspaces).  The library
 *    allocates no device memory.  A workspace pointer must be 256-byte
 *    aligned (cudaMalloc's and PyTorch's allocations are); another one is an
 *    argument error.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *    default stream).  Data-dependent sizes (ray count, pair counts) stay on
 *    the device; no call synchronises with the host, so the sequence can be
 *    captured in a CUDA graph.
 *  - Argument errors are returned synchronously and nothing is launched.
 *    Errors found on the device (capacity exceeded, a wait that timed out)
 *    are recorded in crsh_counters.status (first error wins) and in the
 *    *_needed fields; read them after synchronising.  Results are then
 *    incomplete but every kernel still terminates.
 *  - Results are deterministic: identical inputs give identical bits.
 *  - Ray directions are expected to be finite and non-zero; t is measured in
 *    units of the stored direction vector.
 */
#ifndef CRSH_H
#define CRSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int crsh_status;
#define CRSH_OK                  0
#define CRSH_ERR_INVALID_ARG     1  /* bad pointer, size or parameter (synchronous) */
#define CRSH_ERR_CAPACITY        2  /* an output or workspace was too small (device) */
#define CRSH_ERR_CUDA            3  /* a CUDA runtime call failed (synchronous) */
#define CRSH_ERR_TIMEOUT         4  /* a bounded device-side wait gave up (device) */
#define CRSH_ERR_NOT_IMPLEMENTED 5
#define CRSH_ERR_BAD_INPUT       6  /* input data the method cannot use (device) */

#define CRSH_MAX_LEVELS 8

#define CRSH_RAY_SHADOW     0
#define CRSH_RAY_REFLECTION 1
#define CRSH_RAY_REFRACTION 2
#define CRSH_RAY_PRIMARY    3   /* camera rays from crsh_primary_rays; never hashed */

#define CRSH_MAT_DIFFUSE 0
#define CRSH_MAT_MIRROR  1
#define CRSH_MAT_GLASS   2

/* Primary-hit buffer (Section 3.2: the rasterised G-buffer of position,
 * normal and material that secondary rays start from), one entry per pixel,
 * structure of arrays. */
typedef struct {
    const float *px, *py, *pz;   /* hit position */
    const float *nx, *ny, *nz;   /* unit surface normal facing the viewer */
    const float *ix, *iy, *iz;   /* unit incident (camera ray) direction */
    const uint32_t *material;    /* CRSH_MAT_*; mirror: reflection ray, glass: reflection + refraction */
    const uint8_t *hit;          /* 1 if the pixel saw geometry */
    uint32_t n_pixels;
} crsh_gbuffer;

/* Rays given directly instead of a G-buffer (hashed and sorted as they are). */
typedef struct {
    const float *ox, *oy, *oz, *dx, *dy, *dz, *tmax;
    const uint8_t *type;         /* CRSH_RAY_* */
    const uint8_t *light;        /* light index of shadow rays (ignored otherwise) */
    uint32_t n;
} crsh_rays_in;

/* Hash and sort parameters (Section 3.3.2, Figures 2-3).  Key layout, 32 bits:
 *   [31:30] ray type
 *   shadow:      [29 : tb+pb] light index, [tb+pb-1 : 0] direction code
 *   refl./refr.: [29 : tb+pb] Morton code of the origin cell (cell_bits per
 *                axis over the box lo..hi), [tb+pb-1 : 0] direction code
 * The direction code is the Z-order interleave (phi bit first) of the
 * theta = acos(dz) bin (tb bits) and the phi = atan2(dy, dx) bin (pb bits);
 * bins are decided by comparison with FP32 tables of cos(k pi / 2^tb) and
 * tan(j pi / 2^pb), so every implementation gets the same keys. */
typedef struct {
    float lo[3], hi[3];            /* box of secondary-ray origins quantised into cells */
    uint32_t shadow_theta_bits;    /* default 13 */
    uint32_t shadow_phi_bits;      /* default 13; >= 3; light bits = 30 - theta - phi */
    uint32_t sec_cell_bits;        /* default 5 (per axis) */
    uint32_t sec_theta_bits;       /* default 7 */
    uint32_t sec_phi_bits;         /* default 8; 3*cell + theta + phi <= 30 */
    uint32_t shadow_cull;          /* 1: shadow ray only if n.(P - L) < 0 (light in front) */
    uint32_t sort;                 /* 0: keep generation order (the unsorted-RSH comparison mode) */
    uint32_t compress;             /* 1: compress equal-key runs into chunks before sorting */
} crsh_hash_params;

/* Sorted rays (output of crsh_hash_sort, input of every later call). */
typedef struct {
    float *ox, *oy, *oz, *dx, *dy, *dz, *tmax;
    uint8_t *type;                 /* CRSH_RAY_* */
    uint32_t *ray_id;              /* generation-order index of each sorted ray */
    uint32_t *pixel;               /* pixel (G-buffer input) or input index of each sorted ray */
    uint32_t capacity;             /* entries allocated in every array above */
} crsh_rays;

/* Counters in the schema of the paper's Tables 1-3, plus the device status.
 * Device memory, written by the calls. */
typedef struct {
    unsigned long long rays;       /* secondary rays after trimming */
    unsigned long long chunks;     /* chunks after compression (Section 3.3.3) */
    unsigned long long mesh_tests; /* top nodes x whole-mesh spheres tested */
    unsigned long long mesh_hits;
    unsigned long long tests[CRSH_MAX_LEVELS];        /* sphere-cone tests made, index l-1 = level l */
    unsigned long long hits[CRSH_MAX_LEVELS];         /* accepted (node, triangle) pairs */
    unsigned long long tests_paper[CRSH_MAX_LEVELS];  /* B per parent pair (the tables' convention) */
    unsigned long long final_tests;                   /* ray-triangle tests made */
    unsigned long long final_tests_paper;             /* B per level-1 pair */
    unsigned long long final_hits;                    /* ray-triangle tests that hit */
    unsigned long long needed_pairs;                  /* largest pair list any level produced */
    unsigned int status;                              /* first device-side crsh_status, 0 = OK */
    unsigned int reserved;
} crsh_counters;

/* Triangle meshes.  Meshes are contiguous triangle ranges. */
typedef struct {
    const float *v0x, *v0y, *v0z, *v1x, *v1y, *v1z, *v2x, *v2y, *v2z;
    uint32_t n_tris;
    const uint32_t *mesh_first_tri;  /* n_meshes + 1 entries; mesh m = [first[m], first[m+1]) */
    const float *mesh_sphere;        /* 4 floats per mesh: centre xyz, radius (encloses the mesh) */
    uint32_t n_meshes;
    float *tri_sphere;               /* 4 floats per triangle, written by crsh_prepare_scene */
    float *tri_mt;                   /* 16 floats per triangle (16-byte aligned), written by
                                        crsh_prepare_scene: (v0, n.x), (v1 - v0, n.y),
                                        (v2 - v0, n.z), (c, q): n = normal, c = centre of the
                                        bounding sphere, q = squared radius of the pre-test of
                                        the final tests */
} crsh_scene;

typedef struct {
    uint32_t bundle;                 /* B: children per node, power of two in [2, 64] */
    uint32_t levels;                 /* L: levels built and traversed, 1..CRSH_MAX_LEVELS */
    float sphere_pad_rel, sphere_pad_abs;  /* radius -> r (1 + rel) + abs after each node */
    float cone_pad_rel, cone_pad_abs;      /* spread -> s (1 + rel) + abs (radians) */
} crsh_build_params;

/* Levels of sphere-cone nodes (Section 3.3.6: 8 floats per node). */
typedef struct {
    float *sphere[CRSH_MAX_LEVELS];  /* 4 floats per node: centre xyz, radius */
    float *cone[CRSH_MAX_LEVELS];    /* 4 floats per node: unit axis xyz, spread (half-angle) */
    float *trig[CRSH_MAX_LEVELS];    /* 2 floats per node: tan(spread), 1/cos(spread), for eq. 9 */
    uint32_t capacity[CRSH_MAX_LEVELS]; /* nodes allocated per level: >= ceil(rays / B^l) */
    uint32_t *count;                 /* device, CRSH_MAX_LEVELS entries: nodes per level */
    uint32_t levels, bundle;
} crsh_hierarchy;

typedef struct {
    uint32_t mesh_cull;              /* 1: whole-mesh spheres at the top level (Section 3.3.7) */
    uint32_t block_threads;          /* block shape of the traversal's test and emit passes: 128,
                                        256 or 512 threads (0 = 256); a tuning knob, results do
                                        not depend on it */
    uint32_t level1_words;           /* 1: leave level 1 in word form (crsh_pairs.words) instead
                                        of writing its (node, triangle) pairs; hierarchies of two
                                        or more levels only */
} crsh_traverse_params;

/* Level-1 candidates in word form, written by crsh_traverse with
 * level1_words = 1 and read by crsh_closest_hit: the same set of (node,
 * triangle) pairs as the list form, kept as the 32-bit ballots of the
 * traversal's last test pass.  Work item i is items[4 i .. 4 i + 3] =
 * (level-1 node n, position r in `tri`, first word w, word count c <= 32):
 * for j < c, bit b of words[w + j] set means node n accepted triangle
 * tri[r + 32 j + b].  Every pair belongs to exactly one item.  The arrays
 * live in the traversal's workspace: the form is valid until that workspace
 * is written again. */
typedef struct {
    const uint32_t *words;
    const uint32_t *tri;             /* level-2 pair list, triangle column */
    const uint32_t *items;           /* 4 entries per work item */
    const uint32_t *n_items;         /* device: work items */
    uint32_t valid;                  /* 1 when the fields above describe level 1 */
    uint32_t reserved;
} crsh_pair_words;

/* Level-1 (node, triangle) pairs grouped by node, triangles ascending, or
 * (level1_words) their word form. */
typedef struct {
    uint32_t *node, *tri;            /* capacity entries each (not written in word form) */
    uint32_t *node_offsets;          /* level-1 node count + 1 entries: CSR over nodes (list form) */
    uint32_t *count;                 /* device: pairs written (list form) */
    uint64_t capacity;               /* 1 .. 2^31 */
    crsh_pair_words words;           /* output of crsh_traverse: valid = 1 in word form, else 0 */
} crsh_pairs;

/* Closest hits in generation order (ray_id). tri = -1: no hit (t = u = v = 0). */
typedef struct {
    int32_t *tri;
    float *t, *u, *v;
} crsh_hits;

/* ---- Primary visibility, next bounce, mesh update (NEXT row f3) -------- */

/* Pinhole camera.  Pixel (x, y) looks along fwd + sx right + sy up with
 * sx = (2 (x + 0.5) / width - 1) tan_x and sy = (1 - 2 (y + 0.5) / height)
 * tan_y (y = 0 is the top row). */
typedef struct {
    float eye[3];
    float fwd[3], right[3], up[3];   /* orthonormal */
    float tan_x, tan_y;              /* tangents of half the horizontal / vertical field of view */
    uint32_t width, height;
} crsh_camera;

/* A first-hit buffer the library writes: the crsh_gbuffer layout, n entries
 * (for a camera, n = width x height in row-major pixel order). */
typedef struct {
    float *px, *py, *pz, *nx, *ny, *nz, *ix, *iy, *iz;
    uint32_t *material;
    uint8_t *hit;
    uint32_t n;
} crsh_gbuffer_out;

/* Camera rays for primary visibility through the same hierarchy path (they
 * stand in for the rasterised G-buffer pass of Section 3.2).  Writes
 * width x height rays to `out` in tile order: 8 x 8 pixel blocks in
 * block-row-major order, Z-order inside a block (pixels outside the image
 * skipped), so every aligned run of B <= 64 rays covers a compact tile and the
 * rays need no hashing or sorting before crsh_build.  Origin = eye, direction
 * = d / |d| for the d above (FP32, no contraction), t_max = +inf, type =
 * CRSH_RAY_PRIMARY, ray_id = pixel = y width + x.  *n_out (device) =
 * width x height.  out->capacity must hold width x height rays
 * (CRSH_ERR_INVALID_ARG otherwise, as for a zero size). */
crsh_status crsh_primary_rays(const crsh_camera *cam, crsh_rays *out, uint32_t *n_out, void *stream);

/* First-hit buffer from closest hits (the G-buffer of Section 3.2, for
 * primary rays, and the hit-point buffer next-bounce rays are generated from,
 * Section 3.3.8).  For every ray i < *n_rays of `rays` with g = ray_id[i] <
 * out->n: hits are read at g (crsh_closest_hit's order); on a hit, position =
 * o + t d, normal = (v1 - v0) x (v2 - v0) / |.| turned to face the ray
 * (n.d <= 0), incident = d, material = tri_material[tri], hit = 1; on a miss
 * all zero except incident.  FP32 with a fixed operation order, no
 * contraction.  Feeding `out` (as a crsh_gbuffer of width out->n, height 1)
 * to crsh_hash_sort emits the next bounce's rays. */
crsh_status crsh_gbuffer_from_hits(const crsh_rays *rays, const uint32_t *n_rays, const crsh_hits *hits,
                                   const crsh_scene *scene, const uint32_t *tri_material,
                                   crsh_gbuffer_out *out, void *stream);

/* Writable vertices and mesh spheres of a scene. */
typedef struct {
    float *v0x, *v0y, *v0z, *v1x, *v1y, *v1z, *v2x, *v2y, *v2z;
    float *mesh_sphere;              /* 4 floats per mesh */
} crsh_scene_out;

/* Per-frame bounding-volume update (Section 3.3.1): mesh m's vertices go
 * through the affine map xf[12 m ..]: row-major 3 x 4 [A | b], v -> A v + b;
 * its sphere's centre likewise and its radius scales by the Frobenius norm of
 * A (at least the largest stretch), rounded up, so the sphere still encloses
 * the moved mesh.  `in` and `out` may alias.  Call crsh_prepare_scene on the
 * result before tracing it. */
crsh_status crsh_transform_meshes(const crsh_scene *in, const float *xf, crsh_scene_out *out, void *stream);

/* Shading accumulation (NEXT row f4; Section 3.3.8 turns the closest hits
 * into shading but names no model, so this is a reading).  Grey level per
 * pixel of `gb` (n_pixels entries, row-major), from the frame's secondary
 * rays (`rays`, *n_rays of them, as crsh_hash_sort left them) and their hits
 * (crsh_closest_hit's order):
 *   no primary hit:  color = sky
 *   else, material m (diffuse 0, mirror 1, glass 2) with albedo a = (0.8, 0.2,
 *   0.1), reflectance k_r = (0, 0.8, 0.1), transmittance k_t = (0, 0, 0.8):
 *   color = a (ambient + sum_k S_k) + k_r R + k_t T, summed in this order;
 *   S_k = max(0, n . (-d)) for the shadow ray of light k if it reached the
 *   light (no hit), else 0 (also 0 when no shadow ray was emitted); R, T =
 *   for the reflection / refraction ray, a(hit material) (ambient + 0.5) on a
 *   hit, sky on a miss, 0 when there is no such ray; ambient = 0.1, sky = 0.6.
 * The shadow ray of light k is the one whose origin is lights[3k ..] (as
 * crsh_hash_sort emits them).  FP32, fixed order, deterministic.
 * cells: device scratch of n_pixels x (n_lights + 2) floats.  color: device,
 * n_pixels floats. */
crsh_status crsh_shade(const crsh_gbuffer *gb, const float *lights, uint32_t n_lights, const crsh_rays *rays,
                       const uint32_t *n_rays, const crsh_hits *hits, const uint32_t *tri_material, float *cells,
                       float *color, void *stream);

/* Library version (major * 10000 + minor * 100 + patch). */
int crsh_version(void);
const char *crsh_status_string(crsh_status s);

/* Triangle bounding spheres (centroid centre, largest vertex distance, padded
 * outward for FP32 rounding) and the per-triangle record of the final tests
 * (v0, edges v1 - v0 and v2 - v0, normal, and the bounding sphere the final
 * tests check a ray's line against before Moller-Trumbore: the tightest of
 * the spheres about the centroid, the three edge midpoints and the
 * circumcentre that hold the triangle, padded like the triangle spheres; the
 * traversal keeps the centroid spheres).  Writes
 * scene->tri_sphere and scene->tri_mt. */
crsh_status crsh_prepare_scene(const crsh_scene *scene, void *stream);

/* The FP32 threshold tables the hash's direction bins compare against
 * (Section 3.3.2 reading): cos_out[k] = fl32(cos(k pi / 2^theta_bits)) for
 * k < 2^theta_bits and tan_out[j] = fl32(tan(j (pi/4) / M)) for j < M =
 * 2^phi_bits / 8, each from an FP64 evaluation.  Device pointers (the caller
 * owns them); theta_bits in [1, 13], phi_bits in [3, 13].  Asynchronous on
 * `stream`; crsh_hash_sort builds the same tables in its workspace. */
crsh_status crsh_hash_tables(uint32_t theta_bits, uint32_t phi_bits, float *cos_out, float *tan_out,
                             void *stream);

/* Workspace bytes crsh_hash_sort needs for up to `capacity` rays generated
 * from at most `max_pixels` G-buffer pixels (0 for crsh_rays_in input). */
size_t crsh_hash_sort_workspace(uint32_t capacity, uint32_t max_pixels);

/* Section 3.3.2-3.3.5.  Exactly one of `gbuffer` and `rays_in` is non-NULL.
 * From a G-buffer: for every hit pixel one shadow ray per light (origin at the
 * light, direction to the hit point, t_max = 0.9999 of the distance), a
 * reflection ray for mirror and glass, and a refraction ray for glass (IOR
 * 1.5, none on total internal reflection); empty slots are trimmed, keeping
 * pixel-major order.  Every ray gets its per-type key; rays are then sorted
 * by key, equal keys keeping generation order (optionally through chunk
 * compression, which gives the same order).
 * lights: device, 3 floats per light (n_lights <= 2^(30 - tb - pb)).
 * Outputs: `out` sorted rays, `keys_out` sorted keys (device, capacity
 * entries), `n_out` device ray count, counters->rays/chunks (the call resets
 * the whole counters struct first).  More rays than out->capacity:
 * CRSH_ERR_CAPACITY on the device, first capacity rays kept in order. */
crsh_status crsh_hash_sort(const crsh_gbuffer *gbuffer, const crsh_rays_in *rays_in,
                           const float *lights, uint32_t n_lights, const crsh_hash_params *params,
                           crsh_rays *out, uint32_t *keys_out, uint32_t *n_out,
                           crsh_counters *counters, void *workspace, size_t workspace_bytes,
                           void *stream);

/* Section 3.3.6.  Level-1 node j bounds sorted rays [jB, min(jB + B, n));
 * level-l node j bounds level-(l-1) nodes [jB, ...).  Cones: eqs. 1-4 fold
 * the rays of a level-1 node in order; eqs. 5-6 merge child cones; spheres:
 * eqs. 7-8; children merge as a balanced binary tree in child order.  Nodes
 * are padded outward (params) so the FP32 hierarchy contains its rays.
 * n_rays: device count from crsh_hash_sort.  Writes out->sphere/cone/trig for
 * levels 1..params->levels and out->count; sets out->levels/bundle. */
crsh_status crsh_build(const crsh_rays *rays, const uint32_t *n_rays, const crsh_build_params *params,
                       crsh_hierarchy *out, void *stream);

/* Workspace bytes crsh_traverse needs for pair lists of `pair_capacity`
 * entries per level over hierarchy `h` and `n_tris` triangles. */
size_t crsh_traverse_workspace(const crsh_hierarchy *h, uint32_t n_tris, uint32_t n_meshes,
                               uint64_t pair_capacity);

/* Section 3.3.7, eq. 9.  Top level: each top node against each whole-mesh
 * sphere (all meshes when mesh_cull = 0), then against the triangle spheres of
 * the meshes it meets; levels L-1 .. 1: each pair (p, t) of the level above
 * expands to the children of p, each tested against t.  Every level's list is
 * compacted in order.  Output: level-1 pairs grouped by node (out), counters
 * tests, hits, tests_paper, mesh_tests, mesh_hits and needed_pairs (reset by this call).  A list
 * longer than out->capacity sets CRSH_ERR_CAPACITY and needed_pairs.  With
 * params->level1_words (two or more levels) level 1 is left in word form:
 * out->words is filled (valid = 1), out->node, tri, node_offsets and count are
 * not written, and the workspace must stay untouched until crsh_closest_hit
 * has read it; otherwise out->words.valid is set to 0. */
crsh_status crsh_traverse(const crsh_hierarchy *h, const crsh_scene *scene,
                          const crsh_traverse_params *params, crsh_pairs *out,
                          crsh_counters *counters, void *workspace, size_t workspace_bytes,
                          void *stream);

/* Workspace bytes crsh_closest_hit / crsh_bruteforce_closest_hit need. */
size_t crsh_closest_hit_workspace(uint32_t ray_capacity);

/* Section 3.3.8.  For every level-1 pair (n, t) (the list of pairs->node and
 * pairs->tri, or pairs->words when its valid flag is set) and every ray of n:
 * Moller-Trumbore in FP32 (two-sided, inclusive edges, 0 < t <= t_max); the
 * closest hit per ray is the smallest (t, triangle id).  The (t, u, v) of the
 * winning triangle are then recomputed in double-word (float + float, about
 * 48-bit) arithmetic from the FP32 inputs and rounded to FP32.  Hits are written at each ray's ray_id.  Counters final_*
 * reset and written by this call.  Workspace: crsh_closest_hit_workspace. */
crsh_status crsh_closest_hit(const crsh_hierarchy *h, const crsh_rays *rays, const uint32_t *n_rays,
                             const crsh_scene *scene, const crsh_pairs *pairs, crsh_hits *out,
                             crsh_counters *counters, void *workspace, size_t workspace_bytes,
                             void *stream);

/* Workspace bytes crsh_closest_hit_backward needs. */
size_t crsh_closest_hit_backward_workspace(uint32_t ray_capacity);

/* Gradients of the closest hits with respect to the triangle vertices and the
 * ray origins and directions (the paper has no backward pass: this is the
 * adjoint of the final test of Section 3.3.8, with which-triangle-is-hit held
 * fixed).  For a ray o + t d hitting triangle (V0, V1, V2) at (u, v) and an
 * upstream gradient g = dL/d(t, u, v) (g_t, g_u, g_v: device, generation
 * order, one float per ray), with A = [-d | e1 | e2] and lambda = A^-T g:
 *   g_orig = lambda, g_dir = t lambda,
 *   g_verts: V0 += -(1-u-v) lambda, V1 += -u lambda, V2 += -v lambda,
 * summed over the rays that hit each triangle.
 * rays / n_rays / hits: as produced by crsh_hash_sort and crsh_closest_hit.
 * Outputs (device, overwritten; zero where no hit): g_verts 9 floats per
 * triangle (V0 xyz, V1 xyz, V2 xyz); g_orig and g_dir 3 floats per ray in
 * generation order, sized for rays->capacity.  FP32.  The per-triangle sums
 * are a stable sort by triangle plus a segmented reduction in a fixed order:
 * no atomics, identical bits on every run.  counters may be NULL (it only
 * receives a device status). */
crsh_status crsh_closest_hit_backward(const crsh_rays *rays, const uint32_t *n_rays, const crsh_scene *scene,
                                      const crsh_hits *hits, const float *g_t, const float *g_u, const float *g_v,
                                      float *g_verts, float *g_orig, float *g_dir, crsh_counters *counters,
                                      void *workspace, size_t workspace_bytes, void *stream);

/* crsh_closest_hit without a caller-supplied workspace.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory - code that runs while a CUDA graph is being captured (where
 * cudaMalloc is not allowed), real-time loops that must never reach the
 * allocator (cudaMalloc can synchronise the whole device), or plugins inside
 * a host application whose allocator owns all device memory.
 * The per-ray scratch (8 bytes per ray) is a fixed array inside the library
 * sized for CRSH_NOALLOC_MAX_RAYS rays (16 MiB); every GPU that loads the
 * library holds it until the process exits.  rays->capacity above
 * CRSH_NOALLOC_MAX_RAYS is rejected with CRSH_ERR_INVALID_ARG before anything
 * is launched.  The first call on each device looks up the array's device
 * address, so make that first call before any stream capture.  All calls
 * share the one array (each call resets the part it uses): calls that may
 * overlap on the GPU - other streams or other host threads on the same
 * device - race and must be serialised by the caller.  Arguments and results
 * are those of crsh_closest_hit. */
#define CRSH_NOALLOC_MAX_RAYS (1u << 21)
crsh_status crsh_closest_hit_noalloc(const crsh_hierarchy *h, const crsh_rays *rays, const uint32_t *n_rays,
                                     const crsh_scene *scene, const crsh_pairs *pairs, crsh_hits *out,
                                     crsh_counters *counters, void *stream);

/* Every ray against every triangle with the same test (Section 1's N x M
 * baseline); results bit-identical to crsh_closest_hit when culling is
 * conservative. */
crsh_status crsh_bruteforce_closest_hit(const crsh_rays *rays, const uint32_t *n_rays,
                                        const crsh_scene *scene, crsh_hits *out, void *workspace,
                                        size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CRSH_H */
