"""ctypes binding of include/crsh.h: the same entry points and structs, argument
marshalling only.  Every step runs in libcrsh.so; there is no fallback, and
loading fails loudly when the library cannot be built or found."""
from __future__ import annotations

import ctypes
import os

from . import _build

MAX_LEVELS = 8
P = ctypes.c_void_p
U32 = ctypes.c_uint32
U64 = ctypes.c_uint64
F32 = ctypes.c_float

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_IMPLEMENTED, ERR_BAD_INPUT = range(7)
RAY_SHADOW, RAY_REFLECTION, RAY_REFRACTION, RAY_PRIMARY = 0, 1, 2, 3


class crsh_gbuffer(ctypes.Structure):
    _fields_ = [(k, P) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz", "material", "hit")] + \
               [("n_pixels", U32)]


class crsh_rays_in(ctypes.Structure):
    _fields_ = [(k, P) for k in ("ox", "oy", "oz", "dx", "dy", "dz", "tmax", "type", "light")] + [("n", U32)]


class crsh_hash_params(ctypes.Structure):
    _fields_ = [("lo", F32 * 3), ("hi", F32 * 3), ("shadow_theta_bits", U32), ("shadow_phi_bits", U32),
                ("sec_cell_bits", U32), ("sec_theta_bits", U32), ("sec_phi_bits", U32), ("shadow_cull", U32),
                ("sort", U32), ("compress", U32)]


class crsh_rays(ctypes.Structure):
    _fields_ = [(k, P) for k in ("ox", "oy", "oz", "dx", "dy", "dz", "tmax", "type", "ray_id", "pixel")] + \
               [("capacity", U32)]


class crsh_counters(ctypes.Structure):
    _fields_ = [("rays", U64), ("chunks", U64), ("mesh_tests", U64), ("mesh_hits", U64),
                ("tests", U64 * MAX_LEVELS), ("hits", U64 * MAX_LEVELS), ("tests_paper", U64 * MAX_LEVELS),
                ("final_tests", U64), ("final_tests_paper", U64), ("final_hits", U64), ("needed_pairs", U64),
                ("status", U32), ("reserved", U32)]


class crsh_scene(ctypes.Structure):
    _fields_ = [(k, P) for k in ("v0x", "v0y", "v0z", "v1x", "v1y", "v1z", "v2x", "v2y", "v2z")] + \
               [("n_tris", U32), ("mesh_first_tri", P), ("mesh_sphere", P), ("n_meshes", U32),
                ("tri_sphere", P), ("tri_mt", P)]


class crsh_build_params(ctypes.Structure):
    _fields_ = [("bundle", U32), ("levels", U32), ("sphere_pad_rel", F32), ("sphere_pad_abs", F32),
                ("cone_pad_rel", F32), ("cone_pad_abs", F32)]


class crsh_hierarchy(ctypes.Structure):
    _fields_ = [("sphere", P * MAX_LEVELS), ("cone", P * MAX_LEVELS), ("trig", P * MAX_LEVELS),
                ("capacity", U32 * MAX_LEVELS), ("count", P), ("levels", U32), ("bundle", U32)]


class crsh_traverse_params(ctypes.Structure):
    _fields_ = [("mesh_cull", U32), ("block_threads", U32), ("level1_words", U32)]


class crsh_pair_words(ctypes.Structure):
    _fields_ = [("words", P), ("tri", P), ("items", P), ("n_items", P), ("valid", U32), ("reserved", U32)]


class crsh_pairs(ctypes.Structure):
    _fields_ = [("node", P), ("tri", P), ("node_offsets", P), ("count", P), ("capacity", U64),
                ("words", crsh_pair_words)]


class crsh_hits(ctypes.Structure):
    _fields_ = [("tri", P), ("t", P), ("u", P), ("v", P)]


class crsh_camera(ctypes.Structure):
    _fields_ = [("eye", F32 * 3), ("fwd", F32 * 3), ("right", F32 * 3), ("up", F32 * 3), ("tan_x", F32),
                ("tan_y", F32), ("width", U32), ("height", U32)]


class crsh_gbuffer_out(ctypes.Structure):
    _fields_ = [(k, P) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz", "material", "hit")] + \
               [("n", U32)]


class crsh_scene_out(ctypes.Structure):
    _fields_ = [(k, P) for k in ("v0x", "v0y", "v0z", "v1x", "v1y", "v1z", "v2x", "v2y", "v2z", "mesh_sphere")]


_lib = None

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("crsh_version", ctypes.c_int, []),
    ("crsh_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("crsh_prepare_scene", ctypes.c_int, [ctypes.POINTER(crsh_scene), P]),
    ("crsh_hash_tables", ctypes.c_int, [U32, U32, P, P, P]),
    ("crsh_primary_rays", ctypes.c_int, [ctypes.POINTER(crsh_camera), ctypes.POINTER(crsh_rays), P, P]),
    ("crsh_gbuffer_from_hits", ctypes.c_int,
     [ctypes.POINTER(crsh_rays), P, ctypes.POINTER(crsh_hits), ctypes.POINTER(crsh_scene), P,
      ctypes.POINTER(crsh_gbuffer_out), P]),
    ("crsh_transform_meshes", ctypes.c_int,
     [ctypes.POINTER(crsh_scene), P, ctypes.POINTER(crsh_scene_out), P]),
    ("crsh_shade", ctypes.c_int,
     [ctypes.POINTER(crsh_gbuffer), P, U32, ctypes.POINTER(crsh_rays), P, ctypes.POINTER(crsh_hits), P, P, P, P]),
    ("crsh_fma_probe", ctypes.c_int, [P, U32, U32, ctypes.POINTER(ctypes.c_ulonglong), P]),
    ("crsh_lookback_selftest", ctypes.c_int, [P, P, U32, U32, U32, U32, P, P, P]),
    ("crsh_hash_sort_workspace", ctypes.c_size_t, [U32, U32]),
    ("crsh_hash_sort", ctypes.c_int,
     [ctypes.POINTER(crsh_gbuffer), ctypes.POINTER(crsh_rays_in), P, U32, ctypes.POINTER(crsh_hash_params),
      ctypes.POINTER(crsh_rays), P, P, P, P, ctypes.c_size_t, P]),
    ("crsh_build", ctypes.c_int,
     [ctypes.POINTER(crsh_rays), P, ctypes.POINTER(crsh_build_params), ctypes.POINTER(crsh_hierarchy), P]),
    ("crsh_traverse_workspace", ctypes.c_size_t, [ctypes.POINTER(crsh_hierarchy), U32, U32, U64]),
    ("crsh_traverse", ctypes.c_int,
     [ctypes.POINTER(crsh_hierarchy), ctypes.POINTER(crsh_scene), ctypes.POINTER(crsh_traverse_params),
      ctypes.POINTER(crsh_pairs), P, P, ctypes.c_size_t, P]),
    ("crsh_closest_hit_workspace", ctypes.c_size_t, [U32]),
    ("crsh_closest_hit", ctypes.c_int,
     [ctypes.POINTER(crsh_hierarchy), ctypes.POINTER(crsh_rays), P, ctypes.POINTER(crsh_scene),
      ctypes.POINTER(crsh_pairs), ctypes.POINTER(crsh_hits), P, P, ctypes.c_size_t, P]),
    ("crsh_closest_hit_backward_workspace", ctypes.c_size_t, [U32]),
    ("crsh_closest_hit_backward", ctypes.c_int,
     [ctypes.POINTER(crsh_rays), P, ctypes.POINTER(crsh_scene), ctypes.POINTER(crsh_hits), P, P, P, P, P, P, P, P,
      ctypes.c_size_t, P]),
    ("crsh_closest_hit_noalloc", ctypes.c_int,
     [ctypes.POINTER(crsh_hierarchy), ctypes.POINTER(crsh_rays), P, ctypes.POINTER(crsh_scene),
      ctypes.POINTER(crsh_pairs), ctypes.POINTER(crsh_hits), P, P]),
    ("crsh_bruteforce_closest_hit", ctypes.c_int,
     [ctypes.POINTER(crsh_rays), P, ctypes.POINTER(crsh_scene), ctypes.POINTER(crsh_hits), P, ctypes.c_size_t, P]),
    ("crsh_closest_hit_timed", ctypes.c_int,
     [ctypes.POINTER(crsh_hierarchy), ctypes.POINTER(crsh_rays), P, ctypes.POINTER(crsh_scene),
      ctypes.POINTER(crsh_pairs), ctypes.POINTER(crsh_hits), P, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_float),
      P]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libcrsh.so (building it first when sources are newer).  Raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libcrsh.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class CrshError(RuntimeError):
    def __init__(self, call: str, status: int):
        msg = load().crsh_status_string(status).decode()
        super().__init__(f"{call}: {msg} (status {status})")
        self.status = status


def _check(call: str, status: int):
    if status != OK:
        raise CrshError(call, status)


def _ref(x):
    return ctypes.byref(x) if x is not None else None


def crsh_version() -> int:
    return load().crsh_version()


def crsh_prepare_scene(scene: crsh_scene, stream: int):
    _check("crsh_prepare_scene", load().crsh_prepare_scene(ctypes.byref(scene), P(stream)))


def crsh_primary_rays(cam: crsh_camera, out: crsh_rays, n_out: int, stream: int):
    _check("crsh_primary_rays", load().crsh_primary_rays(ctypes.byref(cam), ctypes.byref(out), P(n_out), P(stream)))


def crsh_gbuffer_from_hits(rays: crsh_rays, n_rays: int, hits: crsh_hits, scene: crsh_scene, tri_material: int,
                           out: crsh_gbuffer_out, stream: int):
    _check("crsh_gbuffer_from_hits",
           load().crsh_gbuffer_from_hits(ctypes.byref(rays), P(n_rays), ctypes.byref(hits), ctypes.byref(scene),
                                         P(tri_material), ctypes.byref(out), P(stream)))


def crsh_transform_meshes(scene: crsh_scene, xf: int, out: crsh_scene_out, stream: int):
    _check("crsh_transform_meshes",
           load().crsh_transform_meshes(ctypes.byref(scene), P(xf), ctypes.byref(out), P(stream)))


def crsh_shade(gb: crsh_gbuffer, lights: int, n_lights: int, rays: crsh_rays, n_rays: int, hits: crsh_hits,
               tri_material: int, cells: int, color: int, stream: int):
    _check("crsh_shade", load().crsh_shade(ctypes.byref(gb), P(lights), n_lights, ctypes.byref(rays), P(n_rays),
                                           ctypes.byref(hits), P(tri_material), P(cells), P(color), P(stream)))


def crsh_fma_probe(out: int, iters: int, blocks: int, stream: int) -> int:
    """Launches the FP32 FMA probe; returns the flops it performs."""
    f = ctypes.c_ulonglong(0)
    _check("crsh_fma_probe", load().crsh_fma_probe(P(out), iters, blocks, ctypes.byref(f), P(stream)))
    return int(f.value)


def crsh_lookback_selftest(status64: int, status32: int, wide: bool, tile: int, aggregate: int, spin_limit: int,
                           prefix_out: int, counters: int, stream: int):
    """Diagnostics: one tile's look-back against prepared status words with a bounded wait."""
    _check("crsh_lookback_selftest",
           load().crsh_lookback_selftest(P(status64), P(status32), int(bool(wide)), tile, aggregate, spin_limit,
                                         P(prefix_out), P(counters), P(stream)))


def crsh_hash_tables(theta_bits: int, phi_bits: int, cos_out: int, tan_out: int, stream: int):
    _check("crsh_hash_tables", load().crsh_hash_tables(theta_bits, phi_bits, P(cos_out), P(tan_out), P(stream)))


def crsh_hash_sort_workspace(capacity: int, max_pixels: int) -> int:
    return load().crsh_hash_sort_workspace(capacity, max_pixels)


def crsh_hash_sort(gbuffer, rays_in, lights_ptr: int, n_lights: int, params: crsh_hash_params, out: crsh_rays,
                   keys_out: int, n_out: int, counters: int, workspace: int, workspace_bytes: int, stream: int):
    _check("crsh_hash_sort", load().crsh_hash_sort(_ref(gbuffer), _ref(rays_in), P(lights_ptr), n_lights,
                                                   ctypes.byref(params), ctypes.byref(out), P(keys_out), P(n_out),
                                                   P(counters), P(workspace), workspace_bytes, P(stream)))


def crsh_build(rays: crsh_rays, n_rays: int, params: crsh_build_params, out: crsh_hierarchy, stream: int):
    _check("crsh_build", load().crsh_build(ctypes.byref(rays), P(n_rays), ctypes.byref(params), ctypes.byref(out),
                                           P(stream)))


def crsh_traverse_workspace(h: crsh_hierarchy, n_tris: int, n_meshes: int, pair_capacity: int) -> int:
    return load().crsh_traverse_workspace(ctypes.byref(h), n_tris, n_meshes, pair_capacity)


def crsh_traverse(h: crsh_hierarchy, scene: crsh_scene, params: crsh_traverse_params, out: crsh_pairs, counters: int,
                  workspace: int, workspace_bytes: int, stream: int):
    _check("crsh_traverse", load().crsh_traverse(ctypes.byref(h), ctypes.byref(scene), ctypes.byref(params),
                                                 ctypes.byref(out), P(counters), P(workspace), workspace_bytes,
                                                 P(stream)))


def crsh_closest_hit_workspace(ray_capacity: int) -> int:
    return load().crsh_closest_hit_workspace(ray_capacity)


def crsh_closest_hit(h: crsh_hierarchy, rays: crsh_rays, n_rays: int, scene: crsh_scene, pairs: crsh_pairs,
                     out: crsh_hits, counters: int, workspace: int, workspace_bytes: int, stream: int):
    _check("crsh_closest_hit", load().crsh_closest_hit(ctypes.byref(h), ctypes.byref(rays), P(n_rays),
                                                       ctypes.byref(scene), ctypes.byref(pairs), ctypes.byref(out),
                                                       P(counters), P(workspace), workspace_bytes, P(stream)))


def crsh_closest_hit_timed(h: crsh_hierarchy, rays: crsh_rays, n_rays: int, scene: crsh_scene, pairs: crsh_pairs,
                           out: crsh_hits, counters: int, workspace: int, workspace_bytes: int, stream: int) -> float:
    """crsh_closest_hit that also returns its final-test kernel's duration in ms (synchronous;
    measurement only)."""
    ms = ctypes.c_float(0.0)
    _check("crsh_closest_hit_timed",
           load().crsh_closest_hit_timed(ctypes.byref(h), ctypes.byref(rays), P(n_rays), ctypes.byref(scene),
                                         ctypes.byref(pairs), ctypes.byref(out), P(counters), P(workspace),
                                         workspace_bytes, ctypes.byref(ms), P(stream)))
    return float(ms.value)


def crsh_bruteforce_closest_hit(rays: crsh_rays, n_rays: int, scene: crsh_scene, out: crsh_hits, workspace: int,
                                workspace_bytes: int, stream: int):
    _check("crsh_bruteforce_closest_hit",
           load().crsh_bruteforce_closest_hit(ctypes.byref(rays), P(n_rays), ctypes.byref(scene), ctypes.byref(out),
                                              P(workspace), workspace_bytes, P(stream)))


NOALLOC_MAX_RAYS = 1 << 21


def crsh_closest_hit_noalloc(h: crsh_hierarchy, rays: crsh_rays, n_rays: int, scene: crsh_scene, pairs: crsh_pairs,
                             out: crsh_hits, counters: int, stream: int):
    """crsh_closest_hit with the library's own fixed scratch (for callers that cannot allocate)."""
    _check("crsh_closest_hit_noalloc",
           load().crsh_closest_hit_noalloc(ctypes.byref(h), ctypes.byref(rays), P(n_rays), ctypes.byref(scene),
                                           ctypes.byref(pairs), ctypes.byref(out), P(counters), P(stream)))


def crsh_closest_hit_backward_workspace(ray_capacity: int) -> int:
    return load().crsh_closest_hit_backward_workspace(ray_capacity)


def crsh_closest_hit_backward(rays: crsh_rays, n_rays: int, scene: crsh_scene, hits: crsh_hits, g_t: int, g_u: int,
                              g_v: int, g_verts: int, g_orig: int, g_dir: int, counters: int, workspace: int,
                              workspace_bytes: int, stream: int):
    _check("crsh_closest_hit_backward",
           load().crsh_closest_hit_backward(ctypes.byref(rays), P(n_rays), ctypes.byref(scene), ctypes.byref(hits),
                                            P(g_t), P(g_u), P(g_v), P(g_verts), P(g_orig), P(g_dir), P(counters),
                                            P(workspace), workspace_bytes, P(stream)))
