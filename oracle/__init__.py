"""CPU oracle of the Coherent Ray-Space Hierarchy (arXiv 2312.06538).

TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded restatement of the
method (crsh_oracle.c, loaded with ctypes) that the GPU library is checked
against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it; the library never does, and the two share no code.

Every function cites the section or equation it follows; ray generation and
hashing are FP32 with a fixed operation order (their outputs are integers both
sides must decide in the paper's 32-bit precision), the rest is FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crsh_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

RAY_SHADOW, RAY_REFLECTION, RAY_REFRACTION = 0, 1, 2
DEFAULT_BITS = dict(shadow_theta_bits=13, shadow_phi_bits=13, sec_cell_bits=5, sec_theta_bits=7,
                    sec_phi_bits=8)


def compile_native(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, no fast-math."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(os.path.dirname(_LIB), exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                                   "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _HashParams(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3),
                ("shadow_theta_bits", ctypes.c_uint32), ("shadow_phi_bits", ctypes.c_uint32),
                ("sec_cell_bits", ctypes.c_uint32), ("sec_theta_bits", ctypes.c_uint32),
                ("sec_phi_bits", ctypes.c_uint32)]


class _Counters(ctypes.Structure):
    _fields_ = [("mesh_tests", ctypes.c_int64), ("mesh_hits", ctypes.c_int64),
                ("tests", ctypes.c_int64 * 8), ("hits", ctypes.c_int64 * 8),
                ("tests_paper", ctypes.c_int64 * 8), ("final_tests", ctypes.c_int64),
                ("final_tests_paper", ctypes.c_int64), ("final_hits", ctypes.c_int64)]


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(compile_native())
        P, I64, U32, D, F, I = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double,
                                ctypes.c_float, ctypes.c_int)
        L.oracle_generate_rays.restype = I64
        L.oracle_generate_rays.argtypes = [U32] + [P] * 11 + [U32, P, I] + [P] * 10
        L.oracle_hash.restype = I
        L.oracle_hash.argtypes = [I64] + [P] * 8 + [ctypes.POINTER(_HashParams), P]
        L.oracle_primary_rays.restype = I64
        L.oracle_primary_rays.argtypes = [P, U32, U32] + [P] * 7
        L.oracle_gbuffer_from_hits.restype = None
        L.oracle_gbuffer_from_hits.argtypes = [I64] + [P] * 21
        L.oracle_shade.restype = None
        L.oracle_shade.argtypes = [U32] + [P] * 5 + [I64] + [P] * 8 + [U32, P]
        L.oracle_tables.restype = None
        L.oracle_tables.argtypes = [U32, U32, P, P]
        L.oracle_stable_sort.restype = None
        L.oracle_stable_sort.argtypes = [I64, P, P]
        L.oracle_chunk_count.restype = I64
        L.oracle_chunk_count.argtypes = [I64, P]
        L.oracle_build.restype = I64
        L.oracle_build.argtypes = [I64] + [P] * 6 + [U32, U32, D, D, D, D, P, P]
        L.oracle_sphere_cone.restype = I
        L.oracle_sphere_cone.argtypes = [P, D, D, D, D]
        L.oracle_tri_spheres.restype = None
        L.oracle_tri_spheres.argtypes = [I64, P, P]
        L.oracle_traverse.restype = I64
        L.oracle_traverse.argtypes = [P, P, U32, U32, I64, P, U32, P, P, I,
                                      ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(_Counters)]
        L.oracle_free.restype = None
        L.oracle_free.argtypes = [P]
        L.oracle_mt.restype = I
        L.oracle_mt.argtypes = [D] * 7 + [P, P, P, P]
        L.oracle_bruteforce.restype = None
        L.oracle_bruteforce.argtypes = [I64] + [P] * 7 + [I64, P, P, P, P, P]
        L.oracle_final.restype = None
        L.oracle_final.argtypes = [I64, P, P, U32, I64] + [P] * 9 + [P, P, P, P, ctypes.POINTER(_Counters)]
        L.oracle_adjoint.restype = None
        L.oracle_adjoint.argtypes = [I64] + [P] * 6 + [P, P, P, P, P, P, P, I64, P, P, P, P]
        L.oracle_check_hierarchy.restype = I64
        L.oracle_check_hierarchy.argtypes = [I64] + [P] * 6 + [U32, U32, P, P, P, P]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


RAY_FIELDS = ("ox", "oy", "oz", "dx", "dy", "dz", "tmax")


def generate_rays(gbuffer: Dict[str, np.ndarray], lights: np.ndarray, shadow_cull: bool) -> Dict[str, np.ndarray]:
    """Section 3.3.2: secondary rays of a G-buffer in pixel-major slot order, trimmed."""
    g = {k: _c(gbuffer[k], np.float32) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz")}
    mat = _c(gbuffer["material"], np.uint32)
    hit = _c(gbuffer["hit"], np.uint8)
    lights = _c(lights, np.float32).reshape(-1, 3)
    npx = mat.shape[0]
    cap = npx * (lights.shape[0] + 2)
    out = {k: np.empty(cap, np.float32) for k in RAY_FIELDS}
    out["type"] = np.empty(cap, np.uint8)
    out["light"] = np.empty(cap, np.uint8)
    out["pixel"] = np.empty(cap, np.uint32)
    n = lib().oracle_generate_rays(npx, *[_p(g[k]) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz")],
                                   _p(mat), _p(hit), lights.shape[0], _p(lights), int(bool(shadow_cull)),
                                   *[_p(out[k]) for k in RAY_FIELDS + ("type", "light", "pixel")])
    return {k: v[:n].copy() for k, v in out.items()}


def hash_keys(rays: Dict[str, np.ndarray], lo, hi, **bits) -> np.ndarray:
    """Section 3.3.2 / Figures 2-3: per-type 32-bit keys (bit layout in crsh_oracle.c)."""
    b = dict(DEFAULT_BITS)
    b.update(bits)
    hp = _HashParams((ctypes.c_float * 3)(*[float(x) for x in lo]), (ctypes.c_float * 3)(*[float(x) for x in hi]),
                     b["shadow_theta_bits"], b["shadow_phi_bits"], b["sec_cell_bits"], b["sec_theta_bits"],
                     b["sec_phi_bits"])
    r = {k: _c(rays[k], np.float32) for k in ("ox", "oy", "oz", "dx", "dy", "dz")}
    ty = _c(rays["type"], np.uint8)
    li = _c(rays["light"], np.uint8)
    n = ty.shape[0]
    keys = np.empty(n, np.uint32)
    rc = lib().oracle_hash(n, *[_p(r[k]) for k in ("ox", "oy", "oz", "dx", "dy", "dz")], _p(ty), _p(li),
                           ctypes.byref(hp), _p(keys))
    if rc != 0:
        raise ValueError("hash bit layout does not fit 32 bits")
    return keys


def hash_tables(theta_bits: int, phi_bits: int):
    """The hash's FP32 threshold tables: cos(k pi / 2^tb), k < 2^tb, and tan(j (pi/4) / M),
    j < M = 2^pb / 8 (bin readings of Section 3.3.2)."""
    c = np.empty(1 << theta_bits, np.float32)
    t = np.empty((1 << phi_bits) // 8, np.float32)
    lib().oracle_tables(int(theta_bits), int(phi_bits), _p(c), _p(t))
    return c, t


def stable_sort(keys: np.ndarray) -> np.ndarray:
    """Sections 3.3.3-3.3.5: the permutation that sorts rays by key, equal keys in input order."""
    keys = _c(keys, np.uint32)
    perm = np.empty(keys.shape[0], np.uint32)
    lib().oracle_stable_sort(keys.shape[0], _p(keys), _p(perm))
    return perm


def chunk_count(keys: np.ndarray) -> int:
    """Section 3.3.3: number of runs of equal consecutive keys."""
    keys = _c(keys, np.uint32)
    return int(lib().oracle_chunk_count(keys.shape[0], _p(keys)))


def level_counts(n: int, B: int, L: int) -> List[int]:
    out, below = [], n
    for _ in range(L):
        below = (below + B - 1) // B
        out.append(below)
    return out


def build_hierarchy(rays: Dict[str, np.ndarray], B: int, L: int, pads=(1e-5, 1e-4, 1e-5, 1e-5)) -> List[np.ndarray]:
    """Section 3.3.6, eqs. 1-8: hierarchy levels 1..L over sorted rays; (n_l, 8) float64 each
    (sphere centre, radius, cone axis, spread)."""
    r = {k: _c(rays[k], np.float32) for k in ("ox", "oy", "oz", "dx", "dy", "dz")}
    n = r["ox"].shape[0]
    cnt = level_counts(n, B, L)
    out = np.zeros((max(1, sum(cnt)), 8), np.float64)
    counts = np.zeros(L, np.int64)
    lib().oracle_build(n, *[_p(r[k]) for k in ("ox", "oy", "oz", "dx", "dy", "dz")], B, L, *map(float, pads),
                       _p(out), _p(counts))
    levels, base = [], 0
    for c in counts:
        levels.append(out[base:base + c].copy())
        base += c
    return levels


def sphere_cone(node8, P, r) -> bool:
    """Eq. 9 for one node (8 doubles) and one sphere (centre P, radius r)."""
    nd = _c(node8, np.float64)
    return bool(lib().oracle_sphere_cone(_p(nd), float(P[0]), float(P[1]), float(P[2]), float(r)))


def tri_spheres(verts: np.ndarray) -> np.ndarray:
    v = _c(verts, np.float32)
    out = np.empty((v.shape[0], 4), np.float64)
    lib().oracle_tri_spheres(v.shape[0], _p(v), _p(out))
    return out


def _counters_dict(c: _Counters, L: int) -> dict:
    return dict(mesh_tests=c.mesh_tests, mesh_hits=c.mesh_hits, tests=list(c.tests)[:L], hits=list(c.hits)[:L],
                tests_paper=list(c.tests_paper)[:L], final_tests=c.final_tests,
                final_tests_paper=c.final_tests_paper, final_hits=c.final_hits)


def traverse(levels: List[np.ndarray], B: int, scene, mesh_cull: bool = True):
    """Section 3.3.7: top-down traversal.  Returns level-1 (pair_node, pair_tri) grouped by
    node with triangles ascending, and the counters of Tables 1-3."""
    L = len(levels)
    counts = np.array([lv.shape[0] for lv in levels], np.int64)
    nodes = _c(np.concatenate(levels) if sum(counts) else np.zeros((1, 8)), np.float64)
    verts = _c(scene.verts, np.float32)
    first = _c(scene.mesh_first_tri, np.uint32)
    spheres = _c(scene.mesh_sphere, np.float32)
    pn, pt = ctypes.c_void_p(), ctypes.c_void_p()
    ctr = _Counters()
    n = lib().oracle_traverse(_p(nodes), _p(counts), B, L, verts.shape[0], _p(verts), spheres.shape[0], _p(first),
                              _p(spheres), int(bool(mesh_cull)), ctypes.byref(pn), ctypes.byref(pt),
                              ctypes.byref(ctr))
    if n > 0:
        node = np.ctypeslib.as_array(ctypes.cast(pn, ctypes.POINTER(ctypes.c_uint32)), (n,)).copy()
        tri = np.ctypeslib.as_array(ctypes.cast(pt, ctypes.POINTER(ctypes.c_uint32)), (n,)).copy()
    else:
        node = np.zeros(0, np.uint32)
        tri = np.zeros(0, np.uint32)
    lib().oracle_free(pn)
    lib().oracle_free(pt)
    return node, tri, _counters_dict(ctr, L)


def mt(o, d, tmax, tri_verts):
    """Moller-Trumbore [Mol97] in FP64 for one ray and one triangle (3x3 vertices)."""
    v = _c(tri_verts, np.float32).reshape(9)
    t, u, w = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    h = lib().oracle_mt(*[float(x) for x in o], *[float(x) for x in d], float(tmax), _p(v),
                        ctypes.byref(t), ctypes.byref(u), ctypes.byref(w))
    return bool(h), t.value, u.value, w.value


def bruteforce(rays: Dict[str, np.ndarray], verts: np.ndarray):
    """Section 1: every ray against every triangle; closest hit (tri, t, u, v); tri -1 = miss."""
    r = {k: _c(rays[k], np.float32) for k in RAY_FIELDS}
    v = _c(verts, np.float32)
    n = r["ox"].shape[0]
    tri = np.empty(n, np.int32)
    t, u, w = (np.empty(n, np.float64) for _ in range(3))
    lib().oracle_bruteforce(n, *[_p(r[k]) for k in RAY_FIELDS], v.shape[0], _p(v), _p(tri), _p(t), _p(u), _p(w))
    return tri, t, u, w


def final(pair_node, pair_tri, B: int, sorted_rays: Dict[str, np.ndarray], perm: np.ndarray, verts: np.ndarray):
    """Section 3.3.8: closest hit per ray over the level-1 pairs, in original ray order."""
    r = {k: _c(sorted_rays[k], np.float32) for k in RAY_FIELDS}
    pn, pt = _c(pair_node, np.uint32), _c(pair_tri, np.uint32)
    perm = _c(perm, np.uint32)
    v = _c(verts, np.float32)
    n = r["ox"].shape[0]
    tri = np.empty(n, np.int32)
    t, u, w = (np.empty(n, np.float64) for _ in range(3))
    ctr = _Counters()
    lib().oracle_final(pn.shape[0], _p(pn), _p(pt), B, n, *[_p(r[k]) for k in RAY_FIELDS], _p(perm), _p(v),
                       _p(tri), _p(t), _p(u), _p(w), ctypes.byref(ctr))
    return (tri, t, u, w), dict(final_tests=ctr.final_tests, final_tests_paper=ctr.final_tests_paper,
                                final_hits=ctr.final_hits)


def check_hierarchy(sorted_rays, B: int, counts, sphere: np.ndarray, cone: np.ndarray):
    """Containment invariants of an FP32 hierarchy, checked exactly in FP64.
    sphere/cone: (sum(counts), 4) float32, level 1 first.  Returns (violations, worst excess)."""
    r = {k: _c(sorted_rays[k], np.float32) for k in ("ox", "oy", "oz", "dx", "dy", "dz")}
    cnt = np.array(counts, np.int64)
    s = _c(sphere, np.float32)
    c = _c(cone, np.float32)
    worst = ctypes.c_double()
    bad = lib().oracle_check_hierarchy(r["ox"].shape[0], *[_p(r[k]) for k in ("ox", "oy", "oz", "dx", "dy", "dz")],
                                       B, len(counts), _p(cnt), _p(s), _p(c), ctypes.byref(worst))
    return int(bad), worst.value


def gather(rays: Dict[str, np.ndarray], perm: np.ndarray) -> Dict[str, np.ndarray]:
    return {k: np.ascontiguousarray(v[perm]) for k, v in rays.items()}


def run_crsh(gbuffer, lights, shadow_cull, lo, hi, scene, B, L, pads, mesh_cull=True, sort=True, **bits):
    """The whole path on the CPU: generate, hash, sort, build, traverse, final tests."""
    rays = generate_rays(gbuffer, lights, shadow_cull)
    keys = hash_keys(rays, lo, hi, **bits)
    n = keys.shape[0]
    perm = stable_sort(keys) if sort else np.arange(n, dtype=np.uint32)
    srays = gather(rays, perm)
    levels = build_hierarchy(srays, B, L, pads)
    pn, pt, ctr = traverse(levels, B, scene, mesh_cull)
    hits, fctr = final(pn, pt, B, srays, perm, scene.verts)
    ctr.update(fctr)
    ctr["rays"] = n
    ctr["chunks"] = chunk_count(keys)
    return dict(rays=rays, keys=keys, perm=perm, sorted_rays=srays, levels=levels, pair_node=pn,
                pair_tri=pt, hits=hits, counters=ctr)


def adjoint(rays: Dict[str, np.ndarray], hits, g_t, g_u, g_v, verts: np.ndarray):
    """FP64 gradients of the closest hit with the hit assignment fixed (implicit-function
    closed form): returns (g_verts (T, 9), g_orig (N, 3), g_dir (N, 3))."""
    r = {k: _c(rays[k], np.float32) for k in ("ox", "oy", "oz", "dx", "dy", "dz")}
    tri = _c(hits[0], np.int32)
    t, u, w = (_c(x, np.float64) for x in hits[1:4])
    gt, gu, gv = (_c(x, np.float64) for x in (g_t, g_u, g_v))
    v = _c(verts, np.float32)
    n = tri.shape[0]
    g_verts = np.empty((v.shape[0], 9), np.float64)
    g_orig = np.empty((n, 3), np.float64)
    g_dir = np.empty((n, 3), np.float64)
    lib().oracle_adjoint(n, *[_p(r[k]) for k in ("ox", "oy", "oz", "dx", "dy", "dz")], _p(tri), _p(t), _p(u), _p(w),
                         _p(gt), _p(gu), _p(gv), v.shape[0], _p(v), _p(g_verts), _p(g_orig), _p(g_dir))
    return g_verts, g_orig, g_dir


def primary_rays(camera: np.ndarray, width: int, height: int) -> Dict[str, np.ndarray]:
    """Camera rays in tile order (NEXT row f3): camera = eye, fwd, right, up, tan_x, tan_y."""
    cam = _c(np.asarray(camera)[:14], np.float32)
    n = width * height
    out = {k: np.empty(n, np.float32) for k in ("ox", "oy", "oz", "dx", "dy", "dz")}
    pixel = np.empty(n, np.uint32)
    got = lib().oracle_primary_rays(_p(cam), width, height, *[_p(out[k]) for k in ("ox", "oy", "oz", "dx", "dy", "dz")],
                                    _p(pixel))
    assert got == n
    out["pixel"] = pixel
    return out


def gbuffer_from_hits(rays: Dict[str, np.ndarray], tri: np.ndarray, t: np.ndarray, verts: np.ndarray,
                      tri_material: np.ndarray) -> Dict[str, np.ndarray]:
    """First-hit buffer of rays (generation order) from their hits (tri, FP32 t)."""
    r = {k: _c(rays[k], np.float32) for k in ("ox", "oy", "oz", "dx", "dy", "dz")}
    n = r["ox"].shape[0]
    tr, tt = _c(tri, np.int32), _c(t, np.float32)
    v, m = _c(verts, np.float32), _c(tri_material, np.int32)
    out = {k: np.empty(n, np.float32) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz")}
    out["material"] = np.empty(n, np.uint32)
    out["hit"] = np.empty(n, np.uint8)
    lib().oracle_gbuffer_from_hits(n, *[_p(r[k]) for k in ("ox", "oy", "oz", "dx", "dy", "dz")], _p(tr), _p(tt),
                                   _p(v), _p(m), *[_p(out[k]) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix",
                                                                         "iy", "iz", "material", "hit")])
    return out


def shade(gbuffer: Dict[str, np.ndarray], rays: Dict[str, np.ndarray], tri: np.ndarray, tri_material: np.ndarray,
          n_lights: int) -> np.ndarray:
    """Grey-level shading of the frame (NEXT row f4): rays in generation order (with type, light,
    pixel), tri = their closest hits."""
    npx = gbuffer["hit"].shape[0]
    g = {k: _c(gbuffer[k], np.float32) for k in ("nx", "ny", "nz")}
    mat, hit = _c(gbuffer["material"], np.uint32), _c(gbuffer["hit"], np.uint8)
    r = {k: _c(rays[k], np.float32) for k in ("dx", "dy", "dz")}
    ty, li, px = _c(rays["type"], np.uint8), _c(rays["light"], np.uint8), _c(rays["pixel"], np.uint32)
    color = np.empty(npx, np.float32)
    lib().oracle_shade(npx, _p(g["nx"]), _p(g["ny"]), _p(g["nz"]), _p(mat), _p(hit), ty.shape[0], _p(r["dx"]),
                       _p(r["dy"]), _p(r["dz"]), _p(ty), _p(li), _p(px), _p(_c(tri, np.int32)),
                       _p(_c(tri_material, np.int32)), int(n_lights), _p(color))
    return color

