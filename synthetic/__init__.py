"""Seeded synthetic workloads shaped like the paper's test scenes (Section 4.2).

The paper's scenes (OFFICE, CORNELL, SPONZA) are not available; these scenes
take their roles: multi-mesh shadow-heavy interiors, mirror/glass-heavy small
scenes, a large scene of many meshes inside a room.  Everything is drawn from
SplitMix64 with seed 1000 + config id; each object has its own substream.

This module only builds inputs: meshes, whole-mesh bounding spheres (computed
offline, as the paper does), lights, and the primary-hit G-buffer that the
rasterization pass of Section 3.2 would produce.  It holds none of the traced
method's arithmetic and is shared by the oracle tests and the CUDA path.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

from . import meshes
from ._native import min_ball, raster_gbuffer
from .rng import SplitMix64

DIFFUSE, MIRROR, GLASS = 0, 1, 2


@dataclasses.dataclass
class Scene:
    verts: np.ndarray            # (T, 3, 3) float32: triangle t, corner k, xyz
    mesh_first_tri: np.ndarray   # (M + 1,) uint32: triangles of mesh m are [first[m], first[m+1])
    mesh_sphere: np.ndarray      # (M, 4) float32: centre xyz, radius (encloses the mesh's vertices)
    mesh_material: np.ndarray    # (M,) int32
    tri_material: np.ndarray     # (T,) int32

    @property
    def n_tris(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_meshes(self) -> int:
        return int(self.mesh_sphere.shape[0])

    def soa(self) -> Dict[str, np.ndarray]:
        """The 9 per-triangle vertex coordinate arrays v0x .. v2z."""
        out = {}
        for k in range(3):
            for a, ax in enumerate("xyz"):
                out[f"v{k}{ax}"] = np.ascontiguousarray(self.verts[:, k, a])
        return out


@dataclasses.dataclass
class Workload:
    name: str
    width: int
    height: int
    scene: Scene
    camera: np.ndarray           # eye, fwd, right, up (3 each), tanx, tany  (float64[14])
    gbuffer: Dict[str, np.ndarray]
    primary_tri: np.ndarray      # (W*H,) int32 triangle seen by each pixel, -1 = background
    lights: np.ndarray           # (K, 3) float32
    bundle: int
    levels: int
    shadow_cull: bool
    hash_lo: np.ndarray          # float32[3]: box quantised into origin cells
    hash_hi: np.ndarray
    extent: float                # max |coordinate| in the scene, lights and hit points
    description: str = ""

    @property
    def n_pixels(self) -> int:
        return self.width * self.height

    def build_pads(self):
        """(sphere_rel, sphere_abs, cone_rel, cone_abs) node padding for the hierarchy."""
        return 1e-5, 1e-6 * self.extent, 1e-5, 1e-5


def _camera(eye, target, fov_deg, w, h) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    tany = np.tan(np.radians(fov_deg) / 2)
    tanx = tany * w / h
    return np.concatenate([eye, fwd, right, up, [tanx, tany]])


class _SceneBuilder:
    def __init__(self, seed: int):
        self.seed = seed
        self.parts: List[tuple] = []   # (verts (n,3,3) f32, material)

    def add(self, V: np.ndarray, F: np.ndarray, material: int):
        tri = V[F].astype(np.float32)
        self.parts.append((tri, material))

    def finish(self) -> Scene:
        verts = np.concatenate([p[0] for p in self.parts]).astype(np.float32)
        counts = np.array([p[0].shape[0] for p in self.parts], np.int64)
        first = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
        spheres = np.zeros((len(self.parts), 4), np.float32)
        for m, (tri, _) in enumerate(self.parts):
            pts = np.unique(tri.reshape(-1, 3), axis=0)
            c, _ = min_ball(pts, self.seed * 7919 + m)
            c32 = c.astype(np.float32)
            r = float(np.max(np.linalg.norm(pts.astype(np.float64) - c32.astype(np.float64), axis=1)))
            r32 = np.float32(r)
            if float(r32) < r:
                r32 = np.nextafter(r32, np.float32(np.inf))
            spheres[m, :3] = c32
            spheres[m, 3] = r32
        mat = np.array([p[1] for p in self.parts], np.int32)
        tri_mat = np.repeat(mat, counts).astype(np.int32)
        return Scene(verts, first, spheres, mat, tri_mat)


def _material(rng: SplitMix64, mirror_frac: float, glass_frac: float) -> int:
    u = rng.uniform()
    if u < mirror_frac:
        return MIRROR
    if u < mirror_frac + glass_frac:
        return GLASS
    return DIFFUSE


def _place(rng, lo, hi, radius, avoid=None):
    for _ in range(1000):
        p = np.array([rng.uniform(lo, hi), rng.uniform(lo, hi), rng.uniform(lo, hi)])
        if avoid is None or np.linalg.norm(p - avoid) > radius + 0.3:
            return p
    raise RuntimeError("placement failed")


def _lights(root: SplitMix64, n: int, spheres: np.ndarray, xz: float, ylo: float, yhi: float):
    out = []
    for k in range(n):
        rng = root.substream(10_000 + k)
        for _ in range(10_000):
            p = np.array([rng.uniform(-xz, xz), rng.uniform(ylo, yhi), rng.uniform(-xz, xz)])
            if all(np.linalg.norm(p - s[:3]) > s[3] + 0.1 for s in spheres):
                break
        else:
            raise RuntimeError("light placement failed")
        out.append(p)
    return np.array(out, np.float32).reshape(n, 3)


def _finish(name, w, h, scene, cam, lights, bundle, levels, shadow_cull, desc) -> Workload:
    g, prim = raster_gbuffer(w, h, cam, scene.verts, scene.tri_material)
    hitm = g["hit"] == 1
    refl = hitm & (g["material"] != DIFFUSE)
    sel = refl if refl.any() else hitm
    if sel.any():
        pos = np.stack([g["px"][sel], g["py"][sel], g["pz"][sel]], 1)
        lo, hi = pos.min(0), pos.max(0)
        pad = 1e-3 * max(1.0, float(np.max(hi - lo)))
        lo, hi = (lo - pad).astype(np.float32), (hi + pad).astype(np.float32)
    else:
        lo, hi = np.full(3, -1, np.float32), np.full(3, 1, np.float32)
    extent = float(max(np.abs(scene.verts).max(), np.abs(lights).max() if lights.size else 0.0,
                       max(np.abs(g["px"]).max(), np.abs(g["py"]).max(), np.abs(g["pz"]).max())))
    return Workload(name, w, h, scene, cam, g, prim, lights, bundle, levels, shadow_cull,
                    lo, hi, extent, desc)


def config1(res: Optional[int] = None) -> Workload:
    """64x64, ground plane + icosphere(3) + torus 24x16 (2,050 tris), one light, all diffuse,
    no facing cull (every hit pixel emits its shadow ray), B = 8, L = 3."""
    w = h = res or 64
    root = SplitMix64(1001)
    sb = _SceneBuilder(1001)
    sb.add(*meshes.plane(-2.0, 100.0), DIFFUSE)
    r0 = root.substream(0)
    rad = r0.uniform(0.2, 1.0)
    V, F = meshes.icosphere(3)
    sb.add(V @ meshes.random_rotation(r0).T * rad + _place(r0, -2, 2, rad), F, DIFFUSE)
    r1 = root.substream(1)
    rad = r1.uniform(0.2, 1.0)
    V, F = meshes.torus(24, 16, 0.7 * rad, 0.3 * rad)
    sb.add(V @ meshes.random_rotation(r1).T + _place(r1, -2, 2, rad), F, DIFFUSE)
    scene = sb.finish()
    lights = _lights(root, 1, scene.mesh_sphere[1:], 2.0, 1.0, 3.0)
    cam = _camera((0, 6, 6), (0, 0, 0), 60.0, w, h)
    return _finish("plain CRSH 64x64, 2,050 tris, 1 light, shadow rays only (B=8, L=3)", w, h, scene,
                   cam, lights, 8, 3, False, config1.__doc__)


def _objects_scene(seed, n_ico, ico_sub, n_tor, tor_seg, n_disp, lo, hi, mirror, glass, ground,
                   avoid=None, all_material=None):
    root = SplitMix64(seed)
    sb = _SceneBuilder(seed)
    if ground == "plane":
        sb.add(*meshes.plane(-2.0, 100.0), DIFFUSE if all_material is None else all_material)
    elif ground == "room":
        sb.add(*meshes.room_box(4.0), DIFFUSE if all_material is None else all_material)
    k = 0
    for i in range(n_ico + n_tor + n_disp):
        rng = root.substream(k)
        k += 1
        rad = rng.uniform(0.2, 1.0)
        rot = meshes.random_rotation(rng)
        pos = _place(rng, lo, hi, rad, avoid)
        mat = _material(rng, mirror, glass) if all_material is None else all_material
        if i < n_ico:
            V, F = meshes.icosphere(ico_sub)
            V = V * rad
        elif i < n_ico + n_tor:
            V, F = meshes.torus(tor_seg[0], tor_seg[1], 0.7 * rad, 0.3 * rad)
        else:
            V, F = meshes.icosphere(3)
            V = meshes.displace(V, rng) * rad
        sb.add(V @ rot.T + pos, F, mat)
    return root, sb.finish()


def config2(res: Optional[int] = None) -> Workload:
    """512x512, plane + 11 icospheres(4) + 5 tori 24x16 (60,162 tris), 30% mirror / 20% glass,
    2 lights with facing cull, shadow + reflection + refraction rays, B = 16, L = 4."""
    w = h = res or 512
    root, scene = _objects_scene(1002, 11, 4, 5, (24, 16), 0, -2, 2, 0.3, 0.2, "plane")
    lights = _lights(root, 2, scene.mesh_sphere[1:], 2.0, 1.0, 3.0)
    cam = _camera((0, 6, 6), (0, 0, 0), 60.0, w, h)
    return _finish(f"plain CRSH {w}x{h}, 60,162 tris, 2 lights, shadow+reflection+refraction "
                   f"(B=16, L=4)", w, h, scene, cam, lights, 16, 4, True, config2.__doc__)


def config3(res: Optional[int] = None) -> Workload:
    """1024x1024, room box + 24 icospheres(4) + 16 tori 48x32 + 24 displaced icospheres(3)
    (202,764 tris), 4 lights, all ray types, B = 16, L = 4."""
    w = h = res or 1024
    eye = np.array([0.0, 1.0, 3.5])
    root, scene = _objects_scene(1003, 24, 4, 16, (48, 32), 24, -3, 3, 0.3, 0.2, "room", avoid=eye)
    lights = _lights(root, 4, scene.mesh_sphere[1:], 3.5, 1.0, 3.5)
    cam = _camera(eye, (0, 0, 0), 60.0, w, h)
    return _finish(f"plain CRSH {w}x{h}, 202,764 tris, 4 lights, all ray types (B=16, L=4)",
                   w, h, scene, cam, lights, 16, 4, True, config3.__doc__)


def config5(res: Optional[int] = None) -> Workload:
    """1024x1024 render of a 99,842-tri scene (plane + 18 icospheres(4) + 10 tori 24x16), every
    surface a mirror and no light: exactly one reflection ray per pixel (2^20 at full size)."""
    w = h = res or 1024
    root, scene = _objects_scene(1005, 18, 4, 10, (24, 16), 0, -2, 2, 0.0, 0.0, "plane",
                                 all_material=MIRROR)
    lights = np.zeros((0, 3), np.float32)
    cam = _camera((0, 6, 6), (0, 0, 0), 60.0, w, h)
    return _finish(f"adjoint {w}x{h} reflection rays, 99,842 tris (B=16, L=4)", w, h, scene, cam,
                   lights, 16, 4, True, config5.__doc__)


def config4_scene(k: int) -> Scene:
    """Scene k of the batched workload: a room box plus icospheres / tori / displaced spheres,
    about 5,000 * 40^(k/7) triangles (5k .. 200k, log-spaced), 30 % mirror, 20 % glass."""
    target = 5000.0 * 40.0 ** (k / 7.0)
    n_big = int(target * 0.6 // 5120)                      # icospheres(4)
    rest = target - 5120 * n_big
    n_tor = int(rest * 0.5 // 768)                         # tori 24x16
    n_disp = max(1, int((rest - 768 * n_tor) // 1280))     # displaced icospheres(3)
    eye = np.array([0.0, 1.0, 3.5])
    _, scene = _objects_scene(1040 + k, n_big, 4, n_tor, (24, 16), n_disp, -3, 3, 0.3, 0.2, "room", avoid=eye)
    return scene


def config4_frame(k: int, res: int):
    """Primary-hit buffer of scene k at res x res, 2 lights (the camera and lights of config 3)."""
    scene = config4_scene_cached(k)
    root = SplitMix64(1040 + k)
    lights = _lights(root, 2, scene.mesh_sphere[1:], 3.5, 1.0, 3.5)
    cam = _camera(np.array([0.0, 1.0, 3.5]), (0, 0, 0), 60.0, res, res)
    return _finish(f"batched scene {k} at {res}x{res}", res, res, scene, cam, lights, 16, 4, True,
                   config4_frame.__doc__)


_c4_cache: Dict[int, Scene] = {}


def config4_scene_cached(k: int) -> Scene:
    if k not in _c4_cache:
        _c4_cache[k] = config4_scene(k)
    return _c4_cache[k]


def config4_batches(n_batches: int = 32, lo: int = 1 << 11, hi: int = 1 << 20):
    """The batched workload: (ray count, scene index) per batch; sizes floor(exp(U[ln lo, ln hi])),
    scene drawn uniformly from the 8 scenes (seed 1004)."""
    rng = SplitMix64(1004)
    out = []
    for _ in range(n_batches):
        size = int(np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        k = int(rng.uniform() * 8) % 8
        out.append((size, k))
    return out


# ---- scenes shaped like the paper's evaluation (Section 4.2), for the
# depth-2, B = 8, 512x512 study of row f4.  The paper's models are not
# available; these take their roles: OFFICE, an interior of many separate
# meshes lit by one light (shadow rays); CORNELL, a small object inside six
# mirrors (shadow and reflection rays); SPONZA, one undivided mesh (shadow
# rays), which gives the whole-mesh spheres nothing to cull.

def study_office(res: Optional[int] = None) -> Workload:
    """OFFICE-shaped: a room with 20 icospheres(3), 12 tori 24x16 and 1 displaced sphere as
    separate meshes (36,108 tris), all diffuse, one light, shadow rays only, B = 8, L = 2."""
    w = h = res or 512
    eye = np.array([0.0, 1.0, 3.5])
    root, scene = _objects_scene(1101, 20, 3, 12, (24, 16), 1, -3, 3, 0.0, 0.0, "room", avoid=eye,
                                 all_material=DIFFUSE)
    lights = _lights(root, 1, scene.mesh_sphere[1:], 3.0, 2.0, 3.5)
    cam = _camera(eye, (0, 0, 0), 60.0, w, h)
    return _finish(f"OFFICE-shaped {w}x{h}, {scene.n_tris:,} tris in {scene.n_meshes} meshes, 1 light, "
                   f"shadow rays (B=8, L=2)", w, h, scene, cam, lights, 8, 2, True, study_office.__doc__)


def study_cornell(res: Optional[int] = None) -> Workload:
    """CORNELL-shaped: an icosphere(2) and a torus 20x12 (800 tris, diffuse) inside a box whose
    six walls are mirrors (12 tris), one light, shadow and reflection rays, B = 8, L = 2."""
    w = h = res or 512
    root = SplitMix64(1102)
    sb = _SceneBuilder(1102)
    sb.add(*meshes.room_box(2.0), MIRROR)
    V, F = meshes.icosphere(2)
    sb.add(V * 0.6 + np.array([-0.4, -0.9, 0.0]), F, DIFFUSE)
    V, F = meshes.torus(20, 12, 0.5, 0.18)
    sb.add(V @ meshes.random_rotation(root.substream(1)).T + np.array([0.6, -0.6, -0.3]), F, DIFFUSE)
    scene = sb.finish()
    lights = np.array([[0.0, 1.5, 0.5]], np.float32)
    cam = _camera(np.array([0.0, 0.2, 1.8]), (0, -0.4, 0), 70.0, w, h)
    return _finish(f"CORNELL-shaped {w}x{h}, {scene.n_tris:,} tris, six mirrors, 1 light, shadow + reflection "
                   f"rays (B=8, L=2)", w, h, scene, cam, lights, 8, 2, True, study_cornell.__doc__)


def study_sponza(res: Optional[int] = None) -> Workload:
    """SPONZA-shaped: a room with 40 displaced icospheres(3) and 20 tori 24x16 merged into ONE mesh
    (66,572 tris, no object subdivision), all diffuse, one light, shadow rays only, B = 8, L = 2."""
    w = h = res or 512
    eye = np.array([0.0, 1.0, 3.5])
    root, parts = _objects_scene(1103, 0, 3, 20, (24, 16), 40, -3, 3, 0.0, 0.0, "room", avoid=eye,
                                 all_material=DIFFUSE)
    sb = _SceneBuilder(1103)
    sb.parts.append((parts.verts, DIFFUSE))   # one mesh
    scene = sb.finish()
    lights = _lights(root, 1, parts.mesh_sphere[1:], 3.0, 2.0, 3.5)
    cam = _camera(eye, (0, 0, 0), 60.0, w, h)
    return _finish(f"SPONZA-shaped {w}x{h}, {scene.n_tris:,} tris in one mesh, 1 light, shadow rays "
                   f"(B=8, L=2)", w, h, scene, cam, lights, 8, 2, True, study_sponza.__doc__)


STUDY = {"OFFICE": study_office, "CORNELL": study_cornell, "SPONZA": study_sponza}

def tiled_gbuffer(w, tiles: int, seed: int = 77):
    """`tiles` copies of the frame's G-buffer, each shifted (up to 0.05 per axis) and with
    normals and incident directions turned by a small seeded rotation (up to 0.02 rad), so
    keys stay spread like a larger frame's."""
    rng = np.random.default_rng(seed)
    parts = {k: [] for k in w.gbuffer}
    for t in range(tiles):
        shift = rng.uniform(-0.05, 0.05, 3).astype(np.float32) if t else np.zeros(3, np.float32)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        ang = rng.uniform(0, 0.02) if t else 0.0
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = (np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K).astype(np.float32)
        g = w.gbuffer
        P = np.stack([g["px"], g["py"], g["pz"]], 1) + shift
        Nn = np.stack([g["nx"], g["ny"], g["nz"]], 1) @ R.T
        I = np.stack([g["ix"], g["iy"], g["iz"]], 1) @ R.T
        Nn /= np.linalg.norm(Nn, axis=1, keepdims=True).clip(1e-30)
        I /= np.linalg.norm(I, axis=1, keepdims=True).clip(1e-30)
        for k, col in (("px", P[:, 0]), ("py", P[:, 1]), ("pz", P[:, 2]), ("nx", Nn[:, 0]), ("ny", Nn[:, 1]),
                       ("nz", Nn[:, 2]), ("ix", I[:, 0]), ("iy", I[:, 1]), ("iz", I[:, 2])):
            parts[k].append(np.ascontiguousarray(col, np.float32))
        parts["material"].append(g["material"])
        parts["hit"].append(g["hit"])
    return {k: np.concatenate(v) for k, v in parts.items()}


CONFIGS = {1: config1, 2: config2, 3: config3, 5: config5}


def make(cid: int, res: Optional[int] = None) -> Workload:
    return CONFIGS[cid](res)
