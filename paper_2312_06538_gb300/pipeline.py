"""Device buffers and call sequence of the whole path: the four C-ABI calls
(crsh_hash_sort -> crsh_build -> crsh_traverse -> crsh_closest_hit) over
caller-owned torch tensors.  PyTorch provides memory and streams only; every
step runs in libcrsh.so."""
from __future__ import annotations

import ctypes
import math
from typing import Dict, Optional, Tuple

import numpy as np
import torch

from . import crsh as C

GB_FIELDS = ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz")
RAY_FIELDS = ("ox", "oy", "oz", "dx", "dy", "dz", "tmax")


def _ptr(t: Optional[torch.Tensor]) -> int:
    return 0 if t is None else t.data_ptr()


def hash_params(lo, hi, *, shadow_cull=True, sort=True, compress=True, shadow_theta_bits=13, shadow_phi_bits=13,
                sec_cell_bits=5, sec_theta_bits=7, sec_phi_bits=8) -> C.crsh_hash_params:
    return C.crsh_hash_params((C.F32 * 3)(*map(float, lo)), (C.F32 * 3)(*map(float, hi)), shadow_theta_bits,
                              shadow_phi_bits, sec_cell_bits, sec_theta_bits, sec_phi_bits, int(bool(shadow_cull)),
                              int(bool(sort)), int(bool(compress)))


def build_params(bundle, levels, pads) -> C.crsh_build_params:
    sr, sa, cr, ca = pads
    return C.crsh_build_params(bundle, levels, sr, sa, cr, ca)


def counters_from_bytes(b: bytes, levels: int) -> dict:
    c = C.crsh_counters.from_buffer_copy(b)
    return dict(rays=c.rays, chunks=c.chunks, mesh_tests=c.mesh_tests, mesh_hits=c.mesh_hits,
                tests=list(c.tests)[:levels], hits=list(c.hits)[:levels], tests_paper=list(c.tests_paper)[:levels],
                final_tests=c.final_tests, final_tests_paper=c.final_tests_paper, final_hits=c.final_hits,
                needed_pairs=c.needed_pairs, status=c.status)


class Pipeline:
    """Buffers for one scene and up to `ray_capacity` rays; run() issues the path on a stream."""

    def __init__(self, scene, *, max_pixels: int, n_lights: int, bundle: int, levels: int,
                 ray_capacity: Optional[int] = None, pair_capacity: Optional[int] = None, device="cuda",
                 level1_words: bool = False):
        C.load()
        self.device = torch.device(device)
        self.bundle, self.levels = int(bundle), int(levels)
        # level 1 in word form: crsh_traverse leaves it in its ballots and crsh_closest_hit reads them
        # there (no level-1 pair list; hierarchies of two or more levels)
        self.level1_words = bool(level1_words) and self.levels >= 2
        dev = self.device
        f32, u32 = torch.float32, torch.int32
        # scene
        soa = scene.soa()
        self.scene_t = {k: torch.from_numpy(v).to(dev) for k, v in soa.items()}
        self.mesh_first = torch.from_numpy(scene.mesh_first_tri.astype(np.int32)).to(dev)
        self.mesh_sphere = torch.from_numpy(np.ascontiguousarray(scene.mesh_sphere, np.float32)).to(dev)
        self.n_tris, self.n_meshes = scene.n_tris, scene.n_meshes
        self.tri_sphere = torch.empty((self.n_tris, 4), dtype=f32, device=dev)
        self.tri_mt = torch.empty((self.n_tris, 16), dtype=f32, device=dev)
        self.scene = C.crsh_scene(*[_ptr(self.scene_t[k]) for k in ("v0x", "v0y", "v0z", "v1x", "v1y", "v1z",
                                                                   "v2x", "v2y", "v2z")],
                                  self.n_tris, _ptr(self.mesh_first), _ptr(self.mesh_sphere), self.n_meshes,
                                  _ptr(self.tri_sphere), _ptr(self.tri_mt))
        # rays
        self.max_pixels = int(max_pixels)
        cap = int(ray_capacity or max(1, self.max_pixels * (n_lights + 2)))
        self.ray_capacity = cap
        self.rays_t = {k: torch.empty(cap, dtype=f32, device=dev) for k in RAY_FIELDS}
        self.rays_t["type"] = torch.empty(cap, dtype=torch.uint8, device=dev)
        self.rays_t["ray_id"] = torch.empty(cap, dtype=u32, device=dev)
        self.rays_t["pixel"] = torch.empty(cap, dtype=u32, device=dev)
        self.rays = C.crsh_rays(*[_ptr(self.rays_t[k]) for k in RAY_FIELDS + ("type", "ray_id", "pixel")], cap)
        self.keys = torch.empty(cap, dtype=u32, device=dev)
        self.n_rays = torch.zeros(1, dtype=u32, device=dev)
        self.counters = torch.zeros(ctypes.sizeof(C.crsh_counters), dtype=torch.uint8, device=dev)
        self.ws_hash_bytes = C.crsh_hash_sort_workspace(cap, self.max_pixels)
        self.ws_hash = torch.empty(self.ws_hash_bytes, dtype=torch.uint8, device=dev)
        # hierarchy
        self.level_caps = []
        below = cap
        self.sph, self.cone, self.trig = [], [], []
        for _ in range(self.levels):
            below = (below + self.bundle - 1) // self.bundle
            n = max(1, below)
            self.level_caps.append(n)
            self.sph.append(torch.empty((n, 4), dtype=f32, device=dev))
            self.cone.append(torch.empty((n, 4), dtype=f32, device=dev))
            self.trig.append(torch.empty((n, 2), dtype=f32, device=dev))
        self.level_count = torch.zeros(C.MAX_LEVELS, dtype=u32, device=dev)
        pad = [0] * (C.MAX_LEVELS - self.levels)
        self.hier = C.crsh_hierarchy((C.P * C.MAX_LEVELS)(*([_ptr(t) for t in self.sph] + pad)),
                                     (C.P * C.MAX_LEVELS)(*([_ptr(t) for t in self.cone] + pad)),
                                     (C.P * C.MAX_LEVELS)(*([_ptr(t) for t in self.trig] + pad)),
                                     (C.U32 * C.MAX_LEVELS)(*(self.level_caps + pad)), _ptr(self.level_count),
                                     self.levels, self.bundle)
        # hits
        self.hit_tri = torch.empty(cap, dtype=u32, device=dev)
        self.hit_t = torch.empty(cap, dtype=f32, device=dev)
        self.hit_u = torch.empty(cap, dtype=f32, device=dev)
        self.hit_v = torch.empty(cap, dtype=f32, device=dev)
        self.hits = C.crsh_hits(_ptr(self.hit_tri), _ptr(self.hit_t), _ptr(self.hit_u), _ptr(self.hit_v))
        self.ws_hit_bytes = C.crsh_closest_hit_workspace(cap)
        self.ws_hit = torch.empty(self.ws_hit_bytes, dtype=torch.uint8, device=dev)
        self.pair_capacity = 0
        self.set_pair_capacity(int(pair_capacity or max(1 << 20, 64 * cap)))
        stream = torch.cuda.current_stream(dev).cuda_stream
        C.crsh_prepare_scene(self.scene, stream)

    def set_pair_capacity(self, cap: int):
        cap = int(cap)
        if cap == self.pair_capacity:
            return
        dev = self.device
        self.pair_capacity = cap
        self.pair_node = torch.empty(cap, dtype=torch.int32, device=dev)
        self.pair_tri = torch.empty(cap, dtype=torch.int32, device=dev)
        self.pair_off = torch.empty(self.level_caps[0] + 1, dtype=torch.int32, device=dev)
        self.pair_count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.pairs = C.crsh_pairs(_ptr(self.pair_node), _ptr(self.pair_tri), _ptr(self.pair_off),
                                  _ptr(self.pair_count), cap)
        self.ws_trav_bytes = C.crsh_traverse_workspace(self.hier, self.n_tris, self.n_meshes, cap)
        self.ws_trav = None
        torch.cuda.empty_cache()
        self.ws_trav = torch.empty(self.ws_trav_bytes, dtype=torch.uint8, device=dev)

    # ---- inputs ----------------------------------------------------------
    @staticmethod
    def gbuffer_struct(g: Dict[str, torch.Tensor]) -> C.crsh_gbuffer:
        """crsh_gbuffer over device tensors; the struct keeps the tensors alive."""
        s = C.crsh_gbuffer(*[_ptr(g[k]) for k in GB_FIELDS], _ptr(g["material"]), _ptr(g["hit"]),
                           int(g["material"].numel()))
        s.keepalive = g
        return s

    @staticmethod
    def rays_in_struct(r: Dict[str, torch.Tensor]) -> C.crsh_rays_in:
        """crsh_rays_in over device tensors (ox..tmax, type, light); keeps them alive."""
        s = C.crsh_rays_in(*[_ptr(r[k]) for k in RAY_FIELDS], _ptr(r["type"]), _ptr(r.get("light")),
                           int(r["ox"].numel()))
        s.keepalive = r
        return s

    @staticmethod
    def gbuffer_to_device(g: Dict[str, np.ndarray], device="cuda") -> Dict[str, torch.Tensor]:
        out = {k: torch.from_numpy(np.ascontiguousarray(g[k], np.float32)).to(device) for k in GB_FIELDS}
        out["material"] = torch.from_numpy(np.ascontiguousarray(g["material"]).view(np.int32)).to(device)
        out["hit"] = torch.from_numpy(np.ascontiguousarray(g["hit"], np.uint8)).to(device)
        return out

    # ---- the path --------------------------------------------------------
    def hash_sort(self, gbuf: Optional[C.crsh_gbuffer], lights: Optional[torch.Tensor], hp: C.crsh_hash_params,
                  stream: int, rays_in: Optional[C.crsh_rays_in] = None):
        n_lights = 0 if lights is None else int(lights.shape[0])
        C.crsh_hash_sort(gbuf, rays_in, _ptr(lights), n_lights, hp, self.rays, _ptr(self.keys), _ptr(self.n_rays),
                         _ptr(self.counters), _ptr(self.ws_hash), self.ws_hash_bytes, stream)

    def build(self, bp: C.crsh_build_params, stream: int):
        C.crsh_build(self.rays, _ptr(self.n_rays), bp, self.hier, stream)

    def traverse(self, mesh_cull: bool, stream: int, block_threads: int = 0, words: Optional[bool] = None):
        words = self.level1_words if words is None else bool(words)
        C.crsh_traverse(self.hier, self.scene,
                        C.crsh_traverse_params(int(bool(mesh_cull)), int(block_threads), int(words)),
                        self.pairs, _ptr(self.counters), _ptr(self.ws_trav), self.ws_trav_bytes, stream)

    def closest_hit(self, stream: int, hits: Optional[C.crsh_hits] = None):
        """Closest hits into `hits` (default: the pipeline's own hit arrays)."""
        C.crsh_closest_hit(self.hier, self.rays, _ptr(self.n_rays), self.scene, self.pairs,
                           self.hits if hits is None else hits, _ptr(self.counters), _ptr(self.ws_hit),
                           self.ws_hit_bytes, stream)

    def closest_hit_timed(self, stream: int) -> float:
        """closest_hit() that returns the final-test kernel's own duration in ms (synchronous;
        crsh_closest_hit_timed, measurement only)."""
        return C.crsh_closest_hit_timed(self.hier, self.rays, _ptr(self.n_rays), self.scene, self.pairs, self.hits,
                                        _ptr(self.counters), _ptr(self.ws_hit), self.ws_hit_bytes, stream)

    def bruteforce(self, stream: Optional[int] = None):
        stream = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        C.crsh_bruteforce_closest_hit(self.rays, _ptr(self.n_rays), self.scene, self.hits, _ptr(self.ws_hit),
                                      self.ws_hit_bytes, stream)

    def backward(self, g_t: torch.Tensor, g_u: torch.Tensor, g_v: torch.Tensor, stream: Optional[int] = None):
        """Gradients of the current hits (crsh_closest_hit_backward): upstream gradients in
        generation order -> (g_verts (T, 9), g_orig (capacity, 3), g_dir (capacity, 3))."""
        stream = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        dev = self.device
        if getattr(self, "ws_bw", None) is None:
            self.ws_bw_bytes = C.crsh_closest_hit_backward_workspace(self.ray_capacity)
            self.ws_bw = torch.empty(self.ws_bw_bytes, dtype=torch.uint8, device=dev)
        g_verts = torch.empty((self.n_tris, 9), dtype=torch.float32, device=dev)
        g_orig = torch.empty((self.ray_capacity, 3), dtype=torch.float32, device=dev)
        g_dir = torch.empty((self.ray_capacity, 3), dtype=torch.float32, device=dev)
        gt, gu, gv = (x.contiguous().float() for x in (g_t, g_u, g_v))
        C.crsh_closest_hit_backward(self.rays, _ptr(self.n_rays), self.scene, self.hits, _ptr(gt), _ptr(gu), _ptr(gv),
                                    _ptr(g_verts), _ptr(g_orig), _ptr(g_dir), _ptr(self.counters), _ptr(self.ws_bw),
                                    self.ws_bw_bytes, stream)
        return g_verts, g_orig, g_dir

    def run(self, gbuf: C.crsh_gbuffer, lights: Optional[torch.Tensor], hp: C.crsh_hash_params,
            bp: C.crsh_build_params, mesh_cull: bool = True, stream: Optional[int] = None,
            hits: Optional[C.crsh_hits] = None):
        """One pass of the whole path (asynchronous); hits as in closest_hit()."""
        stream = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        self.hash_sort(gbuf, lights, hp, stream)
        self.build(bp, stream)
        self.traverse(mesh_cull, stream)
        self.closest_hit(stream, hits)

    def run_fit(self, gbuf, lights, hp, bp, mesh_cull=True, max_tries=8):
        """run(), growing the pair lists until no level overflows (synchronises)."""
        for _ in range(max_tries):
            self.run(gbuf, lights, hp, bp, mesh_cull)
            c = self.read_counters()
            if c["status"] == C.ERR_CAPACITY and c["needed_pairs"] > self.pair_capacity:
                if c["needed_pairs"] > (1 << 31):
                    raise RuntimeError(f"pair lists of {c['needed_pairs']} entries exceed the 2^31 capacity limit")
                self.set_pair_capacity(min(int(c["needed_pairs"] * 1.25) + 1024, 1 << 31))
                continue
            if c["status"] != C.OK:
                raise C.CrshError("device status", c["status"])
            return c
        raise RuntimeError("pair capacity did not converge")

    # ---- primary visibility and first-hit buffers (NEXT row f3) -----------
    @staticmethod
    def camera_struct(camera: np.ndarray, width: int, height: int) -> C.crsh_camera:
        """camera = eye, fwd, right, up (3 each), tan_x, tan_y."""
        c = np.asarray(camera, np.float64)
        return C.crsh_camera((C.F32 * 3)(*c[0:3]), (C.F32 * 3)(*c[3:6]), (C.F32 * 3)(*c[6:9]),
                             (C.F32 * 3)(*c[9:12]), float(c[12]), float(c[13]), int(width), int(height))

    def primary(self, cam: C.crsh_camera, stream: int):
        """Camera rays into the sorted-ray buffers (they need no hashing or sorting)."""
        C.crsh_primary_rays(cam, self.rays, _ptr(self.n_rays), stream)

    def run_primary(self, cam: C.crsh_camera, bp: C.crsh_build_params, stream: Optional[int] = None):
        """Primary visibility through the hierarchy: camera rays -> build -> traverse -> closest hit."""
        stream = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        self.primary(cam, stream)
        self.build(bp, stream)
        self.traverse(True, stream)
        self.closest_hit(stream)

    def gbuffer_out(self, n: int) -> Tuple[Dict[str, torch.Tensor], C.crsh_gbuffer_out]:
        """A writable first-hit buffer of n entries."""
        dev = self.device
        g = {k: torch.empty(n, dtype=torch.float32, device=dev) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix",
                                                                         "iy", "iz")}
        g["material"] = torch.empty(n, dtype=torch.int32, device=dev)
        g["hit"] = torch.empty(n, dtype=torch.uint8, device=dev)
        s = C.crsh_gbuffer_out(*[_ptr(g[k]) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz",
                                                     "material", "hit")], n)
        s.keepalive = g
        return g, s

    def gbuffer_from_hits(self, tri_material: torch.Tensor, out: C.crsh_gbuffer_out, stream: Optional[int] = None):
        """First-hit buffer of the traced rays, indexed by ray_id (asynchronous)."""
        stream = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        C.crsh_gbuffer_from_hits(self.rays, _ptr(self.n_rays), self.hits, self.scene, _ptr(tri_material), out, stream)

    def shade(self, gbuf: C.crsh_gbuffer, lights: Optional[torch.Tensor], tri_material: torch.Tensor,
              stream: Optional[int] = None) -> torch.Tensor:
        """Grey-level shading of the frame from its secondary rays and hits (asynchronous)."""
        stream = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        npx = int(gbuf.n_pixels)
        nl = 0 if lights is None else int(lights.shape[0])
        cells = torch.empty(npx * (nl + 2), dtype=torch.float32, device=self.device)
        color = torch.empty(npx, dtype=torch.float32, device=self.device)
        C.crsh_shade(gbuf, _ptr(lights), nl, self.rays, _ptr(self.n_rays), self.hits, _ptr(tri_material),
                     _ptr(cells), _ptr(color), stream)
        color.keepalive = cells
        return color

    # ---- results (synchronising) ------------------------------------------
    def read_counters(self) -> dict:
        torch.cuda.synchronize(self.device)
        return counters_from_bytes(self.counters.cpu().numpy().tobytes(), self.levels)

    def n(self) -> int:
        return int(self.n_rays.item())

    def sorted_rays(self) -> Dict[str, np.ndarray]:
        n = self.n()
        out = {k: self.rays_t[k][:n].cpu().numpy() for k in RAY_FIELDS + ("type", "pixel")}
        out["ray_id"] = self.rays_t["ray_id"][:n].cpu().numpy().view(np.uint32)
        out["keys"] = self.keys[:n].cpu().numpy().view(np.uint32)
        return out

    def hits_host(self):
        n = self.n()
        return (self.hit_tri[:n].cpu().numpy().view(np.int32), self.hit_t[:n].cpu().numpy(),
                self.hit_u[:n].cpu().numpy(), self.hit_v[:n].cpu().numpy())

    def levels_host(self):
        cnt = self.level_count.cpu().numpy().view(np.uint32)
        return [(self.sph[l][:cnt[l]].cpu().numpy(), self.cone[l][:cnt[l]].cpu().numpy(),
                 self.trig[l][:cnt[l]].cpu().numpy()) for l in range(self.levels)]

    def pairs_host(self):
        if self.pairs.words.valid:
            raise RuntimeError("level 1 is in word form: no pair list was written")
        p = min(int(self.pair_count.item()), self.pair_capacity)
        cnt = int(self.level_count[0].item())
        return (self.pair_node[:p].cpu().numpy().view(np.uint32), self.pair_tri[:p].cpu().numpy().view(np.uint32),
                self.pair_off[:cnt + 1].cpu().numpy().view(np.uint32))


def workload_pipeline(w, *, device="cuda", pair_capacity=None, level1_words=False) -> "Pipeline":
    return Pipeline(w.scene, max_pixels=w.n_pixels, n_lights=w.lights.shape[0], bundle=w.bundle, levels=w.levels,
                    pair_capacity=pair_capacity, device=device, level1_words=level1_words)


def workload_params(w, *, sort=True, compress=True):
    hp = hash_params(w.hash_lo, w.hash_hi, shadow_cull=w.shadow_cull, sort=sort, compress=compress)
    bp = build_params(w.bundle, w.levels, w.build_pads())
    return hp, bp
