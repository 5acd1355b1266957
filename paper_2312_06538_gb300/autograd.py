"""torch.autograd.Function around the closest hit: differentiable (t, u, v) of
rays against triangles, through the hierarchy path of libcrsh.so forward and
crsh_closest_hit_backward backward (hit assignment held fixed)."""
from __future__ import annotations

import numpy as np
import torch

from . import crsh as C
from .pipeline import Pipeline, RAY_FIELDS, build_params, hash_params


class SceneRays:
    """Static configuration of the differentiable call: mesh layout and spheres, hierarchy and
    hash parameters, and buffers sized for up to `max_rays` rays."""

    def __init__(self, scene, max_rays: int, bundle=16, levels=4, pads=None, hash_lo=None, hash_hi=None,
                 device="cuda"):
        self.p = Pipeline(scene, max_pixels=0, n_lights=0, bundle=bundle, levels=levels, ray_capacity=max_rays,
                          device=device)
        ext = float(np.abs(scene.verts).max())
        self.pads = pads or (1e-5, 1e-6 * max(ext, 1.0), 1e-5, 1e-5)
        lo = np.asarray(hash_lo if hash_lo is not None else scene.verts.reshape(-1, 3).min(0) - 1e-3, np.float32)
        hi = np.asarray(hash_hi if hash_hi is not None else scene.verts.reshape(-1, 3).max(0) + 1e-3, np.float32)
        self.hp = hash_params(lo, hi)
        self.bp = build_params(bundle, levels, self.pads)


class CRSHClosestHit(torch.autograd.Function):
    """forward(origins (N,3), directions (N,3), verts (T,3,3), types (N,) uint8, tmax (N,), cfg)
    -> t (N,), u (N,), v (N,), tri (N,) int32 (not differentiable; -1 = miss)."""

    @staticmethod
    def forward(ctx, origins, directions, verts, types, tmax, cfg: SceneRays):
        p = cfg.p
        n = origins.shape[0]
        if n > p.ray_capacity:
            raise ValueError("more rays than the configuration holds")
        # triangles: the scene's SoA arrays are the differentiable vertices
        v = verts.detach().contiguous().float()
        for k in range(3):
            for a, ax in enumerate("xyz"):
                p.scene_t[f"v{k}{ax}"].copy_(v[:, k, a])
        stream = torch.cuda.current_stream(p.device).cuda_stream
        C.crsh_prepare_scene(p.scene, stream)
        rays = {"ox": origins[:, 0], "oy": origins[:, 1], "oz": origins[:, 2], "dx": directions[:, 0],
                "dy": directions[:, 1], "dz": directions[:, 2], "tmax": tmax}
        rays = {k: x.detach().contiguous().float() for k, x in rays.items()}
        rays["type"] = types.detach().contiguous().to(torch.uint8)
        rays["light"] = torch.zeros_like(rays["type"])
        rin = Pipeline.rays_in_struct(rays)
        for _ in range(8):
            p.hash_sort(None, None, cfg.hp, stream, rays_in=rin)
            p.build(cfg.bp, stream)
            p.traverse(True, stream)
            p.closest_hit(stream)
            c = p.read_counters()
            if c["status"] == C.ERR_CAPACITY and c["needed_pairs"] > p.pair_capacity:
                p.set_pair_capacity(int(c["needed_pairs"] * 1.25) + 1024)
                continue
            break
        if c["status"] != C.OK:
            raise C.CrshError("closest hit", c["status"])
        t, u, w = p.hit_t[:n].clone(), p.hit_u[:n].clone(), p.hit_v[:n].clone()
        tri = p.hit_tri[:n].clone()
        ctx.cfg = cfg
        ctx.n = n
        ctx.mark_non_differentiable(tri)
        return t, u, w, tri

    @staticmethod
    def backward(ctx, g_t, g_u, g_v, g_tri):
        p, n = ctx.cfg.p, ctx.n
        dev = p.device
        z = torch.zeros(p.ray_capacity, dtype=torch.float32, device=dev)
        gt, gu, gv = z.clone(), z.clone(), z.clone()
        if g_t is not None:
            gt[:n] = g_t
        if g_u is not None:
            gu[:n] = g_u
        if g_v is not None:
            gv[:n] = g_v
        g_verts, g_orig, g_dir = p.backward(gt, gu, gv)
        return g_orig[:n], g_dir[:n], g_verts.view(-1, 3, 3), None, None, None


def closest_hit(origins, directions, verts, types, tmax, cfg: SceneRays):
    """Differentiable closest hit: (t, u, v, tri) for each ray, in input order."""
    return CRSHClosestHit.apply(origins, directions, verts, types, tmax, cfg)
