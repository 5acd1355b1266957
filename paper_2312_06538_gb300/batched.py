"""Many ray batches of uneven size over several scenes through one CUDA graph.

Each batch gets its own buffers and its own hierarchy shape (bundle B, depth L)
chosen by an autotuner per size class.  All batches are captured once into a
single CUDA graph, spread over several streams so that small batches overlap;
replaying the graph runs every batch with no host work per launch.  The plain
alternative runs each batch through the four C-ABI calls from Python with the
default B = 16, L = 4, one after the other.  Hits do not depend on B or L
(culling is conservative and the final test is the same function), so both
give identical bits.  (Not a step of the paper, which traces one batch at a
time; it is the paper's per-batch steps 3-7 of Section 3.1 run back to back.)
"""
from __future__ import annotations

import math
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import crsh as C
from .pipeline import Pipeline, RAY_FIELDS, build_params, hash_params

BUNDLES = (4, 8, 16, 32, 64)
DEPTHS = (2, 3, 4, 5, 6)
BLOCKS = (128, 256, 512)   # threads per block of the traversal's test and emit passes


def secondary_rays(scene, gbuffer: Dict[str, np.ndarray], lights: np.ndarray, n: int, hash_lo, hash_hi,
                   shadow_cull=True, device="cuda") -> Tuple[Dict[str, torch.Tensor], int]:
    """The first n secondary rays (generation order) of a primary-hit buffer, generated by the
    library itself (crsh_hash_sort with sorting off).  Returns device tensors and the count."""
    npx = int(gbuffer["material"].shape[0])
    p = Pipeline(scene, max_pixels=npx, n_lights=lights.shape[0], bundle=16, levels=1, device=device,
                 pair_capacity=1 << 10)
    hp = hash_params(hash_lo, hash_hi, shadow_cull=shadow_cull, sort=False, compress=False)
    g = p.gbuffer_struct(p.gbuffer_to_device(gbuffer, device))
    lt = torch.from_numpy(np.ascontiguousarray(lights, np.float32)).to(device) if lights.shape[0] else None
    p.hash_sort(g, lt, hp, torch.cuda.current_stream(p.device).cuda_stream)
    got = min(p.n(), n)
    out = {k: p.rays_t[k][:got].clone() for k in RAY_FIELDS + ("type",)}
    out["light"] = torch.zeros(got, dtype=torch.uint8, device=device)
    # light index of shadow rays: shadow slots of a pixel come in light order
    if lights.shape[0] > 1:
        # recover it from the key: the light bits sit above the shadow direction code
        # (theta + phi bits of the hash parameters)
        code_bits = int(hp.shadow_theta_bits) + int(hp.shadow_phi_bits)
        light_mask = (1 << (30 - code_bits)) - 1
        keys = p.keys[:got].to(torch.int64) & 0xFFFFFFFF
        sh = out["type"] == C.RAY_SHADOW
        out["light"] = torch.where(sh, (keys >> code_bits) & light_mask, torch.zeros_like(keys)).to(torch.uint8)
    del p
    return out, got


class BatchRun:
    """Buffers and calls for one batch of prebuilt rays with a given hierarchy shape."""

    def __init__(self, scene, rays: Dict[str, torch.Tensor], n: int, bundle: int, levels: int, pads, hp,
                 device="cuda", block: int = 256, level1_words: bool = True):
        self.n = n
        self.rays = rays
        self.p = Pipeline(scene, max_pixels=0, n_lights=0, bundle=bundle, levels=levels, ray_capacity=max(1, n),
                          pair_capacity=max(1 << 16, 32 * n), device=device, level1_words=level1_words)
        self.rin = Pipeline.rays_in_struct(rays)
        self.hp = hp
        self.bp = build_params(bundle, levels, pads)
        self.bundle, self.levels, self.block = bundle, levels, block

    def run(self, stream: int):
        p = self.p
        p.hash_sort(None, None, self.hp, stream, rays_in=self.rin)
        p.build(self.bp, stream)
        p.traverse(True, stream, self.block)
        p.closest_hit(stream)

    def fit(self, max_tries=8) -> dict:
        """Run once, growing the pair lists until nothing overflows (synchronises)."""
        stream = torch.cuda.current_stream(self.p.device).cuda_stream
        for _ in range(max_tries):
            self.run(stream)
            c = self.p.read_counters()
            if c["status"] == C.ERR_CAPACITY and c["needed_pairs"] > self.p.pair_capacity:
                self.p.set_pair_capacity(int(c["needed_pairs"] * 1.25) + 1024)
                continue
            if c["status"] != C.OK:
                raise C.CrshError("batch", c["status"])
            return c
        raise RuntimeError("pair capacity did not converge")

    def hits(self):
        n = self.n
        return (self.p.hit_tri[:n], self.p.hit_t[:n], self.p.hit_u[:n], self.p.hit_v[:n])


def _time_ms(fn, reps=3) -> float:
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sorted(ts)[len(ts) // 2]


class Autotuner:
    """Picks (B, L, block) per batch-size class (floor(log2 n)) by timing candidates on a
    representative batch of that class: every (B, L) at the default block shape, then the
    block shapes of the traversal passes for the best (B, L).  Results are reused for the
    other batches of the class."""

    def __init__(self, bundles: Sequence[int] = BUNDLES, depths: Sequence[int] = DEPTHS, reps: int = 3,
                 blocks: Sequence[int] = BLOCKS):
        self.bundles, self.depths, self.reps, self.blocks = tuple(bundles), tuple(depths), reps, tuple(blocks)
        self.table: Dict[int, Tuple[int, int, int]] = {}
        self.log: List[dict] = []

    @staticmethod
    def size_class(n: int) -> int:
        return int(math.floor(math.log2(max(1, n))))

    def choose(self, scene, rays, n, pads, hp, device="cuda") -> Tuple[int, int, int]:
        k = self.size_class(n)
        if k in self.table:
            return self.table[k]
        best, best_ms = (16, 4, 256), float("inf")
        stream = lambda: torch.cuda.current_stream().cuda_stream  # noqa: E731

        def trial(B, L, blk):
            br = BatchRun(scene, rays, n, B, L, pads, hp, device, block=blk)
            br.fit()
            ms = _time_ms(lambda: br.run(stream()), self.reps)
            self.log.append({"size_class": k, "bundle": B, "levels": L, "block": blk, "ms": ms})
            del br
            return ms
        blk0 = 256 if 256 in self.blocks else self.blocks[0]
        for B in self.bundles:
            for L in self.depths:
                if B ** (L - 1) > max(n, 1):   # more levels than the batch can fill
                    continue
                ms = trial(B, L, blk0)
                if ms < best_ms:
                    best, best_ms = (B, L, blk0), ms
        for blk in self.blocks:
            if blk != blk0:
                ms = trial(best[0], best[1], blk)
                if ms < best_ms:
                    best, best_ms = (best[0], best[1], blk), ms
        torch.cuda.empty_cache()
        self.table[k] = best
        return best


class BatchedCRSH:
    """All batches in one CUDA graph over `n_streams` streams."""

    def __init__(self, batches: Sequence[Tuple[object, Dict[str, torch.Tensor], int]], pads_of, hp_of,
                 tuner: Optional[Autotuner] = None, n_streams: int = 8, device="cuda"):
        self.device = torch.device(device)
        self.tuner = tuner or Autotuner()
        self.runs: List[BatchRun] = []
        for scene, rays, n in batches:
            B, L, blk = self.tuner.choose(scene, rays, n, pads_of(scene), hp_of(scene), device)
            br = BatchRun(scene, rays, n, B, L, pads_of(scene), hp_of(scene), device, block=blk)
            br.fit()
            self.runs.append(br)
        self.n_streams = n_streams
        self.graph = None

    def capture(self):
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(self.device)
        side = [torch.cuda.Stream(self.device) for _ in range(self.n_streams)]
        with torch.cuda.graph(g, stream=cap):
            for s in side:
                s.wait_stream(cap)
            # largest batches first, round-robin over the streams
            order = sorted(range(len(self.runs)), key=lambda i: -self.runs[i].n)
            for j, i in enumerate(order):
                s = side[j % self.n_streams]
                self.runs[i].run(s.cuda_stream)
            for s in side:
                cap.wait_stream(s)
        self.graph = g
        self._streams = (cap, side)
        return g

    def replay(self):
        self.graph.replay()

    def check_status(self):
        bad = [i for i, r in enumerate(self.runs) if r.p.read_counters()["status"] != C.OK]
        return bad


class PlainBatches:
    """Reference: each batch through the four calls in turn, default B = 16, L = 4, level 1 as a
    list, one stream.
    capture() records the same calls, in the same order on one stream, as one CUDA graph
    (the ablation that removes only the host's launch gaps)."""

    def __init__(self, batches, pads_of, hp_of, device="cuda", bundle=16, levels=4, level1_words=False):
        self.device = torch.device(device)
        self.runs = []
        for scene, rays, n in batches:
            br = BatchRun(scene, rays, n, bundle, levels, pads_of(scene), hp_of(scene), device,
                          level1_words=level1_words)
            br.fit()
            self.runs.append(br)
        self.graph = None

    def run(self):
        stream = torch.cuda.current_stream().cuda_stream
        for r in self.runs:
            r.run(stream)

    def capture(self):
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(self.device)
        with torch.cuda.graph(g, stream=cap):
            for r in self.runs:
                r.run(cap.cuda_stream)
        self.graph = g
        self._stream = cap
        return g

    def replay(self):
        self.graph.replay()
