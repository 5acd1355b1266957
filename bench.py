"""Benchmark of the CRSH path on GB300: secondary rays per second for one frame.

A step is one pass of the whole path over one frame's primary-hit buffer:
crsh_hash_sort -> crsh_build -> crsh_traverse -> crsh_closest_hit.  Default
workload: 512x512, 60,162 triangles in 17 meshes (30 % mirror, 20 % glass),
2 lights, B = 16, L = 4 (all inputs synthetic, seeded).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 the script runs under torchrun: every rank runs its own replica of
the frame (the path has no exchange step), ranks meet at a barrier around the
timed steps and the slowest rank's time counts (weak scaling).
--impl reference times the CPU oracle (the plain restatement of the method
used by the tests) on the host cores instead; under torchrun only rank 0 runs.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from typing import Optional

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "secondary Mrays/s, batched vs plain at exact hits; tri tests/ray; adjoint ms"
UNIT = "Mrays/s"
MT_FLOPS = 46          # FP32 operations of one Moller-Trumbore test (cross 9, dots 5 each, 1 reciprocal,
                       # 3 subtractions, 3 scalings, u + v 1)
EQ9_FLOPS = 27         # FP32 operations of one sphere-cone test (eq. 9)
L2_FLUSH_BYTES = 512 << 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_over_ranks(local_ms: float, local_units: float, world: int):
    """Max time and total units over ranks (identity when world == 1)."""
    if world <= 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def workload_description(w):
    return (f"plain CRSH frame: {w.width}x{w.height} primary hits, {w.scene.n_tris:,} triangles in "
            f"{w.scene.n_meshes} meshes, {w.lights.shape[0]} lights, shadow+reflection+refraction rays, "
            f"B={w.bundle}, L={w.levels}")


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle on the host cores
# ---------------------------------------------------------------------------

def crop_pixels(w, side: int, x0=None, y0=None):
    """Pixel indices of a side x side crop of the frame (central by default), row-major."""
    W, H = w.width, w.height
    x0 = (W - side) // 2 if x0 is None else x0
    y0 = (H - side) // 2 if y0 is None else y0
    return (np.arange(y0, y0 + side)[:, None] * W + np.arange(x0, x0 + side)[None, :]).reshape(-1)


def crop_gbuffer(w, side: int, x0=None, y0=None):
    """A crop of the frame's G-buffer (same scene, same ray mix)."""
    idx = crop_pixels(w, side, x0, y0)
    return {k: np.ascontiguousarray(v[idx]) for k, v in w.gbuffer.items()}


def oracle_step(w, g):
    import oracle
    t0 = time.perf_counter()
    r = oracle.run_crsh(g, w.lights, w.shadow_cull, w.hash_lo, w.hash_hi, w.scene, w.bundle, w.levels,
                        w.build_pads())
    return time.perf_counter() - t0, r["counters"]["rays"], r


# Worker processes of the all-core oracle timing: each builds the workload once
# and runs the single-threaded oracle over the tiles it is handed.
_WORKER = {}


def _worker_init(config: int, res):
    import oracle
    import synthetic
    oracle.compile_native()
    _WORKER["w"] = synthetic.make(config, res=res)


def _worker_tile(tile):
    side, x0, y0 = tile
    w = _WORKER["w"]
    _, n, _ = oracle_step(w, crop_gbuffer(w, side, x0, y0))
    return n


def tile_grid(w, side: int, count: int):
    """count distinct side x side tiles, nearest the frame centre first."""
    W, H = w.width, w.height
    tiles = [(side, x, y) for y in range(0, H - side + 1, side) for x in range(0, W - side + 1, side)]
    cx, cy = W / 2, H / 2
    tiles.sort(key=lambda t: (t[1] + side / 2 - cx) ** 2 + (t[2] + side / 2 - cy) ** 2)
    return [tiles[i % len(tiles)] for i in range(count)]


class OraclePool:
    """The single-threaded oracle run on every host core at once, one process per core
    (started with spawn, so it is safe after CUDA has been initialised)."""

    def __init__(self, config: int, res, procs=None):
        import multiprocessing as mp
        import oracle
        oracle.compile_native()
        self.procs = int(procs or os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_worker_init, initargs=(config, res))

    def run(self, tiles):
        """Runs the tiles; returns (wall seconds, rays)."""
        t0 = time.perf_counter()
        n = sum(self.pool.map(_worker_tile, tiles, chunksize=1))
        return time.perf_counter() - t0, n

    def close(self):
        self.pool.close()
        self.pool.join()


def flagged_vs_oracle(w, ref, crop_idx, gpu_hits, gpu_gen_pixel):
    """Closest hits of the GPU frame against the oracle's for the rays of one crop (the
    rays of the crop are, in order, the frame's rays whose pixel lies in the crop)."""
    from tests import parity
    sel = np.nonzero(np.isin(gpu_gen_pixel, crop_idx))[0]
    n_ref = ref["hits"][0].shape[0]
    if sel.shape[0] != n_ref:
        return {"error": f"crop has {n_ref} oracle rays, the frame {sel.shape[0]}"}
    rep = parity.compare_hits(tuple(h[sel] for h in gpu_hits), ref["hits"], ref["rays"], w.scene.verts)
    return {"rays_compared": int(n_ref), "hits": rep["hits"], "flagged_ties": rep["ties"],
            "flagged_edges": rep["edges"], "flagged_order": rep["order"], "unexplained": len(rep["unexplained"]),
            "t_beyond_tol": rep["t_viol"], "uv_beyond_tol": rep["uv_viol"], "max_t_rel": rep["max_t_rel"],
            "max_uv_abs": rep["max_uv_abs"], "rules": "tests/parity.py (tie, FP32-decision edge, FP32 t order)"}


def cpu_baseline(w, config: int, res, budget_s: float = 15.0, side: int = 128, gpu_hits=None, gpu_gen_pixel=None):
    """The oracle on the host: single-threaded over the central crop (grown until one pass
    costs about budget_s / 6), and on every core at once over distinct tiles of that size.
    The single-threaded pass's hits also check the GPU frame's (flagged counts)."""
    import oracle
    oracle.compile_native()
    g = crop_gbuffer(w, side)
    dt, n, ref = oracle_step(w, g)
    while dt < budget_s / 6 and side * 2 <= min(w.width, w.height):
        side *= 2
        g = crop_gbuffer(w, side)
        dt, n, ref = oracle_step(w, g)
    out = {"value": n / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"central {side}x{side} crop of the frame ({n} rays), one pass, single-threaded C"}
    if gpu_hits is not None:
        out["parity_sample"] = flagged_vs_oracle(w, ref, crop_pixels(w, side), gpu_hits, gpu_gen_pixel)
    try:
        pool = OraclePool(config, res)
        tiles = tile_grid(w, side, pool.procs)
        pool.run(tile_grid(w, 16, pool.procs))          # warm-up: workers built
        wall, rays = pool.run(tiles)
        pool.close()
        out["all_cores"] = {"value": rays / wall / 1e6, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                            "sample": f"{len(tiles)} distinct {side}x{side} tiles of the frame ({rays} rays), one "
                                      f"single-threaded oracle process per core, wall clock"}
    except Exception as e:  # the all-core leg must not cost the line
        out["all_cores"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_reference(args, w):
    """The reference arm: the oracle on all host cores, each step one tile per core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    side = args.ref_crop
    pool = OraclePool(args.config, args.res)
    tiles = tile_grid(w, side, pool.procs)
    for _ in range(args.warmup):
        pool.run(tiles)
    times, rays = [], 0
    for _ in range(args.steps):
        dt, n = pool.run(tiles)
        times.append(dt)
        rays += n
    pool.close()
    tot = sum(times)
    value = rays / tot / 1e6
    sample = (f"{len(tiles)} distinct {side}x{side} tiles of the frame per step ({rays // args.steps} rays), one "
              f"single-threaded oracle process per core")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_description(w), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def closest_traffic(kernel: str, config: int, res) -> Optional[float]:
    """DRAM bytes per launch of the final-test kernel from the committed ncu summary, or None
    when the record is of another workload or the kernel source changed since those counters
    were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        if rec["config"] != config or res is not None:
            return None
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
            return None
        return rec["bytes_per_launch"]
    except Exception:
        return None


def launches_per_step(levels: int, compress: bool, words: bool = False) -> int:
    """Kernels of libcrsh.so launched by one pass (count of <<<>>> in the call sequence)."""
    # tables, zeroing, gen, chunk (which also counts the digits) or hist, plan, 4 passes, pos, gather
    hash_sort = 1 + 1 + 1 + 1 + 1 + 4 + (1 if compress else 0) + 1
    build = max(1, levels - 1)   # level 1 (with level 2 merged in), then one per level above
    if words and levels >= 2:    # zeroing, mesh stage, top stage, 5 kernels per level above 1; unit scan, count, items at 1
        traverse = 1 + 1 + 5 + 5 * (levels - 2) + 3
    else:                        # zeroing, mesh stage, top stage, 5 kernels per level, csr
        traverse = 1 + 1 + 5 + 5 * (levels - 1) + 1
    closest = 3
    return hash_sort + build + traverse + closest


def time_path(run, flush, stream, reps: int, warmup: int = 3) -> float:
    """Mean ms of run() over reps, CUDA events on the stream, L2 flushed before each."""
    import torch
    for _ in range(warmup):
        flush.fill_(1)
        run()
    ts = []
    for k in range(reps):
        flush.fill_(k & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ts) / reps


def comparators(w, p, gstruct, lights, hp, bp, flush, stream, dev, n_rays):
    """Same frame through the N x M brute force (after the same hash/sort) and through
    the unsorted, no-mesh-culling mode (the RAH comparison of the paper)."""
    import torch
    from paper_2312_06538_gb300 import pipeline as pl
    sh = stream.cuda_stream
    out = {}

    def brute():
        p.hash_sort(gstruct, lights, hp, sh)
        p.bruteforce(sh)
    ms = time_path(brute, flush, stream, reps=3, warmup=1)
    out["bruteforce"] = {"mrays_per_s": n_rays / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                         "tri_tests_per_ray": w.scene.n_tris}
    hp_rah, _ = pl.workload_params(w, sort=False)
    # Unsorted nodes accept far more triangles: the pair lists of the whole frame may not
    # fit the 2^31-entry pair capacity; then the mode runs on the largest central crop
    # (512, 256 or 128 pixels square) whose lists fit.
    sample = "the whole frame"
    q, c, why = None, None, ""
    try:
        q = pl.workload_pipeline(w, device=dev)
        g_rah = gstruct
        c = q.run_fit(g_rah, lights, hp_rah, bp, mesh_cull=False)
    except Exception as e:
        why = f"{type(e).__name__} on the whole frame: {e}"
        q = None
    for side in (512, 256, 128):
        if c is not None or side > min(w.width, w.height):
            continue
        torch.cuda.empty_cache()
        try:
            g_crop = pl.Pipeline.gbuffer_to_device(crop_gbuffer(w, side), dev)
            q = pl.Pipeline(w.scene, max_pixels=side * side, n_lights=w.lights.shape[0], bundle=w.bundle,
                            levels=w.levels, device=dev)
            g_rah = q.gbuffer_struct(g_crop)
            c = q.run_fit(g_rah, lights, hp_rah, bp, mesh_cull=False)
            sample = f"central {side}x{side} crop ({why})"
        except Exception as e:
            why += f"; {type(e).__name__} on the {side}x{side} crop"
            q = None
    ms = time_path(lambda: q.run(g_rah, lights, hp_rah, bp, mesh_cull=False, stream=sh), flush, stream, reps=5)
    out["unsorted_no_mesh_cull"] = {"mrays_per_s": c["rays"] / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                                    "tri_tests_per_ray": c["final_tests"] / max(1, c["rays"]),
                                    "all_tests_per_ray": (c["final_tests"] + sum(c["tests"])) / max(1, c["rays"]),
                                    "rays": c["rays"], "sample": sample}
    del q
    torch.cuda.empty_cache()
    return out


def adjoint_timing(dev, flush, stream, reps: int = 10):
    """Backward (crsh_closest_hit_backward) vs forward closest hit on the adjoint workload:
    2^20 reflection rays of a 1024x1024 all-mirror frame, 99,842 triangles (config 5)."""
    import synthetic
    import torch
    from paper_2312_06538_gb300 import pipeline as pl
    w5 = synthetic.make(5)
    p5 = pl.workload_pipeline(w5, device=dev)
    hp5, bp5 = pl.workload_params(w5)
    g5 = p5.gbuffer_struct(p5.gbuffer_to_device(w5.gbuffer, dev))
    c5 = p5.run_fit(g5, None, hp5, bp5)
    n = c5["rays"]
    z = torch.randn((3, p5.ray_capacity), generator=torch.Generator().manual_seed(1005)).to(dev)
    sh = stream.cuda_stream
    fwd = time_path(lambda: p5.closest_hit(sh), flush, stream, reps)
    bwd = time_path(lambda: p5.backward(z[0], z[1], z[2], sh), flush, stream, reps)
    out = {"workload": f"{n} reflection rays, {w5.scene.n_tris:,} triangles (1024x1024 all-mirror frame)",
           "backward_ms": bwd, "forward_closest_hit_ms": fwd, "backward_over_forward": bwd / fwd,
           "hit_rays": int((p5.hit_tri[:n] >= 0).sum().item())}
    del p5
    torch.cuda.empty_cache()
    return out


def batched_comparison(dev, n_batches=32, reps=5):
    """32 ray batches of log-uniform size (2^11 .. 2^20 rays) over 8 scenes of 5k..200k
    triangles: the batched pipeline (autotuned B, L per size class, one CUDA graph over 8
    streams) against the plain pipeline run per batch (B = 16, L = 4, one stream)."""
    import math
    import synthetic
    import torch
    from paper_2312_06538_gb300 import batched as bt
    from paper_2312_06538_gb300 import pipeline as pl
    spec = synthetic.config4_batches(n_batches)
    batches, frames = [], {}
    t0 = time.perf_counter()
    for n, k in spec:
        res = max(16, int(math.ceil(math.sqrt(n))))
        while True:
            wk = synthetic.config4_frame(k, res)
            rays, got = bt.secondary_rays(wk.scene, wk.gbuffer, wk.lights, n, wk.hash_lo, wk.hash_hi, device=dev)
            if got >= n:
                break
            res = int(res * 1.3) + 1
        frames[id(wk.scene)] = wk
        batches.append((wk.scene, rays, n))
    prep_s = time.perf_counter() - t0
    pads_of = lambda sc: frames[id(sc)].build_pads()  # noqa: E731
    hp_of = lambda sc: pl.hash_params(frames[id(sc)].hash_lo, frames[id(sc)].hash_hi)  # noqa: E731
    t0 = time.perf_counter()
    tuner = bt.Autotuner()
    bat = bt.BatchedCRSH(batches, pads_of, hp_of, tuner=tuner, n_streams=8, device=dev)
    tune_s = time.perf_counter() - t0
    plain = bt.PlainBatches(batches, pads_of, hp_of, device=dev)
    plain_g = bt.PlainBatches(batches, pads_of, hp_of, device=dev)
    plain_w = bt.PlainBatches(batches, pads_of, hp_of, device=dev, level1_words=True)
    fixed = bt.BatchedCRSH(batches, pads_of, hp_of, tuner=bt.Autotuner(bundles=(16,), depths=(4,), reps=1, blocks=(256,)),
                           n_streams=8, device=dev)
    bat.capture()
    plain_g.capture()
    plain_w.capture()
    fixed.capture()
    total = sum(n for _, _, n in batches)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        """Median of reps, CUDA events on the launching stream (the graph replays run
        their side streams between the events)."""
        fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b) * 1e-3)
        return sorted(ts)[len(ts) // 2]
    tp = timed(plain.run)
    tpg = timed(plain_g.replay)
    tpw = timed(plain_w.replay)
    tf = timed(fixed.replay)
    tb = timed(bat.replay)
    identical = all(torch.equal(x.view(torch.int32), y.view(torch.int32))
                    for runs in (bat.runs, plain_g.runs, plain_w.runs, fixed.runs)
                    for a, b in zip(runs, plain.runs) for x, y in zip(a.hits(), b.hits()))
    out = {"workload": f"{len(batches)} batches, {total:,} rays, sizes {min(n for n, _ in spec)}..{max(n for n, _ in spec)}, "
                       f"8 scenes of 5k..200k triangles",
           "plain_mrays_per_s": total / tp / 1e6, "batched_mrays_per_s": total / tb / 1e6,
           "batched_over_plain": tp / tb, "identical_hits": bool(identical),
           "plain_ms": 1e3 * tp, "batched_ms": 1e3 * tb,
           "ablation": {
               "plain_eager_ms": 1e3 * tp,
               "plain_one_graph_one_stream_ms": 1e3 * tpg,
               "plain_words_one_graph_one_stream_ms": 1e3 * tpw,
               "untuned_B16_L4_graph_8_streams_ms": 1e3 * tf,
               "tuned_graph_8_streams_ms": 1e3 * tb,
               "what": "plain calls issued from Python on one stream (level 1 as a list); the same calls "
                       "captured in one graph on one stream (removes host launch gaps); the same with level 1 "
                       "in word form (adds the word form); every batch at B=16, L=4 in one graph over 8 streams "
                       "(adds concurrency); the autotuned B, L, block in that graph (adds tuning)"},
           "timing": "CUDA events on the launching stream, median of reps",
           "tuned": {str(k): list(v) for k, v in sorted(tuner.table.items())},
           "prep_s": prep_s, "tune_s": tune_s}
    del bat, plain, plain_g, fixed
    torch.cuda.empty_cache()
    return out


def fp32_probe(dev, stream, reps: int = 5):
    """Measured FP32 FMA throughput (crsh_fma_probe: 8 independent FMA chains per thread,
    full occupancy), best of reps, CUDA events on the stream."""
    import torch
    from paper_2312_06538_gb300 import crsh as C
    props = torch.cuda.get_device_properties(dev)
    blocks = props.multi_processor_count * 8
    out = torch.empty(blocks, dtype=torch.float32, device=dev)
    sh = stream.cuda_stream
    C.crsh_fma_probe(out.data_ptr(), 1000, blocks, sh)       # warm-up
    best = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        flops = C.crsh_fma_probe(out.data_ptr(), 50000, blocks, sh)
        b.record(stream)
        torch.cuda.synchronize(dev)
        best = max(best, flops / (a.elapsed_time(b) * 1e-3) / 1e12)
    return best


def hbm_sweep(args, tiles_list=(1, 2, 4, 8, 16, 22), reps: int = 20):
    """Hash+sort (one crsh_hash_sort call: generation, hashing, trimming, compression, 4-pass
    radix sort, decompression + gather) and build (crsh_build) at 3M..70M rays: G-buffers of
    1..22 perturbed tiles of the 1024x1024 frame of config 3.  Algorithmic bytes per call:
    hash 40 B per pixel read + 41 B per ray written, sort 16 B per sorted chunk (one read and
    one write of key and value), decompress + gather 4 + 28 + 28 B per ray; build 28 B per ray
    read + 40 B per level-1 node written.  Median of reps, L2 flushed before each."""
    import synthetic
    import torch
    from paper_2312_06538_gb300 import pipeline as pl
    dev = torch.device("cuda", torch.cuda.current_device())
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    w = synthetic.make(3)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    lights = torch.from_numpy(w.lights).to(dev)
    for tiles in tiles_list:
        g = synthetic.tiled_gbuffer(w, tiles)
        npx = g["hit"].shape[0]
        p = pl.Pipeline(w.scene, max_pixels=npx, n_lights=w.lights.shape[0], bundle=w.bundle, levels=w.levels,
                        ray_capacity=npx * 4, pair_capacity=1 << 16, device=dev)
        hp, bp = pl.workload_params(w)
        gd = p.gbuffer_to_device(g, dev)
        gs = p.gbuffer_struct(gd)
        p.hash_sort(gs, lights, hp, sh)
        p.build(bp, sh)
        c = p.read_counters()
        n, chunks = c["rays"], c["chunks"]

        def med(fn):
            ts = []
            warm = 3 if reps >= 3 else 1
            for k in range(reps + warm):
                flush.fill_(k & 0xff)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize(dev)
                if k >= warm:
                    ts.append(a.elapsed_time(b))
            return statistics.median(ts)
        t_hash = med(lambda: p.hash_sort(gs, lights, hp, sh))
        t_build = med(lambda: p.build(bp, sh))
        # the algorithmic bytes of the method's steps: hash 40 B per pixel read (the G-buffer's
        # position, normal, incident direction and material) + 41 B per ray written; sort 16 B per
        # sorted element; decompression + gather 4 B (permutation) + 28 B read + 28 B written per ray
        b_hash = 40 * npx + 41 * n + 16 * chunks + (4 + 28 + 28) * n
        b_build = 28 * n + 40 * ((n + w.bundle - 1) // w.bundle)
        line = {"sweep": "hash_sort+build HBM", "pixels": npx, "rays": n, "chunks": chunks,
                "hash_sort_ms": t_hash, "hash_sort_gbs": b_hash / (t_hash * 1e-3) / 1e9,
                "hash_sort_frac": b_hash / (t_hash * 1e-3) / 1e9 / hbm,
                "build_ms": t_build, "build_gbs": b_build / (t_build * 1e-3) / 1e9,
                "build_frac": b_build / (t_build * 1e-3) / 1e9 / hbm,
                "peak_gbs": hbm, "peak_source": src,
                "mrays_per_s_hash_sort_build": n / ((t_hash + t_build) * 1e-3) / 1e6}
        print(json.dumps(line), flush=True)
        del p, gd, gs
        torch.cuda.empty_cache()


def f3_timing(w, p, gstruct, lights, hp, flush, stream, dev, reps: int = 20):
    """NEXT row f3 on the bench frame: primary visibility through the hierarchy (camera rays ->
    build -> traverse -> closest hit -> G-buffer), and the next bounce (first-hit buffer of the
    frame's secondary hits -> crsh_hash_sort)."""
    import torch
    from paper_2312_06538_gb300 import pipeline as pl
    sh = stream.cuda_stream
    npx = w.width * w.height
    q = pl.Pipeline(w.scene, max_pixels=npx, n_lights=1, bundle=16, levels=4, ray_capacity=npx, device=dev)
    _, bp = pl.workload_params(w)
    cam = q.camera_struct(w.camera, w.width, w.height)
    mat = torch.from_numpy(w.scene.tri_material.astype(np.int32)).to(dev)
    gq, gqs = q.gbuffer_out(npx)
    for _ in range(6):
        q.run_primary(cam, bp, sh)
        c = q.read_counters()
        if c["status"] == 2 and c["needed_pairs"] > q.pair_capacity:
            q.set_pair_capacity(int(1.25 * c["needed_pairs"]) + 1024)
            continue
        break

    def primary():
        q.run_primary(cam, bp, sh)
        q.gbuffer_from_hits(mat, gqs, sh)
    ms_p = time_path(primary, flush, stream, reps)
    tri = q.hit_tri[:npx].cpu().numpy().view(np.int32)
    agree = float((tri == w.primary_tri).mean())
    # next bounce from the frame's secondary hits (p holds them after the main timing)
    n = p.n()
    gn, gns = p.gbuffer_out(n)
    nb = pl.Pipeline(w.scene, max_pixels=n, n_lights=w.lights.shape[0], bundle=16, levels=4, device=dev,
                     pair_capacity=1 << 16)
    gstruct_n = nb.gbuffer_struct(gn)

    def bounce():
        p.gbuffer_from_hits(mat, gns, sh)
        nb.hash_sort(gstruct_n, lights, hp, sh)
    ms_b = time_path(bounce, flush, stream, reps)
    n_next = nb.n()
    ms_s = time_path(lambda: p.shade(gstruct, lights, mat, sh), flush, stream, reps)
    out = {"primary": {"workload": f"{w.width}x{w.height} camera rays, B=16, L=4, through the hierarchy",
                       "mrays_per_s": npx / (ms_p * 1e-3) / 1e6, "ms": ms_p,
                       "tri_tests_per_ray": c["final_tests"] / npx,
                       "same_triangle_as_fp64_raster": agree},
           "next_bounce": {"rays_in": n, "rays_out": n_next, "ms": ms_b,
                           "mrays_per_s": n_next / (ms_b * 1e-3) / 1e6,
                           "what": "first-hit buffer of the secondary hits + hash/sort of the next bounce's rays"},
           "shade": {"pixels": npx, "rays": n, "ms": ms_s,
                     "what": "crsh_shade: Lambert + hard shadows + one mirror/glass bounce from the frame's hits"}}
    del q, nb
    torch.cuda.empty_cache()
    return out


# Table 4 of the paper (GTX TITAN, their scenes), quoted as context: total intersections
TABLE4 = {"OFFICE": {"brute_force": 9133132168, "rah": 469683524, "crsh": 170070948},
          "CORNELL": {"brute_force": 606911976, "rah": 72869648, "crsh": 53578192},
          "SPONZA": {"brute_force": 17058578850, "rah": 632408864, "crsh": 405619896}}


def paper_total(c: dict) -> int:
    """Total intersections in the paper's convention: every level's B x parent-hit tests plus the
    final B x level-1-hit tests (the identity that reproduces Table 4 from Tables 1-3)."""
    return int(sum(c["tests_paper"]) + c["final_tests_paper"])


def study(args):
    """Row f4: the paper's evaluation shape (Section 4) on OFFICE-, CORNELL- and SPONZA-shaped
    synthetic scenes at 512x512, hierarchy depth 2, B = 8: total intersections of CRSH (sorted,
    whole-mesh culling), RAH (unsorted, no mesh culling) and the brute force, one JSON line per
    scene."""
    import synthetic
    import torch
    from paper_2312_06538_gb300 import pipeline as pl
    dev = torch.device("cuda", torch.cuda.current_device())
    for name, make in synthetic.STUDY.items():
        w = make()
        row = {"study": name, "scene": w.name, "triangles": w.scene.n_tris}
        for mode, sort, cull in (("crsh", True, True), ("rah", False, False)):
            p = pl.workload_pipeline(w, device=dev)
            hp, bp = pl.workload_params(w, sort=sort)
            g = p.gbuffer_struct(p.gbuffer_to_device(w.gbuffer, dev))
            lights = torch.from_numpy(w.lights).to(dev)
            c = p.run_fit(g, lights, hp, bp, mesh_cull=cull)
            tri = p.hits_host()[0]
            types = np.bincount(p.sorted_rays()["type"], minlength=3)
            row[mode] = {"total_isect": paper_total(c), "level_tests_paper": list(map(int, c["tests_paper"])),
                         "level_hits": list(map(int, c["hits"])), "final_tests_paper": int(c["final_tests_paper"]),
                         "final_hits": int(c["final_hits"]), "hit_rays": int((tri >= 0).sum())}
            row["rays"] = int(c["rays"])
            row["rays_by_type"] = {"shadow": int(types[0]), "reflection": int(types[1]), "refraction": int(types[2])}
            del p
            torch.cuda.empty_cache()
        bf = row["rays"] * w.scene.n_tris
        row["brute_force"] = {"total_isect": bf}
        row["relative"] = {"crsh": row["crsh"]["total_isect"] / bf, "rah": row["rah"]["total_isect"] / bf,
                           "crsh_vs_rah": row["crsh"]["total_isect"] / row["rah"]["total_isect"]}
        t = TABLE4[name]
        row["paper_table4_context"] = {"crsh_relative": t["crsh"] / t["brute_force"],
                                       "rah_relative": t["rah"] / t["brute_force"],
                                       "crsh_vs_rah": t["crsh"] / t["rah"]}
        print(json.dumps(row), flush=True)


def run_gpu(args, w):
    import ctypes

    import torch
    import torch.distributed as dist

    from paper_2312_06538_gb300 import crsh as C
    from paper_2312_06538_gb300 import frames as fr
    from paper_2312_06538_gb300 import pipeline as pl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)

    p = pl.workload_pipeline(w, device=dev, level1_words=args.level1 == "words")
    hp, bp = pl.workload_params(w)
    g_host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
              pl.Pipeline.gbuffer_to_device(w.gbuffer, "cpu").items()}
    g_dev = {k: v.to(dev) for k, v in g_host.items()}
    lights = torch.from_numpy(w.lights).to(dev)
    gstruct = p.gbuffer_struct(g_dev)
    c = p.run_fit(gstruct, lights, hp, bp)          # sizes the pair lists, checks the status
    n_rays = c["rays"]
    if args.profile_steps:
        # for profilers: the path's calls issued directly, nothing timed; prints the counters
        for _ in range(args.profile_steps):
            p.run(gstruct, lights, hp, bp)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_steps": args.profile_steps, "workload": workload_description(w),
                          "pixels": w.n_pixels, "counters": {k: v for k, v in c.items()}}), flush=True)
        return
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    def step(ev):
        ev[0].record(stream)
        p.hash_sort(gstruct, lights, hp, sh)
        ev[1].record(stream)
        p.build(bp, sh)
        ev[2].record(stream)
        p.traverse(True, sh)
        ev[3].record(stream)
        p.closest_hit(sh)
        ev[4].record(stream)

    warm = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for _ in range(args.warmup):
        flush.fill_(1)
        step(warm)
    torch.cuda.synchronize(dev)
    # The timed steps replay one CUDA graph of the four calls (the API is capture-safe: sizes stay
    # on the device), which removes the host launch gaps between the path's kernels.
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(dev)
    with torch.cuda.graph(graph, stream=cap):
        p.hash_sort(gstruct, lights, hp, cap.cuda_stream)
        p.build(bp, cap.cuda_stream)
        p.traverse(True, cap.cuda_stream)
        p.closest_hit(cap.cuda_stream)
    for _ in range(args.warmup):
        flush.fill_(1)
        graph.replay()
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    with ClockSampler(props.index if hasattr(props, "index") else local) as clk:
        torch.cuda.synchronize(dev)
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xff)       # L2 (129 MB) flushed between timed steps, outside the events
            evs[k][0].record(stream)
            graph.replay()
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall0
        if world > 1:
            dist.barrier()
    step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    local_ms = float(step_ms.sum())
    # per-stage breakdown: the same calls issued directly, events between them
    n_stage = min(args.steps, 100)
    sevs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(n_stage)]
    for k in range(n_stage):
        flush.fill_(k & 0xff)
        step(sevs[k])
    torch.cuda.synchronize(dev)
    stage = np.array([[sevs[k][i].elapsed_time(sevs[k][i + 1]) for i in range(4)] for k in range(n_stage)])
    # the final-test kernel alone: CUDA events recorded on its launching stream around its launch
    # (crsh_closest_hit_timed), each time after the same hash, build and traversal as a step
    n_kern = min(args.steps, 50)
    kern = []
    for k in range(n_kern):
        flush.fill_(k & 0xff)
        p.hash_sort(gstruct, lights, hp, sh)
        p.build(bp, sh)
        p.traverse(True, sh)
        kern.append(p.closest_hit_timed(sh))
    kern_ms = float(np.mean(kern))
    c_after = p.read_counters()
    assert c_after["status"] == 0 and c_after["rays"] == n_rays
    tot_ms, tot_units = reduce_over_ranks(local_ms, float(n_rays) * args.steps, world)
    value = tot_units / (tot_ms * 1e-3) / 1e6

    # end to end through the API with host buffers: every frame's G-buffer and lights go up from one
    # pinned staging buffer and its hits come back to pinned host memory, two frames in flight
    # (frames.FrameStream: one frame's copies overlap the other's kernels).  The wall clock spans
    # the first upload to the last read-back; the L2 flush runs before each frame, inside it.
    fields = dict(g_host)
    fields["lights"] = torch.from_numpy(np.ascontiguousarray(w.lights, np.float32))
    layout = fr.HostLayout(fields)
    stage_host = layout.pack(fields, layout.host_buffer())
    fs = fr.FrameStream(p, layout, hp, bp, stream=stream, before_frame=lambda: flush.fill_(3))
    h2d = layout.nbytes
    for k in range(args.warmup):
        fs.push(stage_host)
    last = fs.drain()
    assert last.n == n_rays
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(args.steps):
        fs.push(stage_host)
    last = fs.drain()
    torch.cuda.synchronize(dev)
    e2e_local_ms = 1e3 * (time.perf_counter() - t0)
    assert last.n == n_rays and torch.equal(last.tri, p.hit_tri[:n_rays].cpu())
    d2h = ctypes.sizeof(C.crsh_counters) + 16 * n_rays
    e2e_ms, e2e_units = reduce_over_ranks(e2e_local_ms, float(n_rays) * args.steps, world)
    e2e_value = e2e_units / (e2e_ms * 1e-3) / 1e6

    # roofline of the dominant kernel (final tests): achieved FP32 flops per launch / event time
    peaks, peak_src = _peaks()
    clocks = clk.summary()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_derived = fp32_peak_tflops(props.multi_processor_count, sm_max)
    peak_tf = fp32_probe(dev, stream)
    ch_ms = float(stage[:, 3].mean())
    achieved = c["final_tests"] * MT_FLOPS / (kern_ms * 1e-3) / 1e12
    tr_ms = float(stage[:, 2].mean())
    eq9_tests = sum(c["tests"]) + c["mesh_tests"]
    traffic = closest_traffic("k_closest_words" if p.level1_words else "k_closest", args.config, args.res)
    words = bool(p.level1_words)
    roofline = {"kernel": ("k_closest_words (crsh_closest_hit's final-test kernel: level-1 ballots gathered "
                           "into groups, then tested)") if words else "k_closest (crsh_closest_hit's final-test kernel)",
                "bound": "alu",
                "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved / peak_tf,
                "traffic": traffic,
                "kernel_ms": kern_ms,
                "timing": f"CUDA events recorded on the launching stream around the kernel's launch "
                          f"(crsh_closest_hit_timed), mean of {n_kern} steps, L2 flushed before each",
                "call_ms": ch_ms,
                "achieved_call": c["final_tests"] * MT_FLOPS / (ch_ms * 1e-3) / 1e12,
                "peak_source": "measured: crsh_fma_probe (FP32 FMA chains at full occupancy, best of 5, burst)",
                "peak_derived": peak_derived,
                "peak_derived_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                       f"(max SM clock, {peak_src} peaks file)",
                "algorithmic": f"{MT_FLOPS} FP32 flops (one Moller-Trumbore test) per candidate ray-triangle test x "
                               f"{c['final_tests']} candidate tests per launch"}
    # the traversal stage (its count, scan and emit kernels; k_count is its top kernel) against the
    # same FP32 peak: eq. 9 work of the tests the paper's count makes, per call
    roofline_traverse = {"kernel": ("crsh_traverse (k_count + k_emit + scans above level 1; level 1: count pass "
                                    "and item descriptors)") if words else
                                   "crsh_traverse (k_count + k_emit + scans, all levels)", "bound": "alu",
                         "achieved": eq9_tests * EQ9_FLOPS / (tr_ms * 1e-3) / 1e12, "peak": peak_tf,
                         "unit": "TFLOP/s", "frac": eq9_tests * EQ9_FLOPS / (tr_ms * 1e-3) / 1e12 / peak_tf,
                         "traffic": None,
                         "algorithmic": f"{EQ9_FLOPS} FP32 flops per eq. 9 test x {eq9_tests} tests per call "
                                        f"(every child x parent triangle, mesh tests included)"}
    total_tests = c["final_tests"] + eq9_tests
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scene, software-rasterised G-buffer)",
        "config": {"workload": workload_description(w), "pixels": w.n_pixels, "triangles": w.scene.n_tris,
                   "rays_per_step": n_rays, "bundle": w.bundle, "levels": w.levels,
                   "level1": "words" if p.level1_words else "list",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed between timed steps (512 MiB write outside the step events)"},
        "level_counts": {"levels": "index l-1 = level l (Tables 1-3 schema)", "tests": list(map(int, c["tests"])),
                         "hits": list(map(int, c["hits"])), "tests_paper": list(map(int, c["tests_paper"])),
                         "mesh_tests": int(c["mesh_tests"]), "mesh_hits": int(c["mesh_hits"]),
                         "final_tests": int(c["final_tests"]), "final_hits": int(c["final_hits"]),
                         "chunks": int(c["chunks"])},
        "tri_tests_per_ray": c["final_tests"] / max(1, n_rays),
        "all_tests_per_ray": total_tests / max(1, n_rays),
        "bruteforce_tests_per_ray": w.scene.n_tris,
        "stage_ms": {"hash_sort": float(stage[:, 0].mean()), "build": float(stage[:, 1].mean()),
                     "traverse": tr_ms, "closest_hit": ch_ms,
                     "note": "the four calls issued directly with events between them; the timed steps "
                             "replay them as one CUDA graph"},
        "traverse_eq9_tflops": eq9_tests * EQ9_FLOPS / (tr_ms * 1e-3) / 1e12,
        "wall_ms_timed_region": 1e3 * t_wall,
        "roofline": roofline,
        "roofline_traverse": roofline_traverse,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step(w.levels, True, bool(p.level1_words)) * args.steps,
        "clocks": clocks,
    }
    if not args.no_comparators:
        try:
            line["comparators"] = comparators(w, p, gstruct, lights, hp, bp, flush, stream, dev, n_rays)
        except Exception as e:  # a comparator must not cost the main line
            line["comparators"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_f3:
        try:
            line.update(f3_timing(w, p, gstruct, lights, hp, flush, stream, dev))
        except Exception as e:
            line["primary"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_batched:
        try:
            line["batched"] = batched_comparison(dev)
        except Exception as e:
            line["batched"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_adjoint:
        try:
            line["adjoint"] = adjoint_timing(dev, flush, stream)
        except Exception as e:
            line["adjoint"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_cpu_baseline:
        sr = p.sorted_rays()
        gen_pixel = np.empty(n_rays, np.int64)
        gen_pixel[sr["ray_id"].astype(np.int64)] = sr["pixel"]
        line["cpu_baseline"] = cpu_baseline(w, args.config, args.res, budget_s=args.cpu_budget,
                                            gpu_hits=p.hits_host(), gpu_gen_pixel=gen_pixel)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--res", type=int, default=None)
    ap.add_argument("--level1", default="words", choices=["words", "list"],
                    help="level 1 of the traversal in word form (read by the final tests from the ballots) "
                         "or as a written (node, triangle) list")
    ap.add_argument("--ref-crop", type=int, default=64)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run the path this many times after sizing it, time nothing, print nothing (for ncu)")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-f3", action="store_true", help="skip primary visibility / next bounce timing")
    ap.add_argument("--sweep", action="store_true",
                    help="hash/sort/build HBM sweep at 3M..70M rays (one JSON line per size) instead of the step")
    ap.add_argument("--sweep-tiles", type=int, nargs="*", default=None, help="sweep sizes in frame tiles")
    ap.add_argument("--sweep-reps", type=int, default=20)
    ap.add_argument("--study", action="store_true",
                    help="the paper-shaped depth-2, B=8 study (CRSH vs RAH vs brute force) instead of the step")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)   # at least 3 untimed warm-up steps
    if args.study:
        study(args)
        return
    if args.sweep:
        if args.sweep_tiles:
            hbm_sweep(args, tiles_list=tuple(args.sweep_tiles), reps=args.sweep_reps)
        else:
            hbm_sweep(args, reps=args.sweep_reps)
        return
    import synthetic
    w = synthetic.make(args.config, res=args.res)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
