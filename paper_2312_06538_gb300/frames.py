"""Frames from pinned host memory through the whole path and back, two frames in
flight.

A frame's inputs (the G-buffer fields and the lights) travel as one pinned
staging buffer, each field at a 256-byte aligned offset.  Its upload and the
read-back of the previous frame's hits run on a copy stream while the path's
kernels of the other frame run on the compute stream, so a stream of frames
pays for its copies only where they exceed the path's own time.  The order is
kept with CUDA events per slot:

    upload(k)     waits for the path of frame k-2 (it read the same device slot)
    path(k)       waits for upload(k) and for the read-back of frame k-2 (same hit slot)
    read-back(k)  waits for path(k); the host waits for it before handing the hits out

Every step of the path still runs in libcrsh.so; this module orders copies and
C-ABI calls only."""
from __future__ import annotations

import ctypes
from typing import Callable, Dict, Optional, Tuple

import torch

from . import crsh as C
from .pipeline import Pipeline, _ptr, counters_from_bytes

ALIGN = 256


class HostLayout:
    """Offsets of named fields in one staging buffer, each field 256-byte aligned."""

    def __init__(self, fields: Dict[str, torch.Tensor]):
        self.spans: Dict[str, Tuple[int, int, torch.dtype, Tuple[int, ...]]] = {}
        off = 0
        for k, v in fields.items():
            nb = int(v.numel() * v.element_size())
            self.spans[k] = (off, nb, v.dtype, tuple(v.shape))
            off = (off + nb + ALIGN - 1) & ~(ALIGN - 1)
        self.nbytes = off

    def host_buffer(self) -> torch.Tensor:
        return torch.empty(self.nbytes, dtype=torch.uint8).pin_memory()

    def pack(self, fields: Dict[str, torch.Tensor], out: torch.Tensor) -> torch.Tensor:
        """Copy host tensors of the layout's shapes and types into `out` (a host_buffer())."""
        for k, (o, nb, dt, shape) in self.spans.items():
            v = fields[k]
            if v.dtype != dt or tuple(v.shape) != shape:
                raise ValueError(f"field {k}: {v.dtype} {tuple(v.shape)}, layout has {dt} {shape}")
            out[o:o + nb].copy_(v.contiguous().reshape(-1).view(torch.uint8))
        return out

    def views(self, buf: torch.Tensor) -> Dict[str, torch.Tensor]:
        return {k: buf[o:o + nb].view(dt).view(shape) for k, (o, nb, dt, shape) in self.spans.items()}


class Frame:
    """Hits of one frame in pinned host memory, in the path's ray order; valid until the
    stream reuses the slot (two pushes later)."""

    def __init__(self, n: int, counters: dict, tri, t, u, v):
        self.n, self.counters = n, counters
        self.tri, self.t, self.u, self.v = tri, t, u, v


class FrameStream:
    """Double-buffered executor of the path over frames of one scene.

    `layout` holds the G-buffer fields of Pipeline.gbuffer_to_device() and "lights" (an
    (n_lights, 3) float tensor).  push() uploads a packed frame, issues the path and returns
    the previous frame's hits (None for the first); drain() returns the last one.  The
    pipeline's pair lists must already be sized (Pipeline.run_fit on a like frame): a frame
    whose status is not CRSH_OK raises CrshError when its hits are read back."""

    def __init__(self, p: Pipeline, layout: HostLayout, hp: C.crsh_hash_params, bp: C.crsh_build_params,
                 *, mesh_cull: bool = True, stream: Optional[torch.cuda.Stream] = None,
                 before_frame: Optional[Callable[[], None]] = None):
        dev = p.device
        self.p, self.layout, self.hp, self.bp, self.mesh_cull = p, layout, hp, bp, mesh_cull
        self.compute = stream if stream is not None else torch.cuda.current_stream(dev)
        self.copy = torch.cuda.Stream(dev)
        self.before_frame = before_frame
        cap = p.ray_capacity
        n_ctr = ctypes.sizeof(C.crsh_counters)
        self.slots = []
        for _ in range(2):
            stage = torch.empty(layout.nbytes, dtype=torch.uint8, device=dev)
            g = layout.views(stage)
            lights = g.pop("lights")
            hits_dev = [torch.empty(cap, dtype=dt, device=dev)
                        for dt in (torch.int32, torch.float32, torch.float32, torch.float32)]
            self.slots.append({
                "stage": stage, "gbuf": Pipeline.gbuffer_struct(g), "lights": lights,
                "hits_dev": hits_dev, "hits": C.crsh_hits(*[_ptr(x) for x in hits_dev]),
                "hits_host": [torch.empty(cap, dtype=x.dtype).pin_memory() for x in hits_dev],
                "ctr_host": torch.empty(n_ctr, dtype=torch.uint8).pin_memory(),
                "uploaded": torch.cuda.Event(), "computed": torch.cuda.Event(), "read": torch.cuda.Event(),
                "busy_compute": False, "busy_read": False,
            })
        self.k = 0
        self.pending: Optional[int] = None

    def push(self, host: torch.Tensor) -> Optional[Frame]:
        """Upload `host` (a pinned buffer of the layout), issue the path on it, and return the
        hits of the frame pushed before (None if there is none)."""
        if host.numel() != self.layout.nbytes or host.dtype != torch.uint8:
            raise ValueError("host buffer does not match the layout")
        s = self.k & 1
        sl = self.slots[s]
        if sl["busy_compute"]:
            self.copy.wait_event(sl["computed"])
        with torch.cuda.stream(self.copy):
            sl["stage"].copy_(host, non_blocking=True)
        sl["uploaded"].record(self.copy)
        self.compute.wait_event(sl["uploaded"])
        if sl["busy_read"]:
            self.compute.wait_event(sl["read"])
        with torch.cuda.stream(self.compute):
            if self.before_frame is not None:
                self.before_frame()
            self.p.run(sl["gbuf"], sl["lights"], self.hp, self.bp, self.mesh_cull,
                       stream=self.compute.cuda_stream, hits=sl["hits"])
            sl["ctr_host"].copy_(self.p.counters, non_blocking=True)
        sl["computed"].record(self.compute)
        sl["busy_compute"] = True
        prev, self.pending = self.pending, s
        self.k += 1
        return None if prev is None else self._read_back(prev)

    def drain(self) -> Optional[Frame]:
        """Hits of the last pushed frame (None if all were returned)."""
        prev, self.pending = self.pending, None
        return None if prev is None else self._read_back(prev)

    def _read_back(self, s: int) -> Frame:
        sl = self.slots[s]
        sl["computed"].synchronize()
        ctr = counters_from_bytes(sl["ctr_host"].numpy().tobytes(), self.p.levels)
        if ctr["status"] != C.OK:
            raise C.CrshError("frame status", ctr["status"])
        n = int(ctr["rays"])
        self.copy.wait_event(sl["computed"])
        with torch.cuda.stream(self.copy):
            for h, d in zip(sl["hits_host"], sl["hits_dev"]):
                h[:n].copy_(d[:n], non_blocking=True)
        sl["read"].record(self.copy)
        sl["busy_read"] = True
        sl["read"].synchronize()
        tri, t, u, v = (h[:n] for h in sl["hits_host"])
        return Frame(n, ctr, tri, t, u, v)
