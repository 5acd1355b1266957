"""Builds and loads synthetic/native.c (primary visibility and minimum balls)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "native.c")
_LIB = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile native.c with gcc (no FMA contraction) if it is missing or stale."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(os.path.dirname(_LIB), exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                                   _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.synth_raster_gbuffer.restype = ctypes.c_int
        _lib.synth_raster_gbuffer.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P] + [P] * 12
        _lib.synth_min_ball.restype = ctypes.c_int
        _lib.synth_min_ball.argtypes = [ctypes.c_int, P, ctypes.c_uint64, P, P]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def raster_gbuffer(w: int, h: int, cam: np.ndarray, verts: np.ndarray, tri_material: np.ndarray):
    """verts: (n_tri, 3, 3) float32; returns the G-buffer dict and per-pixel triangle id."""
    n_tri = verts.shape[0]
    verts = np.ascontiguousarray(verts, dtype=np.float32)
    tri_material = np.ascontiguousarray(tri_material, dtype=np.int32)
    cam = np.ascontiguousarray(cam, dtype=np.float64)
    npx = w * h
    f = {k: np.empty(npx, np.float32) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz")}
    material = np.empty(npx, np.uint32)
    hit = np.empty(npx, np.uint8)
    tri = np.empty(npx, np.int32)
    n = lib().synth_raster_gbuffer(w, h, _p(cam), n_tri, _p(verts), _p(tri_material),
                                   *[_p(f[k]) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz")],
                                   _p(material), _p(hit), _p(tri))
    if n < 0:
        raise MemoryError("synth_raster_gbuffer: allocation failed")
    g = dict(f)
    g["material"] = material
    g["hit"] = hit
    return g, tri


def min_ball(points: np.ndarray, seed: int):
    """Smallest enclosing ball of (n, 3) float32 points: (centre float64[3], radius)."""
    pts = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    c = np.zeros(3, np.float64)
    r = np.zeros(1, np.float64)
    if lib().synth_min_ball(pts.shape[0], _p(pts), seed & ((1 << 64) - 1), _p(c), _p(r)) != 0:
        raise ValueError("synth_min_ball failed")
    return c, float(r[0])
