"""Triangle-mesh generators for the synthetic scenes (vertices + index triples)."""
from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=8)
def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4**subdiv outward-facing triangles."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts, np.float64)
    F = np.array(faces, np.int64)
    V.setflags(write=False)
    F.setflags(write=False)
    return V, F


def torus(nu: int, nv: int, R: float, r: float):
    """Torus about the y axis: 2 * nu * nv triangles."""
    u = np.arange(nu) * (2 * np.pi / nu)
    v = np.arange(nv) * (2 * np.pi / nv)
    uu, vv = np.meshgrid(u, v, indexing="ij")
    x = (R + r * np.cos(vv)) * np.cos(uu)
    z = (R + r * np.cos(vv)) * np.sin(uu)
    y = r * np.sin(vv)
    V = np.stack([x, y, z], -1).reshape(-1, 3)
    F = []
    for i in range(nu):
        for j in range(nv):
            a = i * nv + j
            b = ((i + 1) % nu) * nv + j
            c = ((i + 1) % nu) * nv + (j + 1) % nv
            d = i * nv + (j + 1) % nv
            F += [(a, b, c), (a, c, d)]
    return V, np.array(F, np.int64)


def plane(y: float, half: float):
    """Two triangles spanning x, z in [-half, half] at height y."""
    V = np.array([(-half, y, -half), (half, y, -half), (half, y, half), (-half, y, half)], np.float64)
    F = np.array([(0, 2, 1), (0, 3, 2)], np.int64)
    return V, F


def room_box(half: float):
    """Axis-aligned box [-half, half]^3, two triangles per wall (12 in all)."""
    h = half
    V = np.array([(x, y, z) for x in (-h, h) for y in (-h, h) for z in (-h, h)], np.float64)
    idx = lambda x, y, z: x * 4 + y * 2 + z  # noqa: E731
    quads = [
        (idx(0, 0, 0), idx(0, 0, 1), idx(0, 1, 1), idx(0, 1, 0)),  # x = -h
        (idx(1, 0, 0), idx(1, 1, 0), idx(1, 1, 1), idx(1, 0, 1)),  # x = +h
        (idx(0, 0, 0), idx(1, 0, 0), idx(1, 0, 1), idx(0, 0, 1)),  # y = -h
        (idx(0, 1, 0), idx(0, 1, 1), idx(1, 1, 1), idx(1, 1, 0)),  # y = +h
        (idx(0, 0, 0), idx(0, 1, 0), idx(1, 1, 0), idx(1, 0, 0)),  # z = -h
        (idx(0, 0, 1), idx(1, 0, 1), idx(1, 1, 1), idx(0, 1, 1)),  # z = +h
    ]
    F = []
    for a, b, c, d in quads:
        F += [(a, b, c), (a, c, d)]
    return V, np.array(F, np.int64)


def random_rotation(rng) -> np.ndarray:
    """Uniform random rotation matrix from a unit quaternion (Shoemake)."""
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    q = np.array([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2), np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3), np.sqrt(u1) * np.cos(2 * np.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def displace(V: np.ndarray, rng, amp: float = 0.15, terms: int = 3) -> np.ndarray:
    """Radial noise: scale each vertex of a unit sphere by 1 + amp * mean_k sin(f_k . v + p_k)."""
    s = np.zeros(V.shape[0])
    for _ in range(terms):
        f = np.array([rng.uniform(-4, 4), rng.uniform(-4, 4), rng.uniform(-4, 4)])
        p = rng.uniform(0, 2 * np.pi)
        s += np.sin(V @ f + p)
    return V * (1.0 + amp * s / terms)[:, None]
