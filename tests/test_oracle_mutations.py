"""Pins of the oracle's triangle bounding sphere (Section 3.3.7 reading: centroid
centre, largest vertex distance) on worked triangles whose spheres are known in
closed form, and mutation tests: the oracle is recompiled on the CPU with a
planted mistake in that function, and the pins must catch it (a sphere that is
too large would change pair counts without breaking hierarchy == brute force,
so the pins must fix it from above as well as from below).  CPU only."""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "crsh_oracle.c")

# (vertices, centre, radius): closed forms
S3 = math.sqrt(3.0)
WORKED = [
    # equilateral triangle of side 2 in the plane z = 1: centroid, radius = side / sqrt(3)
    ([[0, 0, 1], [2, 0, 1], [1, S3, 1]], [1, S3 / 3, 1], 2 / S3),
    # right isosceles triangle with legs 3: centroid (1, 1, 0); farthest corners at sqrt(5)
    ([[0, 0, 0], [3, 0, 0], [0, 3, 0]], [1, 1, 0], math.sqrt(5.0)),
    # collinear corners: centroid is the middle one, radius half the length
    ([[0, 0, 0], [1, 0, 0], [2, 0, 0]], [1, 0, 0], 1.0),
    # a scalene triangle: centroid (2, 1, 0); distances sqrt(5), sqrt(5), 2 -> sqrt(5)
    ([[0, 0, 0], [4, 0, 0], [2, 3, 0]], [2, 1, 0], math.sqrt(5.0)),
    # a point triangle: radius 0
    ([[0.5, -1.5, 2], [0.5, -1.5, 2], [0.5, -1.5, 2]], [0.5, -1.5, 2], 0.0),
    # off-axis: the same right isosceles triangle moved and turned into the plane x = 4
    ([[4, 0, 0], [4, 3, 0], [4, 0, 3]], [4, 1, 1], math.sqrt(5.0)),
]


def _tri_sphere_errors(tri_spheres):
    """Pin violations of a tri_spheres implementation (verts (T,3,3) -> (T,4))."""
    verts = np.array([w[0] for w in WORKED], np.float32)
    got = tri_spheres(verts)
    bad = []
    for k, (v, c, r) in enumerate(WORKED):
        if not np.allclose(got[k, :3], c, rtol=0, atol=1e-6):
            bad.append((k, "centre", got[k, :3].tolist(), c))
        if abs(got[k, 3] - r) > 1e-6 * max(1.0, r):
            bad.append((k, "radius", float(got[k, 3]), r))
    # random triangles: the sphere holds every corner and one corner lies on it
    rng = np.random.default_rng(7)
    vr = rng.uniform(-3, 3, size=(200, 3, 3)).astype(np.float32)
    s = tri_spheres(vr)
    dist = np.linalg.norm(vr.astype(np.float64) - s[:, None, :3], axis=2)
    if not np.all(dist <= s[:, 3:4] * (1 + 1e-12) + 1e-12):
        bad.append(("random", "corner outside"))
    if not np.allclose(dist.max(axis=1), s[:, 3], rtol=1e-12, atol=1e-12):
        bad.append(("random", "no corner on the sphere"))
    if not np.allclose(s[:, :3], vr.astype(np.float64).mean(axis=1), rtol=0, atol=1e-6):
        bad.append(("random", "centre is not the centroid"))
    return bad


def test_tri_sphere_worked_triangles():
    assert _tri_sphere_errors(oracle.tri_spheres) == []


def _compile_mutant(tmp_path, old: str, new: str):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", str(path), "-o",
                           str(lib), "-lm"])
    L = ctypes.CDLL(str(lib))
    L.oracle_tri_spheres.restype = None
    L.oracle_tri_spheres.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]

    def tri_spheres(verts):
        v = np.ascontiguousarray(verts, np.float32)
        out = np.empty((v.shape[0], 4), np.float64)
        L.oracle_tri_spheres(v.shape[0], v.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p))
        return out
    return tri_spheres


RADIUS_LINE = "double r = fmax(dlen(dsub(a, m)), fmax(dlen(dsub(b, m)), dlen(dsub(c, m))));"
CENTRE_LINE = "d3 m = dscl(dadd(dadd(a, b), c), 1.0 / 3.0);"
MUTANTS = {
    # oversized: the radius doubled
    "radius_doubled": (RADIUS_LINE, RADIUS_LINE.replace("double r = ", "double r = 2.0 * ")),
    # oversized: the radius of the bounding box around the centroid (half the box diagonal)
    "radius_from_box": (RADIUS_LINE,
                        "double r = 0.5 * dlen(D3(fmax(a.x, fmax(b.x, c.x)) - fmin(a.x, fmin(b.x, c.x)), "
                        "fmax(a.y, fmax(b.y, c.y)) - fmin(a.y, fmin(b.y, c.y)), "
                        "fmax(a.z, fmax(b.z, c.z)) - fmin(a.z, fmin(b.z, c.z))));"),
    # slightly oversized: a 1 % margin
    "radius_one_percent": (RADIUS_LINE, RADIUS_LINE.replace("double r = ", "double r = 1.01 * ")),
    # undersized: the nearest corner instead of the farthest
    "radius_min": (RADIUS_LINE, RADIUS_LINE.replace("fmax", "fmin")),
    # wrong centre: the first corner
    "centre_v0": (CENTRE_LINE, "d3 m = a;"),
    # wrong centre: an index slip (b counted twice)
    "centre_index": (CENTRE_LINE, "d3 m = dscl(dadd(dadd(a, b), b), 1.0 / 3.0);"),
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_tri_sphere_mutants_fail_the_pins(tmp_path, name):
    old, new = MUTANTS[name]
    mutant = _compile_mutant(tmp_path, old, new)
    assert _tri_sphere_errors(mutant), f"mutant {name} passed the triangle-sphere pins"
