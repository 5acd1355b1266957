"""The GPU-vs-oracle comparison rules themselves (tests/parity.py), on the CPU:
a correct result passes, and planted mistakes are reported, not excused."""
import numpy as np
import pytest

import oracle
from tests import parity


def _c1(wl1):
    r = oracle.run_crsh(wl1.gbuffer, wl1.lights, wl1.shadow_cull, wl1.hash_lo, wl1.hash_hi, wl1.scene, wl1.bundle,
                        wl1.levels, wl1.build_pads())
    tri, t, u, v = r["hits"]
    return r, (tri.copy(), t.astype(np.float32), u.astype(np.float32), v.astype(np.float32))


def test_oracle_against_itself_passes(wl1):
    r, gpu = _c1(wl1)
    rep = parity.compare_hits(gpu, r["hits"], r["rays"], wl1.scene.verts)
    parity.check_report(rep)
    assert rep["ties"] == rep["edges"] == 0 and rep["hits"] > 50


def test_planted_wrong_triangle_is_unexplained(wl1):
    r, gpu = _c1(wl1)
    tri = gpu[0]
    hit = np.nonzero(tri >= 0)[0]
    i = hit[len(hit) // 2]
    tri[i] = (tri[i] + 1) % wl1.scene.n_tris        # a neighbour id the ray does not hit there
    miss = np.nonzero(r["hits"][0] < 0)[0]
    tri[miss[0]] = 5                                 # a hit where there is none
    rep = parity.compare_hits(gpu, r["hits"], r["rays"], wl1.scene.verts)
    bad = {u[0] for u in rep["unexplained"]}
    assert i in bad and miss[0] in bad


def test_planted_distance_error_is_caught(wl1):
    r, gpu = _c1(wl1)
    hit = np.nonzero(gpu[0] >= 0)[0]
    gpu[1][hit[0]] *= 1.0 + 3e-5
    gpu[2][hit[1]] += 3e-5
    rep = parity.compare_hits(gpu, r["hits"], r["rays"], wl1.scene.verts)
    assert rep["t_viol"] == 1 and rep["uv_viol"] == 1


# --------------------------------------------------------------------------
# The FP32 error band of the edge rule: sound, capped, and not a free pass
# --------------------------------------------------------------------------

def _rays(o, d, tmax=np.inf):
    o = np.asarray(o, np.float32).reshape(-1, 3)
    d = np.asarray(d, np.float32).reshape(-1, 3)
    n = o.shape[0]
    return {"ox": o[:, 0].copy(), "oy": o[:, 1].copy(), "oz": o[:, 2].copy(), "dx": d[:, 0].copy(),
            "dy": d[:, 1].copy(), "dz": d[:, 2].copy(), "tmax": np.full(n, tmax, np.float32)}


def _grazing_case():
    """A ray meeting the plane z = 0 at (0.2, 0.3) at grazing incidence (cos = 1e-4),
    5 units from its origin.  Triangle 0 contains that point; triangle 1 (same plane)
    misses it by 0.5 in barycentric units."""
    d = np.array([1.0, 0.0, -1e-4])
    d /= np.linalg.norm(d)
    o = np.array([0.2, 0.3, 0.0]) - 5.0 * d
    verts = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0]],
                      [[0.7, 0, 0], [1.7, 0, 0], [0.7, 1, 0]]], np.float32)
    return _rays(o, d), verts


def test_planted_wrong_triangle_at_grazing_incidence_is_unexplained():
    rays, verts = _grazing_case()
    ref = oracle.bruteforce(rays, verts)
    assert ref[0][0] == 0
    gpu = (np.array([1], np.int32), np.float32(ref[1]).reshape(1), np.zeros(1, np.float32), np.zeros(1, np.float32))
    rep = parity.compare_hits(gpu, ref, rays, verts)
    assert rep["unexplained"] == [(0, 1, 0)] and rep["edges"] == 0
    # the FP32 band of triangle 1 at this incidence, in barycentric units, is far below
    # its 0.5 miss (a band of 1e-4 / cos(incidence) would have reached 1.0 here)
    q = parity.fp32_decision((rays["ox"][0], rays["oy"][0], rays["oz"][0]),
                             (rays["dx"][0], rays["dy"][0], rays["dz"][0]), np.inf, verts[1])
    assert q["u"][1] / abs(q["D"][0]) < 1e-3 and q["u"][0] / abs(q["D"][0]) == pytest.approx(-0.5, abs=1e-4)
    # a planted miss of the hit triangle is unexplained too (the point is 0.2 inside)
    gpu = (np.array([-1], np.int32), np.zeros(1, np.float32), np.zeros(1, np.float32), np.zeros(1, np.float32))
    rep = parity.compare_hits(gpu, ref, rays, verts)
    assert rep["unexplained"] == [(0, -1, 0)]


def test_planted_order_flip_is_unexplained():
    """Two parallel triangles 1e-3 apart along the ray: picking the farther one is no tie,
    no edge and far outside the FP32 error of t."""
    verts = np.array([[[0, 0, 5], [1, 0, 5], [0, 1, 5]], [[0, 0, 5.005], [1, 0, 5.005], [0, 1, 5.005]]], np.float32)
    rays = _rays([0.2, 0.3, 0.0], [0, 0, 1])
    ref = oracle.bruteforce(rays, verts)
    assert ref[0][0] == 0
    gpu = (np.array([1], np.int32), np.array([5.005], np.float32), np.array([0.2], np.float32),
           np.array([0.3], np.float32))
    rep = parity.compare_hits(gpu, ref, rays, verts)
    assert rep["unexplained"] == [(0, 1, 0)]


def test_exact_edge_hit_is_excused_as_edge():
    """A ray through a shared edge of two triangles: both FP32 answers are possible, and
    the one the oracle did not pick is counted as an edge (or a tie), not unexplained."""
    verts = np.array([[[0, 0, 3], [1, 0, 3], [0, 1, 3]], [[1, 0, 3], [1, 1, 3], [0, 1, 3]]], np.float32)
    rays = _rays([0.5, 0.5, 0.0], [0, 0, 1])
    ref = oracle.bruteforce(rays, verts)
    other = 1 - int(ref[0][0])
    gpu = (np.array([other], np.int32), np.float32(ref[1]).reshape(1), np.float32(ref[2]).reshape(1),
           np.float32(ref[3]).reshape(1))
    rep = parity.compare_hits(gpu, ref, rays, verts)
    assert rep["unexplained"] == [] and rep["ties"] + rep["edges"] == 1


def _fp32_decision_numpy(o, d, tmax, v):
    """The library's FP32 Cramer-form decision restated with numpy float32 (every
    operation rounded separately, no fused multiply-add): one of the evaluation orders
    the error bound must cover."""
    f = np.float32
    o, d, v = np.asarray(o, f), np.asarray(d, f), np.asarray(v, f)
    a = v[0]
    e1, e2 = v[1] - a, v[2] - a
    n = np.array([e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]], f)
    dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2]
    s = o - a
    q = np.array([s[1] * d[2] - s[2] * d[1], s[2] * d[0] - s[0] * d[2], s[0] * d[1] - s[1] * d[0]], f)
    tn = s[0] * n[0] + s[1] * n[1] + s[2] * n[2]
    un = e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]
    wn = e1[0] * q[0] + e1[1] * q[1] + e1[2] * q[2]
    sg = f(1) if dn < 0 else f(-1)
    u, w, tp, ad = un * sg, -wn * sg, tn * sg, abs(dn)
    if not (u >= 0 and w >= 0 and f(u + w) <= ad and tp > 0 and tp <= f(f(tmax) * ad)):
        return False
    t = f(tp / ad)
    return bool(t > 0 and t <= tmax)


def test_fp32_band_is_sound_on_near_edge_rays(monkeypatch):
    """Rays aimed within 1e-6 of a triangle's edges and corners at random incidence:
    wherever an FP32 evaluation of the decision differs from the FP64 one, the
    uncapped error bound calls the decision uncertain."""
    monkeypatch.setattr(parity, "EDGE_CAP", np.inf)
    monkeypatch.setattr(parity, "TMAX_CAP", np.inf)
    rng = np.random.default_rng(11)
    flips = 0
    for k in range(4000):
        v = rng.uniform(-2, 2, size=(3, 3)).astype(np.float32)
        # a point on an edge (or a corner), nudged by up to 1e-6 of the edge length
        i, j = rng.integers(0, 3, size=2)
        lam = rng.choice([0.0, 1.0, rng.uniform()])
        p = v[i].astype(np.float64) * (1 - lam) + v[j].astype(np.float64) * lam
        p += rng.normal(size=3) * 1e-6
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        dist = rng.uniform(0.1, 50.0)
        o = (p - dist * d).astype(np.float32)
        d32 = d.astype(np.float32)
        tmax = np.float32(dist * (1 + rng.choice([0.0, 1e-7, -1e-7]))) if k % 3 == 0 else np.inf
        exact = oracle.mt(o, d32, tmax, v)[0]
        fp32 = _fp32_decision_numpy(o, d32, tmax, v)
        if exact != fp32:
            flips += 1
            q = parity.fp32_decision(o, d32, tmax, v)
            assert parity.decision_band(q) == "uncertain", (k, exact, fp32, q)
    assert flips > 10   # the sample does reach FP32's limits
