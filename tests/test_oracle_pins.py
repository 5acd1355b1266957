"""Pins of the CPU oracle against facts fixed outside it: closed forms, library
routines, brute force on tiny inputs, invariants, and the numbers printed in
the paper's Tables 1-4.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def rays_from(o, d, tmax=None, types=None):
    o = np.asarray(o, np.float32).reshape(-1, 3)
    d = np.asarray(d, np.float32).reshape(-1, 3)
    n = o.shape[0]
    r = {"ox": o[:, 0].copy(), "oy": o[:, 1].copy(), "oz": o[:, 2].copy(),
         "dx": d[:, 0].copy(), "dy": d[:, 1].copy(), "dz": d[:, 2].copy(),
         "tmax": np.full(n, np.inf, np.float32) if tmax is None else np.asarray(tmax, np.float32),
         "type": np.zeros(n, np.uint8) if types is None else np.asarray(types, np.uint8),
         "light": np.zeros(n, np.uint8)}
    return r


# --------------------------------------------------------------------------
# Moller-Trumbore (Section 3.3.8) and brute force (Section 1)
# --------------------------------------------------------------------------

def test_mt_axis_aligned_known_t():
    tri = np.array([[0, 0, 5], [1, 0, 5], [0, 1, 5]], np.float32)
    h, t, u, v = oracle.mt((0.2, 0.3, 0.0), (0, 0, 1), np.inf, tri)
    assert h and t == pytest.approx(5.0, abs=1e-12)
    assert u == pytest.approx(0.2, abs=1e-7) and v == pytest.approx(0.3, abs=1e-7)
    # direction of length 2: t is measured in units of the stored direction
    h, t, _, _ = oracle.mt((0.2, 0.3, 0.0), (0, 0, 2), np.inf, tri)
    assert h and t == pytest.approx(2.5, abs=1e-12)


@pytest.mark.parametrize("corner,uv", [(0, (0.0, 0.0)), (1, (1.0, 0.0)), (2, (0.0, 1.0))])
def test_mt_vertex_hits(corner, uv):
    tri = np.array([[0, 0, 3], [2, 0, 3], [0, 2, 3]], np.float32)
    o = tri[corner].astype(np.float64) - np.array([0, 0, 3.0])
    h, t, u, v = oracle.mt(o, (0, 0, 1), np.inf, tri)
    assert h and t == pytest.approx(3.0) and (u, v) == pytest.approx(uv, abs=1e-12)


def test_mt_range_and_parallel():
    tri = np.array([[0, 0, 5], [1, 0, 5], [0, 1, 5]], np.float32)
    assert not oracle.mt((0.2, 0.3, 0.0), (0, 0, 1), 4.999, tri)[0]      # beyond t_max
    assert oracle.mt((0.2, 0.3, 0.0), (0, 0, 1), 5.0, tri)[0]            # t == t_max is inside
    assert not oracle.mt((0.2, 0.3, 6.0), (0, 0, 1), np.inf, tri)[0]     # behind the origin
    assert not oracle.mt((0.2, 0.3, 0.0), (1, 0, 0), np.inf, tri)[0]     # parallel: det == 0
    assert not oracle.mt((0.8, 0.3, 0.0), (0, 0, 1), np.inf, tri)[0]     # u + v > 1
    h, t, _, _ = oracle.mt((0.2, 0.3, 10.0), (0, 0, -1), np.inf, tri)   # back side: two-sided
    assert h and t == pytest.approx(5.0)


def _solve_hit(o, d, tri):
    """Independent: solve o + t d = v0 + u e1 + v e2 with numpy.linalg."""
    v0, v1, v2 = (tri[k].astype(np.float64) for k in range(3))
    A = np.stack([-np.asarray(d, np.float64), v1 - v0, v2 - v0], 1)
    t, u, v = np.linalg.solve(A, np.asarray(o, np.float64) - v0)
    return t, u, v


def test_mt_matches_linear_solve_random():
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(3000):
        tri = rng.uniform(-1, 1, (3, 3)).astype(np.float32)
        o = rng.uniform(-3, 3, 3).astype(np.float32)
        w = rng.uniform(-0.3, 1.0, 3)
        aim = (w / w.sum()) @ tri.astype(np.float64)          # some inside, some outside
        d = unit(aim - o).astype(np.float32)
        t, u, v = _solve_hit(o, d, tri)
        margin = min(u, v, 1 - u - v)
        h, tt, uu, vv = oracle.mt(o, d, np.inf, tri)
        if abs(margin) < 1e-6 or abs(t) < 1e-6:
            continue
        inside = margin > 0 and t > 0
        assert h == inside
        if inside:
            checked += 1
            assert tt == pytest.approx(t, rel=1e-9, abs=1e-9)
            assert uu == pytest.approx(u, abs=1e-9) and vv == pytest.approx(v, abs=1e-9)
    assert checked > 100


def test_bruteforce_matches_independent_closest():
    rng = np.random.default_rng(2)
    verts = rng.uniform(-1, 1, (40, 3, 3)).astype(np.float32)
    o = rng.uniform(-3, 3, (60, 3)).astype(np.float32)
    tgt = rng.uniform(-0.5, 0.5, (60, 3))
    d = np.array([unit(a - b) for a, b in zip(tgt, o)], np.float32)
    tri, t, u, v = oracle.bruteforce(rays_from(o, d), verts)
    for i in range(60):
        best = None
        for k in range(40):
            tt, uu, vv = _solve_hit(o[i], d[i], verts[k])
            if min(uu, vv, 1 - uu - vv) >= 0 and tt > 0 and (best is None or tt < best[0]):
                best = (tt, k)
        if best is None:
            assert tri[i] == -1
        else:
            assert tri[i] == best[1] and t[i] == pytest.approx(best[0], rel=1e-9)
    assert (tri >= 0).sum() > 10


def test_bruteforce_tie_goes_to_smaller_id():
    tri = np.array([[0, 0, 5], [1, 0, 5], [0, 1, 5]], np.float32)
    verts = np.stack([tri, tri, tri])
    res = oracle.bruteforce(rays_from([[0.2, 0.3, 0]], [[0, 0, 1]]), verts)
    assert res[0][0] == 0


# --------------------------------------------------------------------------
# Eq. 9: sphere-cone test
# --------------------------------------------------------------------------

def _exact_dist_to_cone(P, C, x, alpha):
    """Textbook distance from point P to the solid one-sided cone (apex C, unit axis x,
    half-angle alpha)."""
    v = np.asarray(P, np.float64) - C
    lv = np.linalg.norm(v)
    if lv == 0:
        return 0.0
    ang = math.atan2(np.linalg.norm(np.cross(v, x)), float(v @ x))
    if ang <= alpha:
        return 0.0
    if ang >= alpha + math.pi / 2:
        return lv
    return lv * math.sin(ang - alpha)


def test_eq9_never_rejects_an_intersecting_sphere():
    rng = np.random.default_rng(3)
    accepted = rejected = 0
    for _ in range(4000):
        C = rng.uniform(-2, 2, 3)
        x = unit(rng.normal(size=3))
        alpha = rng.uniform(0, 1.4)
        d = rng.uniform(0, 0.5)
        P = rng.uniform(-6, 6, 3)
        r = rng.uniform(0, 0.7)
        node = np.concatenate([C, [d], x, [alpha]])
        eq9 = oracle.sphere_cone(node, P, r)
        exact = _exact_dist_to_cone(P, C, x, alpha) <= d + r
        if exact:
            assert eq9, "eq. 9 rejected a sphere that meets the node"
        accepted += eq9
        rejected += not eq9
    assert rejected > 500 and accepted > 500


def test_eq9_is_monotone_under_sphere_containment():
    """Eq. 9 accepts iff the sphere meets the region |s| tan(a) + d sec(a) >= distance to the
    axis, so a sphere that contains another is accepted whenever the inner one is (the GPU
    traversal tests a chunk's bounding sphere first and skips children that reject it)."""
    rng = np.random.default_rng(11)
    tested = 0
    for _ in range(20000):
        C = rng.uniform(-2, 2, 3)
        x = unit(rng.normal(size=3))
        alpha = rng.uniform(0, 1.5)
        d = rng.uniform(0, 0.3)
        node = np.concatenate([C, [d], x, [alpha]])
        K = rng.uniform(-6, 6, 3)
        R = rng.uniform(0.01, 1.5)
        # inner sphere, often touching the outer one from inside
        r = R * rng.uniform(0, 1)
        off = (R - r) * (1.0 if rng.uniform() < 0.5 else rng.uniform())
        P = K + off * unit(rng.normal(size=3))
        if oracle.sphere_cone(node, P, r):
            tested += 1
            assert oracle.sphere_cone(node, K, R), (node, K, R, P, r)
    assert tested > 2000


def test_eq9_closed_cases():
    node = np.array([0, 0, 0, 0.1, 0, 0, 1, 0.2])
    assert oracle.sphere_cone(node, (0, 0, 10), 0.0)                      # on the axis
    lim = 10 * math.tan(0.2) + 0.1 / math.cos(0.2)                        # radial reach at z = 10
    assert oracle.sphere_cone(node, (lim - 1e-9, 0, 10), 0.0)
    assert not oracle.sphere_cone(node, (lim + 1e-6, 0, 10), 0.0)
    assert oracle.sphere_cone(np.array([0, 0, 0, 0, 0, 0, 1, math.pi / 2]), (0, 0, -50), 0.0)


# --------------------------------------------------------------------------
# Section 3.3.6: cones (eqs. 1-6), spheres (eqs. 7-8), tree merge order
# --------------------------------------------------------------------------

def _build(o, d, B, L, pads=(0, 0, 0, 0)):
    return oracle.build_hierarchy(rays_from(o, d), B, L, pads)


@pytest.mark.parametrize("theta", [1e-4, 0.01, 0.3, 1.0, 2.5])
def test_two_rays_give_half_angle_about_bisector(theta):
    a = np.array([1.0, 0, 0])
    b = np.array([math.cos(theta), math.sin(theta), 0])
    lv = _build(np.zeros((2, 3)), np.stack([a, b]), 2, 1)
    node = lv[0][0]
    assert node[7] == pytest.approx(theta / 2, rel=1e-6)
    assert node[4:7] == pytest.approx(unit(a + b), abs=1e-6)


def test_identical_rays_zero_spread_and_points_zero_radius():
    d = np.tile(unit([1, 2, 3]), (8, 1))
    o = np.tile([0.5, -1, 2], (8, 1))
    node = _build(o, d, 8, 1)[0][0]
    assert node[7] == 0.0 and node[3] == 0.0
    assert node[:3] == pytest.approx([0.5, -1, 2])


def _rotate_toward(x, r, angle):
    """Rodrigues rotation of unit x by angle toward unit r (in their common plane)."""
    k = np.cross(x, r)
    k = k / np.linalg.norm(k)
    return x * math.cos(angle) + np.cross(k, x) * math.sin(angle) + k * (k @ x) * (1 - math.cos(angle))


def test_fold_matches_closed_form_recurrence():
    """Independent closed form of eqs. 1-4: when r lies outside (x, phi) at angle theta,
    the new spread is (phi + theta) / 2 and the axis turns toward r by (theta - phi) / 2."""
    rng = np.random.default_rng(4)
    for trial in range(40):
        base = unit(rng.normal(size=3))
        d = np.array([unit(base + 0.4 * rng.normal(size=3)) for _ in range(16)])
        d32 = d.astype(np.float32).astype(np.float64)
        d32 = np.array([unit(v) for v in d32])
        x, phi = d32[0], 0.0
        for r in d32[1:]:
            th = math.atan2(np.linalg.norm(np.cross(x, r)), x @ r)
            if th <= phi:
                continue
            x = _rotate_toward(x, r, (th - phi) / 2)
            phi = (phi + th) / 2
        node = _build(np.zeros((16, 3)), d, 16, 1)[0][0]
        assert node[7] == pytest.approx(phi, abs=1e-9)
        assert node[4:7] == pytest.approx(x, abs=1e-9)


def test_cone_union_same_axis_is_max_and_two_axes_bisect():
    a, b = unit([1, 0, 0]), unit([0, 1, 0])
    e = 0.05
    # level 1: node 0 = two rays around a (spread e), node 1 = two identical rays b
    da = [unit([math.cos(e), math.sin(e), 0]), unit([math.cos(e), -math.sin(e), 0])]
    d = np.stack(da + [b, b])
    lv = _build(np.zeros((4, 3)), d, 2, 2)
    top = lv[1][0]
    # (directions are stored in FP32, hence the 1e-7 tolerances)
    assert lv[0][0][7] == pytest.approx(e, abs=1e-7) and lv[0][1][7] == 0.0
    assert top[4:7] == pytest.approx(unit(a + b), abs=1e-7)
    assert top[7] == pytest.approx(math.pi / 4 + e, abs=1e-7)       # half the axis angle + max
    d2 = np.stack(da + da[::-1])
    top2 = _build(np.zeros((4, 3)), d2, 2, 2)[1][0]
    assert top2[7] == pytest.approx(e, abs=1e-7)                      # same axes: max spread


def test_sphere_union_worked_examples():
    # two points: midpoint and half the distance (eqs. 7-8)
    o = np.array([[1, 2, 3], [3, 2, 7]], np.float64)
    n = _build(o, np.tile([0, 0, 1.0], (2, 1)), 2, 1)[0][0]
    assert n[:3] == pytest.approx([2, 2, 5]) and n[3] == pytest.approx(math.sqrt(20) / 2)
    # four collinear points 0, 1, 2, 10 merged as a balanced tree:
    # (0 u 1) = (0.5, 0.5), (2 u 10) = (6, 4), union = (3.25, 5.5/2 + 4 = 6.75).
    # A left-to-right fold would give (5.625, 5.625) instead.
    o = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [10, 0, 0]], np.float64)
    n = _build(o, np.tile([0, 0, 1.0], (4, 1)), 4, 1)[0][0]
    assert n[:3] == pytest.approx([3.25, 0, 0]) and n[3] == pytest.approx(6.75)


def test_padding_and_level_counts():
    rng = np.random.default_rng(5)
    o = rng.uniform(-1, 1, (1000, 3))
    d = np.array([unit(v) for v in rng.normal(size=(1000, 3))])
    lv0 = _build(o, d, 8, 3)
    lv1 = _build(o, d, 8, 3, pads=(1e-3, 1e-2, 1e-3, 1e-2))
    assert [x.shape[0] for x in lv0] == [125, 16, 2] == oracle.level_counts(1000, 8, 3)
    assert lv1[0][:, 3] == pytest.approx(lv0[0][:, 3] * 1.001 + 1e-2)
    sp = np.minimum(np.pi, lv0[0][:, 7] * 1.001 + 1e-2)
    assert lv1[0][:, 7] == pytest.approx(sp)


def test_hierarchy_invariants_hold_on_oracle_nodes():
    rng = np.random.default_rng(6)
    n = 3001  # ragged: partial last nodes at every level
    o = rng.uniform(-2, 2, (n, 3)).astype(np.float32)
    d = np.array([unit(v) for v in rng.normal(size=(n, 3)) + [0, 0, 2]]).astype(np.float32)
    r = rays_from(o, d)
    lv = oracle.build_hierarchy(r, 16, 3, (1e-5, 1e-5, 1e-5, 1e-5))
    sph = np.concatenate([x[:, :4] for x in lv]).astype(np.float32)
    con = np.concatenate([x[:, 4:] for x in lv]).astype(np.float32)
    bad, worst = oracle.check_hierarchy(r, 16, [x.shape[0] for x in lv], sph, con)
    assert bad == 0 and worst <= 0
    # planting a shrunken node must be caught
    sph2 = sph.copy()
    sph2[3, 3] *= 0.5
    assert oracle.check_hierarchy(r, 16, [x.shape[0] for x in lv], sph2, con)[0] > 0


# --------------------------------------------------------------------------
# Section 3.3.2: ray generation and hashing
# --------------------------------------------------------------------------

def _gbuffer(P, N, I, mat):
    P, N, I = (np.asarray(a, np.float32).reshape(-1, 3) for a in (P, N, I))
    g = {k: np.ascontiguousarray(a[:, j]) for a, ks in ((P, "pxyz"), (N, "nxyz"), (I, "ixyz"))
         for j, k in enumerate([ks[0] + c for c in "xyz"])}
    g["material"] = np.asarray(mat, np.uint32)
    g["hit"] = np.ones(len(mat), np.uint8)
    return g


def test_ray_generation_geometry():
    rng = np.random.default_rng(7)
    n = 300
    N = np.array([unit(v) for v in rng.normal(size=(n, 3))])
    I = np.array([unit(v) for v in rng.normal(size=(n, 3))])
    I = np.where((np.sum(I * N, 1) < 0)[:, None], I, -I)          # incident against the normal
    P = rng.uniform(-1, 1, (n, 3))
    lights = np.array([[0, 5, 0], [3, 3, 3]], np.float32)
    g = _gbuffer(P, N, I, np.full(n, 2))                            # glass: every ray type
    r = oracle.generate_rays(g, lights, shadow_cull=False)
    assert r["ox"].shape[0] == n * 4                                # 2 shadow + refl + refr
    for k in range(n):
        base = 4 * k
        assert list(r["type"][base:base + 4]) == [0, 0, 1, 2] and list(r["light"][base:base + 2]) == [0, 1]
        assert (r["pixel"][base:base + 4] == k).all()
        p, nn, ii = P[k].astype(np.float32).astype(np.float64), g["nx"][k], None
        nv = np.array([g["nx"][k], g["ny"][k], g["nz"][k]], np.float64)
        iv = np.array([g["ix"][k], g["iy"][k], g["iz"][k]], np.float64)
        for j in range(2):   # shadow: from the light toward P, stopping just short of it
            o = np.array([r["ox"][base + j], r["oy"][base + j], r["oz"][base + j]], np.float64)
            d = np.array([r["dx"][base + j], r["dy"][base + j], r["dz"][base + j]], np.float64)
            assert o == pytest.approx(lights[j].astype(np.float64))
            dist = np.linalg.norm(p - o)
            assert o + d * dist == pytest.approx(p, abs=1e-5)
            assert r["tmax"][base + j] == pytest.approx(0.9999 * dist, rel=1e-6)
        # reflection: equal angles, in the plane of i and n
        d = np.array([r["dx"][base + 2], r["dy"][base + 2], r["dz"][base + 2]], np.float64)
        assert np.linalg.norm(d) == pytest.approx(1, abs=1e-6)
        assert d @ nv == pytest.approx(-(iv @ nv), abs=1e-5)
        assert np.cross(d - iv, nv) == pytest.approx(np.zeros(3), abs=1e-5)
        o = np.array([r["ox"][base + 2], r["oy"][base + 2], r["oz"][base + 2]], np.float64)
        assert (o - p) @ nv > 0                                      # offset to the incident side
        # refraction entering glass: Snell sin(t) = sin(i) / 1.5, bending toward -n
        d = np.array([r["dx"][base + 3], r["dy"][base + 3], r["dz"][base + 3]], np.float64)
        sin_i = np.linalg.norm(np.cross(iv, nv))
        sin_t = np.linalg.norm(np.cross(d, nv))
        assert sin_t == pytest.approx(sin_i / 1.5, abs=2e-6)
        assert d @ nv < 0
        o = np.array([r["ox"][base + 3], r["oy"][base + 3], r["oz"][base + 3]], np.float64)
        assert (o - p) @ nv < 0


def test_shadow_cull_and_total_internal_reflection():
    N = [[0, 1, 0]] * 3
    I = [[0, -1, 0], [0, -1, 0], unit([1, 0.2, 0])]                  # last: leaving glass at grazing angle
    P = [[0, 0, 0]] * 3
    lights = np.array([[0, 2, 0], [0, -2, 0]], np.float32)           # above and below the surface
    g = _gbuffer(P, N, I, [0, 1, 2])
    r = oracle.generate_rays(g, lights, shadow_cull=True)
    # pixel 0: only the light above survives; pixel 1: + reflection; pixel 2: shadow + reflection, no refraction (TIR)
    assert list(r["type"]) == [0, 0, 1, 0, 1]
    assert list(r["pixel"]) == [0, 1, 1, 2, 2]
    assert (r["light"][r["type"] == 0] == 0).all()
    # entering at the same grazing angle refracts (no TIR from the thin side)
    g2 = _gbuffer([[0, 0, 0]], [[0, 1, 0]], [unit([1, -0.2, 0])], [2])
    assert list(oracle.generate_rays(g2, np.zeros((0, 3)), True)["type"]) == [1, 2]


def _deinterleave(keys, tb, pb):
    """Undo the Z-order of the direction code bit by bit (phi bit, theta bit, ...)."""
    th = np.zeros_like(keys)
    ph = np.zeros_like(keys)
    pos = 0
    for b in range(min(tb, pb)):
        ph |= ((keys >> pos) & 1) << b
        pos += 1
        th |= ((keys >> pos) & 1) << b
        pos += 1
    for b in range(min(tb, pb), pb):
        ph |= ((keys >> pos) & 1) << b
        pos += 1
    for b in range(min(tb, pb), tb):
        th |= ((keys >> pos) & 1) << b
        pos += 1
    return th, ph


def _exact_bins(d, tb, pb):
    th = math.acos(max(-1.0, min(1.0, d[2]))) * (1 << tb) / math.pi
    ph = (math.atan2(d[1], d[0]) % (2 * math.pi)) * (1 << pb) / (2 * math.pi)
    return th, ph


@pytest.mark.parametrize("tb,pb", [(13, 13), (7, 8), (3, 3)])
def test_spherical_bins_match_acos_atan2(tb, pb):
    rng = np.random.default_rng(8)
    d = np.array([unit(v) for v in rng.normal(size=(20000, 3))], np.float32)
    r = rays_from(np.zeros_like(d), d)
    keys = oracle.hash_keys(r, (-1, -1, -1), (1, 1, 1), shadow_theta_bits=tb, shadow_phi_bits=pb)
    th_bin, ph_bin = _deinterleave(keys, tb, pb)
    checked = 0
    for k in range(d.shape[0]):
        th, ph = _exact_bins(d[k].astype(np.float64), tb, pb)
        if min(th - math.floor(th), math.ceil(th) - th) < 1e-3 or min(ph - math.floor(ph), math.ceil(ph) - ph) < 1e-3:
            continue
        assert th_bin[k] == int(th) and ph_bin[k] == int(ph) % (1 << pb)
        checked += 1
    assert checked > 15000


def test_hash_special_directions_and_layout():
    d = np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]], np.float32)
    r = rays_from(np.zeros_like(d), d)
    r["light"][:] = 5
    k = oracle.hash_keys(r, (-1, -1, -1), (1, 1, 1))
    th, ph = _deinterleave(k & ((1 << 26) - 1), 13, 13)
    assert list(k >> 26) == [5] * 6                                  # light index in the high bits, type 0
    assert th[0] == 0 and th[1] == 8191 and (th[2:] == 4096).all()   # acos(0) = pi/2 lands on bin 4096
    assert ph[0] == 0 and ph[1] == 0                                  # poles
    assert list(ph[2:]) == [0, 2048, 4096, 6144]


def test_origin_cell_morton():
    # secondary ray, 5 bits/axis over [0, 32)^3: cell (x, y, z) = floor(origin)
    o = np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5], [0.5, 1.5, 0.5], [0.5, 0.5, 1.5], [31.5, 31.5, 31.5],
                  [5.5, 17.5, 30.5], [-3, 40, 2.5]], np.float32)
    d = np.tile([0, 0, 1], (o.shape[0], 1)).astype(np.float32)
    r = rays_from(o, d, types=np.ones(o.shape[0]))
    k = oracle.hash_keys(r, (0, 0, 0), (32, 32, 32))
    cell = (k >> 15) & 0x7FFF

    def morton(x, y, z):
        c = 0
        for b in range(5):
            c |= ((x >> b) & 1) << (3 * b) | ((y >> b) & 1) << (3 * b + 1) | ((z >> b) & 1) << (3 * b + 2)
        return c
    exp = [morton(0, 0, 0), morton(1, 0, 0), morton(0, 1, 0), morton(0, 0, 1), morton(31, 31, 31),
           morton(5, 17, 30), morton(0, 31, 2)]
    assert list(cell) == exp
    assert list(cell[:4]) == [0, 1, 2, 4]
    assert (k >> 30 == 1).all()


def test_stable_sort_and_chunks():
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 50, 5000).astype(np.uint32)
    perm = oracle.stable_sort(keys)
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))
    assert oracle.chunk_count(keys) == 1 + int(np.count_nonzero(np.diff(keys)))
    assert oracle.chunk_count(np.zeros(0, np.uint32)) == 0
    assert oracle.chunk_count(np.full(7, 3, np.uint32)) == 1


# --------------------------------------------------------------------------
# Section 3.3.7-3.3.8 and Tables 1-4
# --------------------------------------------------------------------------

def test_paper_tables_counting_convention():
    """Tables 1-4: level-1 tests = B x level-2 hits, final tests = B x level-1 hits, total =
    top tests + level-1 tests + final tests; tests = misses + hits.  These are the conventions the
    oracle's paper-style counters follow."""
    g = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))
    B = g["bundle"]
    tot = {}
    for name, row in g.items():
        if not name.startswith("table") or name == "table4_totals":
            continue
        for alg in ("rah", "crsh"):
            t = row[alg]
            for lvl in range(2):
                assert t["tests"][lvl] == t["misses"][lvl] + t["hits"][lvl]
            assert t["tests"][0] == B * t["hits"][1]
            scene = name.split("_")[1]
            tot.setdefault((scene, alg), 0)
            tot[(scene, alg)] += t["tests"][1] + t["tests"][0] + B * t["hits"][0]
    t4 = g["table4_totals"]
    for scene in ("office", "cornell", "sponza"):
        for alg in ("rah", "crsh"):
            assert tot[(scene, alg)] == t4[scene][alg]
    assert t4["office"]["brute"] == 251546 * 36308            # N x M with M = 36,308 triangles
    assert t4["sponza"]["brute"] == 256713 * 66450
    assert g["table1_office_shadow_251546_rays"]["rah"]["tests"][1] == math.ceil(251546 / 64) * 36308


def _oracle_run(w, **kw):
    return oracle.run_crsh(w.gbuffer, w.lights, w.shadow_cull, w.hash_lo, w.hash_hi, w.scene, w.bundle,
                           w.levels, w.build_pads(), **kw)


def test_crsh_equals_bruteforce_config1(wl1):
    res = _oracle_run(wl1)
    assert res["rays"]["ox"].shape[0] == 4096
    bf = oracle.bruteforce(res["rays"], wl1.scene.verts)
    assert np.array_equal(bf[0], res["hits"][0])
    hit = bf[0] >= 0
    assert hit.sum() > 50
    assert np.array_equal(bf[1][hit], res["hits"][1][hit])
    c = res["counters"]
    B = wl1.bundle
    for l in range(wl1.levels - 1):
        assert c["tests_paper"][l] == B * c["hits"][l + 1]
    assert c["final_tests_paper"] == B * c["hits"][0]
    assert c["final_tests"] <= c["final_tests_paper"]


def test_crsh_equals_bruteforce_all_ray_types(wl2_small):
    res = _oracle_run(wl2_small)
    types = np.bincount(res["rays"]["type"], minlength=3)
    assert (types > 0).all()
    bf = oracle.bruteforce(res["rays"], wl2_small.scene.verts)
    assert np.array_equal(bf[0], res["hits"][0])
    # unsorted, no mesh culling (the RAH comparison mode) reaches the same hits with more tests
    rah = _oracle_run(wl2_small, sort=False, mesh_cull=False)
    assert np.array_equal(bf[0], rah["hits"][0])
    top = wl2_small.levels - 1
    n_top = rah["levels"][top].shape[0]
    assert rah["counters"]["tests"][top] == n_top * wl2_small.scene.n_tris
    assert rah["counters"]["final_tests"] > res["counters"]["final_tests"]


def test_traversal_pairs_equal_ancestor_brute_force():
    """Level-1 pairs = every (node, triangle) whose whole ancestor chain (and mesh sphere)
    passes eq. 9, found here by direct enumeration."""
    import synthetic
    w = synthetic.make(1, res=12)
    res = _oracle_run(w)
    lv = res["levels"]
    B, L = w.bundle, w.levels
    ts = oracle.tri_spheres(w.scene.verts)
    mesh_of = np.repeat(np.arange(w.scene.n_meshes), np.diff(w.scene.mesh_first_tri.astype(np.int64)))
    want = set()
    for n1 in range(lv[0].shape[0]):
        chain = [n1 // B ** l for l in range(L)]
        for t in range(w.scene.n_tris):
            ms = w.scene.mesh_sphere[mesh_of[t]]
            if not oracle.sphere_cone(lv[L - 1][chain[L - 1]], ms[:3], ms[3]):
                continue
            if all(oracle.sphere_cone(lv[l][chain[l]], ts[t, :3], ts[t, 3]) for l in range(L)):
                want.add((n1, t))
    got = set(zip(res["pair_node"].tolist(), res["pair_tri"].tolist()))
    assert got == want and len(want) > 0
    order = list(zip(res["pair_node"].tolist(), res["pair_tri"].tolist()))
    assert order == sorted(order)


# --------------------------------------------------------------------------
# Adjoint of the closest hit (hit assignment fixed): central finite differences
# --------------------------------------------------------------------------

def _loss_fd(o, d, tri_v, w):
    h, t, u, v = oracle.mt(o, d, np.inf, tri_v)
    assert h
    return w[0] * t + w[1] * u + w[2] * v


def test_adjoint_matches_central_differences():
    """dL/d(o, d, V) of L = w_t t + w_u u + w_v v against FP64 central differences of the oracle's own
    Moller-Trumbore (h = 1e-5 on float64 inputs, where truncation is far below the tolerance)."""
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(60):
        tri_v = rng.uniform(-1, 1, (3, 3))
        bary = rng.dirichlet([2, 2, 2])
        target = bary @ tri_v
        o = rng.uniform(-3, 3, 3)
        d = target - o
        d = d / np.linalg.norm(d)
        h, t, u, v = oracle.mt(o, d, np.inf, tri_v.astype(np.float32))
        if not h or min(u, v, 1 - u - v) < 5e-2:
            continue
        w = rng.normal(size=3)
        rays = {"ox": np.array([o[0]], np.float32), "oy": np.array([o[1]], np.float32),
                "oz": np.array([o[2]], np.float32), "dx": np.array([d[0]], np.float32),
                "dy": np.array([d[1]], np.float32), "dz": np.array([d[2]], np.float32)}
        o32 = np.array([rays[k][0] for k in ("ox", "oy", "oz")], np.float64)
        d32 = np.array([rays[k][0] for k in ("dx", "dy", "dz")], np.float64)
        v32 = tri_v.astype(np.float32)
        h, t, u, v = oracle.mt(o32, d32, np.inf, v32)
        gv_, go, gd = oracle.adjoint(rays, (np.array([0], np.int32), np.array([t]), np.array([u]), np.array([v])),
                                     [w[0]], [w[1]], [w[2]], v32[None])

        def fd(f, x, eps=1e-5):
            g = np.zeros_like(x)
            for k in range(x.size):
                a, b = x.copy(), x.copy()
                a.flat[k] += eps
                b.flat[k] -= eps
                g.flat[k] = (f(a) - f(b)) / (2 * eps)
            return g

        # float64 finite differences through a float64 copy of the test (oracle.mt reads float64 rays,
        # float32 vertices: perturb vertices through exact float64 -> the vertex FD uses numpy's solve)
        def mt64(oo, dd, vv):
            A = np.stack([-dd, vv[1] - vv[0], vv[2] - vv[0]], 1)
            tt, uu, ww = np.linalg.solve(A, oo - vv[0])
            return w[0] * tt + w[1] * uu + w[2] * ww
        V = v32.astype(np.float64)
        ref_o = fd(lambda x: mt64(x, d32, V), o32)
        ref_d = fd(lambda x: mt64(o32, x, V), d32)
        ref_v = fd(lambda x: mt64(o32, d32, x.reshape(3, 3)), V.reshape(-1))
        scale = max(1.0, np.abs(ref_v).max(), np.abs(ref_o).max(), np.abs(ref_d).max())
        assert np.abs(go[0] - ref_o).max() <= 1e-4 * scale
        assert np.abs(gd[0] - ref_d).max() <= 1e-4 * scale
        assert np.abs(gv_[0] - ref_v).max() <= 1e-4 * scale
        checked += 1
    assert checked > 20


def test_adjoint_accumulates_per_triangle_and_skips_misses():
    tri_v = np.array([[0, 0, 5], [1, 0, 5], [0, 1, 5]], np.float32)
    rays = {"ox": np.array([0.2, 0.1, 5.0], np.float32), "oy": np.array([0.3, 0.1, 5.0], np.float32),
            "oz": np.zeros(3, np.float32), "dx": np.zeros(3, np.float32), "dy": np.zeros(3, np.float32),
            "dz": np.ones(3, np.float32)}
    hits = (np.array([0, 0, -1], np.int32), np.array([5.0, 5.0, 0]), np.array([0.2, 0.1, 0]), np.array([0.3, 0.1, 0]))
    gv_, go, gd = oracle.adjoint(rays, hits, np.ones(3), np.zeros(3), np.zeros(3), tri_v[None])
    # dt/do_z = -1 for a plane z = 5 hit from below along +z; dt/do_x = dt/do_y = 0
    assert go[0] == pytest.approx([0, 0, -1]) and go[1] == pytest.approx([0, 0, -1])
    assert (go[2] == 0).all() and (gd[2] == 0).all()
    assert gd[0] == pytest.approx([0, 0, -5])
    # translating the triangle by +z moves t by +1: the three corner gradients sum to (0, 0, 1) per ray
    assert gv_[0].reshape(3, 3).sum(0) == pytest.approx([0, 0, 2])


# --------------------------------------------------------------------------
# NEXT row f3: camera rays and first-hit buffers
# --------------------------------------------------------------------------

def _cam(eye, fwd, right, up, tx, ty):
    return np.array(list(eye) + list(fwd) + list(right) + list(up) + [tx, ty], np.float64)


def test_primary_rays_cover_every_pixel_once_in_compact_tiles():
    cam = _cam((0, 1, 5), (0, 0, -1), (1, 0, 0), (0, 1, 0), 0.6, 0.45)
    for w, h in ((16, 8), (19, 13), (64, 64)):
        r = oracle.primary_rays(cam, w, h)
        assert np.array_equal(np.sort(r["pixel"]), np.arange(w * h))
        x, y = r["pixel"] % w, r["pixel"] // w
        full_w, full_h = (w // 8) * 8, (h // 8) * 8
        for start in range(0, r["pixel"].size - 16 + 1, 16):
            xs, ys = x[start:start + 16], y[start:start + 16]
            if xs.max() < full_w and ys.max() < full_h:      # inside full blocks: a 4x4 square
                assert xs.max() - xs.min() == 3 and ys.max() - ys.min() == 3
        assert np.all(r["ox"] == np.float32(0)) and np.all(r["oz"] == np.float32(5))


def test_primary_ray_directions_against_fp64():
    fwd = np.array([0.3, -0.2, -1.0]); fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, [0, 1, 0]); right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    cam = _cam((1, 2, 3), fwd, right, up, 0.7, 0.5)
    w, h = 24, 16
    r = oracle.primary_rays(cam, w, h)
    x, y = (r["pixel"] % w).astype(np.float64), (r["pixel"] // w).astype(np.float64)
    c32 = cam.astype(np.float32).astype(np.float64)
    sx = (2 * (x + 0.5) / w - 1) * c32[12]
    sy = (1 - 2 * (y + 0.5) / h) * c32[13]
    d = c32[3:6][None] + sx[:, None] * c32[6:9][None] + sy[:, None] * c32[9:12][None]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = np.stack([r["dx"], r["dy"], r["dz"]], 1).astype(np.float64)
    assert np.abs(got - d).max() < 8 * np.finfo(np.float32).eps
    # the corner pixel's angle to the axis matches the field of view
    k = int(np.nonzero(r["pixel"] == 0)[0][0])
    ang_x = math.atan(abs(np.dot(got[k], c32[6:9])) / np.dot(got[k], c32[3:6]))
    assert abs(ang_x - math.atan((1 - 1 / w) * c32[12])) < 1e-6


def test_odd_image_centre_ray_is_the_axis():
    cam = _cam((0, 0, 0), (0, 0, -1), (1, 0, 0), (0, 1, 0), 0.5, 0.5)
    r = oracle.primary_rays(cam, 9, 7)
    k = int(np.nonzero(r["pixel"] == 3 * 9 + 4)[0][0])
    assert (r["dx"][k], r["dy"][k], r["dz"][k]) == (0.0, 0.0, -1.0)


def test_gbuffer_from_hits_worked_cases():
    verts = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0]],      # normal +z
                      [[0, 0, 0], [0, 1, 0], [1, 0, 0]]],     # same plane, normal -z
                     np.float32)
    rays = rays_from([[0.25, 0.25, 1.0], [0.25, 0.25, 1.0], [0.25, 0.25, -2.0], [5, 5, 5]],
                     [[0, 0, -1], [0, 0, -1], [0, 0, 1], [0, 0, 1]])
    tri = np.array([0, 1, 0, -1], np.int32)
    t = np.array([1.0, 1.0, 2.0, 0.0], np.float32)
    g = oracle.gbuffer_from_hits(rays, tri, t, verts, np.array([7, 9], np.int32))
    assert list(g["hit"]) == [1, 1, 1, 0]
    for i in range(3):
        assert (g["px"][i], g["py"][i], g["pz"][i]) == (0.25, 0.25, 0.0)
    # normals face the incoming ray whatever the winding
    assert (g["nx"][0], g["ny"][0], g["nz"][0]) == (0.0, 0.0, 1.0)
    assert (g["nx"][1], g["ny"][1], g["nz"][1]) == (0.0, 0.0, 1.0)
    assert (g["nx"][2], g["ny"][2], g["nz"][2]) == (0.0, 0.0, -1.0)
    assert list(g["material"]) == [7, 9, 7, 0]
    assert (g["ix"][3], g["iy"][3], g["iz"][3]) == (0.0, 0.0, 1.0) and g["px"][3] == 0 and g["nx"][3] == 0


def test_gbuffer_from_hits_reproduces_the_raster_gbuffer():
    """On config 1, the first-hit buffer of the camera rays, with the FP64 brute-force hits of
    those rays, matches the software rasteriser's G-buffer: the same pixels hit the same
    triangles (except where the FP32 ray direction decides an edge), with positions and normals
    within FP32 rounding."""
    w = synthetic.make(1)
    r = oracle.primary_rays(w.camera, w.width, w.height)
    tri, t, _, _ = oracle.bruteforce({**r, "tmax": np.full(r["ox"].shape, np.inf, np.float32)}, w.scene.verts)
    g = oracle.gbuffer_from_hits(r, tri, t.astype(np.float32), w.scene.verts, w.scene.tri_material)
    px = r["pixel"]
    same = tri == w.primary_tri[px]
    assert same.mean() > 0.995
    both = same & (tri >= 0)
    for k, kk in (("px", "px"), ("py", "py"), ("pz", "pz")):
        assert np.allclose(g[k][both], w.gbuffer[kk][px][both], rtol=1e-5, atol=1e-5)
    for k in ("nx", "ny", "nz"):
        assert np.allclose(g[k][both], w.gbuffer[k][px][both], atol=1e-5)
    assert np.array_equal(g["material"][both], w.gbuffer["material"][px][both])


# --------------------------------------------------------------------------
# NEXT row f4: shading accumulation (a stated reading; the paper names no model)
# --------------------------------------------------------------------------

def test_shade_worked_pixels():
    s2 = math.sqrt(0.5)
    # pixel 0: diffuse, normal +y, light 0 visible at 45 degrees, light 1 occluded
    # pixel 1: mirror, normal +y, no shadow rays, reflection ray hits a diffuse triangle
    # pixel 2: glass, reflection misses (sky), refraction hits glass
    # pixel 3: background
    gb = {"nx": np.array([0, 0, 0, 0], np.float32), "ny": np.array([1, 1, 1, 0], np.float32),
          "nz": np.array([0, 0, 0, 0], np.float32), "material": np.array([0, 1, 2, 0], np.uint32),
          "hit": np.array([1, 1, 1, 0], np.uint8)}
    rays = {"dx": np.array([s2, 0, 0, 0, 0, 0], np.float32), "dy": np.array([-s2, -1, 1, 1, -1, -1], np.float32),
            "dz": np.array([0, 0, 0, 0, 0, 0], np.float32),
            "type": np.array([0, 0, 1, 1, 2, 0], np.uint8), "light": np.array([0, 1, 0, 0, 0, 0], np.uint8),
            "pixel": np.array([0, 0, 1, 2, 2, 3], np.uint32)}
    tri = np.array([-1, 5, 0, -1, 1, -1], np.int32)          # triangle 0 diffuse, 1 glass
    tm = np.array([0, 2] + [0] * 4, np.int32)
    c = oracle.shade(gb, rays, tri, tm, 2)
    f = np.float32
    assert c[0] == f(0.8) * (f(0.1) + f(s2) + f(0))          # n . (-d) = cos 45 degrees
    assert c[1] == f(0.2) * f(0.1) + f(0.8) * (f(0.8) * (f(0.1) + f(0.5)))
    assert c[2] == (f(0.1) * f(0.1) + f(0.1) * f(0.6)) + f(0.8) * (f(0.1) * (f(0.1) + f(0.5)))
    assert c[3] == f(0.6)
    # a back-facing light contributes nothing
    rays["dy"][0] = np.float32(s2)
    assert oracle.shade(gb, rays, tri, tm, 2)[0] == f(0.8) * f(0.1)
