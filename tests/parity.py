"""Shared comparison logic of the GPU parity tests (the oracle decides)."""
from __future__ import annotations

import numpy as np

import oracle

T_REL = 1e-5      # hit distance, relative
UV_ABS = 1e-5     # barycentrics, absolute
TIE_REL = 1e-6    # two triangles this close in t are a near-tie (either id is correct)
EDGE = 1e-4       # barycentric margin inside which FP32 and FP64 may disagree on a hit (normal incidence)
TMAX_REL = 2e-6   # relative band around t = t_max (and t = 0) where they may disagree (normal incidence)


def _fp64_hit(rays, i, tri, verts):
    o = (rays["ox"][i], rays["oy"][i], rays["oz"][i])
    d = (rays["dx"][i], rays["dy"][i], rays["dz"][i])
    return oracle.mt(o, d, float(rays["tmax"][i]), verts[tri])


def _crossing(rays, i, tri, verts):
    """FP64 plane crossing of ray i with a triangle, ignoring every range test:
    (barycentric margin min(u, v, 1-u-v), t, |cos| of the incidence angle)."""
    v = verts[tri].astype(np.float64)
    o = np.array([rays["ox"][i], rays["oy"][i], rays["oz"][i]], np.float64)
    d = np.array([rays["dx"][i], rays["dy"][i], rays["dz"][i]], np.float64)
    e1, e2 = v[1] - v[0], v[2] - v[0]
    n = np.cross(e1, e2)
    cos = abs(d @ n) / max(np.linalg.norm(n) * np.linalg.norm(d), 1e-300)
    A = np.stack([-d, e1, e2], 1)
    try:
        t, u, w = np.linalg.solve(A, o - v[0])
    except np.linalg.LinAlgError:
        return -np.inf, np.inf, 0.0
    return min(u, w, 1 - u - w), t, cos


def _uncertain(rays, i, tri, verts):
    """True when FP32 cannot decide whether ray i hits this triangle: the FP64
    crossing lies within the FP32 error band of an edge, of t = t_max or of
    t = 0.  FP32 errors of the barycentrics and of t grow like 1/cos(incidence),
    so the bands do too (EDGE and TMAX_REL at normal incidence)."""
    m, t, cos = _crossing(rays, i, tri, verts)
    c = max(cos, 1e-4)
    if not np.isfinite(t):
        return True
    tmax = float(rays["tmax"][i])
    near_edge = abs(m) <= EDGE / c
    inside = m >= -EDGE / c
    near_tmax = np.isfinite(tmax) and abs(t - tmax) <= TMAX_REL * tmax / c
    near_zero = abs(t) <= TMAX_REL * max(1.0, abs(t)) / c
    return near_edge or (inside and (near_tmax or near_zero))


def compare_hits(gpu, ref, rays, verts):
    """gpu: (tri, t, u, v) FP32 arrays; ref: FP64 closest hits of the same rays (same order).
    A different triangle is accepted (and counted) only when it is a near-tie in t or when
    FP32 cannot decide one of the two triangles (edge, t_max or t = 0 within the FP32
    error band); anything else is listed as unexplained.  Returns a report."""
    gtri, gt, gu, gv = gpu
    rtri, rt, ru, rv = ref
    n = gtri.shape[0]
    same = gtri == rtri
    hit = same & (rtri >= 0)
    rep = dict(n=int(n), hits=int((rtri >= 0).sum()), ties=0, edges=0, unexplained=[])
    t_rel = np.abs(gt[hit].astype(np.float64) - rt[hit]) / np.maximum(np.abs(rt[hit]), 1e-30)
    uv = np.maximum(np.abs(gu[hit] - ru[hit]), np.abs(gv[hit] - rv[hit]))
    rep["max_t_rel"] = float(t_rel.max()) if t_rel.size else 0.0
    rep["max_uv_abs"] = float(uv.max()) if uv.size else 0.0
    rep["t_viol"] = int((t_rel > T_REL).sum())
    rep["uv_viol"] = int((uv > UV_ABS).sum())
    # misses must agree exactly in (t, u, v) = 0
    miss = same & (rtri < 0)
    rep["miss_nonzero"] = int(((gt[miss] != 0) | (gu[miss] != 0) | (gv[miss] != 0)).sum())
    for i in np.nonzero(~same)[0]:
        g, r = int(gtri[i]), int(rtri[i])
        if g >= 0 and r >= 0:
            h, t64, _, _ = _fp64_hit(rays, i, g, verts)
            if h and abs(t64 - rt[i]) <= TIE_REL * abs(rt[i]):
                rep["ties"] += 1
                continue
        if (r >= 0 and _uncertain(rays, i, r, verts)) or (g >= 0 and _uncertain(rays, i, g, verts)):
            rep["edges"] += 1
            continue
        rep["unexplained"].append((int(i), g, r))
    return rep


def check_report(rep, max_flagged_frac=2e-3):
    assert not rep["unexplained"], f"unexplained closest-hit mismatches: {rep['unexplained'][:10]}"
    assert rep["t_viol"] == 0, f"t beyond {T_REL} relative: {rep}"
    assert rep["uv_viol"] == 0, f"barycentrics beyond {UV_ABS}: {rep}"
    assert rep["miss_nonzero"] == 0
    assert rep["ties"] + rep["edges"] <= max(3, max_flagged_frac * rep["n"]), rep


def within(a, b, rel):
    return abs(a - b) <= rel * max(abs(b), 1)
