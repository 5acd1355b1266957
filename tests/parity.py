"""Shared comparison logic of the GPU parity tests (the oracle decides).

Closest hits (Section 3.3.8) are compared element by element with the oracle's
FP64 hits of the same rays.  Where the triangle differs, the mismatch is
accepted only in three cases, each counted and reported:

- tie:   both triangles are hit (FP64) at distances within TIE_REL of each
         other, the near-tie the tolerances allow;
- edge:  the FP32 hit/miss decision of one of the two triangles can differ
         from the exact one.  The band is a rigorous forward error bound of
         the kernel's FP32 Cramer-form Moller-Trumbore (below), evaluated per
         ray and triangle, and capped at EDGE_CAP (barycentric units) and
         TMAX_CAP (relative distance): a mismatch outside the capped band is
         unexplained however grazing the ray.  TMAX_CAP is 10x the 1e-4 by
         which a shadow ray stops short of its own surface (t_max = 0.9999
         of the distance): at grazing incidence on small triangles the FP32
         error of t exceeds that 1e-4, and the kernel may then find the ray's
         own surface triangle; the cap still rejects any t-range flip more
         than 1e-3 of the distance away;
- order: both triangles are hit, and their distances are closer than the
         FP32 error bound of t (capped at ORDER_CAP relative).

Error bound.  The library decides a hit from FP32 inputs o, d, t_max, v0, v1,
v2 with e1 = fl(v1 - v0), e2 = fl(v2 - v0), n = fl(e1 x e2), s = fl(o - v0),
q = fl(s x d) and the dot products D = -(d.n), t' = s.n, u' = e2.q,
v' = -(e1.q), accepting when u' >= 0, v' >= 0, u' + v' <= |D|, t' > 0 and
t' <= t_max |D| (signs folded by sign(D)).  Each quantity is carried as its
exact value x (FP64 from the FP32 inputs) and a bound e on |fl(x) - x| under
the standard model fl(a op b) = (a op b)(1 + delta), |delta| <= u = 2^-24:
a sum of k products computed with fused multiply-adds has error at most
gamma_k sum |a_i b_i| (gamma_k = k u / (1 - k u), Higham, "Accuracy and
Stability of Numerical Algorithms", 2nd ed., section 3.1), plus the
propagated errors of its operands, sum (|a_i| e(b_i) + |b_i| e(a_i) +
e(a_i) e(b_i)).  A comparison x >= 0 can come out differently in FP32 only
when |x| <= e(x).
"""
from __future__ import annotations

import os

import numpy as np

import oracle

T_REL = 1e-5      # hit distance, relative
UV_ABS = 1e-5     # barycentrics, absolute
TIE_REL = 1e-6    # two triangles this close in t are a near-tie (either id is correct)
EDGE_CAP = 1e-3   # largest barycentric band an FP32 edge decision may be excused in
TMAX_CAP = 1e-3   # largest relative band around t = t_max / t = 0 that may be excused
ORDER_CAP = 1e-5  # largest relative t difference an FP32 ordering flip may be excused at

U32 = 2.0 ** -24          # unit roundoff of FP32
FP64_SLACK = 1e-12        # relative slack for the FP64 evaluation of the exact values


def _gamma(k):
    return k * U32 / (1 - k * U32)


def _sub(a, b):
    """fl(a - b) of two FP32 inputs: exact value and error bound."""
    x = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return x, U32 * np.abs(x)


def _dot(pairs):
    """Sum of len(pairs) products computed with fused multiply-adds: pairs of
    ((a, ea), (b, eb)).  Returns (exact value, error bound)."""
    k = len(pairs)
    x = 0.0
    prop = 0.0
    mag = 0.0
    for (a, ea), (b, eb) in pairs:
        x = x + a * b
        p = np.abs(a) * eb + np.abs(b) * ea + ea * eb
        prop = prop + p
        mag = mag + np.abs(a * b) + p
    return x, prop + _gamma(k) * mag + FP64_SLACK * mag


def _neg(a):
    return -a[0], a[1]


def fp32_decision(o, d, tmax, v):
    """The FP32 Moller-Trumbore decision quantities of ray (o, d, t_max) and
    triangle v (3x3, rows v0, v1, v2) with their error bounds.  Returns a dict
    of exact values and bounds: D, u (= u'), v (= v'), w (= |D| - u' - v'),
    t (= t'), m (= t_max |D| - t', inf for an infinite t_max)."""
    v = np.asarray(v, np.float64)
    o = [float(x) for x in o]
    d = [(float(x), 0.0) for x in d]
    e1 = [_sub(v[1, i], v[0, i]) for i in range(3)]
    e2 = [_sub(v[2, i], v[0, i]) for i in range(3)]
    n = [_dot([(e1[1], e2[2]), (_neg(e1[2]), e2[1])]),
         _dot([(e1[2], e2[0]), (_neg(e1[0]), e2[2])]),
         _dot([(e1[0], e2[1]), (_neg(e1[1]), e2[0])])]
    dn = _dot([(d[0], n[0]), (d[1], n[1]), (d[2], n[2])])
    s = [_sub(o[i], v[0, i]) for i in range(3)]
    q = [_dot([(s[1], d[2]), (_neg(s[2]), d[1])]),
         _dot([(s[2], d[0]), (_neg(s[0]), d[2])]),
         _dot([(s[0], d[1]), (_neg(s[1]), d[0])])]
    tn = _dot([(s[0], n[0]), (s[1], n[1]), (s[2], n[2])])
    un = _dot([(e2[0], q[0]), (e2[1], q[1]), (e2[2], q[2])])
    wn = _dot([(e1[0], q[0]), (e1[1], q[1]), (e1[2], q[2])])
    D = -dn[0]
    sg = 1.0 if D >= 0 else -1.0
    uu = (sg * un[0], un[1])
    vv = (-sg * wn[0], wn[1])
    aD = abs(D)
    # fl(u' + v') <= |D|: the sum's own rounding plus both operands' and |D|'s errors
    w_err = uu[1] + vv[1] + U32 * (abs(uu[0] + vv[0]) + uu[1] + vv[1]) + dn[1]
    ww = (aD - uu[0] - vv[0], w_err)
    tt = (sg * tn[0], tn[1])
    tmax = float(tmax)
    if np.isfinite(tmax):
        # fl(t_max |D|) and the division t = t'/|D| checked again against t_max
        m_err = tn[1] + tmax * dn[1] + U32 * tmax * (aD + dn[1]) + 2 * U32 * tmax * aD
        mm = (tmax * aD - tt[0], m_err)
    else:
        mm = (np.inf, 0.0)
    return dict(D=(D, dn[1]), u=uu, v=vv, w=ww, t=tt, m=mm)


def decision_band(q):
    """Classify one FP32 decision: 'hit' or 'miss' when FP32 must agree with the
    exact decision, 'uncertain' when it may differ within the capped band."""
    D, eD = q["D"]
    aD = abs(D)
    cap_bary = EDGE_CAP * aD
    def band(key, cap):
        x, e = q[key]
        return x, min(e, cap)
    if aD <= eD:
        # the sign of D itself is uncertain: a hit needs u' + v' <= |D| for some sign
        big = (abs(q["u"][0]) - q["u"][1]) + (abs(q["v"][0]) - q["v"][1])
        return "uncertain" if big <= 2 * eD else "miss"
    checks = [band("u", cap_bary), band("v", cap_bary), band("w", cap_bary)]
    # t' and t_max |D| - t' are distances times |D|: the cap is TMAX_CAP of the
    # distance (at least of one unit of the direction vector)
    tx, te = q["t"]
    checks.append((tx, min(te, TMAX_CAP * max(aD, abs(tx)))))
    mx, me = q["m"]
    if np.isfinite(mx):
        checks.append((mx, min(me, TMAX_CAP * max(aD, abs(tx)))))
    if any(x < -e for x, e in checks):
        return "miss"
    if all(x > e for x, e in checks):
        return "hit"
    return "uncertain"


def t_error(q):
    """Bound on |fl32(t) - t| of the kernel's t = t'/|D| (given a certain D)."""
    D, eD = q["D"]
    tx, te = q["t"]
    aD = abs(D)
    if aD <= eD:
        return np.inf
    t = tx / aD
    return (te + abs(t) * eD) / (aD - eD) + U32 * abs(t)


def _ray(rays, i):
    o = (rays["ox"][i], rays["oy"][i], rays["oz"][i])
    d = (rays["dx"][i], rays["dy"][i], rays["dz"][i])
    return o, d, float(rays["tmax"][i])


def explain(rays, i, g, r, verts):
    """Why ray i may pick triangle g on the GPU where the oracle picks r (-1 = miss).
    Returns 'tie', 'edge', 'order' or None (unexplained)."""
    o, d, tmax = _ray(rays, i)
    hg = oracle.mt(o, d, tmax, verts[g]) if g >= 0 else (False, 0.0, 0.0, 0.0)
    hr = oracle.mt(o, d, tmax, verts[r]) if r >= 0 else (False, 0.0, 0.0, 0.0)
    if g >= 0 and r >= 0 and hg[0] and hr[0] and abs(hg[1] - hr[1]) <= TIE_REL * abs(hr[1]):
        return "tie"
    # the GPU may have missed the oracle's triangle
    if r >= 0 and decision_band(fp32_decision(o, d, tmax, verts[r])) == "uncertain":
        return "edge"
    if g >= 0:
        qg = fp32_decision(o, d, tmax, verts[g])
        # the GPU may have hit a triangle the exact test misses
        if not hg[0] and decision_band(qg) == "uncertain":
            return "edge"
        # both hit: FP32 may order their distances the other way
        if hg[0] and r >= 0 and hr[0]:
            qr = fp32_decision(o, d, tmax, verts[r])
            band = min(t_error(qg) + t_error(qr), ORDER_CAP * abs(hr[1]))
            if hg[1] - hr[1] <= band:
                return "order"
    return None


def compare_hits(gpu, ref, rays, verts):
    """gpu: (tri, t, u, v) FP32 arrays; ref: FP64 closest hits of the same rays (same order).
    Returns a report with the counts of ties, edges and order flips and the list of
    unexplained mismatches (ray, gpu triangle, oracle triangle)."""
    gtri, gt, gu, gv = gpu
    rtri, rt, ru, rv = ref
    n = gtri.shape[0]
    same = gtri == rtri
    hit = same & (rtri >= 0)
    rep = dict(n=int(n), hits=int((rtri >= 0).sum()), ties=0, edges=0, order=0, unexplained=[])
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
        why = explain(rays, i, g, r, verts)
        if why == "tie":
            rep["ties"] += 1
        elif why == "edge":
            rep["edges"] += 1
        elif why == "order":
            rep["order"] += 1
        else:
            rep["unexplained"].append((int(i), g, r))
    return rep


def summary(rep) -> str:
    """One line with the flagged counts, printed by every parity test."""
    return (f"rays={rep['n']} hits={rep['hits']} ties={rep['ties']} edges={rep['edges']} order={rep['order']} "
            f"unexplained={len(rep['unexplained'])} max_t_rel={rep['max_t_rel']:.2e} "
            f"max_uv_abs={rep['max_uv_abs']:.2e}")


# every report checked in this process, printed at the end of the pytest run
REPORTS = []


def check_report(rep, max_flagged_frac=2e-3, label=""):
    label = label or os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    REPORTS.append((label, summary(rep)))
    print(f"closest-hit parity {label}: {summary(rep)}")
    assert not rep["unexplained"], f"unexplained closest-hit mismatches: {rep['unexplained'][:10]}"
    assert rep["t_viol"] == 0, f"t beyond {T_REL} relative: {rep}"
    assert rep["uv_viol"] == 0, f"barycentrics beyond {UV_ABS}: {rep}"
    assert rep["miss_nonzero"] == 0
    flagged = rep["ties"] + rep["edges"] + rep["order"]
    assert flagged <= max(3, max_flagged_frac * rep["n"]), rep


def within(a, b, rel):
    return abs(a - b) <= rel * max(abs(b), 1)
