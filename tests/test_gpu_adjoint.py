"""crsh_closest_hit_backward against the FP64 oracle gradient and central
finite differences, on the hits the GPU found (the hit assignment is fixed).

Loss L = sum_i w_i t_i + sum_i (a_i u_i + b_i v_i) with seeded N(0, 1) weights
over hit rays.  Bars: per output tensor, norm-wise relative error <= 1e-4 and
element-wise |err| <= 1e-4 |ref| + 1e-3 max|ref| against the FP64 closed form;
against central differences (FP64 forward, hit fixed; h = 1e-3 for origins and
directions, 1e-3 x the shortest edge for a triangle's vertices, Richardson-
extrapolated from steps h and h/2 so that the truncation error, O(h^4), sits far
below the bar; rays within 1e-2 of an edge are excluded and counted) the same
bars at 1e-4."""
import numpy as np
import pytest

import oracle
import synthetic
from synthetic import rng as srng

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _run(w):
    from paper_2312_06538_gb300 import pipeline as pl
    p = pl.workload_pipeline(w)
    hp, bp = pl.workload_params(w)
    g = p.gbuffer_struct(p.gbuffer_to_device(w.gbuffer))
    lights = torch.from_numpy(w.lights).cuda() if w.lights.shape[0] else None
    p.run_fit(g, lights, hp, bp)
    return p


def _weights(n, seed=1005):
    z = srng.normal_array(seed, 3 * n).reshape(3, n)
    return z[0], z[1], z[2]


def _gpu_grads(p, gw):
    n = p.n()
    dev = p.device
    gt = torch.from_numpy(np.ascontiguousarray(gw[0], np.float32)).to(dev)
    gu = torch.from_numpy(np.ascontiguousarray(gw[1], np.float32)).to(dev)
    gv = torch.from_numpy(np.ascontiguousarray(gw[2], np.float32)).to(dev)
    gverts, gorig, gdir = p.backward(gt, gu, gv)
    torch.cuda.synchronize()
    return gverts.cpu().numpy(), gorig[:n].cpu().numpy(), gdir[:n].cpu().numpy()


def _gen_order_rays(w):
    return oracle.generate_rays(w.gbuffer, w.lights, w.shadow_cull)


def _close(got, ref, rel=1e-4):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    scale = np.abs(ref).max()
    if scale == 0:
        assert np.abs(got).max() == 0
        return
    assert np.linalg.norm(got - ref) <= rel * np.linalg.norm(ref), (np.linalg.norm(got - ref), np.linalg.norm(ref))
    assert (np.abs(got - ref) <= rel * np.abs(ref) + 1e-3 * scale).all()


@pytest.fixture(scope="module", params=[(5, 128), (2, 96)])
def case(request):
    cid, res = request.param
    w = synthetic.make(cid, res=res)
    p = _run(w)
    rays = _gen_order_rays(w)
    hits = p.hits_host()
    gw = _weights(p.n())
    return w, p, rays, hits, gw


def test_backward_matches_fp64_closed_form(case):
    w, p, rays, hits, gw = case
    tri = hits[0]
    assert (tri >= 0).sum() > 1000
    gv, go, gd = _gpu_grads(p, gw)
    rv, ro, rd = oracle.adjoint(rays, (tri, hits[1].astype(np.float64), hits[2].astype(np.float64),
                                       hits[3].astype(np.float64)), *gw, w.scene.verts)
    _close(gv, rv)
    _close(go, ro)
    _close(gd, rd)
    miss = tri < 0
    assert (go[miss] == 0).all() and (gd[miss] == 0).all()
    unhit = np.setdiff1d(np.arange(w.scene.n_tris), tri[tri >= 0])
    assert (gv[unhit] == 0).all()


def test_backward_is_deterministic(case):
    w, p, rays, hits, gw = case
    a = _gpu_grads(p, gw)
    b = _gpu_grads(p, gw)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def unit3(k):
    e = np.zeros(3)
    e[k] = 1.0
    return e


def richardson(f, h):
    """Central difference of f at 0, Richardson-extrapolated from steps h and h/2:
    (4 D(h/2) - D(h)) / 3 cancels the h^2 term of the truncation error."""
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


def test_backward_matches_central_differences():
    """FD on config 1 (2,050 triangles, 4,096 rays), FP64 forward with the hit fixed."""
    w = synthetic.make(1)
    p = _run(w)
    rays = _gen_order_rays(w)
    tri, _, _, _ = p.hits_host()
    gw = _weights(p.n(), seed=77)
    gv, go, gd = _gpu_grads(p, gw)
    hit = np.nonzero(tri >= 0)[0]
    V = w.scene.verts.astype(np.float64)
    h = 1e-3

    def solve(o, d, vv):
        A = np.stack([-d, vv[1] - vv[0], vv[2] - vv[0]], 1)
        return np.linalg.solve(A, o - vv[0])

    def loss_ray(i, o, d, vv):
        t, u, v = solve(o, d, vv)
        return gw[0][i] * t + gw[1][i] * u + gw[2][i] * v

    keep, excluded = [], 0
    fo, fd_ = np.zeros((hit.size, 3)), np.zeros((hit.size, 3))
    fv = np.zeros_like(V.reshape(-1, 9))
    for n_, i in enumerate(hit):
        o = np.array([rays["ox"][i], rays["oy"][i], rays["oz"][i]], np.float64)
        d = np.array([rays["dx"][i], rays["dy"][i], rays["dz"][i]], np.float64)
        vv = V[tri[i]]
        t, u, v = solve(o, d, vv)
        if min(u, v, 1 - u - v) < 1e-2:
            excluded += 1
            continue
        keep.append(n_)
        for k in range(3):
            fo[n_, k] = richardson(lambda x: loss_ray(i, o + x * unit3(k), d, vv), h)
            fd_[n_, k] = richardson(lambda x: loss_ray(i, o, d + x * unit3(k), vv), h)
        # vertex steps relative to the triangle's size (a fixed 1e-3 would move small triangles by
        # percent and put second-order terms above the tolerance)
        hv = h * min(np.linalg.norm(vv[1] - vv[0]), np.linalg.norm(vv[2] - vv[1]), np.linalg.norm(vv[0] - vv[2]))
        for c in range(9):
            def moved(x, c=c):
                a = vv.copy().reshape(-1)
                a[c] += x
                return loss_ray(i, o, d, a.reshape(3, 3))
            fv[tri[i], c] += richardson(moved, hv)
    keep = np.array(keep)
    assert keep.size > 100 and excluded < 0.5 * hit.size
    # vertex gradients: compare triangles whose hits were all kept
    bad_tris = np.unique(tri[hit[np.setdiff1d(np.arange(hit.size), keep)]]) if keep.size < hit.size else []
    ok_tris = np.setdiff1d(np.unique(tri[hit]), bad_tris)
    _close(go[hit[keep]], fo[keep], rel=1e-4)
    _close(gd[hit[keep]], fd_[keep], rel=1e-4)
    _close(gv[ok_tris], fv[ok_tris], rel=1e-4)


def test_autograd_function_matches_direct_call():
    from paper_2312_06538_gb300 import autograd as ag
    w = synthetic.make(5, res=64)
    rays = _gen_order_rays(w)
    n = rays["ox"].shape[0]
    cfg = ag.SceneRays(w.scene, max_rays=n, bundle=w.bundle, levels=w.levels, pads=w.build_pads(),
                       hash_lo=w.hash_lo, hash_hi=w.hash_hi)
    dev = cfg.p.device
    o = torch.from_numpy(np.stack([rays["ox"], rays["oy"], rays["oz"]], 1)).to(dev).requires_grad_()
    d = torch.from_numpy(np.stack([rays["dx"], rays["dy"], rays["dz"]], 1)).to(dev).requires_grad_()
    V = torch.from_numpy(w.scene.verts.copy()).to(dev).requires_grad_()
    types = torch.from_numpy(rays["type"]).to(dev)
    tmax = torch.from_numpy(rays["tmax"]).to(dev)
    t, u, v, tri = ag.closest_hit(o, d, V, types, tmax, cfg)
    wt, wu, wv = (torch.from_numpy(x.astype(np.float32)).to(dev) for x in _weights(n, seed=9))
    hitm = (tri >= 0).float()
    loss = ((wt * t + wu * u + wv * v) * hitm).sum()
    loss.backward()
    tri_np = tri.cpu().numpy()
    assert (tri_np >= 0).sum() > 500
    hits = (tri_np, t.detach().cpu().numpy().astype(np.float64), u.detach().cpu().numpy().astype(np.float64),
            v.detach().cpu().numpy().astype(np.float64))
    m = tri_np >= 0
    rv, ro, rd = oracle.adjoint(rays, hits, *(x * m for x in _weights(n, seed=9)), w.scene.verts)
    _close(V.grad.cpu().numpy().reshape(-1, 9), rv)
    _close(o.grad.cpu().numpy(), ro)
    _close(d.grad.cpu().numpy(), rd)


def test_backward_full_config5_against_fp64():
    """The adjoint workload at full size (config 5: 2^20 reflection rays of a 1024x1024
    all-mirror frame, 99,842 triangles): every ray's gradient and every triangle's summed
    gradient against the FP64 closed form, at 1e-4.  The hit assignment is the GPU's forward
    pass (held fixed, as the adjoint defines); a seeded sample of it is checked against the
    oracle's brute force, and (t, u, v) of every hit are re-solved in FP64."""
    from tests import parity
    w = synthetic.make(5)
    p = _run(w)
    rays = _gen_order_rays(w)
    n = p.n()
    assert n == rays["ox"].shape[0] == 1 << 20
    tri, _, _, _ = p.hits_host()
    hit = np.nonzero(tri >= 0)[0]
    assert hit.size > 100_000
    idx = np.sort(np.random.default_rng(5).choice(n, size=600, replace=False))
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in rays.items()}
    rep = parity.compare_hits(tuple(x[idx] for x in p.hits_host()), oracle.bruteforce(sub, w.scene.verts), sub,
                              w.scene.verts)
    parity.check_report(rep)
    # FP64 (t, u, v) of every hit: A (t, u, v) = o - v0, A = [-d | e1 | e2]
    V = w.scene.verts.astype(np.float64)[tri[hit]]
    o = np.stack([rays["ox"], rays["oy"], rays["oz"]], 1).astype(np.float64)[hit]
    d = np.stack([rays["dx"], rays["dy"], rays["dz"]], 1).astype(np.float64)[hit]
    A = np.stack([-d, V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]], 2)
    tuv = np.linalg.solve(A, (o - V[:, 0])[:, :, None])[:, :, 0]
    t64, u64, v64 = (np.zeros(n) for _ in range(3))
    t64[hit], u64[hit], v64[hit] = tuv[:, 0], tuv[:, 1], tuv[:, 2]
    gw = _weights(n)
    gv, go, gd = _gpu_grads(p, gw)
    rv, ro, rd = oracle.adjoint(rays, (tri, t64, u64, v64), *gw, w.scene.verts)
    _close(gv, rv)
    _close(go, ro)
    _close(gd, rd)
