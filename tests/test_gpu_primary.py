"""NEXT row f3 on the GPU: camera rays, primary visibility through the hierarchy, first-hit
buffers, the next bounce, and the per-frame mesh update.

- Camera rays and first-hit buffers are bit-exact against the oracle (same FP32 operation
  order; first-hit buffers from the same hits).
- Primary visibility through CRSH (camera rays -> build -> traverse -> closest hit) hits the
  same triangles as the FP64 software rasteriser except where the FP32 ray direction decides an
  edge (< 0.5 % of pixels), and equals the GPU brute force bit for bit.
- The next bounce (first-hit buffer of secondary rays -> crsh_hash_sort) equals the oracle's,
  ray for ray, wherever both sides start from the same hit.
- The mesh update moves vertices like numpy and keeps every moved vertex inside its sphere."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pipe(w, capacity=None):
    from paper_2312_06538_gb300 import pipeline as pl
    n = w.width * w.height
    return pl.Pipeline(w.scene, max_pixels=n, n_lights=max(1, w.lights.shape[0]), bundle=16, levels=4,
                       ray_capacity=capacity or max(n, 4 * n), device="cuda")


def _cam(p, w):
    return p.camera_struct(w.camera, w.width, w.height)


@pytest.mark.parametrize("cid,res", [(2, 512), (1, 61)])
def test_camera_rays_bit_exact(cid, res):
    w = synthetic.make(cid, res=res)
    p = _pipe(w)
    p.primary(_cam(p, w), torch.cuda.current_stream().cuda_stream)
    n = p.n()
    assert n == w.width * w.height
    got = p.sorted_rays()
    ref = oracle.primary_rays(w.camera, w.width, w.height)
    for k in ("ox", "oy", "oz", "dx", "dy", "dz"):
        assert np.array_equal(got[k].view(np.uint32), ref[k].view(np.uint32)), k
    assert np.array_equal(got["pixel"], ref["pixel"]) and np.array_equal(got["ray_id"], ref["pixel"])
    assert np.all(np.isinf(got["tmax"])) and np.all(got["type"] == 3)


def test_first_hit_buffer_bit_exact_from_the_same_hits():
    w = synthetic.make(1)
    p = _pipe(w)
    p.primary(_cam(p, w), torch.cuda.current_stream().cuda_stream)
    ref_rays = oracle.primary_rays(w.camera, w.width, w.height)
    rays = {**ref_rays, "tmax": np.full(ref_rays["ox"].shape, np.inf, np.float32)}
    tri, t, u, v = oracle.bruteforce(rays, w.scene.verts)
    # hits in ray_id (pixel) order, as crsh_closest_hit writes them
    order = np.argsort(ref_rays["pixel"])
    n = w.width * w.height
    p.hit_tri[:n] = torch.from_numpy(tri[order].astype(np.int32)).cuda()
    p.hit_t[:n] = torch.from_numpy(t[order].astype(np.float32)).cuda()
    mat = torch.from_numpy(w.scene.tri_material.astype(np.int32)).cuda()
    g, gs = p.gbuffer_out(n)
    p.gbuffer_from_hits(mat, gs)
    torch.cuda.synchronize()
    by_pixel = {k: np.ascontiguousarray(v_[order]) for k, v_ in ref_rays.items()}
    ref = oracle.gbuffer_from_hits(by_pixel, tri[order], t[order].astype(np.float32), w.scene.verts,
                                   w.scene.tri_material)
    for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz"):
        assert np.array_equal(g[k].cpu().numpy().view(np.uint32), ref[k].view(np.uint32)), k
    assert np.array_equal(g["material"].cpu().numpy().view(np.uint32), ref["material"])
    assert np.array_equal(g["hit"].cpu().numpy(), ref["hit"])


def test_primary_visibility_through_the_hierarchy():
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(2)
    p = _pipe(w)
    _, bp = pl.workload_params(w)
    cam = _cam(p, w)
    for _ in range(6):   # size the pair lists
        p.run_primary(cam, bp)
        c = p.read_counters()
        if c["status"] == 2 and c["needed_pairs"] > p.pair_capacity:
            p.set_pair_capacity(int(1.25 * c["needed_pairs"]) + 1024)
            continue
        break
    assert c["status"] == 0
    n = w.width * w.height
    tri = p.hit_tri[:n].cpu().numpy().view(np.int32)
    agree = tri == w.primary_tri
    assert agree.mean() > 0.995, agree.mean()
    # the disagreements sit on edges or silhouettes: the raster's own triangle is hit by an
    # FP64 ray within 1e-3 (barycentric) of one of its edges, or the raster saw background
    bad = np.nonzero(~agree)[0]
    verts = w.scene.verts.astype(np.float64)
    cam = w.camera
    near_edge = 0
    for px in bad[:2000]:
        t_r = w.primary_tri[px]
        x, y = px % w.width, px // w.width
        sx = (2 * (x + 0.5) / w.width - 1) * cam[12]
        sy = (1 - 2 * (y + 0.5) / w.height) * cam[13]
        d = cam[3:6] + sx * cam[6:9] + sy * cam[9:12]
        d /= np.linalg.norm(d)
        cand = [t_r, tri[px]]
        ok = False
        for tt in cand:
            if tt < 0:
                continue
            a, b, c_ = verts[tt]
            A = np.stack([-d, b - a, c_ - a], 1)
            try:
                s_, u_, v_ = np.linalg.solve(A, cam[0:3] - a)
            except np.linalg.LinAlgError:
                continue
            if min(u_, v_, 1 - u_ - v_) > -2e-3 and min(u_, v_, 1 - u_ - v_) < 2e-3:
                ok = True
        near_edge += ok
    assert near_edge >= 0.9 * min(len(bad), 2000), (near_edge, len(bad))
    # the hierarchy path equals the brute force on the same camera rays, bit for bit
    crsh = [x.copy() for x in p.hits_host()]
    p.bruteforce()
    bf = p.hits_host()
    for a, b in zip(crsh, bf):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    # and the first-hit buffer matches the raster's positions where both hit the same triangle
    mat = torch.from_numpy(w.scene.tri_material.astype(np.int32)).cuda()
    g, gs = p.gbuffer_out(n)
    p.hit_tri[:n] = torch.from_numpy(crsh[0].astype(np.int32)).cuda()
    p.hit_t[:n] = torch.from_numpy(crsh[1]).cuda()
    p.gbuffer_from_hits(mat, gs)
    both = agree & (tri >= 0)
    for k in ("px", "py", "pz"):
        assert np.allclose(g[k].cpu().numpy()[both], w.gbuffer[k][both], rtol=1e-4, atol=1e-4), k
    assert np.array_equal(g["material"].cpu().numpy().view(np.uint32)[both], w.gbuffer["material"][both])


def test_next_bounce_matches_the_oracle():
    """Secondary rays of a 96x96 config-2 frame: first-hit buffer of their hits, then
    crsh_hash_sort of that buffer (the next bounce).  Where the GPU and the oracle hit the same
    triangle at the same FP32 t, the buffer entries and every ray generated from them are
    bit-identical."""
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(2, res=96)
    p = pl.workload_pipeline(w)
    hp, bp = pl.workload_params(w)
    gs_in = p.gbuffer_struct(p.gbuffer_to_device(w.gbuffer))
    lights = torch.from_numpy(w.lights).cuda()
    p.run_fit(gs_in, lights, hp, bp)
    n = p.n()
    tri_g, t_g, _, _ = p.hits_host()
    mat = torch.from_numpy(w.scene.tri_material.astype(np.int32)).cuda()
    g, gs = p.gbuffer_out(n)
    p.gbuffer_from_hits(mat, gs)
    torch.cuda.synchronize()
    gpu_gb = {k: v_.cpu().numpy() for k, v_ in g.items()}
    gpu_gb["material"] = gpu_gb["material"].view(np.uint32)
    # oracle: its own secondary rays and hits, then its first-hit buffer and next bounce
    ref = oracle.run_crsh(w.gbuffer, w.lights, w.shadow_cull, w.hash_lo, w.hash_hi, w.scene, w.bundle,
                          w.levels, w.build_pads())
    tri_o, t_o = ref["hits"][0], ref["hits"][1].astype(np.float32)
    ref_gb = oracle.gbuffer_from_hits(ref["rays"], tri_o, t_o, w.scene.verts, w.scene.tri_material)
    same = (tri_o == tri_g) & (t_o.view(np.uint32) == t_g.view(np.uint32))
    assert same.mean() > 0.99
    for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz", "material", "hit"):
        a, b = gpu_gb[k][same], ref_gb[k][same]
        assert np.array_equal(a.view(np.uint32) if a.dtype == np.float32 else a,
                              b.view(np.uint32) if b.dtype == np.float32 else b), k
    # next bounce on the GPU
    q = pl.Pipeline(w.scene, max_pixels=n, n_lights=w.lights.shape[0], bundle=16, levels=4, device="cuda")
    q.hash_sort(q.gbuffer_struct(g), lights, hp, torch.cuda.current_stream().cuda_stream)
    nb = q.sorted_rays()
    ref_nb = oracle.generate_rays(ref_gb, w.lights, w.shadow_cull)
    # compare the rays generated from identical buffer entries, in generation order
    keep_g = np.isin(nb["pixel"], np.nonzero(same)[0])
    keep_o = np.isin(ref_nb["pixel"], np.nonzero(same)[0])
    order_g = np.argsort(nb["ray_id"][keep_g], kind="stable")
    assert keep_g.sum() == keep_o.sum() > 1000
    for k in ("ox", "oy", "oz", "dx", "dy", "dz", "tmax"):
        a = nb[k][keep_g][order_g]
        b = ref_nb[k][keep_o]
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), k
    assert np.array_equal(nb["pixel"][keep_g][order_g], ref_nb["pixel"][keep_o])


def test_mesh_update_moves_vertices_and_keeps_them_in_their_spheres():
    from paper_2312_06538_gb300 import crsh as C
    w = synthetic.make(2, res=32)
    p = _pipe(w)
    M = w.scene.n_meshes
    rng = np.random.default_rng(5)
    xf = np.zeros((M, 12), np.float32)
    for m in range(M):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        a, b, c, d = q
        R = np.array([[1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)],
                      [2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)],
                      [2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)]]) * rng.uniform(0.5, 2)
        xf[m, [0, 1, 2, 4, 5, 6, 8, 9, 10]] = R.reshape(-1)
        xf[m, [3, 7, 11]] = rng.uniform(-1, 1, 3)
    xf_t = torch.from_numpy(xf.reshape(-1)).cuda()
    out_v = {k: torch.empty_like(t_) for k, t_ in p.scene_t.items()}
    out_s = torch.empty_like(p.mesh_sphere)
    so = C.crsh_scene_out(*[out_v[k].data_ptr() for k in ("v0x", "v0y", "v0z", "v1x", "v1y", "v1z", "v2x", "v2y",
                                                          "v2z")], out_s.data_ptr())
    C.crsh_transform_meshes(p.scene, xf_t.data_ptr(), so, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    first = w.scene.mesh_first_tri.astype(np.int64)
    mesh = np.searchsorted(first, np.arange(w.scene.n_tris), side="right") - 1
    V = w.scene.verts.astype(np.float64)
    A = xf.astype(np.float64).reshape(M, 3, 4)
    moved = np.einsum("tij,tkj->tki", A[mesh][:, :, :3], V) + A[mesh][:, None, :, 3]
    got = np.stack([np.stack([out_v[f"v{k}{a}"].cpu().numpy() for a in "xyz"], 1) for k in range(3)], 1)
    assert np.allclose(got, moved, rtol=1e-5, atol=1e-5)
    sph = out_s.cpu().numpy().astype(np.float64)
    for m in range(M):
        pts = moved[first[m]:first[m + 1]].reshape(-1, 3)
        assert np.all(np.linalg.norm(pts - sph[m, :3], axis=1) <= sph[m, 3]), m


def test_shading_matches_the_oracle_where_the_hits_agree():
    """crsh_shade on a 96x96 config-2 frame: bit-exact against the oracle's shading for every
    pixel whose secondary rays all hit the same triangles on both sides (the only input the
    two do not share)."""
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(2, res=96)
    p = pl.workload_pipeline(w)
    hp, bp = pl.workload_params(w)
    gs = p.gbuffer_struct(p.gbuffer_to_device(w.gbuffer))
    lights = torch.from_numpy(w.lights).cuda()
    p.run_fit(gs, lights, hp, bp)
    mat = torch.from_numpy(w.scene.tri_material.astype(np.int32)).cuda()
    color = p.shade(gs, lights, mat).cpu().numpy()
    tri_g = p.hits_host()[0]
    ref = oracle.run_crsh(w.gbuffer, w.lights, w.shadow_cull, w.hash_lo, w.hash_hi, w.scene, w.bundle,
                          w.levels, w.build_pads())
    tri_o = ref["hits"][0]
    rc = oracle.shade(w.gbuffer, ref["rays"], tri_o, w.scene.tri_material, w.lights.shape[0])
    px = ref["rays"]["pixel"]
    bad = np.zeros(w.width * w.height, bool)
    bad[px[tri_o != tri_g]] = True
    assert (~bad).mean() > 0.99
    assert np.array_equal(color[~bad].view(np.uint32), rc[~bad].view(np.uint32))
    assert np.all(np.isfinite(color)) and color.min() >= 0.0
