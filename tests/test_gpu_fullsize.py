"""Full-size workloads in the launch configuration bench.py times.

Config 2 (512x512, 60,162 triangles, ~0.5 M rays, B = 16, L = 4): every ray
against the oracle (keys, order, hierarchy containment, per-level pair counts
of the oracle's own full traversal, closest hits).  Config 3 (1024x1024,
202,764 triangles, ~3 M rays): keys and order bit-exact, containment, the
paper's counting identities, a seeded sample of rays against the oracle's
brute force, and the hierarchy result bit-identical to the GPU brute force
for every ray; on the central 256x256 crop of its frame (whole scene), per-level
pair counts and every closest hit against the oracle's full CRSH."""
import numpy as np
import pytest

import oracle
import synthetic
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gpu(w, pair_capacity=None):
    from paper_2312_06538_gb300 import pipeline as pl
    p = pl.workload_pipeline(w, pair_capacity=pair_capacity)
    hp, bp = pl.workload_params(w)
    g = p.gbuffer_struct(p.gbuffer_to_device(w.gbuffer))
    lights = torch.from_numpy(w.lights).cuda() if w.lights.shape[0] else None
    c = p.run_fit(g, lights, hp, bp)
    return p, c


def _front(w):
    """Oracle ray generation, hash and sort (fast at any size)."""
    rays = oracle.generate_rays(w.gbuffer, w.lights, w.shadow_cull)
    keys = oracle.hash_keys(rays, w.hash_lo, w.hash_hi)
    perm = oracle.stable_sort(keys)
    return rays, keys, perm


@pytest.fixture(scope="module")
def c2():
    w = synthetic.make(2)
    p, c = _gpu(w)
    ref = oracle.run_crsh(w.gbuffer, w.lights, w.shadow_cull, w.hash_lo, w.hash_hi, w.scene, w.bundle, w.levels,
                          w.build_pads())
    return w, p, c, ref


def test_c2_keys_order_and_counts(c2):
    w, p, c, ref = c2
    got = p.sorted_rays()
    assert c["rays"] == ref["counters"]["rays"] > 400_000
    assert c["chunks"] == ref["counters"]["chunks"]
    assert np.array_equal(got["ray_id"], ref["perm"])
    assert np.array_equal(got["keys"], ref["keys"][ref["perm"]])
    rc = ref["counters"]
    for l in range(w.levels):
        assert parity.within(c["hits"][l], rc["hits"][l], 1e-3), (l, c["hits"], rc["hits"])
        assert parity.within(c["tests"][l], rc["tests"][l], 1e-3), (l, c["tests"], rc["tests"])
    assert parity.within(c["final_tests"], rc["final_tests"], 1e-3)
    assert c["mesh_tests"] == rc["mesh_tests"]


def test_c2_hierarchy_contains_its_rays(c2):
    w, p, c, ref = c2
    lv = p.levels_host()
    counts = [x[0].shape[0] for x in lv]
    bad, worst = oracle.check_hierarchy(ref["sorted_rays"], w.bundle, counts, np.concatenate([x[0] for x in lv]),
                                        np.concatenate([x[1] for x in lv]))
    assert bad == 0, (bad, worst)


def test_c2_closest_hits_every_ray(c2):
    w, p, c, ref = c2
    rep = parity.compare_hits(p.hits_host(), ref["hits"], ref["rays"], w.scene.verts)
    parity.check_report(rep)
    idx = np.random.default_rng(2).choice(c["rays"], size=1500, replace=False)
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in ref["rays"].items()}
    assert np.array_equal(oracle.bruteforce(sub, w.scene.verts)[0], ref["hits"][0][idx])


def test_c2_equals_gpu_bruteforce(c2):
    w, p, c, ref = c2
    a = [x.copy() for x in p.hits_host()]
    p.bruteforce()
    for x, y in zip(a, p.hits_host()):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


@pytest.fixture(scope="module")
def c3():
    w = synthetic.make(3)
    p, c = _gpu(w, pair_capacity=1 << 27)
    return w, p, c


def test_c3_keys_order_identities_and_containment(c3):
    w, p, c = c3
    rays, keys, perm = _front(w)
    got = p.sorted_rays()
    assert c["rays"] == rays["ox"].shape[0] > 2_000_000
    assert np.array_equal(got["ray_id"], perm)
    assert np.array_equal(got["keys"], keys[perm])
    assert c["chunks"] == oracle.chunk_count(keys)
    for l in range(w.levels - 1):
        assert c["tests_paper"][l] == w.bundle * c["hits"][l + 1]
    assert c["final_tests_paper"] == w.bundle * c["hits"][0]
    srays = oracle.gather(rays, perm)
    lv = p.levels_host()
    bad, worst = oracle.check_hierarchy(srays, w.bundle, [x[0].shape[0] for x in lv],
                                        np.concatenate([x[0] for x in lv]), np.concatenate([x[1] for x in lv]))
    assert bad == 0, (bad, worst)


def test_c3_sampled_hits_and_gpu_bruteforce(c3):
    w, p, c = c3
    rays, _, _ = _front(w)
    hits = [x.copy() for x in p.hits_host()]
    idx = np.sort(np.random.default_rng(3).choice(c["rays"], size=800, replace=False))
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in rays.items()}
    bf = oracle.bruteforce(sub, w.scene.verts)
    rep = parity.compare_hits(tuple(h[idx] for h in hits), bf, sub, w.scene.verts)
    parity.check_report(rep)
    assert rep["hits"] > 100
    p.bruteforce()
    for x, y in zip(hits, p.hits_host()):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


@pytest.mark.parametrize("compress", [True, False])
def test_sort_at_12m_rays_bit_exact(compress):
    """The hash/sort path at the size of the HBM sweep (4 perturbed tiles of the config-3 frame,
    12.8 M rays, 3,100 radix tiles per pass): keys and order bit-exact against the oracle's
    generation, hash and stable sort, with and without compression."""
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(3)
    g = synthetic.tiled_gbuffer(w, 4)
    npx = g["hit"].shape[0]
    p = pl.Pipeline(w.scene, max_pixels=npx, n_lights=w.lights.shape[0], bundle=16, levels=4,
                    ray_capacity=npx * 4, pair_capacity=1 << 16, device="cuda")
    hp = pl.hash_params(w.hash_lo, w.hash_hi, shadow_cull=w.shadow_cull, compress=compress)
    gs = p.gbuffer_struct(p.gbuffer_to_device(g))
    p.hash_sort(gs, torch.from_numpy(w.lights).cuda(), hp, torch.cuda.current_stream().cuda_stream)
    c = p.read_counters()
    assert c["status"] == 0
    rays = oracle.generate_rays(g, w.lights, w.shadow_cull)
    keys = oracle.hash_keys(rays, w.hash_lo, w.hash_hi)
    perm = oracle.stable_sort(keys)
    n = p.n()
    assert n == keys.shape[0] > 12_000_000
    got = p.sorted_rays()
    assert np.array_equal(got["keys"], keys[perm])
    assert np.array_equal(got["ray_id"], perm.astype(np.uint32))
    for k in ("ox", "dx", "tmax"):
        assert np.array_equal(got[k].view(np.uint32), rays[k][perm].view(np.uint32)), k
    if compress:
        assert c["chunks"] == oracle.chunk_count(keys)


def test_build_at_12m_rays_equals_its_prefix_build():
    """The level-1 build at 12.8 M rays (800 K nodes: every warp builds several blocks of 32 nodes,
    which takes the fully unrolled fold and sphere tree and the 16-byte staging loads) against the
    build of a 153,600-ray prefix of the same sorted rays (one block per warp: the rolled loops):
    the nodes the two share, at level 1 and at level 2 (merged in the level-1 kernel), are
    bit-identical, since every node depends on its own rays only."""
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(3)
    g = synthetic.tiled_gbuffer(w, 4)
    npx = g["hit"].shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    p = pl.Pipeline(w.scene, max_pixels=npx, n_lights=w.lights.shape[0], bundle=16, levels=4,
                    ray_capacity=npx * 4, pair_capacity=1 << 16, device="cuda")
    hp = pl.hash_params(w.hash_lo, w.hash_hi, shadow_cull=w.shadow_cull)
    bp = pl.build_params(16, 4, w.build_pads())
    p.hash_sort(p.gbuffer_struct(p.gbuffer_to_device(g)), torch.from_numpy(w.lights).cuda(), hp, stream)
    p.build(bp, stream)
    assert p.read_counters()["status"] == 0
    n = p.n()
    assert n > 12_000_000
    big = p.levels_host()
    P = 16 * 32 * 300
    q = pl.Pipeline(w.scene, max_pixels=1, n_lights=w.lights.shape[0], bundle=16, levels=4, ray_capacity=P,
                    pair_capacity=1 << 16, device="cuda")
    for k in pl.RAY_FIELDS:
        q.rays_t[k][:P].copy_(p.rays_t[k][:P])
    q.n_rays.fill_(P)
    q.build(bp, stream)
    small = q.levels_host()
    assert small[0][0].shape[0] == P // 16 and small[1][0].shape[0] == P // 256
    for lvl, m in ((0, P // 16), (1, P // 256)):
        for a, b in zip(big[lvl], small[lvl]):
            assert np.array_equal(a[:m].view(np.uint32), b[:m].view(np.uint32)), lvl


def test_c3_crop_level_counts_and_hits_against_the_oracle():
    """The config-3 scene at full size (202,764 triangles in 65 meshes, 4 lights) seen through
    the central 256x256 crop of its frame: keys and order bit-exact, per-level pair counts
    (hits, tests, paper-convention tests) within 0.1 % of the oracle's FP64 traversal, mesh
    tests exact, and every closest hit against the oracle's."""
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(3)
    side = 256
    x0, y0 = (w.width - side) // 2, (w.height - side) // 2
    idx = (np.arange(y0, y0 + side)[:, None] * w.width + np.arange(x0, x0 + side)[None, :]).reshape(-1)
    g = {k: np.ascontiguousarray(v[idx]) for k, v in w.gbuffer.items()}
    p = pl.Pipeline(w.scene, max_pixels=side * side, n_lights=w.lights.shape[0], bundle=w.bundle, levels=w.levels,
                    device="cuda")
    hp, bp = pl.workload_params(w)
    c = p.run_fit(p.gbuffer_struct(p.gbuffer_to_device(g)), torch.from_numpy(w.lights).cuda(), hp, bp)
    ref = oracle.run_crsh(g, w.lights, w.shadow_cull, w.hash_lo, w.hash_hi, w.scene, w.bundle, w.levels,
                          w.build_pads())
    rc = ref["counters"]
    assert c["rays"] == rc["rays"] > 150_000
    assert c["chunks"] == rc["chunks"]
    got = p.sorted_rays()
    assert np.array_equal(got["ray_id"], ref["perm"])
    assert np.array_equal(got["keys"], ref["keys"][ref["perm"]])
    assert c["mesh_tests"] == rc["mesh_tests"]
    for l in range(w.levels):
        assert parity.within(c["hits"][l], rc["hits"][l], 1e-3), (l, c["hits"], rc["hits"])
        assert parity.within(c["tests"][l], rc["tests"][l], 1e-3), (l, c["tests"], rc["tests"])
        assert parity.within(c["tests_paper"][l], rc["tests_paper"][l], 1e-3)
    assert parity.within(c["final_tests"], rc["final_tests"], 1e-3)
    print(f"config-3 crop: GPU hits per level {c['hits']}, oracle {rc['hits']}; final tests "
          f"{c['final_tests']} vs {rc['final_tests']}")
    rep = parity.compare_hits(p.hits_host(), ref["hits"], ref["rays"], w.scene.verts)
    parity.check_report(rep)
