"""crsh_closest_hit_noalloc: the closest-hit call for callers that cannot
allocate device memory (graph capture, allocator-free real-time loops, hosts
that own all device memory).  It uses a fixed array inside the library
instead of a workspace; its results must equal those of crsh_closest_hit.
This file is collected last so that a failure here comes after every other
test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pipeline():
    import synthetic
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(2, res=96)
    p = pl.workload_pipeline(w)
    hp, bp = pl.workload_params(w)
    g = p.gbuffer_struct(p.gbuffer_to_device(w.gbuffer))
    lights = torch.from_numpy(w.lights).cuda()
    c = p.run_fit(g, lights, hp, bp)
    return p, c


def test_noalloc_matches_workspace_call_twice_in_a_row():
    from paper_2312_06538_gb300 import crsh as C
    p, c = _pipeline()
    ref = [x.copy() for x in p.hits_host()]
    assert (ref[0] >= 0).sum() > 0
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        # poison the outputs so that a call that writes nothing cannot pass
        for t in (p.hit_tri, p.hit_t, p.hit_u, p.hit_v):
            t.fill_(-7)
        C.crsh_closest_hit_noalloc(p.hier, p.rays, p.n_rays.data_ptr(), p.scene, p.pairs, p.hits,
                                   p.counters.data_ptr(), stream)
        c2 = p.read_counters()
        assert c2["status"] == C.OK
        assert c2["final_tests"] == c["final_tests"] and c2["final_hits"] == c["final_hits"]
        tri, t, u, v = p.hits_host()
        assert np.array_equal(tri, ref[0])
        hit = tri >= 0
        assert np.allclose(t[hit], ref[1][hit], rtol=1e-5, atol=0)
        assert np.allclose(u[hit], ref[2][hit], rtol=0, atol=1e-5)
        assert np.allclose(v[hit], ref[3][hit], rtol=0, atol=1e-5)
        assert (t[~hit] == 0).all()


def test_noalloc_rejects_more_rays_than_its_array_holds():
    import ctypes
    from paper_2312_06538_gb300 import crsh as C
    p, _ = _pipeline()
    big = C.crsh_rays.from_buffer_copy(p.rays)
    big.capacity = C.NOALLOC_MAX_RAYS + 1
    stream = torch.cuda.current_stream().cuda_stream
    rc = C.load().crsh_closest_hit_noalloc(ctypes.byref(p.hier), ctypes.byref(big), C.P(p.n_rays.data_ptr()),
                                           ctypes.byref(p.scene), ctypes.byref(p.pairs), ctypes.byref(p.hits),
                                           C.P(p.counters.data_ptr()), C.P(stream))
    assert rc == C.ERR_INVALID_ARG
    torch.cuda.synchronize()
