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


def _pipeline(words=False):
    import synthetic
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(2, res=96)
    p = pl.workload_pipeline(w, level1_words=words)
    hp, bp = pl.workload_params(w)
    g = p.gbuffer_struct(p.gbuffer_to_device(w.gbuffer))
    lights = torch.from_numpy(w.lights).cuda()
    c = p.run_fit(g, lights, hp, bp)
    return p, c


@pytest.mark.parametrize("words", [False, True])
def test_noalloc_matches_workspace_call_twice_in_a_row(words):
    from paper_2312_06538_gb300 import crsh as C
    p, c = _pipeline(words)
    assert bool(p.pairs.words.valid) == words
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
        # the same deterministic kernels run on the same inputs: the results are
        # compared bit for bit, so a scratch-aliasing error of any size shows
        got = p.hits_host()
        for x, y in zip(got, ref):
            assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


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


def test_noalloc_clamps_a_device_count_above_the_capacity():
    """A device ray count larger than rays->capacity must not make the kernels walk past
    the shared array: they stop at the capacity and report CRSH_ERR_CAPACITY."""
    from paper_2312_06538_gb300 import crsh as C
    p, c = _pipeline()
    ref = [x.copy() for x in p.hits_host()]
    n = p.n()
    stream = torch.cuda.current_stream().cuda_stream
    # slots past the real rays get valid generation indices (the hits are scattered
    # through them), then the count is raised past the capacity
    cap = p.ray_capacity
    p.rays_t["ray_id"][n:cap] = torch.arange(n, cap, dtype=torch.int64, device="cuda").to(torch.uint32)
    p.n_rays.fill_(cap + 1000)
    C.crsh_closest_hit_noalloc(p.hier, p.rays, p.n_rays.data_ptr(), p.scene, p.pairs, p.hits,
                               p.counters.data_ptr(), stream)
    torch.cuda.synchronize()
    st = p.read_counters()["status"]
    p.n_rays.fill_(n)
    assert st == C.ERR_CAPACITY
    # the real rays still got their hits
    got = p.hits_host()
    assert np.array_equal(got[0], ref[0])
