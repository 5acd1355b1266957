"""Level 1 in word form (crsh_traverse with level1_words, crsh_closest_hit
reading the traversal's last ballots) against the list form on the same
inputs: hits bit for bit, and the level counts and final-test counts equal.
Covers every bundle size, one to six levels, the unsorted no-mesh-culling
mode, a frame's capacity retry, both full-size frames and the oracle on a
sample of config 3."""
import dataclasses

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _both(w, sort=True, mesh_cull=True, pair_capacity=None):
    from paper_2312_06538_gb300 import pipeline as pl
    out = []
    for words in (False, True):
        p = pl.workload_pipeline(w, pair_capacity=pair_capacity, level1_words=words)
        hp, bp = pl.workload_params(w, sort=sort)
        g = p.gbuffer_struct(p.gbuffer_to_device(w.gbuffer))
        lights = torch.from_numpy(w.lights).cuda() if w.lights.shape[0] else None
        c = p.run_fit(g, lights, hp, bp, mesh_cull=mesh_cull)
        out.append((p, c))
    return out


def _same(a, b):
    (pa, ca), (pb, cb) = a, b
    assert not pa.pairs.words.valid and (pb.pairs.words.valid or pb.levels < 2)
    for x, y in zip(pa.hits_host(), pb.hits_host()):
        assert np.array_equal(np.asarray(x).view(np.uint32), np.asarray(y).view(np.uint32))
    for k in ("rays", "tests", "hits", "tests_paper", "mesh_tests", "mesh_hits", "final_tests", "final_hits",
              "final_tests_paper"):
        assert ca[k] == cb[k], (k, ca[k], cb[k])
    assert cb["status"] == 0


@pytest.mark.parametrize("cid,res", [(1, None), (2, 96), (2, 200), (5, 64), (3, 128)])
def test_words_equal_list_form(cid, res):
    w = synthetic.make(cid, res=res) if res else synthetic.make(cid)
    _same(*_both(w))


@pytest.mark.parametrize("B,L", [(2, 3), (4, 2), (8, 5), (32, 2), (16, 1), (64, 2), (64, 3), (4, 6)])
def test_words_every_bundle_and_depth(B, L):
    w = dataclasses.replace(synthetic.make(2, res=64), bundle=B, levels=L)
    _same(*_both(w))


def test_words_unsorted_no_mesh_cull():
    w = synthetic.make(2, res=48)
    _same(*_both(w, sort=False, mesh_cull=False))


def test_words_after_a_capacity_retry():
    w = synthetic.make(2, res=96)
    _same(*_both(w, pair_capacity=4096))


def test_words_full_size_config2():
    _same(*_both(synthetic.make(2)))


def test_words_full_size_config3_against_oracle_sample():
    import oracle
    from tests import parity
    w = synthetic.make(3)
    a, b = _both(w, pair_capacity=1 << 27)
    _same(a, b)
    pb = b[0]
    rays = oracle.generate_rays(w.gbuffer, w.lights, w.shadow_cull)
    n = rays["ox"].shape[0]
    assert n == b[1]["rays"]
    idx = np.sort(np.random.default_rng(2024).choice(n, size=800, replace=False))
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in rays.items()}
    got = tuple(np.asarray(x)[idx] for x in pb.hits_host())
    rep = parity.compare_hits(got, oracle.bruteforce(sub, w.scene.verts), sub, w.scene.verts)
    parity.check_report(rep, label="config 3, word form, 800 sampled rays")
    assert rep["hits"] > 100


def test_timed_closest_hit_matches_the_plain_call():
    """crsh_closest_hit_timed (the bench's kernel timing) gives the plain call's hits and counters bit
    for bit, in both forms of level 1, and a positive kernel time."""
    w = synthetic.make(2, res=96)
    for p, c in _both(w):
        s = torch.cuda.current_stream().cuda_stream
        ref = [np.array(x, copy=True) for x in p.hits_host()]
        ms = p.closest_hit_timed(s)
        assert ms > 0.0
        for x, y in zip(ref, p.hits_host()):
            assert np.array_equal(np.asarray(x).view(np.uint32), np.asarray(y).view(np.uint32))
        c2 = p.read_counters()
        for k in ("final_tests", "final_hits", "final_tests_paper", "status"):
            assert c2[k] == c[k], (k, c2[k], c[k])
