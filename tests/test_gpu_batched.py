"""Batched pipeline (one CUDA graph over several streams, autotuned B and L per
batch-size class) against the plain per-batch pipeline: identical hits, bit
for bit, for every batch, across graph replays."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _batches(spec):
    import synthetic
    from paper_2312_06538_gb300 import batched as bt
    out, meta = [], []
    for n, k in spec:
        res = max(16, int(math.ceil(math.sqrt(n))))
        while True:
            w = synthetic.config4_frame(k, res)
            rays, got = bt.secondary_rays(w.scene, w.gbuffer, w.lights, n, w.hash_lo, w.hash_hi)
            if got >= n:
                break
            res = int(res * 1.3) + 1
        out.append((w.scene, rays, n))
        meta.append(w)
    return out, meta


def test_batched_graph_equals_plain_bitwise():
    from paper_2312_06538_gb300 import batched as bt
    from paper_2312_06538_gb300 import pipeline as pl
    spec = [(2100, 0), (9000, 3), (33000, 1), (5000, 2), (60000, 3), (2500, 1)]
    batches, meta = _batches(spec)
    by_scene = {id(w.scene): w for w in meta}
    pads_of = lambda s: by_scene[id(s)].build_pads()  # noqa: E731
    hp_of = lambda s: pl.hash_params(by_scene[id(s)].hash_lo, by_scene[id(s)].hash_hi)  # noqa: E731
    tuner = bt.Autotuner(bundles=(8, 16), depths=(2, 4), reps=1)
    bat = bt.BatchedCRSH(batches, pads_of, hp_of, tuner=tuner, n_streams=4)
    plain = bt.PlainBatches(batches, pads_of, hp_of)
    plain.run()
    bat.capture()
    for rep in range(2):
        bat.replay()
        torch.cuda.synchronize()
        assert bat.check_status() == []
        for a, b in zip(bat.runs, plain.runs):
            for x, y in zip(a.hits(), b.hits()):
                assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    assert set(tuner.table) == {bt.Autotuner.size_class(n) for n, _ in spec}
    assert all((b, l) in [(8, 2), (8, 4), (16, 2), (16, 4)] and blk in (128, 256, 512)
               for b, l, blk in tuner.table.values())
    assert sum(int((r.hits()[0] >= 0).sum().item()) for r in bat.runs) > 1000


def test_batched_hits_match_the_oracle_on_every_batch():
    """Every batch of the batched graph against the oracle's brute force (Section 1's
    definition) on a seeded sample of 500 of its rays, with the closest-hit rules of
    tests/parity.py.  Batches cover the four smallest config-4 scenes and both ray
    sources (one light and several lights)."""
    import oracle
    from paper_2312_06538_gb300 import batched as bt
    from paper_2312_06538_gb300 import pipeline as pl
    from tests import parity
    spec = [(2100, 0), (9000, 3), (33000, 1), (5000, 2), (60000, 3), (2500, 1)]
    batches, meta = _batches(spec)
    by_scene = {id(w.scene): w for w in meta}
    pads_of = lambda s: by_scene[id(s)].build_pads()  # noqa: E731
    hp_of = lambda s: pl.hash_params(by_scene[id(s)].hash_lo, by_scene[id(s)].hash_hi)  # noqa: E731
    tuner = bt.Autotuner(bundles=(4, 16), depths=(2, 3), reps=1)
    bat = bt.BatchedCRSH(batches, pads_of, hp_of, tuner=tuner, n_streams=4)
    bat.capture()
    bat.replay()
    torch.cuda.synchronize()
    assert bat.check_status() == []
    rng = np.random.default_rng(1004)
    for k, ((scene, rays, n), run) in enumerate(zip(batches, bat.runs)):
        idx = np.sort(rng.choice(n, size=min(500, n), replace=False))
        sub = {f: np.ascontiguousarray(rays[f][:n].cpu().numpy()[idx]) for f in pl.RAY_FIELDS}
        ref = oracle.bruteforce(sub, scene.verts)
        tri, t, u, v = (x[:n].cpu().numpy() for x in run.hits())
        got = (tri.view(np.int32)[idx], t[idx], u[idx], v[idx])
        rep = parity.compare_hits(got, ref, sub, scene.verts)
        parity.check_report(rep, label=f"batch {k} ({n} rays, scene {spec[k][1]}, B={run.bundle}, L={run.levels})")
        assert rep["hits"] > 20
