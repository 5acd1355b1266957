"""The frame executor (two frames in flight, uploads and read-backs on their own
stream) against the plain pipeline: every frame's hits bit-identical to a direct
run of the path on the same inputs, with a different ray count per frame; a
frame whose pair lists overflow raises on read-back."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _frames(w, n):
    from paper_2312_06538_gb300 import pipeline as pl
    g = pl.Pipeline.gbuffer_to_device(w.gbuffer, "cpu")
    out = []
    for k in range(n):
        f = dict(g)
        # lights move from frame to frame, so the shadow-ray count (and n) changes
        f["lights"] = torch.from_numpy((w.lights + np.float32(0.07 * k)).astype(np.float32))
        out.append(f)
    return out


@pytest.mark.parametrize("words", [False, True])
def test_frames_match_direct_runs_bitwise(words):
    from paper_2312_06538_gb300 import frames as fr
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(2, res=96)
    p = pl.workload_pipeline(w, level1_words=words)
    hp, bp = pl.workload_params(w)
    frames = _frames(w, 5)
    refs = []
    for f in frames:
        gs = p.gbuffer_struct({k: v.cuda() for k, v in f.items() if k != "lights"})
        c = p.run_fit(gs, f["lights"].cuda(), hp, bp)
        refs.append(tuple(x[:c["rays"]].cpu() for x in (p.hit_tri, p.hit_t, p.hit_u, p.hit_v)))
    assert len({r[0].numel() for r in refs}) > 1
    layout = fr.HostLayout(frames[0])
    bufs = [layout.pack(f, layout.host_buffer()) for f in frames]
    fs = fr.FrameStream(p, layout, hp, bp)
    got = []
    for rep in range(2):
        for b in bufs:
            out = fs.push(b)
            if out is not None:
                got.append(tuple(x.clone() for x in (out.tri, out.t, out.u, out.v)))
        out = fs.drain()
        got.append(tuple(x.clone() for x in (out.tri, out.t, out.u, out.v)))
    assert fs.drain() is None
    assert len(got) == 2 * len(frames)
    for k, g in enumerate(got):
        for a, b in zip(g, refs[k % len(frames)]):
            assert torch.equal(a.view(torch.int32), b.view(torch.int32)), k


def test_frame_overflow_raises_on_read_back():
    from paper_2312_06538_gb300 import crsh as C
    from paper_2312_06538_gb300 import frames as fr
    from paper_2312_06538_gb300 import pipeline as pl
    w = synthetic.make(1)
    p = pl.workload_pipeline(w, pair_capacity=1 << 12)
    hp, bp = pl.workload_params(w)
    f = _frames(w, 1)[0]
    layout = fr.HostLayout(f)
    fs = fr.FrameStream(p, layout, hp, bp)
    assert fs.push(layout.pack(f, layout.host_buffer())) is None
    with pytest.raises(C.CrshError) as e:
        fs.drain()
    assert e.value.status == C.ERR_CAPACITY
