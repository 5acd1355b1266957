"""Host side of the frame executor: the staging layout (256-byte aligned fields, pack
and views round-trip, shape and type checks).  Needs no GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_06538_gb300 import frames as fr  # noqa: E402


def _fields(n=1000, n_lights=3, seed=0):
    g = torch.Generator().manual_seed(seed)
    f = {k: torch.rand(n, generator=g) for k in ("px", "py", "pz", "nx", "ny", "nz", "ix", "iy", "iz")}
    f["material"] = torch.randint(0, 1 << 30, (n,), generator=g, dtype=torch.int32)
    f["hit"] = torch.randint(0, 2, (n,), generator=g, dtype=torch.uint8)
    f["lights"] = torch.rand((n_lights, 3), generator=g)
    return f


@pytest.mark.parametrize("n", [1, 63, 1000, 4097])
def test_layout_aligns_and_round_trips(n):
    f = _fields(n)
    lay = fr.HostLayout(f)
    offs = [o for o, _, _, _ in lay.spans.values()]
    assert all(o % 256 == 0 for o in offs) and offs == sorted(offs)
    ends = [o + nb for o, nb, _, _ in lay.spans.values()]
    assert all(e <= o for e, o in zip(ends, offs[1:])) and ends[-1] <= lay.nbytes and lay.nbytes % 256 == 0
    buf = lay.pack(f, torch.zeros(lay.nbytes, dtype=torch.uint8))
    back = lay.views(buf)
    for k, v in f.items():
        assert back[k].dtype == v.dtype and back[k].shape == v.shape
        assert np.array_equal(back[k].numpy().view(np.uint8), v.numpy().view(np.uint8))


def test_layout_refuses_a_mismatched_field():
    f = _fields(100)
    lay = fr.HostLayout(f)
    buf = torch.zeros(lay.nbytes, dtype=torch.uint8)
    bad = dict(f)
    bad["px"] = torch.zeros(101)
    with pytest.raises(ValueError):
        lay.pack(bad, buf)
    bad = dict(f)
    bad["hit"] = torch.zeros(100, dtype=torch.int32)
    with pytest.raises(ValueError):
        lay.pack(bad, buf)
