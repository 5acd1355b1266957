"""Failure detection on the GPU without a GPU fault: the bounded waits of the
decoupled look-back (single-pass scans, radix sort) run out when a predecessor
tile never publishes, record CRSH_ERR_TIMEOUT and return.  The status words are
prepared on the host; nothing here hangs or faults (each wait is limited to a
few thousand polls).  The positive controls check the look-back's sum."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LB_AGG, LB_INC = 1 << 62, 2 << 62
LB32_AGG, LB32_INC = 1 << 30, 2 << 30


def _run(wide, words, tile, aggregate, limit):
    from paper_2312_06538_gb300 import crsh as C
    dev = torch.device("cuda")
    s64 = torch.zeros(max(1, tile + 1), dtype=torch.int64, device=dev)
    s32 = torch.zeros(max(1, tile + 1), dtype=torch.int32, device=dev)
    if wide:
        s64[:len(words)] = torch.tensor(np.array(words, np.uint64).view(np.int64), device=dev)
    else:
        s32[:len(words)] = torch.tensor(np.array(words, np.uint32).view(np.int32), device=dev)
    out = torch.full((1,), -1, dtype=torch.int64, device=dev)
    import ctypes
    ctr = torch.zeros(ctypes.sizeof(C.crsh_counters), dtype=torch.uint8, device=dev)
    C.crsh_lookback_selftest(s64.data_ptr(), s32.data_ptr(), wide, tile, aggregate, limit, out.data_ptr(),
                             ctr.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    c = C.crsh_counters.from_buffer_copy(bytes(ctr.cpu().numpy()))
    final = (s64 if wide else s32).cpu().numpy().view(np.uint64 if wide else np.uint32)[tile]
    return int(out.item()), c.status, int(final)


@pytest.mark.parametrize("wide", [True, False])
def test_lookback_sums_published_predecessors(wide):
    from paper_2312_06538_gb300 import crsh as C
    tile = 40
    if wide:
        words = [LB_INC | 5] + [LB_AGG | 3] * (tile - 1)
    else:
        words = [LB32_INC | 5] + [LB32_AGG | 3] * (tile - 1)
    prefix, status, final = _run(wide, words, tile, 7, 1 << 10)
    assert status == C.OK
    assert prefix == 5 + 3 * (tile - 1)
    assert final == (LB_INC if wide else LB32_INC) | (prefix + 7)


@pytest.mark.parametrize("wide", [True, False])
@pytest.mark.parametrize("silent", [0, 17, 39])
def test_lookback_wait_runs_out_when_a_predecessor_never_publishes(wide, silent):
    """Tile 40 waits on tile `silent`, whose word stays 0 (never published): after the
    spin limit the kernel records CRSH_ERR_TIMEOUT, publishes its own word and returns."""
    from paper_2312_06538_gb300 import crsh as C
    tile = 40
    if wide:
        words = [LB_AGG | 3] * tile
        words[0] = LB_AGG | 3
    else:
        words = [LB32_AGG | 3] * tile
    words[silent] = 0
    _, status, final = _run(wide, words, tile, 7, 1 << 10)
    assert status == C.ERR_TIMEOUT
    assert final >> (62 if wide else 30) == 2      # the tile still published its inclusive word
