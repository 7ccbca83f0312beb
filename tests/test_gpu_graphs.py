"""After the first call (lane-layout tuning, scratch sizing), an evaluation on device
buffers is a fixed sequence of stream-ordered launches with no allocation or host
synchronisation, so it can be captured in a CUDA graph and replayed."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def me():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_07439_gb300 as m
    return m


@pytest.mark.parametrize("name,entry,prec,queues", [("gg_ttg", "real_subtracted", "mixed", 0),
                                                    ("gg_tt", "born", "mixed", 0), ("gg_ttgg", "born", "mixed", 0),
                                                    ("uu_ttg", "real_subtracted", "fp64", 0),
                                                    ("gg_ttg", "real_subtracted", "mixed", 1),
                                                    ("ee_uug", "real_subtracted", "fp64", 1)])
def test_capture_and_replay(me, name, entry, prec, queues):
    """queues 1: the per-term path (a counter reset and six kernels) is captured too."""
    b = synth.flat_points(name, 3000, 17)
    p = torch.from_numpy(b.p).cuda()
    w = torch.from_numpy(b.wgt).cuda()
    out = torch.empty(b.n, dtype=torch.float64, device="cuda")
    h = me.Handle(name, precision=me.ME_PREC_MIXED if prec == "mixed" else me.ME_PREC_FP64, term_queues=queues)
    s = torch.cuda.Stream()
    h.set_stream(s.cuda_stream)
    f = getattr(h, entry)
    with torch.cuda.stream(s):
        f(p, w, out)  # first call: tuning and scratch sizing, outside the capture
    torch.cuda.synchronize()
    ref = out.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        f(p, w, out)
    out.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    acc = h.accumulators()
    assert acc[2] == 4 * b.n  # first call + 3 replays
