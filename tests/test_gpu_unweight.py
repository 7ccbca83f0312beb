"""Unweighting on the device (me_unweight) against the oracle (oracle/unweight.py) on the
same uniforms: the oracle takes them from the host Philox4x32-10 generator (synth), the
device draws its own from the same published definition.  The kept indices, the event
weights, the applied w_max and the overweight count are compared exactly (the decision
u * w_max < |w| is the same float64 operation on both sides).  Sizes: one point, one
block boundary either side, a ragged tail, and an empty batch."""
import numpy as np
import pytest

import synth
from oracle.unweight import unweight

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


@pytest.fixture(scope="module")
def h(me):
    return me.Handle("gg_ttg", precision=me.ME_PREC_MIXED)


def _weights(n, seed):
    x = synth.uniforms(seed, 0, n, 2)
    return np.where(x[1] < 0.3, -1.0, 1.0) * np.exp(4.0 * x[0])  # signed, spread over e^4


@pytest.mark.parametrize("n", [1, 255, 256, 257, 100003])
@pytest.mark.parametrize("w_max", [0.0, 20.0])
def test_device_unweighting_equals_oracle(h, n, w_max):
    seed, stream, first = 21, 5, 1000
    w = _weights(n, seed)
    u = synth.uniforms(seed, stream, n, 1, first_point=first)[0]
    idx, ew, wm, nover = unweight(w, w_max, u)
    kept, kw, wm_d, nover_d = h.unweight(torch.from_numpy(w).cuda(), w_max=w_max, seed=seed, stream=stream,
                                         first_point=first)
    np.testing.assert_array_equal(kept.cpu().numpy(), idx)
    np.testing.assert_array_equal(kw.cpu().numpy(), ew)
    assert wm_d == wm and nover_d == nover
    if w_max > 0 and n > 1000:
        assert nover > 0  # e^4 > 20: the overweight branch is exercised


def test_offsets_select_the_same_events(h):
    """A batch unweighted in two parts with first_point offsets gives the events of the whole."""
    n, seed, stream = 50000, 22, 6
    w = torch.from_numpy(_weights(n, seed)).cuda()
    kept, kw, _, _ = h.unweight(w, w_max=30.0, seed=seed, stream=stream)
    a, _, _, _ = h.unweight(w[:20000].contiguous(), w_max=30.0, seed=seed, stream=stream, first_point=0)
    b, _, _, _ = h.unweight(w[20000:].contiguous(), w_max=30.0, seed=seed, stream=stream, first_point=20000)
    both = np.concatenate([a.cpu().numpy(), b.cpu().numpy() + 20000])
    np.testing.assert_array_equal(both, kept.cpu().numpy())


def test_unweighted_subtracted_real_is_unbiased(h):
    """Events from the subtracted real weights of 2^18 flat g g -> t tbar g points: the sum
    of the event weights equals the sum of the weights within its statistical error."""
    b = synth.flat_points("gg_ttg", 1 << 18, 31)
    w = h.real_subtracted(torch.from_numpy(b.p).cuda(), torch.from_numpy(b.wgt).cuda())
    kept, kw, wm, _ = h.unweight(w, seed=31, stream=9)
    wn = w.cpu().numpy()
    sigma = np.sqrt(np.sum(wm * np.abs(wn) - wn * wn))
    assert abs(kw.cpu().numpy().sum() - wn.sum()) < 5 * sigma
    assert 0 < kept.shape[0] < wn.size


def test_empty_and_bad_arguments(me, h):
    kept, kw, wm, no = h.unweight(torch.empty(0, dtype=torch.float64, device="cuda"), w_max=3.0)
    assert kept.shape[0] == 0 and wm == 3.0 and no == 0
    with pytest.raises(me.MEError) as e:
        h.unweight(torch.ones(10, dtype=torch.float64), w_max=1.0)  # host buffer
    assert e.value.code == me.ME_ERR_ARG
    with pytest.raises(me.MEError) as e:
        h.unweight(torch.ones(10, dtype=torch.float64, device="cuda"), w_max=float("nan"))
    assert e.value.code == me.ME_ERR_ARG
