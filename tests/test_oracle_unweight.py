"""Pins of the unweighting oracle (oracle/unweight.py) by what the accept/reject step
must satisfy, independently of how it is written: the expected event weight of every
point is its weight (the sum over a large sample agrees within its statistical error,
also bin by bin in a kinematic variable); the number of events is the sum of |w| / w_max;
and the exact special cases (|w| = w_max always kept, w = 0 never, overweight points kept
with their own weight, w_max <= 0 taking the batch maximum, NaN never kept)."""
import numpy as np

import synth
from oracle.unweight import unweight


def _sample(n, seed):
    x = synth.uniforms(seed, 0, n, 1)[0]
    # a signed weight with a sign change and a peak, like a subtracted real weight
    w = (np.cos(6.0 * x) + 0.3) / (0.05 + (x - 0.7) ** 2)
    u = synth.uniforms(seed, 3, n, 1)[0]
    return x, w, u


def test_expected_event_weight_is_the_weight():
    x, w, u = _sample(400000, 11)
    w_max = np.abs(w).max()
    idx, ew, wm, nover = unweight(w, 0.0, u)
    assert wm == w_max and nover == 0
    sigma = np.sqrt(np.sum(w_max * np.abs(w) - w * w))
    assert abs(ew.sum() - w.sum()) < 5 * sigma
    # bin by bin in x
    bins = np.minimum((x * 10).astype(int), 9)
    for b in range(10):
        sel = bins == b
        sb = np.sqrt(np.sum(w_max * np.abs(w[sel]) - w[sel] ** 2))
        kb = bins[idx] == b
        assert abs(ew[kb].sum() - w[sel].sum()) < 5 * sb + 1e-300
    # the event weights are +-w_max
    assert np.all(np.abs(ew) == w_max)
    assert np.all(np.sign(ew) == np.sign(w[idx]))


def test_number_of_events():
    _, w, u = _sample(400000, 12)
    w_max = 1.5 * np.abs(w).max()
    idx, _, _, _ = unweight(w, w_max, u)
    p = np.abs(w) / w_max
    assert abs(idx.size - p.sum()) < 5 * np.sqrt(np.sum(p * (1 - p)))
    assert np.all(np.diff(idx) > 0)


def test_special_cases():
    u = np.array([1e-9, 0.5, 0.999999, 0.3, 0.7, 0.2, 0.9])
    w = np.array([2.0, -2.0, 2.0, 0.0, 5.0, np.nan, -0.5])
    idx, ew, wm, nover = unweight(w, 2.0, u)
    # |w| = w_max: kept for any u < 1; w = 0 never; 5 > w_max kept as itself; NaN never;
    # -0.5: kept iff 0.9 * 2 < 0.5 (no)
    assert list(idx) == [0, 1, 2, 4]
    assert list(ew) == [2.0, -2.0, 2.0, 5.0]
    assert wm == 2.0 and nover == 1
    idx, ew, wm, nover = unweight(w, 0.0, u)  # batch maximum, NaN ignored
    assert wm == 5.0 and nover == 0
    # kept iff 5 u < |w|: 5e-9 < 2 yes, 2.5 < 2 no, 5.0 < 2 no, 3.5 < 5 yes, 4.5 < 0.5 no
    assert list(idx) == [0, 4] and list(ew) == [5.0, 5.0]
