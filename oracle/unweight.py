"""Unweighted event generation (oracle; test infrastructure, not the product path).

The accept/reject step of Sec. 3.1, which turns points weighted by the integrand into
events distributed like it, for signed NLO weights.  It is written directly from its
definition:
- point i is kept iff u_i w_max < |w_i|;
- a kept point carries the event weight sign(w_i) max(w_max, |w_i|).
The uniforms u_i are an input, drawn by the caller.  Then E[event weight of point i]
= (|w_i| / w_max) sign(w_i) w_max = w_i for |w_i| <= w_max, and w_i for overweight
points, which are always kept.  Pinned in tests/test_oracle_unweight.py.
"""
from __future__ import annotations

import numpy as np


def unweight(w: np.ndarray, w_max: float, u: np.ndarray):
    """(indices of kept points in increasing order, their event weights, number overweight).
    w_max <= 0 takes max |w| (NaN ignored); NaN weights are never kept."""
    w = np.asarray(w, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    aw = np.abs(w)
    if not w_max > 0.0:
        finite = aw[~np.isnan(aw)]
        w_max = float(finite.max()) if finite.size else 0.0
    with np.errstate(invalid="ignore"):
        keep = u * w_max < aw
        over = aw > w_max
    idx = np.nonzero(keep)[0]
    ew = np.where(aw[idx] > w_max, w[idx], np.copysign(w_max, w[idx]))
    return idx, ew, w_max, int(np.count_nonzero(over))
