"""Phase-space cuts of each term (oracle, FP64).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU baseline,
never by the library.

Algorithm 2 (Sec. 4.3) ends by zeroing every term a of {Born, real, soft, collinear}
whose cuts fail at that term's own kinematics (passCuts(a, p)); the "smarter" variant
discussed after it stores the points that pass each term's cuts separately and
evaluates each kind of amplitude once enough have passed.  The paper names no cuts.
The readings here are two infrared-safe families, each applied to the momenta of the
term it masks (the real event, or the Born counter-event of a soft or collinear term):

  * heavy-quark final states (t tbar, t tbar g, t tbar g g): both heavy quarks (legs
    2 and 3) need transverse momentum p_T >= pt_min and |rapidity| <= abs_y_max,
    rapidity y = (1/2) ln((E + p_z)/(E - p_z)) along the beam axis z;
  * e+e- -> massless partons: thrust T <= thrust_max and |cos theta_T| <= abs_cos_axis_max
    for the thrust axis.  For two or three massless partons in their centre-of-mass
    frame the thrust is T = max_i 2 E_i / sqrt(s) and the thrust axis is the direction of
    the most energetic parton (three partons: T(n) = sum_i |p_i.n| / sum_i |p_i| is
    largest along a parton's direction, and with p_a = -(p_b + p_c) that value is
    2 |p_a| / sqrt(s)).  A soft gluon or a collinear pair leaves both unchanged, so the
    cuts are infrared safe.

A cut with pt_min = 0, abs_y_max = inf, abs_cos_axis_max >= 1 or thrust_max >= 1 is off.

Each decision is an integer result taken in float64.  It is written without square
roots or logarithms, as a fixed sequence of correctly rounded operations, so that any
implementation doing the same operations on the same momenta takes the same decision:
  p_T:       px*px + py*py >= pt_min^2
  rapidity:  E + |pz| <= exp(2 y_max) * (E - |pz|)
  axis:      pz*pz <= c^2 * ((px*px + py*py) + pz*pz),   m = most energetic final parton
  thrust:    2 E_m <= T_max * (E_0 + E_1)
(the most energetic parton is the first of the largest energies, in leg order).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .matrix_element import PROCESSES


@dataclass(frozen=True)
class Cuts:
    pt_min: float = 0.0
    abs_y_max: float = math.inf
    abs_cos_axis_max: float = 1.0
    thrust_max: float = 1.0

    def active(self, name: str) -> bool:
        fam = family(name)
        if fam == "heavy":
            return self.pt_min > 0.0 or math.isfinite(self.abs_y_max)
        if fam == "ee":
            return self.abs_cos_axis_max < 1.0 or self.thrust_max < 1.0
        return False


def family(name: str) -> str:
    legs = PROCESSES[name].legs
    if legs[2:4] == ("t", "t~"):
        return "heavy"
    if legs[0] in ("e+", "e-"):
        return "ee"
    return "none"


def passes(name: str, k: np.ndarray, cuts: Cuts | None) -> np.ndarray:
    """Boolean (N,) for momenta k (N, n, 4) of process ``name`` (or of a Born
    counter-event of it: the final state's legs are 2, 3, ...)."""
    N = k.shape[0]
    ok = np.ones(N, dtype=bool)
    if cuts is None or not cuts.active(name):
        return ok
    if family(name) == "heavy":
        for leg in (2, 3):
            E, px, py, pz = (k[:, leg, c] for c in range(4))
            if cuts.pt_min > 0.0:
                ok &= (px * px + py * py) >= cuts.pt_min * cuts.pt_min
            if math.isfinite(cuts.abs_y_max):
                a = np.abs(pz)
                ok &= (E + a) <= math.exp(2.0 * cuts.abs_y_max) * (E - a)
        return ok
    # e+e-: the most energetic final parton (first one on ties)
    E = k[:, 2:, 0]
    m = np.argmax(E, axis=1) + 2
    km = k[np.arange(N), m]
    if cuts.abs_cos_axis_max < 1.0:
        c2 = cuts.abs_cos_axis_max * cuts.abs_cos_axis_max
        ok &= km[:, 3] * km[:, 3] <= c2 * ((km[:, 1] * km[:, 1] + km[:, 2] * km[:, 2]) + km[:, 3] * km[:, 3])
    if cuts.thrust_max < 1.0:
        ok &= 2.0 * km[:, 0] <= cuts.thrust_max * (k[:, 0, 0] + k[:, 1, 0])
    return ok


def tree_weights(name: str, k: np.ndarray, cuts: Cuts | None, cp=None) -> np.ndarray:
    """|M|^2 of the points that pass the cuts, 0 elsewhere (the n-body term of
    Algorithm 2)."""
    from .matrix_element import Couplings, me2
    return np.where(passes(name, k, cuts), me2(name, k, cp or Couplings()), 0.0)
