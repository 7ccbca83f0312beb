"""Pins for the extended-precision use of the oracle and for the float64 parity rule.

The float64 parity tests arbitrate a disagreement between the CUDA float64 path and the
float64 oracle by evaluating the oracle in np.longdouble at the same inputs and by
estimating the condition number of the value in its float64 inputs
(tests/fp64_arbiter.py).  These tests pin both pieces to something other than
themselves:
  * every step of the oracle really runs in extended precision: at exactly on-shell
    points built in extended precision, the squared matrix elements equal textbook
    closed forms to a few hundred extended-precision rounding errors -- far below the
    float64 rounding error, so one float64 step anywhere in the chain would fail;
  * the condition-number estimate reproduces closed-form condition numbers;
  * the rule accepts errors of the size conditioning explains and rejects larger ones.
"""
import math

import numpy as np
import pytest

from oracle import fks
from oracle import matrix_element as me
from oracle.matrix_element import Couplings
from tests import fp64_arbiter as arb

L = np.longdouble
pytestmark = pytest.mark.skipif(not arb.extended_precision_available(),
                                reason="np.longdouble is not wider than float64 here")
EPS = float(np.finfo(L).eps)
CP = Couplings()


def _two_body(rs, mass, cth, phi):
    """Exactly on-shell 2 -> 2 points (N, 4, 4) in extended precision, beams along z."""
    n = cth.size
    e = L(rs) / 2
    pa = e * np.sqrt(L(1) - L(4) * L(mass) ** 2 / L(rs) ** 2)
    sth = np.sqrt(L(1) - cth * cth)
    p = np.zeros((n, 4, 4), dtype=L)
    p[:, 0] = [e, 0, 0, e]
    p[:, 1] = [e, 0, 0, -e]
    p[:, 2, 0] = e
    p[:, 2, 1] = pa * sth * np.cos(phi)
    p[:, 2, 2] = pa * sth * np.sin(phi)
    p[:, 2, 3] = pa * cth
    p[:, 3, 0] = e
    p[:, 3, 1:] = -p[:, 2, 1:]
    return p


def _angles(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, n).astype(L), rng.uniform(0, 2 * np.pi, n).astype(L)


def test_extended_ee_uu_equals_closed_form():
    """(4 pi alpha)^2 N_c Q_u^2 (1 + cos^2 theta).  The vertex factors are the oracle's
    float64 constants e and e Q_u (the CUDA path forms the same float64 products), so
    the closed form takes them as given: e^2 (e Q_u)^2 N_c (1 + cos^2 theta)."""
    cth, phi = _angles(64, 1)
    p = _two_body(100.0, 0.0, cth, phi)
    got = me.me2("ee_uu", p)
    assert got.dtype == L
    e = CP.as_dict()["e"]
    ref = L(e) ** 2 * L(e * (2.0 / 3.0)) ** 2 * 3 * (1 + cth ** 2)
    rel = np.abs(got / ref - 1).astype(float)
    assert rel.max() < 100 * EPS, rel.max()


def test_extended_gg_tt_equals_closed_form():
    """Combridge's g g -> t tbar form g^4 (1/(6 t1 t2) - 3/8)(t1^2 + t2^2 + rho - rho^2/(4 t1 t2))."""
    cth, phi = _angles(64, 2)
    p = _two_body(900.0, 173.0, cth, phi)
    got = me.me2("gg_tt", p)
    s = (p[:, 0, 0] + p[:, 1, 0]) ** 2
    dot = lambda a, b: a[:, 0] * b[:, 0] - (a[:, 1:] * b[:, 1:]).sum(axis=1)
    t1 = 2 * dot(p[:, 0], p[:, 2]) / s
    t2 = 2 * dot(p[:, 1], p[:, 2]) / s
    rho = 4 * L(173.0) ** 2 / s
    g2 = L(CP.as_dict()["gs"]) ** 2
    ref = g2 ** 2 * (1 / (6 * t1 * t2) - L(3) / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))
    rel = np.abs(got / ref - 1).astype(float)
    assert rel.max() < 500 * EPS, rel.max()


def test_extended_agrees_with_float64_on_generic_points():
    """At generic points the float64 oracle and its extended-precision evaluation agree
    to float64 rounding, and the subtracted real is evaluated in extended precision too."""
    import synth
    b = synth.flat_points("gg_ttg", 32, 4)
    k = me.to_points(b.p)
    a = me.me2("gg_ttg", k)
    x = me.me2("gg_ttg", k.astype(L))
    assert np.max(np.abs(a / x - 1)) < 1e-13
    w = fks.real_subtracted("gg_ttg", k.astype(L))
    assert w.dtype == L


def test_condition_estimate_matches_closed_forms():
    """f = x - y has condition number (|x| + |y|) / |x - y| in its inputs.  The estimate
    (eight random sign vectors, each input moved by half a float64 ulp, i.e. between 1/2
    and 1 of u relative) never exceeds it and reaches at least half of it whenever one
    sample gives x and y opposite signs (all but about 1 in 128 points); f = x y z has 3."""
    rng = np.random.default_rng(11)
    x = rng.uniform(0.5, 2.0, 512)
    y = x * (1 - 10.0 ** rng.uniform(-9, -1, 512))
    k = np.stack([x, y, np.full(512, 0.7)], axis=1)[:, :, None] * np.ones((1, 1, 4))
    _, c = arb.extended(lambda q: q[:, 0, 0] - q[:, 1, 0], k)
    exact = (np.abs(x) + np.abs(y)) / np.abs(x - y)
    assert np.all(c <= exact * (1 + 1e-6))
    assert np.mean(c >= 0.5 * exact) > 0.97
    _, c3 = arb.extended(lambda q: q[:, 0, 0] * q[:, 1, 0] * q[:, 2, 0], k)
    assert np.all(c3 <= 3 * (1 + 1e-6)) and np.all(c3 >= 0.5 - 1e-6)
    assert np.mean(c3 > 1.5) > 0.8


def test_rule_accepts_conditioning_and_rejects_mistakes():
    """A relative error of 1e-13 passes everywhere; 1e-9 fails at well-conditioned
    points; at an ill-conditioned point an error of 10 cond u passes and 1000 cond u
    fails."""
    f = lambda q: q[:, 0, 0] - q[:, 1, 0]
    x = np.array([1.0, 2.0, 1.0])
    y = np.array([0.5, 0.3, 1.0 - 1e-8])
    k = np.stack([x, y], axis=1)[:, :, None] * np.ones((1, 1, 4))
    ref = x - y
    cond = (np.abs(x) + np.abs(y)) / np.abs(x - y)
    arb.check_fp64(ref * (1 + 1e-13), f, k)
    with pytest.raises(AssertionError):
        arb.check_fp64(ref * (1 + 1e-9), f, k)
    ok = ref.copy()
    ok[2] = ref[2] * (1 + 10 * cond[2] * arb.U)
    st = arb.check_fp64(ok, f, k)
    assert st["arbitrated"] == 1
    bad = ref.copy()
    bad[2] = ref[2] * (1 + 1000 * cond[2] * arb.U)
    with pytest.raises(AssertionError):
        arb.check_fp64(bad, f, k)
