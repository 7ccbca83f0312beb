"""Pins for the per-term cuts of the oracle (Algorithm 2: each term of Born, real, soft
and collinear is zeroed where its own kinematics fail the cuts): the decisions against
the textbook definitions of p_T, rapidity and thrust; closed forms of the terms that
survive; the O(alpha_s) thrust distribution of e+e- -> 3 partons; infrared safety of
the subtracted real with cuts."""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import colour, fks
from oracle import matrix_element as me
from oracle.cuts import Cuts, passes, tree_weights
from oracle.matrix_element import Couplings, to_points

CP = Couplings()
GS2 = 4 * math.pi * CP.alpha_s
E2 = 4 * math.pi * CP.alpha
SQRT_S = {"ee_uu": 100.0, "ee_uug": 100.0, "gg_tt": 1000.0, "gg_ttg": 1000.0, "uu_tt": 1000.0,
          "uu_ttg": 1000.0, "gg_ttgg": 2000.0}


def _flat(name, n, seed):
    b = synth.flat_points(name, n, seed)
    return to_points(b.p), b.wgt


@pytest.mark.parametrize("name", ["ee_uug", "gg_ttg", "uu_ttg"])
def test_inactive_cuts_change_nothing(name):
    k, _ = _flat(name, 300, 11)
    ref = fks.real_subtracted(name, k)
    for c in (Cuts(), Cuts(abs_cos_axis_max=1.0, thrust_max=1.0),
              Cuts(pt_min=500.0, abs_y_max=0.1) if name == "ee_uug" else Cuts(abs_cos_axis_max=0.1, thrust_max=0.7)):
        assert np.array_equal(fks.real_subtracted(name, k, cuts=c), ref)
    np.testing.assert_array_equal(tree_weights("gg_tt", _flat("gg_tt", 50, 3)[0], Cuts()),
                                  me.me2("gg_tt", _flat("gg_tt", 50, 3)[0]))


def _rapidity(p):
    return 0.5 * np.log((p[..., 0] + p[..., 3]) / (p[..., 0] - p[..., 3]))


@pytest.mark.parametrize("name", ["gg_tt", "gg_ttg", "gg_ttgg"])
def test_heavy_quark_decisions_follow_the_definitions(name):
    """Both heavy quarks need p_T = hypot(px, py) >= pt_min and |y| <= y_max,
    y = (1/2) ln((E+pz)/(E-pz)); points within 1e-9 of a threshold are not judged."""
    k, _ = _flat(name, 4000, 21)
    cut = Cuts(pt_min=0.3 * SQRT_S[name] / 2, abs_y_max=0.8)
    got = passes(name, k, cut)
    pt = np.hypot(k[:, 2:4, 1], k[:, 2:4, 2])
    y = np.abs(_rapidity(k[:, 2:4]))
    want = np.all((pt >= cut.pt_min) & (y <= cut.abs_y_max), axis=1)
    clear = np.all((np.abs(pt / cut.pt_min - 1) > 1e-9) & (np.abs(y / cut.abs_y_max - 1) > 1e-9), axis=1)
    assert clear.mean() > 0.99
    assert np.array_equal(got[clear], want[clear])
    assert 0.05 < want.mean() < 0.95  # the cut is neither empty nor everything


def _thrust_brute_force(k):
    """Thrust T = max over unit n of sum_i |p_i.n| / sum_i |p_i| by the exact subset
    form: the maximum lies along sum_i e_i p_i for a choice of signs e_i = +-1."""
    p = k[:, 2:, 1:]
    tot = np.linalg.norm(p, axis=2).sum(axis=1)
    best = np.zeros(k.shape[0])
    axis = np.zeros((k.shape[0], 3))
    for signs in itertools.product((1.0, -1.0), repeat=p.shape[1]):
        v = (np.array(signs)[None, :, None] * p).sum(axis=1)
        t = np.linalg.norm(v, axis=1) / tot
        better = t > best
        best = np.where(better, t, best)
        axis = np.where(better[:, None], v, axis)
    return best, np.abs(axis[:, 2]) / np.linalg.norm(axis, axis=1)


@pytest.mark.parametrize("name", ["ee_uu", "ee_uug"])
def test_thrust_decisions_follow_the_definition(name):
    k, _ = _flat(name, 4000, 22)
    T, cosT = _thrust_brute_force(k)
    for cut in (Cuts(abs_cos_axis_max=0.7), Cuts(thrust_max=0.9), Cuts(abs_cos_axis_max=0.5, thrust_max=0.85)):
        got = passes(name, k, cut)
        want = (cosT <= cut.abs_cos_axis_max) & ((T <= cut.thrust_max) | (cut.thrust_max >= 1.0))
        clear = (np.abs(cosT / cut.abs_cos_axis_max - 1) > 1e-9) & (
            (np.abs(T / cut.thrust_max - 1) > 1e-9) | (cut.thrust_max >= 1.0))
        assert clear.mean() > 0.99
        assert np.array_equal(got[clear], want[clear]), cut
    if name == "ee_uu":
        assert np.all(np.abs(T - 1) < 1e-12)  # two partons: T = 1, so every thrust cut fails
        assert not passes(name, k, Cuts(thrust_max=0.99)).any()


def test_thrust_cut_keeps_only_the_real():
    """With T <= T_max < 1 every Born counter-event (T = 1) fails: the subtracted real is
    the real |M|^2 inside the cut and 0 outside, for any (xi_c, delta)."""
    k, _ = _flat("ee_uug", 2000, 23)
    T, _ = _thrust_brute_force(k)
    cut = Cuts(thrust_max=0.9)
    for fp in (fks.FKSParams(), fks.FKSParams(1.0, 2.0)):
        W = fks.real_subtracted("ee_uug", k, fp, cuts=cut)
        inside = T <= 0.9
        np.testing.assert_allclose(W[inside], me.me2("ee_uug", k[inside]), rtol=1e-13)
        assert np.all(W[~inside] == 0.0)
        assert 0.05 < inside.mean() < 0.95


def _born_closed(kb):
    """e+e- -> u ubar: (4 pi alpha)^2 N_c Q_u^2 (1 + cos^2 theta)."""
    c = kb[:, 2, 3] / np.linalg.norm(kb[:, 2, 1:], axis=1)
    return E2 ** 2 * 3 * (2 / 3) ** 2 * (1 + c * c)


def test_axis_cut_masks_the_real_and_keeps_the_counterterms():
    """Points whose most energetic parton is the gluon, along the beam (the real fails
    |cos theta_T| <= 0.6), with both Born counter-events' axes inside: the subtracted real
    is minus the counterterms, each in closed form -- soft g^2 C_F B_j/(8 pi^3), collinear
    g^2 C_F (1+(1-xi)^2) B_j/(16 pi^3), soft-collinear g^2 C_F B_j/(8 pi^3), B_j the
    closed-form Born of sector j, over xi^2 (1-y_j) K_j."""
    rs = 100.0
    rng = np.random.default_rng(31)
    n = 20000
    k = to_points(synth.fsr_emission_points(rs, rng.uniform(-0.3, 0.3, n), rng.uniform(0, 2 * np.pi, n),
                                            rng.uniform(0.7, 0.95, n), rng.uniform(-0.85, -0.3, n),
                                            rng.uniform(0, 2 * np.pi, n), 2))
    cut = Cuts(abs_cos_axis_max=0.6)
    gl = k[:, 4]
    is_max = (gl[:, 0] > k[:, 2, 0]) & (gl[:, 0] > k[:, 3, 0])
    gl_out = np.abs(gl[:, 3]) / np.linalg.norm(gl[:, 1:], axis=1) > 0.6 + 1e-9
    n3 = np.abs(k[:, 2, 3]) / np.linalg.norm(k[:, 2, 1:], axis=1)
    n4 = np.abs(k[:, 3, 3]) / np.linalg.norm(k[:, 3, 1:], axis=1)
    sel = is_max & gl_out & (n3 < 0.6 - 1e-9) & (n4 < 0.6 - 1e-9)
    assert sel.sum() > 150
    k = k[sel]
    s = rs * rs
    for fp in (fks.FKSParams(0.8, 1.0), fks.FKSParams(1.0, 2.0), fks.FKSParams(0.75, 1.6)):
        W = fks.real_subtracted("ee_uug", k, fp, cuts=cut)
        xi = 2 * k[:, 4, 0] / rs
        ref = np.zeros(k.shape[0])
        for j in (2, 3):
            kin = fks.fsr_map(k, 4, j, 5 - j)
            B = _born_closed(kin.born_soft)
            y = kin.y
            K = s * (1 - xi) / (16 * math.pi ** 3 * (2 - xi * (1 - y)) ** 2)
            ts = (xi < fp.xi_cut).astype(float)
            tc = (y > 1 - fp.delta).astype(float)
            G0 = GS2 * colour.CF * B / (8 * math.pi ** 3)
            G1 = GS2 * colour.CF * (1 + (1 - xi) ** 2) * B / (16 * math.pi ** 3)
            ref -= (ts * G0 + tc * G1 - ts * tc * G0) / (xi * xi * (1 - y) * K)
        assert np.any(ref != 0)
        np.testing.assert_allclose(W, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_axis_cut_masks_the_counterterms_and_keeps_the_real():
    """Both Born axes outside |cos theta_T| <= 0.5, the real's thrust axis (its most
    energetic parton) inside: the subtracted real is the real |M|^2 alone."""
    k, _ = _flat("ee_uug", 6000, 24)
    cut = Cuts(abs_cos_axis_max=0.5)
    W = fks.real_subtracted("ee_uug", k, fks.FKSParams(1.0, 2.0), cuts=cut)
    m = np.argmax(k[:, 2:, 0], axis=1) + 2
    km = k[np.arange(k.shape[0]), m]
    real_in = np.abs(km[:, 3]) / np.linalg.norm(km[:, 1:], axis=1) < 0.5 - 1e-9
    n3 = np.abs(k[:, 2, 3]) / np.linalg.norm(k[:, 2, 1:], axis=1)
    n4 = np.abs(k[:, 3, 3]) / np.linalg.norm(k[:, 3, 1:], axis=1)
    sel = real_in & (n3 > 0.5 + 1e-9) & (n4 > 0.5 + 1e-9)
    assert sel.sum() > 20
    np.testing.assert_allclose(W[sel], me.me2("ee_uug", k[sel]), rtol=1e-13)


def _thrust_distribution(T):
    """O(alpha_s) thrust distribution of e+e- -> q qbar g, (1/sigma_0) d sigma/dT over
    C_F alpha_s / (2 pi) (De Rujula, Ellis, Floratos, Gaillard 1978)."""
    return 2 * (3 * T * T - 3 * T + 2) / (T * (1 - T)) * math.log((2 * T - 1) / (1 - T)) - 3 * (3 * T - 2) * (2 - T) / (1 - T)


def test_three_parton_rate_below_a_thrust_cut():
    """sigma(T <= 0.9) / sigma_0 from the oracle's subtracted real with the thrust cut,
    integrated over flat RAMBO points, against (a) the Dalitz-plot integral of
    (x1^2 + x2^2)/((1-x1)(1-x2)) and (b) the integrated textbook thrust distribution."""
    T = 0.9
    a = colour.CF * CP.alpha_s / (2 * math.pi)
    dal, _ = integrate.dblquad(lambda x2, x1: (x1 * x1 + x2 * x2) / ((1 - x1) * (1 - x2)), 2 - 2 * T, T,
                               lambda x1: 2 - T - x1, lambda x1: T, epsabs=1e-12, epsrel=1e-11)
    txt, _ = integrate.quad(_thrust_distribution, 2 / 3, T, epsabs=1e-12, epsrel=1e-11)
    assert abs(dal / txt - 1) < 1e-9
    rs = 100.0
    s = rs * rs
    sig0 = 4 * math.pi * CP.alpha ** 2 * 3 * (4 / 9) / (3 * s)
    k, wgt = _flat("ee_uug", 1 << 15, 25)
    w = fks.real_subtracted("ee_uug", k, cuts=Cuts(thrust_max=T)) * wgt / (2 * s) / sig0
    est, err = w.mean(), w.std() / math.sqrt(w.size)
    assert err < 0.02 * est
    assert abs(est - a * dal) < 4 * err, (est, err, a * dal)


def _isr_pair_points(n, xi, cos_beam, cos_pair, seed):
    rng = np.random.default_rng(seed)
    return to_points(synth.emission_points(1000.0, 173.0, np.full(n, xi), np.full(n, cos_beam),
                                           rng.uniform(0, 2 * np.pi, n), np.full(n, cos_pair),
                                           rng.uniform(0, 2 * np.pi, n)))


@pytest.mark.parametrize("name", ["gg_ttg", "uu_ttg"])
@pytest.mark.parametrize("sector,cut,cos_pair", [
    # p_T cut: the soft Born's heavy quarks (p = beta sqrt(s)/2) pass, the collinear
    # Born's (p = beta_Q sqrt(s z)/2, smaller) fail; p_T is invariant along the beam
    (0, Cuts(pt_min=300.0), math.sqrt(1 - 0.7 ** 2)),
    (1, Cuts(pt_min=300.0), math.sqrt(1 - 0.7 ** 2)),
    # rapidity cut: sector 2's collinear Born is boosted towards +z, so its quark fails
    (1, Cuts(abs_y_max=1.0), 0.7867),
])
def test_isr_cuts_are_infrared_safe(name, sector, cut, cos_pair):
    """Approaching a sector's collinear limit at xi = 0.3 where the collinear counter-event
    fails the cut and the soft one passes: the real (whose kinematics tend to the
    collinear counter-event's) fails too, and W (1 - y) -> 0.  Masking the collinear term
    with the soft counter-event's cut instead (a plausible wiring mistake) leaves
    W (1 - y) finite."""
    fp = fks.FKSParams(0.5, 1.0)
    born = fks.REAL_PROCESSES[name][0]
    res, wrong = [], []
    for r in (1e-3, 1e-5, 1e-7):
        cb = (1 - r) if sector == 0 else -(1 - r)
        k = _isr_pair_points(8, 0.3, cb, cos_pair, seed=41)
        kin = fks.isr_map(k, 4, sector, me.MT)
        assert np.all(passes(born, kin.born_soft, cut))
        assert not np.any(passes(born, kin.born_coll, cut)) and not np.any(passes(name, k, cut))
        W = fks.real_subtracted(name, k, fp, cuts=cut)
        _, parts = fks.real_subtracted(name, k, fp, detail=True)
        p = parts[sector]
        den = p["xi"] ** 2 * p["K"]
        scale = np.abs(p["G_coll"]) / den  # the collinear term's size times (1 - y)
        res.append(np.max(np.abs(W) * r / scale))
        wrong_W = W - p["G_coll"] / (den * r)
        wrong.append(np.min(np.abs(wrong_W) * r / scale))
    assert res[-1] < 1e-3 and res[0] > res[-1]
    assert min(wrong) > 0.5


def test_tree_weights_and_nbody_with_cuts():
    k, _ = _flat("gg_tt", 500, 26)
    cut = Cuts(pt_min=150.0, abs_y_max=1.2)
    w = tree_weights("gg_tt", k, cut)
    m = passes("gg_tt", k, cut)
    assert 0.05 < m.mean() < 0.95
    np.testing.assert_array_equal(w[m], me.me2("gg_tt", k[m]))
    assert np.all(w[~m] == 0)
