"""Pins for the oracle's FKS pieces: sector functions, maps, Jacobians, soft/collinear limits,
the integrated counterterms and the e+e- K-factor."""
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from oracle import colour, fks, nlo_ee
from oracle import matrix_element as me
from oracle.matrix_element import Couplings, to_points

CP = Couplings()
GS2 = 4 * math.pi * CP.alpha_s


def _isr_points(n, xi, cos_beam, seed=0):
    rng = np.random.default_rng(seed)
    return to_points(synth.emission_points(1000.0, 173.0, np.broadcast_to(xi, n).copy(),
                                           np.broadcast_to(cos_beam, n).copy(),
                                           rng.uniform(0, 2 * np.pi, n), rng.uniform(-1, 1, n),
                                           rng.uniform(0, 2 * np.pi, n)))


def _fsr_points(n, xi, y, partner=2, seed=0):
    rng = np.random.default_rng(seed)
    return to_points(synth.fsr_emission_points(100.0, rng.uniform(-1, 1, n), rng.uniform(0, 2 * np.pi, n),
                                               np.broadcast_to(xi, n).copy(), np.broadcast_to(y, n).copy(),
                                               rng.uniform(0, 2 * np.pi, n), partner))


def test_sector_functions_partition_unity():
    for name, pts in [("ee_uug", to_points(synth.flat_points("ee_uug", 200, 1).p)),
                      ("gg_ttg", to_points(synth.flat_points("gg_ttg", 200, 1).p))]:
        born, i, partners, _ = fks.REAL_PROCESSES[name]
        S = fks.sector_functions(pts, i, partners)
        np.testing.assert_allclose(S.sum(axis=0), 1.0, rtol=1e-14)
        assert np.all(S >= 0)
    k = _fsr_points(10, 0.3, 1 - 1e-9)
    S = fks.sector_functions(k, 4, fks.REAL_PROCESSES["ee_uug"][2])
    np.testing.assert_allclose(S[0], 1.0, atol=1e-8)


def test_fsr_map_roundtrip_and_born():
    rng = np.random.default_rng(4)
    xi = rng.uniform(0, 1, 50)
    y = rng.uniform(-1, 1, 50)
    k = _fsr_points(50, xi, y)
    kin = fks.fsr_map(k, 4, 2, 3)
    np.testing.assert_allclose(kin.xi, xi, atol=1e-14)
    np.testing.assert_allclose(kin.y, y, atol=1e-13)
    b = kin.born_soft
    np.testing.assert_allclose(b[:, 2:].sum(axis=1), b[:, :2].sum(axis=1), atol=1e-12)
    m2 = b[..., 0] ** 2 - (b[..., 1:] ** 2).sum(axis=-1)
    np.testing.assert_allclose(m2, 0, atol=1e-10)


def test_isr_map_roundtrip_and_borns():
    rng = np.random.default_rng(5)
    n = 40
    xi = rng.uniform(0.01, 0.85, n)
    cb = rng.uniform(-1, 1, n)
    k = _isr_points(n, xi, cb)
    for j, sgn in ((0, 1.0), (1, -1.0)):
        kin = fks.isr_map(k, 4, j, 173.0)
        np.testing.assert_allclose(kin.xi, xi, atol=1e-13)
        np.testing.assert_allclose(kin.y, sgn * cb, atol=1e-13)
        for b, rs in ((kin.born_soft, 1000.0), (kin.born_coll, None)):
            np.testing.assert_allclose(b[:, 2:].sum(axis=1), b[:, :2].sum(axis=1), atol=1e-9)
            m2 = b[..., 0] ** 2 - (b[..., 1:] ** 2).sum(axis=-1)
            np.testing.assert_allclose(m2[:, 2:], 173.0 ** 2, rtol=1e-9)
        s_coll = (kin.born_coll[:, 0, 0] + kin.born_coll[:, 1, 0]) ** 2 - kin.born_coll[:, :2, 3].sum(axis=1) ** 2
        np.testing.assert_allclose(s_coll, 1e6 * (1 - xi), rtol=1e-12)


def test_fsr_jacobian_integrates_to_three_body_volume():
    """int xi K dxi dy dphi = (s/(256 pi^3)) / (1/(8 pi)) for the massless final-state map."""
    s = 1e4
    val, _ = integrate.dblquad(lambda y, xi: xi * s * (1 - xi) / (16 * math.pi ** 3 * (2 - xi * (1 - y)) ** 2),
                               0, 1, -1, 1)
    assert abs(2 * math.pi * val / (8 * math.pi) / (s / (256 * math.pi ** 3)) - 1) < 1e-10


def test_isr_jacobian_matches_massive_rambo_volume():
    """int dPhi_B xi K dxi dy dphi (Born volume beta/(8 pi)) == <massive RAMBO weight>."""
    m, rs = 173.0, 1000.0
    s = rs * rs
    beta = math.sqrt(1 - 4 * m * m / s)
    xmax = 1 - 4 * m * m / s
    val, _ = integrate.quad(lambda xi: xi * s * math.sqrt(max(0.0, 1 - 4 * m * m / (s * (1 - xi))))
                            / (64 * math.pi ** 3 * beta), 0, xmax)
    vol = beta / (8 * math.pi) * val * 2 * 2 * math.pi
    b = synth.flat_points("gg_ttg", 400000, 77)
    mc, err = b.wgt.mean(), b.wgt.std() / math.sqrt(b.n)
    assert abs(mc - vol) < 4 * err and err < 2e-3 * vol


@pytest.mark.parametrize("name", ["gg_ttg", "uu_ttg"])
def test_isr_soft_limit_ratio(name):
    """G(xi,y)/G(0,y) -> 1 linearly in xi (colour-correlated eikonal with massive terms)."""
    dev = []
    for xi in (1e-3, 1e-4, 1e-5):
        k = _isr_points(6, xi, np.linspace(-0.9, 0.9, 6), seed=1)
        _, parts = fks.real_subtracted(name, k, detail=True)
        dev.append(np.abs(parts[0]["G"] / parts[0]["G_soft"] - 1).max())
    assert dev[-1] < 1e-4
    assert dev[0] / dev[-1] > 50


@pytest.mark.parametrize("name", ["gg_ttg", "uu_ttg"])
def test_isr_collinear_limit_ratio(name):
    """G(xi,y)/G(xi,1) -> 1 as 1-y -> 0 at fixed xi, for every azimuth (spin correlations)."""
    for j, side in ((0, 1.0), (1, -1.0)):
        dev = []
        for om in (1e-4, 1e-6, 1e-8):
            k = _isr_points(8, 0.35, side * (1 - om), seed=2)
            _, parts = fks.real_subtracted(name, k, detail=True)
            p = parts[j]
            dev.append(np.abs(p["G"] / p["G_coll"] - 1).max())
        assert dev[-1] < 2e-3
        assert dev[0] / dev[-1] > 30


def test_isr_collinear_spin_correlation_matters():
    """With the azimuthal (B_perp) term dropped the gg collinear ratio does not tend to 1."""
    k = _isr_points(8, 0.35, 1 - 1e-8, seed=2)
    _, parts = fks.real_subtracted("gg_ttg", k, detail=True)
    kin = fks.isr_map(k, 4, 0, 173.0)
    B = me.me2("gg_tt", kin.born_coll)
    z = 0.65
    s = 1e6
    avg = (2 / s) / z * 2 * GS2 * 2 * colour.CA * (z + 0.35 ** 2 * z + 0.35 ** 2 / z) * B * kin.K_coll
    assert np.abs(parts[0]["G"] / avg - 1).max() > 1e-2
    assert np.abs(parts[0]["G"] / parts[0]["G_coll"] - 1).max() < 2e-3


def test_fsr_limits_and_closed_forms():
    for partner, isec in ((2, 0), (3, 1)):
        dev_s, dev_c = [], []
        for v in (1e-4, 1e-6, 1e-8):
            k = _fsr_points(6, v, np.linspace(-0.9, 0.9, 6), partner)
            _, parts = fks.real_subtracted("ee_uug", k, detail=True)
            p = parts[isec]
            dev_s.append(np.abs(p["G"] / p["G_soft"] - 1).max())
            B = me.me2("ee_uu", fks.fsr_map(k, 4, partner, 5 - partner).born_soft)
            # G(0,y) = g^2 C_F B / (8 pi^3), independent of y
            np.testing.assert_allclose(p["G_soft"], GS2 * colour.CF * B / (8 * math.pi ** 3), rtol=1e-12)
            k = _fsr_points(6, 0.4, 1 - v, partner)
            _, parts = fks.real_subtracted("ee_uug", k, detail=True)
            p = parts[isec]
            dev_c.append(np.abs(p["G"] / p["G_coll"] - 1).max())
            B = me.me2("ee_uu", fks.fsr_map(k, 4, partner, 5 - partner).born_soft)
            np.testing.assert_allclose(p["G_coll"], GS2 * colour.CF * (1 + 0.6 ** 2) * B / (16 * math.pi ** 3),
                                       rtol=1e-12)
        assert dev_s[-1] < 1e-6 and dev_c[-1] < 1e-4
        assert dev_s[0] / dev_s[1] > 50 and dev_c[0] / dev_c[-1] > 30


def _closed_form_subtracted(xi, y, xc, dl):
    """Sector (q,g) FKS integrand [G - ...]/(xi(1-y)) with the orientation-averaged real
    (x1^2+x2^2)/((1-x1)(1-x2)), in units of g^2 C_F B_avg (s = 1)."""
    x1 = 2 * (1 - xi) / (2 - xi * (1 - y))
    x2 = 2 - x1 - xi
    if x1 >= 1.0 or x2 >= 1.0:  # measure-zero edge hit by the quadrature rule
        return 0.0
    R = 2 * (x1 * x1 + x2 * x2) / ((1 - x1) * (1 - x2))
    d53 = 1 - y
    d54 = 2 * (1 - x1) / (x2 * xi)
    S = d54 / (d53 + d54)
    K = (1 - xi) / (16 * math.pi ** 3 * (2 - xi * (1 - y)) ** 2)
    G = xi * xi * (1 - y) * R * S * K
    G0 = 1 / (8 * math.pi ** 3)
    G1 = (1 + (1 - xi) ** 2) / (16 * math.pi ** 3)
    ts = 1.0 if xi < xc else 0.0
    tc = 1.0 if y > 1 - dl else 0.0
    return (G - ts * G0 - tc * G1 + ts * tc * G0) / (xi * (1 - y))


def test_oracle_fsr_weight_matches_orientation_averaged_closed_form():
    """Averaging the oracle's per-point weight over beams along x, y, z reproduces the
    closed-form integrand exactly (both the real and the Born-proportional counterterms
    average exactly over three orthogonal axes)."""
    rs, xc, dl = 100.0, 0.5, 1.0
    rng = np.random.default_rng(8)
    n = 30
    xi = rng.uniform(0.01, 0.99, n)
    y = rng.uniform(-0.99, 0.99, n)
    k0 = _fsr_points(n, xi, y, 2, seed=9)
    vals = []
    for ax in (1, 2, 3):
        k = k0.copy()
        k[:, 0, 1:] = 0
        k[:, 1, 1:] = 0
        k[:, 0, ax] = rs / 2
        k[:, 1, ax] = -rs / 2
        _, parts = fks.real_subtracted("ee_uug", k, fks.FKSParams(xc, dl), detail=True)
        p = parts[0]
        vals.append(p["W"] * p["xi"] * p["K"])
    avg = np.mean(vals, axis=0)
    B_avg = (4 * math.pi * CP.alpha) ** 2 * 3 * (4 / 9) * (4 / 3)
    ref = np.array([_closed_form_subtracted(a, b, xc, dl) for a, b in zip(xi, y)]) * GS2 * colour.CF * B_avg
    np.testing.assert_allclose(avg, ref, rtol=1e-10)


@pytest.mark.parametrize("xc,dl", [(1.0, 2.0), (0.5, 1.0), (0.1, 0.5), (0.3, 1.5)])
def test_integrated_counterterms_by_quadrature(xc, dl):
    """Virtual + integrated CTs + quadrature of the 4-d subtracted real = sigma_LO (3/2) a_s,
    i.e. sigma_NLO/sigma_LO = 1 + alpha_s/pi, for any (xi_c, delta)."""
    tot = 0.0
    for a, b in ([(0, xc), (xc, 1)] if xc < 1 else [(0, 1)]):
        for c, d in ([(-1, 1 - dl), (1 - dl, 1)] if dl < 2 else [(-1, 1)]):
            def g(y, xi):
                if xi <= 0 or y >= 1 or y <= -1 or xi >= 1:
                    return 0.0
                return _closed_form_subtracted(xi, y, xc, dl)
            v, _ = integrate.dblquad(g, a, b, c, d, epsabs=1e-11, epsrel=1e-10)
            tot += v
    X = 2 * tot * 2 * math.pi * 8 * math.pi ** 2  # both sectors, units of a_s sigma_LO
    c = nlo_ee.nbody_coefficient(xc, dl)
    # the adaptive quadrature reaches 3e-9 for three of the choices and 3e-7 for
    # (0.1, 0.5), where the cut-offs put kinks close to the integrable singularities
    assert abs(X + c - 1.5) < 1e-6


def test_kfactor_monte_carlo():
    """Flat RAMBO points: sigma_LO (1 + a_s c) + <real - CT> = sigma_LO (1 + alpha_s/pi)."""
    rs = 100.0
    s = rs * rs
    sig_lo = 4 * math.pi * CP.alpha ** 2 * 3 * (4 / 9) / (3 * s)
    a_s = CP.alpha_s * colour.CF / (2 * math.pi)
    b = synth.flat_points("ee_uug", 32768, 2)
    w = fks.real_subtracted("ee_uug", to_points(b.p)) * b.wgt / (2 * s)
    ratio = 1 + a_s * nlo_ee.nbody_coefficient(0.5, 1.0) + w.mean() / sig_lo
    err = w.std() / math.sqrt(w.size) / sig_lo
    assert abs(ratio - (1 + CP.alpha_s / math.pi)) < 4 * err + 1e-4, (ratio, err)
    # n-body weights from the oracle agree with B (1 + a_s c)
    bb = synth.flat_points("ee_uu", 64, 1)
    pb = to_points(bb.p)
    np.testing.assert_allclose(nlo_ee.nbody_nlo(pb), me.me2("ee_uu", pb) * (1 + a_s * nlo_ee.nbody_coefficient(0.5, 1)),
                               rtol=1e-14)


def test_isr_sector_collinear_borns_are_related_by_a_beam_boost():
    """The collinear counter-kinematics of the two ISR sectors (beam 1 or beam 2 scaled by
    1 - xi) differ by a boost along the beam axis: the unpolarised Born and the Born with
    either gluon polarised along the transverse direction (0, cos phi, sin phi, 0) take the
    same values at both.  The kernels rely on this to evaluate both sectors' collinear
    pieces at one kinematics."""
    rng = np.random.default_rng(9)
    n = 30
    k = _isr_points(n, rng.uniform(0.01, 0.85, n), rng.uniform(-1, 1, n), seed=9)
    k1, k2 = fks.isr_map(k, 4, 0, 173.0), fks.isr_map(k, 4, 1, 173.0)
    np.testing.assert_allclose(k1.e_perp, k2.e_perp, atol=0)
    np.testing.assert_allclose(me.me2("gg_tt", k2.born_coll), me.me2("gg_tt", k1.born_coll), rtol=1e-12)
    for leg in (0, 1):
        np.testing.assert_allclose(me.spin_correlated("gg_tt", k2.born_coll, leg, k2.e_perp),
                                   me.spin_correlated("gg_tt", k1.born_coll, leg, k1.e_perp), rtol=1e-12)
    # not a property of any two kinematics: the soft Born (at sqrt(s)) differs
    assert np.median(np.abs(me.me2("gg_tt", k1.born_soft) / me.me2("gg_tt", k1.born_coll) - 1)) > 1e-2


def _boundary_points():
    """Four g g -> t tbar g points: an ordinary one, one with no emitted energy (xi = 0
    exactly), and two with the gluon exactly along a beam (y = 1 in sector 1 or 2)."""
    xi = np.array([0.3, 0.0, 0.3, 0.3])
    cb = np.array([0.2, 0.2, 1.0, -1.0])
    return synth.emission_points(1000.0, 173.0, xi, cb, np.full(4, 0.4), np.full(4, 0.3), np.full(4, 1.1))


def test_domain_boundary_points_carry_zero_weight():
    """Points on the boundary of the FKS domain have measure zero and no defined subtracted
    weight: the oracle gives them weight 0, and the other points of the batch are
    unaffected."""
    p = _boundary_points()
    with np.errstate(all="ignore"):
        w = fks.real_subtracted("gg_ttg", to_points(p))
        w0 = fks.real_subtracted("gg_ttg", to_points(p[:, :, :1]))
    assert np.all(np.isfinite(w))
    assert list(w[1:]) == [0.0, 0.0, 0.0]
    assert w[0] == w0[0] and w[0] != 0.0
