"""Pins for the oracle's squared matrix elements: closed forms, traces, symmetries."""
import math

import numpy as np
import pytest

import synth
from oracle import matrix_element as me
from oracle.diagrams import Diagrams, Process, helicities
from oracle.dirac import GAMMA, METRIC, dot, slash
from oracle.matrix_element import Couplings, to_points

CP = Couplings()
GS2 = 4 * math.pi * CP.alpha_s
E2 = 4 * math.pi * CP.alpha


def _inv(p, a, b):
    return p[:, a, 0] * p[:, b, 0] - (p[:, a, 1:] * p[:, b, 1:]).sum(axis=1)


def test_diagram_counts():
    """Tree diagram counts (the four-gluon vertex counted once per diagram)."""
    expect = {"ee_uu": 1, "ee_uug": 2, "gg_tt": 3, "gg_ttg": 16, "gg_ttgg": 123,
              "uu_tt": 1, "uu_ttg": 5}
    for name, n in expect.items():
        assert me.diagrams(name).n_diagrams == n, name


def test_paper_example_ee_to_two_photons():
    """Sec. 2.1, Eq. (born): e+e- -> 2 photons has two LO diagrams (tests/golden/paper_counts.txt);
    the textbook massless result is (1/4) sum|M|^2 = 2 e^4 (u/t + t/u)."""
    proc = Process("ee_aa", ("e+", "e-", "a", "a"), frozenset({("e", "a")}))
    d = Diagrams(proc)
    golden = dict(l.split()[:2] for l in open(__file__.replace("test_oracle_me.py", "golden/paper_counts.txt"))
                  if l.strip() and not l.startswith("#"))
    assert d.n_diagrams == int(golden["ee_aa_lo_diagrams"])
    p = to_points(synth.flat_points("ee_uu", 16, 9).p)
    hel = helicities(4)
    A = d.amplitudes(p, hel, CP.as_dict())
    val = np.einsum("nht,ts,nhs->n", A.conj(), d.gram(), A).real / 4.0
    t = -2 * _inv(p, 0, 2)
    u = -2 * _inv(p, 0, 3)
    np.testing.assert_allclose(val, 2 * E2 ** 2 * (u / t + t / u), rtol=1e-12)


def test_ee_uu_angular_distribution():
    p = to_points(synth.flat_points("ee_uu", 100, 1).p)
    cth = p[:, 2, 3] / np.linalg.norm(p[:, 2, 1:], axis=1)
    ref = E2 ** 2 * 3 * (2 / 3) ** 2 * (1 + cth ** 2)
    np.testing.assert_allclose(me.me2("ee_uu", p), ref, rtol=1e-12)


def test_ee_uu_total_cross_section():
    """sigma_LO = 4 pi alpha^2 N_c Q_u^2 / (3 s) = 3.18090e-8 GeV^-2 at sqrt(s)=100 GeV, by
    Gauss-Legendre quadrature of the oracle over the angle."""
    rs = 100.0
    x, w = np.polynomial.legendre.leggauss(16)
    N = len(x)
    c = x
    sn = np.sqrt(1 - c * c)
    p = np.zeros((N, 4, 4))
    p[:, 0] = [rs / 2, 0, 0, rs / 2]
    p[:, 1] = [rs / 2, 0, 0, -rs / 2]
    p[:, 2] = np.stack([np.full(N, rs / 2), rs / 2 * sn, 0 * c, rs / 2 * c], axis=1)
    p[:, 3] = p[:, 2] * np.array([1, -1, -1, -1])
    m2 = me.me2("ee_uu", p)
    sigma = (w * m2).sum() * 2 * math.pi / (32 * math.pi ** 2) / (2 * rs * rs)
    assert abs(sigma / (4 * math.pi * CP.alpha ** 2 * 3 * (4 / 9) / (3 * rs * rs)) - 1) < 1e-13
    assert abs(sigma - 3.18090e-8) < 1e-12


def _lepton_tensor(p1, p2):
    """Tr[p1slash gamma^mu p2slash gamma^nu] for massless leptons (upper indices)."""
    return np.einsum("nab,mbc,ncd,kda->nmk", slash(p1), GAMMA, slash(p2), GAMMA)


def test_ee_uu_trace_brute_force():
    p = to_points(synth.flat_points("ee_uu", 20, 3).p)
    L = _lepton_tensor(p[:, 0], p[:, 1])
    H = _lepton_tensor(p[:, 2], p[:, 3])
    g = np.diag(METRIC)
    LH = np.einsum("nmk,nmk,m,k->n", L, H, g, g).real
    s = 2 * _inv(p, 0, 1)
    ref = 0.25 * 3 * E2 ** 2 * (2 / 3) ** 2 * LH / s ** 2
    np.testing.assert_allclose(me.me2("ee_uu", p), ref, rtol=1e-12)


def test_ee_uug_trace_brute_force():
    """Sum over spins by traces with -g_{ab} for the gluon (valid for one external gluon)."""
    p = to_points(synth.flat_points("ee_uug", 12, 4).p)
    p1, p2, p3, p4, k = (p[:, i] for i in range(5))
    L = _lepton_tensor(p1, p2)
    g = np.diag(METRIC)
    d3 = 2 * dot(p3, k)
    d4 = 2 * dot(p4, k)
    # O^{nu alpha} = gamma^a (p3+k)slash gamma^nu / d3 - gamma^nu (p4+k)slash gamma^a / d4
    O = (np.einsum("aij,njk,vkl->nvail", GAMMA, slash(p3 + k), GAMMA) / d3[:, None, None, None, None]
         - np.einsum("vij,njk,akl->nvail", GAMMA, slash(p4 + k), GAMMA) / d4[:, None, None, None, None])
    Obar = np.einsum("ij,nvakj,kl->nvail", GAMMA[0], O.conj(), GAMMA[0])
    H = np.einsum("nij,nvajk,nkl,nwali,a->nvw", slash(p3), O, slash(p4), Obar, -g)
    LH = np.einsum("nvw,nvw,v,w->n", L, H, g, g).real
    s = 2 * _inv(p, 0, 1)
    ref = 0.25 * E2 ** 2 * (2 / 3) ** 2 * GS2 * 4.0 * LH / s ** 2  # colour: Tr(T^a T^a) = 4
    np.testing.assert_allclose(me.me2("ee_uug", p), ref, rtol=1e-12)


def test_ee_uug_orientation_average_closed_form():
    """Averaging the beam over x, y, z gives the orientation-averaged
    (2 g^2 C_F/s) e^4 N_c Q^2 (4/3) (x1^2+x2^2)/((1-x1)(1-x2)) exactly."""
    rs = 100.0
    p = to_points(synth.flat_points("ee_uug", 40, 2).p)
    vals = []
    for ax in (1, 2, 3):
        q = p.copy()
        q[:, 0, 1:] = 0
        q[:, 1, 1:] = 0
        q[:, 0, ax] = rs / 2
        q[:, 1, ax] = -rs / 2
        vals.append(me.me2("ee_uug", q))
    avg = np.mean(vals, axis=0)
    x1 = 2 * p[:, 2, 0] / rs
    x2 = 2 * p[:, 3, 0] / rs
    ref = (2 * GS2 * (4 / 3) / rs ** 2) * E2 ** 2 * 3 * (4 / 9) * (4 / 3) * (x1 ** 2 + x2 ** 2) / ((1 - x1) * (1 - x2))
    np.testing.assert_allclose(avg, ref, rtol=1e-12)


def _taus(p):
    s = 2 * _inv(p, 0, 1)
    return 2 * _inv(p, 0, 2) / s, 2 * _inv(p, 1, 2) / s, 4 * 173.0 ** 2 / s


def test_gg_tt_closed_form():
    p = to_points(synth.gg_tt_scan(200, 3).p)
    t1, t2, rho = _taus(p)
    ref = GS2 ** 2 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))
    np.testing.assert_allclose(me.me2("gg_tt", p), ref, rtol=1e-12)


def test_uu_tt_closed_form():
    p = to_points(synth.flat_points("uu_tt", 200, 3).p)
    t1, t2, rho = _taus(p)
    np.testing.assert_allclose(me.me2("uu_tt", p), 4 / 9 * GS2 ** 2 * (t1 ** 2 + t2 ** 2 + rho / 2), rtol=1e-12)


@pytest.mark.parametrize("name,legs,n", [("gg_tt", [0, 1], 6), ("gg_ttg", [0, 1, 4], 6),
                                         ("uu_ttg", [4], 6), ("ee_uug", [4], 6),
                                         ("gg_ttgg", [0, 5], 2)])
def test_gauge_invariance(name, legs, n):
    """eps -> k/k0 for one gluon: every colour component of the amplitude vanishes."""
    d = me.diagrams(name)
    p = to_points(synth.flat_points(name, n, 21).p)
    C = d.colour_tensors()
    for leg in legs:
        hel = helicities(d.n, {leg: 1})
        A = d.amplitudes(p, hel, CP.as_dict(), override={leg: p[:, leg] / p[:, leg, 0:1]})
        M = np.einsum("nht,td->nhd", A, C)
        scale = np.einsum("nht,td->nhd", np.abs(A), np.abs(C)).max()
        assert np.abs(M).max() < 1e-13 * scale


def _lorentz(p, rng):
    """Random rotation followed by a random boost of all momenta (N, n, 4)."""
    q = p.copy()
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    th = rng.uniform(0, np.pi)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    R = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    q[..., 1:] = q[..., 1:] @ R.T
    b = rng.normal(size=3) * 0.3
    g = 1 / math.sqrt(1 - b @ b)
    bp = q[..., 1:] @ b
    out = q.copy()
    out[..., 0] = g * (q[..., 0] + bp)
    out[..., 1:] = q[..., 1:] + (((g - 1) * bp / (b @ b) + g * q[..., 0])[..., None]) * b
    return out


@pytest.mark.parametrize("name,n", [("gg_ttg", 6), ("uu_ttg", 6), ("gg_ttgg", 2), ("ee_uug", 6)])
def test_lorentz_invariance(name, n):
    p = to_points(synth.flat_points(name, n, 5).p)
    q = _lorentz(p, np.random.default_rng(1))
    np.testing.assert_allclose(me.me2(name, q), me.me2(name, p), rtol=1e-12)


def test_bose_symmetry():
    p = to_points(synth.flat_points("gg_ttgg", 3, 8).p)
    ref = me.me2("gg_ttgg", p)
    q = p.copy()
    q[:, [4, 5]] = q[:, [5, 4]]
    np.testing.assert_allclose(me.me2("gg_ttgg", q), ref, rtol=1e-12)
    for name in ("gg_tt", "gg_ttg"):
        p = to_points(synth.flat_points(name, 6, 8).p)
        q = p.copy()
        q[:, [0, 1]] = q[:, [1, 0]]
        np.testing.assert_allclose(me.me2(name, q), me.me2(name, p), rtol=1e-12)


@pytest.mark.parametrize("name", ["ee_uug", "gg_tt", "gg_ttg", "uu_ttg", "gg_ttgg"])
def test_helicity_flip_symmetry(name):
    """Flipping every helicity leaves the colour-summed |M|^2 unchanged (tree amplitudes,
    real couplings); the same holds for colour correlators and for one gluon polarised
    along a real transverse vector.  The CUDA path sums one member of each pair and doubles."""
    d = me.diagrams(name)
    k = to_points(synth.flat_points(name, 3, 12).p)
    hel = helicities(d.n)
    A = d.amplitudes(k, hel, CP.as_dict())
    idx = {tuple(h): i for i, h in enumerate(hel)}
    flip = np.array([idx[tuple(-h)] for h in hel])
    per = np.einsum("nht,ts,nhs->nh", A.conj(), me.gram(name), A).real
    np.testing.assert_allclose(per, per[:, flip], rtol=1e-11, atol=1e-14 * np.abs(per).max())
    if name in ("gg_tt",):
        for kk in range(4):
            for ll in range(kk, 4):
                pc = np.einsum("nht,ts,nhs->nh", A.conj(), me.gram(name, kk, ll), A).real
                np.testing.assert_allclose(pc, pc[:, flip], atol=1e-12 * np.abs(pc).max())
        ep = np.zeros((3, 4))
        ep[:, 1], ep[:, 2] = 0.6, 0.8
        for leg in (0, 1):
            hl = helicities(4, {leg: 1})
            Ap = d.amplitudes(k, hl, CP.as_dict(), override={leg: ep})
            pp = np.einsum("nht,ts,nhs->nh", Ap.conj(), me.gram(name), Ap).real
            ix = {tuple(np.delete(h, leg)): i for i, h in enumerate(hl)}
            fl = np.array([ix[tuple(-np.delete(h, leg))] for h in hl])
            np.testing.assert_allclose(pp, pp[:, fl], atol=1e-12 * np.abs(pp).max())
