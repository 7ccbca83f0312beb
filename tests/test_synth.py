"""Pins for the seeded input generators (Philox4x32-10, RAMBO, 2-body, emission points)."""
import math

import numpy as np

import synth


def _philox_reference(c, k):
    """Philox4x32-10 restated with Python integers from its published definition."""
    M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    c = list(c)
    k0, k1 = k
    for r in range(10):
        if r:
            k0 = (k0 + W0) % 2 ** 32
            k1 = (k1 + W1) % 2 ** 32
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) % 2 ** 32, p1 % 2 ** 32,
             ((p0 >> 32) ^ c[3] ^ k1) % 2 ** 32, p0 % 2 ** 32]
    return c


def test_philox_matches_integer_restatement():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4, 50), dtype=np.uint64).astype(np.uint32)
    for key in [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (12345, 678)]:
        out = synth.philox4x32_10(ctr, key)
        for i in range(ctr.shape[1]):
            ref = _philox_reference([int(x) for x in ctr[:, i]], key)
            assert [int(x) for x in out[:, i]] == ref


# Known-answer vectors published with the generator's reference implementation
# (Salmon et al., SC'11; Random123 distribution): (counter c0..c3, key k0 k1) -> output.
PHILOX_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF), (0xFFFFFFFF, 0xFFFFFFFF),
     (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


def test_philox_known_answer_vectors():
    """The generator reproduces the published known answers: a misreading of the round
    function, the multipliers, the Weyl constants or the word order fails here."""
    for ctr, key, expect in PHILOX_KAT:
        out = synth.philox4x32_10(np.array(ctr, dtype=np.uint32).reshape(4, 1), key)
        assert [int(x) for x in out[:, 0]] == list(expect), [hex(int(x)) for x in out[:, 0]]


def test_uniforms_open_interval_and_moments():
    u = synth.uniforms(7, 3, 200000, 4)
    assert np.all(u > 0) and np.all(u < 1)
    assert abs(u.mean() - 0.5) < 3e-3
    assert abs((u * u).mean() - 1 / 3) < 3e-3
    # different streams / seeds / offsets give different numbers, same inputs the same
    assert not np.allclose(u, synth.uniforms(7, 4, 200000, 4))
    assert np.array_equal(u[:, 100:], synth.uniforms(7, 3, 199900, 4, first_point=100))


def _check_momenta(p, masses, rs):
    E, px, py, pz = p[0], p[1], p[2], p[3]
    m2 = E * E - px * px - py * py - pz * pz
    for i, m in enumerate(masses):
        np.testing.assert_allclose(m2[i], m * m, atol=1e-9 * rs * rs)
    np.testing.assert_allclose(E.sum(axis=0), rs, rtol=1e-12)
    for c in (px, py, pz):
        np.testing.assert_allclose(c.sum(axis=0), 0.0, atol=1e-11 * rs)


def test_rambo_massless_weights_closed_form():
    for n, rs in [(2, 100.0), (3, 100.0), (4, 500.0)]:
        u = synth.uniforms(1, 0, 1000, 4 * n)
        p, w = synth.rambo_massless(rs, n, u)
        _check_momenta(p, [0.0] * n, rs)
        s = rs * rs
        if n == 2:
            np.testing.assert_allclose(w, 1.0 / (8.0 * math.pi), rtol=1e-14)
        if n == 3:
            np.testing.assert_allclose(w, s / (256.0 * math.pi ** 3), rtol=1e-14)


def test_rambo_massless_is_flat():
    """Flat 2-body: cos(theta) of the first particle is uniform."""
    u = synth.uniforms(11, 0, 100000, 8)
    p, _ = synth.rambo_massless(100.0, 2, u)
    c = p[3, 0] / p[0, 0]
    hist, _ = np.histogram(c, bins=10, range=(-1, 1))
    assert np.all(np.abs(hist / 1e4 - 1.0) < 0.05)


def test_rambo_massive_two_body_weight():
    m = 173.0
    rs = 1000.0
    u = synth.uniforms(2, 0, 500, 8)
    p, w = synth.rambo_massive(rs, [m, m], u)
    _check_momenta(p, [m, m], rs)
    beta = math.sqrt(1 - 4 * m * m / rs ** 2)
    np.testing.assert_allclose(w, beta / (8 * math.pi), rtol=1e-12)


def test_rambo_massive_three_body_onshell():
    u = synth.uniforms(4, 0, 500, 12)
    p, w = synth.rambo_massive(1000.0, [173.0, 173.0, 0.0], u)
    _check_momenta(p, [173.0, 173.0, 0.0], 1000.0)
    assert np.all(w > 0)


def test_flat_points_layout():
    b = synth.flat_points("gg_ttg", 33, 4)
    assert b.p.shape == (4, 5, 33) and b.p.flags["C_CONTIGUOUS"]
    np.testing.assert_allclose(b.p[0, 0], 500.0)
    np.testing.assert_allclose(b.p[3, 1], -500.0)


def test_two_body_scan():
    b = synth.gg_tt_scan(1000, 3)
    rs = b.p[0, 0] + b.p[0, 1]
    assert rs.min() >= 400 and rs.max() <= 2000
    m2 = b.p[0, 2] ** 2 - (b.p[1:, 2] ** 2).sum(axis=0)
    np.testing.assert_allclose(m2, 173.0 ** 2, rtol=1e-10)


def test_emission_points_conserve_momentum():
    N = 64
    rng = np.random.default_rng(3)
    p = synth.emission_points(1000.0, 173.0, rng.uniform(1e-6, 0.8, N), rng.uniform(-1, 1, N),
                              rng.uniform(0, 6, N), rng.uniform(-1, 1, N), rng.uniform(0, 6, N))
    np.testing.assert_allclose(p[:, 2:].sum(axis=1), p[:, :2].sum(axis=1), atol=1e-9)
    m2 = p[0] ** 2 - (p[1:] ** 2).sum(axis=0)
    np.testing.assert_allclose(m2[2:4], 173.0 ** 2, rtol=1e-9)
    q = synth.fsr_emission_points(100.0, rng.uniform(-1, 1, N), rng.uniform(0, 6, N),
                                  rng.uniform(0, 1, N), rng.uniform(-1, 1, N), rng.uniform(0, 6, N))
    np.testing.assert_allclose(q[:, 2:].sum(axis=1), q[:, :2].sum(axis=1), atol=1e-10)
    m2 = q[0] ** 2 - (q[1:] ** 2).sum(axis=0)
    np.testing.assert_allclose(m2[2:], 0.0, atol=1e-9)


def test_approach_points_labels():
    b, lab = synth.approach_points("gg_ttg", 8, 5)
    assert b.n == 8 * 16
    assert set(np.unique(lab["kind"])) == {0, 1, 2}


def test_fks_points_invert_to_their_sector_variables():
    """Points from a sector channel map back, through the oracle's inverse sector maps, to
    the variables they were built from; every point is on shell and balanced."""
    from oracle import fks
    from oracle.matrix_element import to_points
    n = 2048
    a_f, a_s = synth.FKS_ALPHA_FLAT, 0.5 * (1.0 - synth.FKS_ALPHA_FLAT)
    vmin = math.sqrt(0.5 * synth.FKS_Y_CUT)
    b = synth.fks_points("gg_ttg", n, 3)
    u = synth.uniforms(3, 0, n, 18)
    k = to_points(b.p)
    ximax = 1.0 - 4.0 * synth.MT ** 2 / 1e6
    for beam, sel in ((0, (u[0] >= a_f) & (u[0] < a_f + a_s)), (1, u[0] >= a_f + a_s)):
        kin = fks.isr_map(k[sel], 4, beam, synth.MT)
        np.testing.assert_allclose(kin.xi, ximax * u[1][sel], rtol=1e-12)
        v = vmin + (1.0 - vmin) * u[2][sel]
        np.testing.assert_allclose(kin.y, 1.0 - 2.0 * v * v, atol=1e-12)
    _check_momenta(b.p[:, 2:], [synth.MT, synth.MT, 0.0], 1000.0)
    e = synth.fks_points("ee_uug", n, 3)
    ke = to_points(e.p)
    for partner, sel in ((2, (u[0] >= a_f) & (u[0] < a_f + a_s)), (3, u[0] >= a_f + a_s)):
        kin = fks.fsr_map(ke[sel], 4, partner, 5 - partner)
        np.testing.assert_allclose(kin.xi, u[3][sel], rtol=1e-12)
        v = vmin + (1.0 - vmin) * u[4][sel]
        np.testing.assert_allclose(kin.y, 1.0 - 2.0 * v * v, atol=1e-12)
    _check_momenta(e.p[:, 2:], [0.0, 0.0, 0.0], 100.0)


def test_fks_point_weights_are_the_oracle_jacobians():
    """Each weight is the phase-space measure over the summed channel densities, with the
    sector Jacobians K of the oracle's maps (pinned there by quadrature and the RAMBO
    volumes) and the RAMBO weight of the point: 1 / (a_flat / w_RAMBO + sum_j a_j h_j),
    h_j = 4 g(y_j) / (xi_max beta(s) xi K) (initial state, dPhi_2(s) = beta(s)/(8 pi) x
    dOmega*/(4 pi)) or 4 g(y_j) / (xi K_j) (final state), g(y) = 1 / (4 v (1 - v_min)),
    v = sqrt((1 - y)/2), for 1 - y >= the cut."""
    from oracle import fks
    from oracle.matrix_element import to_points
    n = 1024
    a_f, a_s = synth.FKS_ALPHA_FLAT, 0.5 * (1.0 - synth.FKS_ALPHA_FLAT)
    vmin = math.sqrt(0.5 * synth.FKS_Y_CUT)
    g = lambda y: np.where(1 - y >= synth.FKS_Y_CUT, 1.0 / (4.0 * np.sqrt(0.5 * (1.0 - y)) * (1.0 - vmin)), 0.0)
    s = 1e6
    beta = math.sqrt(1.0 - 4.0 * synth.MT ** 2 / s)
    ximax = 1.0 - 4.0 * synth.MT ** 2 / s
    b = synth.fks_points("uu_ttg", n, 8)
    k = to_points(b.p)
    h = a_f / synth.rambo_weight(1000.0, [synth.MT, synth.MT, 0.0], b.p[:, 2:])
    for beam in (0, 1):
        kin = fks.isr_map(k, 4, beam, synth.MT)
        h = h + a_s * 4.0 * g(kin.y) / (ximax * beta * kin.xi * kin.K)
    # (the map recovers y from the momenta: 1 - |y| near 0 carries the momenta's rounding
    # relative to 1 - |y|, hence 1e-10 rather than 1e-12; a wrong Jacobian is off by O(1))
    np.testing.assert_allclose(b.wgt, 1.0 / h, rtol=1e-10)
    e = synth.fks_points("ee_uug", n, 8)
    ke = to_points(e.p)
    h = a_f / (100.0 ** 2 / (256 * math.pi ** 3))
    for kk in (fks.fsr_map(ke, 4, 2, 3), fks.fsr_map(ke, 4, 3, 2)):
        h = h + a_s * 4.0 * g(kk.y) / (kk.xi * kk.K)
    np.testing.assert_allclose(e.wgt, 1.0 / h, rtol=1e-10)


def test_fks_point_weights_integrate_to_the_phase_space_volume():
    """Mean weight = three-body volume: s/(256 pi^3) for massless partons, the massive
    RAMBO volume for t tbar g (within 4 combined standard errors)."""
    n = 1 << 18
    e = synth.fks_points("ee_uug", n, 12)
    vol = 100.0 ** 2 / (256 * math.pi ** 3)
    assert abs(e.wgt.mean() - vol) <= 4 * e.wgt.std() / math.sqrt(n)
    b = synth.fks_points("gg_ttg", n, 12)
    r = synth.flat_points("gg_ttg", n, 12)
    err = math.hypot(b.wgt.std(), r.wgt.std()) / math.sqrt(n)
    assert abs(b.wgt.mean() - r.wgt.mean()) <= 4 * err
