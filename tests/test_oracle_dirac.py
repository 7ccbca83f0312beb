"""Pins for the oracle's Dirac algebra, spinors and polarisation vectors."""
import numpy as np

from oracle.dirac import GAMMA, METRIC, bar, dot, polarisation, slash, spinor_u, spinor_v


def _momenta(m, n=20, seed=0):
    rng = np.random.default_rng(seed)
    p3 = rng.normal(size=(n, 3)) * 50
    p3[0] = [0, 0, -30.0]  # exactly along -z
    p3[1] = [0, 0, 30.0]
    E = np.sqrt(m * m + (p3 ** 2).sum(axis=1))
    return np.concatenate([E[:, None], p3], axis=1)


def test_clifford_algebra():
    for mu in range(4):
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            np.testing.assert_allclose(ac, 2 * METRIC[mu, nu] * np.eye(4), atol=1e-15)


def test_dirac_equation():
    for m in (0.0, 173.0):
        p = _momenta(m)
        ps = slash(p)
        for lam in (-1, 1):
            u = spinor_u(p, m, lam)
            v = spinor_v(p, m, lam)
            scale = p[:, 0:1]
            np.testing.assert_allclose(np.einsum("nij,nj->ni", ps, u) - m * u, 0, atol=1e-12 * scale.max() ** 1.5)
            np.testing.assert_allclose(np.einsum("nij,nj->ni", ps, v) + m * v, 0, atol=1e-12 * scale.max() ** 1.5)


def test_spin_sums():
    for m in (0.0, 173.0):
        p = _momenta(m)
        su = sum(np.einsum("ni,nj->nij", spinor_u(p, m, l), bar(spinor_u(p, m, l))) for l in (-1, 1))
        sv = sum(np.einsum("ni,nj->nij", spinor_v(p, m, l), bar(spinor_v(p, m, l))) for l in (-1, 1))
        np.testing.assert_allclose(su, slash(p) + m * np.eye(4), atol=1e-11 * p[:, 0].max())
        np.testing.assert_allclose(sv, slash(p) - m * np.eye(4), atol=1e-11 * p[:, 0].max())


def test_helicity_eigenstates_massless():
    """Massless u(p,+) is right-handed: P_L u = 0 (lower components only)."""
    p = _momenta(0.0)
    u = spinor_u(p, 0.0, 1)
    np.testing.assert_allclose(u[:, :2], 0, atol=1e-12)
    u = spinor_u(p, 0.0, -1)
    np.testing.assert_allclose(u[:, 2:], 0, atol=1e-12)


def test_polarisation_vectors():
    k = _momenta(0.0)
    khat = k[:, 1:] / k[:, 0:1]
    for lam in (-1, 1):
        e = polarisation(k, lam)
        np.testing.assert_allclose(dot(e, k), 0, atol=1e-12)
        np.testing.assert_allclose(dot(e, e.conj()), -1, atol=1e-14)
        np.testing.assert_allclose(dot(e, e), 0, atol=1e-14)
    tot = sum(np.einsum("ni,nj->nij", polarisation(k, l)[:, 1:], polarisation(k, l)[:, 1:].conj())
              for l in (-1, 1))
    ref = np.eye(3)[None] - np.einsum("ni,nj->nij", khat, khat)
    np.testing.assert_allclose(tot, ref, atol=1e-14)
