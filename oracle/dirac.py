"""Minkowski metric, Dirac matrices and helicity wavefunctions (oracle, FP64).

Conventions (standard QFT, e.g. Peskin & Schroeder; the paper fixes none):
  * metric (+,-,-,-); four-vectors carry upper indices, last axis = (E,px,py,pz);
  * chiral (Weyl) representation: gamma^0 = [[0,1],[1,0]],
    gamma^k = [[0,sigma^k],[-sigma^k,0]];
  * helicity spinors (lambda = +-1), with chi_lambda the two-spinor of helicity
    lambda along p/|p| and omega_+- = sqrt(E +- |p|):
        u(p,l) = ( omega_{-l} chi_l ,  omega_{+l} chi_l )
        v(p,l) = ( -l omega_{+l} chi_{-l} ,  l omega_{-l} chi_{-l} )
    chi_+ = (|p|+pz, px+i py)/sqrt(2|p|(|p|+pz)),
    chi_- = (-px+i py, |p|+pz)/sqrt(2|p|(|p|+pz)); for p along -z the limits
    chi_+ = (0,1), chi_- = (-1,0) are used;
  * polarisation vectors eps(k,l) = (-l e1 - i e2)/sqrt(2) with
    e1 = (0, cos(th)cos(ph), cos(th)sin(ph), -sin(th)), e2 = (0, -sin(ph), cos(ph), 0).
All arrays broadcast over leading (point) axes.  The working precision follows the
momenta: float64 momenta give float64/complex128 results (the oracle proper);
np.longdouble momenta carry every step in extended precision, which the tests use to
arbitrate between two float64 evaluations that differ.
"""
from __future__ import annotations

import numpy as np

METRIC = np.diag([1.0, -1.0, -1.0, -1.0])

_s1 = np.array([[0, 1], [1, 0]], dtype=complex)
_s2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
_s3 = np.array([[1, 0], [0, -1]], dtype=complex)
_I2 = np.eye(2, dtype=complex)
_Z2 = np.zeros((2, 2), dtype=complex)


def _blk(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.stack([
    _blk(_Z2, _I2, _I2, _Z2),
    _blk(_Z2, _s1, -_s1, _Z2),
    _blk(_Z2, _s2, -_s2, _Z2),
    _blk(_Z2, _s3, -_s3, _Z2),
])  # GAMMA[mu] = gamma^mu
GAMMA5 = 1j * GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def ctype(x) -> np.dtype:
    """Complex dtype of the precision of array x (complex128 for float64 input)."""
    return np.result_type(np.asarray(x).dtype, np.complex64)


def dot(a, b):
    """Minkowski product a.b over the last axis (works for complex arrays, no conjugation)."""
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def lower(a):
    """a_mu = g_{mu nu} a^nu."""
    return a * np.array([1.0, -1.0, -1.0, -1.0])


def slash(a):
    """gamma^mu a_mu as [..., 4, 4]."""
    return np.einsum("...m,mij->...ij", lower(a), GAMMA)


def _chi(p, lam):
    """Helicity two-spinor chi_lam(p_hat), shape [..., 2]."""
    px, py, pz = p[..., 1], p[..., 2], p[..., 3]
    pa = np.sqrt(px * px + py * py + pz * pz)
    s = pa + pz
    ok = s > 0.0  # p exactly along -z: explicit limits below
    den = np.sqrt(np.where(ok, 2.0 * pa * s, 1.0))
    out = np.zeros(p.shape[:-1] + (2,), dtype=ctype(p))
    if lam > 0:
        out[..., 0] = np.where(ok, s / den, 0.0)
        out[..., 1] = np.where(ok, (px + 1j * py) / den, 1.0)
    else:
        out[..., 0] = np.where(ok, (-px + 1j * py) / den, -1.0)
        out[..., 1] = np.where(ok, s / den, 0.0)
    return out


def _omegas(p, mass):
    pa = np.sqrt(p[..., 1] ** 2 + p[..., 2] ** 2 + p[..., 3] ** 2)
    e = p[..., 0]
    wp = np.sqrt(np.maximum(e + pa, 0.0))
    wm = np.sqrt(np.maximum(e - pa, 0.0))
    if mass == 0.0:
        wm = np.zeros_like(wm)
    else:
        # E - |p| = m^2/(E + |p|) without cancellation
        wm = mass / np.where(wp > 0, wp, 1.0)
    return wp, wm


def spinor_u(p, mass, lam):
    """Dirac spinor u(p, lam) (column), shape [..., 4]."""
    wp, wm = _omegas(p, mass)
    chi = _chi(p, lam)
    top = (wm if lam > 0 else wp)[..., None] * chi
    bot = (wp if lam > 0 else wm)[..., None] * chi
    return np.concatenate([top, bot], axis=-1)


def spinor_v(p, mass, lam):
    """Dirac spinor v(p, lam) (column), shape [..., 4]."""
    wp, wm = _omegas(p, mass)
    chi = _chi(p, -lam)
    w_l = wp if lam > 0 else wm      # omega_{+lam}
    w_ml = wm if lam > 0 else wp     # omega_{-lam}
    top = (-lam * w_l)[..., None] * chi
    bot = (lam * w_ml)[..., None] * chi
    return np.concatenate([top, bot], axis=-1)


def bar(psi):
    """Dirac adjoint psi^dagger gamma^0 (row), shape [..., 4]."""
    return np.einsum("...i,ij->...j", psi.conj(), GAMMA[0])


def polarisation(k, lam):
    """Polarisation vector eps^mu(k, lam) of a massless vector boson, shape [..., 4]."""
    kx, ky, kz = k[..., 1], k[..., 2], k[..., 3]
    ka = np.sqrt(kx * kx + ky * ky + kz * kz)
    pt = np.sqrt(kx * kx + ky * ky)
    ct = kz / ka
    st = pt / ka
    has_pt = pt > 0.0
    cp = np.where(has_pt, kx / np.where(has_pt, pt, 1.0), 1.0)
    sp = np.where(has_pt, ky / np.where(has_pt, pt, 1.0), 0.0)
    zero = np.zeros_like(ka)
    e1 = np.stack([zero, ct * cp, ct * sp, -st], axis=-1)
    e2 = np.stack([zero, -sp, cp, zero], axis=-1)
    return (-lam * e1 - 1j * e2) / np.sqrt(ka.dtype.type(2))
