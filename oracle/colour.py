"""Explicit SU(3) colour algebra (oracle, FP64).

T^a = lambda^a / 2 with the eight Gell-Mann matrices, so Tr(T^a T^b) = delta^ab/2;
f^abc is obtained numerically from the commutator, f^abc = -2i Tr([T^a,T^b] T^c).
Colour-charge operators on an external leg in the all-outgoing convention:
  * fundamental index (outgoing quark, incoming antiquark):   (T^a)_{i i'}
  * antifundamental index (outgoing antiquark, incoming quark): -(T^a)_{i' i}
  * adjoint index (gluon):                                       -i f^{a b b'}
so that every colour-invariant tensor c satisfies sum_legs T_leg c = 0.
The generators exist in complex128 (the oracle proper) and, for the extended-precision
evaluations that arbitrate float64 disagreements, in the complex type of np.longdouble
(generators(dtype)); both are built by the same steps.
"""
from __future__ import annotations

import numpy as np

NC = 3
CF = (NC * NC - 1) / (2.0 * NC)
CA = float(NC)
TR = 0.5


def gell_mann(dtype=complex) -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=dtype)
    r3 = np.sqrt(np.zeros(1, dtype=dtype).real.dtype.type(3))  # sqrt(3) in that precision
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / r3
    lam[7][2, 2] = -2 / r3
    return lam


def _structure_constants(T: np.ndarray) -> np.ndarray:
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    f = -2j * np.einsum("abik,cki->abc", comm, T)
    assert np.max(np.abs(f.imag)) < 1e-14
    return f.real


_GENS: dict = {}


def generators(dtype=complex):
    """(T^a, f^abc, -i f^abc) with T^a = lambda^a / 2, in the given complex type."""
    key = np.dtype(dtype)
    if key not in _GENS:
        T_ = gell_mann(key) / 2
        F_ = _structure_constants(T_)
        _GENS[key] = (T_, F_, -1j * F_)
    return _GENS[key]


T, F, ADJ = generators(complex)  # ADJ: (T_adj^a)_{b c} = -i f^{abc}


def charge_matrices(kind: str, dtype=complex) -> np.ndarray:
    """Colour-charge generators acting on one leg's index: (8, d, d) with
    (T_leg^a c)[i] = sum_i' M[a, i, i'] c[i']."""
    T_, _, ADJ_ = generators(dtype)
    if kind == "fund":
        return T_
    if kind == "antifund":
        return -np.transpose(T_, (0, 2, 1))
    if kind == "adj":
        return ADJ_
    raise ValueError(kind)
