"""Explicit SU(3) colour algebra (oracle, FP64).

T^a = lambda^a / 2 with the eight Gell-Mann matrices, so Tr(T^a T^b) = delta^ab/2;
f^abc is obtained numerically from the commutator, f^abc = -2i Tr([T^a,T^b] T^c).
Colour-charge operators on an external leg in the all-outgoing convention:
  * fundamental index (outgoing quark, incoming antiquark):   (T^a)_{i i'}
  * antifundamental index (outgoing antiquark, incoming quark): -(T^a)_{i' i}
  * adjoint index (gluon):                                       -i f^{a b b'}
so that every colour-invariant tensor c satisfies sum_legs T_leg c = 0.
"""
from __future__ import annotations

import numpy as np

NC = 3
CF = (NC * NC - 1) / (2.0 * NC)
CA = float(NC)
TR = 0.5


def gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=complex)
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
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


T = gell_mann() / 2.0


def _structure_constants() -> np.ndarray:
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    f = -2j * np.einsum("abik,cki->abc", comm, T)
    assert np.max(np.abs(f.imag)) < 1e-14
    return f.real


F = _structure_constants()
ADJ = -1j * F  # (T_adj^a)_{b c} = -i f^{abc}


def charge_matrices(kind: str) -> np.ndarray:
    """Colour-charge generators acting on one leg's index: (8, d, d) with
    (T_leg^a c)[i] = sum_i' M[a, i, i'] c[i']."""
    if kind == "fund":
        return T
    if kind == "antifund":
        return -np.transpose(T, (0, 2, 1))
    if kind == "adj":
        return ADJ
    raise ValueError(kind)
