"""Pins for the oracle's explicit SU(3) colour algebra and diagram colour tensors."""
import itertools

import numpy as np
import pytest

import synth
from oracle import colour
from oracle import matrix_element as me
from oracle.diagrams import helicities
from oracle.matrix_element import Couplings, to_points

T, F = colour.T, colour.F


def test_generator_normalisation_and_casimirs():
    np.testing.assert_allclose(np.einsum("aij,bji->ab", T, T), 0.5 * np.eye(8), atol=1e-15)
    np.testing.assert_allclose(np.einsum("aij,ajk->ik", T, T), colour.CF * np.eye(3), atol=1e-15)
    np.testing.assert_allclose(np.einsum("acd,bcd->ab", F, F), colour.CA * np.eye(8), atol=1e-14)
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    np.testing.assert_allclose(comm, 1j * np.einsum("abc,cik->abik", F, T), atol=1e-15)
    for p in itertools.permutations(range(3)):
        sign = np.linalg.det(np.eye(3)[list(p)])
        np.testing.assert_allclose(np.transpose(F, p), sign * F, atol=1e-15)
    # Jacobi identity
    jac = (np.einsum("abe,ecd->abcd", F, F) + np.einsum("bce,ead->abcd", F, F)
           + np.einsum("cae,ebd->abcd", F, F))
    np.testing.assert_allclose(jac, 0, atol=1e-14)


@pytest.mark.parametrize("name", ["ee_uug", "gg_tt", "gg_ttg", "uu_tt", "uu_ttg", "gg_ttgg"])
def test_colour_conservation_on_every_diagram(name):
    d = me.diagrams(name)
    legs = me.coloured_legs(name)
    tot = sum(d.charge_on_leg(k) for k in legs)
    scale = np.abs(d.colour_tensors()).max()
    assert np.abs(tot).max() < 1e-13 * scale


@pytest.mark.parametrize("name,seed", [("gg_tt", 1), ("gg_ttg", 2), ("uu_ttg", 3)])
def test_brute_force_colour_sum(name, seed):
    """sum over every colour assignment of |sum_t c_t A_t|^2 == A^dag G A."""
    d = me.diagrams(name)
    k = to_points(synth.flat_points(name, 3, seed).p)
    hel = helicities(d.n)
    A = d.amplitudes(k, hel, Couplings().as_dict())
    C = d.colour_tensors()
    brute = (np.abs(np.einsum("nht,td->nhd", A, C)) ** 2).sum(axis=(1, 2))
    gram = np.einsum("nht,ts,nhs->n", A.conj(), me.gram(name), A).real
    np.testing.assert_allclose(gram, brute, rtol=1e-12)


def _strings(order_legs, shape, q_axis, qb_axis):
    """Colour tensors (T^{a_s1} ... T^{a_sk})_{i j} for every ordering of the gluon legs."""
    out = []
    for perm in itertools.permutations(order_legs):
        M = np.zeros(shape, dtype=complex)
        for idx in itertools.product(*[range(8)] * len(perm)):
            prod = np.eye(3, dtype=complex)
            for a in idx:
                prod = prod @ T[a]
            sl = [slice(None)] * len(shape)
            for leg, a in zip(perm, idx):
                sl[leg] = a
            M[tuple(sl)] = prod if q_axis < qb_axis else prod.T
        out.append(M.reshape(-1))
    return np.array(out)


def test_gg_tt_colour_matrix():
    """Strings (T^a T^b)_{ij}, (T^b T^a)_{ij}: C = (1/3) [[16,-2],[-2,16]]."""
    S = _strings([0, 1], (8, 8, 3, 3), 2, 3)
    C = S.conj() @ S.T
    np.testing.assert_allclose(3 * C, [[16, -2], [-2, 16]], atol=1e-13)


@pytest.mark.parametrize("name,gluons,shape", [
    ("gg_tt", [0, 1], (8, 8, 3, 3)),
    ("gg_ttg", [0, 1, 4], (8, 8, 3, 3, 8)),
])
def test_diagram_colour_in_string_span(name, gluons, shape):
    S = _strings(gluons, shape, 2, 3)
    C = me.diagrams(name).colour_tensors()
    coef, *_ = np.linalg.lstsq(S.T, C.T, rcond=None)
    resid = C.T - S.T @ coef
    assert np.abs(resid).max() < 1e-13


def test_gg_ttgg_string_colour_matrix_is_integer_over_54():
    """The 24 strings of four gluons: diag = N_c C_F^4 = 512/54, 54 C integral, and every
    diagram's colour tensor lies in their span."""
    d = me.diagrams("gg_ttgg")
    shape = d.colour_shape()  # (8,8,3,3,8,8)
    gl = [0, 1, 4, 5]
    # build strings via einsum chains (faster than loops)
    out = []
    for perm in itertools.permutations(gl):
        M = np.einsum("aij,bjk,ckl,dlm->abcdim", T, T, T, T)  # (a,b,c,d,i,m)
        # place gluon index of perm[r] at leg perm[r]
        full = np.zeros(shape, dtype=complex)
        # axes of M: (g_perm0, g_perm1, g_perm2, g_perm3, i, j); target legs (0,1,2,3,4,5)
        src = {perm[0]: 0, perm[1]: 1, perm[2]: 2, perm[3]: 3, 2: 4, 3: 5}
        full = np.transpose(M, [src[l] for l in range(6)])
        out.append(full.reshape(-1))
    S = np.array(out)
    C = S.conj() @ S.T
    np.testing.assert_allclose(np.diag(C).real, 512 / 54, atol=1e-12)
    C54 = 54 * C.real
    np.testing.assert_allclose(C54, np.round(C54), atol=1e-10)
    assert np.abs(C.imag).max() < 1e-13
    coef, *_ = np.linalg.lstsq(S.T, d.colour_tensors().T, rcond=None)
    assert np.abs(d.colour_tensors().T - S.T @ coef).max() < 1e-12
