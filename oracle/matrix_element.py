"""Squared tree matrix elements, colour- and spin-correlated Borns (oracle, FP64).

|M|^2 = (1/avg) sum_helicities sum_colours |sum_diagrams|^2  (Sec. 2.1, Eq. (born);
Sec. 2.2, Eq. (real)).  avg = initial spins (2 each) x initial colours (3 or 8 each)
divided by the identical-final-particle factor.  Couplings: g_s = sqrt(4 pi alpha_s),
e = sqrt(4 pi alpha).  Units: GeV, |M|^2 for 2->n in GeV^(4-2n).

Colour-correlated Born (needed by the soft counterterm, Sec. 2.2 / Sec. 4.2):
  B_kl = (1/avg) sum_hel <M| T_k . T_l |M>, k,l over coloured legs (k = l allowed).
Spin-correlated Born (needed by the g -> g g collinear counterterm):
  B_perp = (1/avg) sum_{other hel} sum_colours |M(eps_leg = e_perp)|^2 with a real
  unit space-like polarisation vector e_perp for one gluon leg.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .diagrams import Diagrams, Process, helicities
from .dirac import ctype

MT = 173.0
_QCD_T = frozenset({("t", "g"), "ggg", "gggg"})

PROCESSES = {
    "ee_uu": Process("ee_uu", ("e+", "e-", "u", "u~"), frozenset({("e", "a"), ("u", "a")})),
    "ee_uug": Process("ee_uug", ("e+", "e-", "u", "u~", "g"),
                      frozenset({("e", "a"), ("u", "a"), ("u", "g")})),
    "gg_tt": Process("gg_tt", ("g", "g", "t", "t~"), _QCD_T, {"t": MT}),
    "gg_ttg": Process("gg_ttg", ("g", "g", "t", "t~", "g"), _QCD_T, {"t": MT}),
    "gg_ttgg": Process("gg_ttgg", ("g", "g", "t", "t~", "g", "g"), _QCD_T, {"t": MT},
                       ident_factor=0.5),
    "uu_tt": Process("uu_tt", ("u", "u~", "t", "t~"), _QCD_T | {("u", "g")}, {"t": MT}),
    "uu_ttg": Process("uu_ttg", ("u", "u~", "t", "t~", "g"), _QCD_T | {("u", "g")}, {"t": MT}),
}


@dataclass
class Couplings:
    alpha: float = 1.0 / 132.507
    alpha_s: float = 0.118

    def as_dict(self):
        return {"gs": math.sqrt(4.0 * math.pi * self.alpha_s),
                "e": math.sqrt(4.0 * math.pi * self.alpha)}


_DIAG_CACHE: dict = {}


def diagrams(name: str) -> Diagrams:
    if name not in _DIAG_CACHE:
        _DIAG_CACHE[name] = Diagrams(PROCESSES[name])
    return _DIAG_CACHE[name]


_GRAM_CACHE: dict = {}


def gram(name: str, k: int | None = None, l: int | None = None, dtype=complex) -> np.ndarray:
    """Colour Gram matrix (or colour-correlated one for legs k, l) in the given complex
    type: complex128 for the oracle proper, that of np.longdouble for extended precision."""
    key = (name, k, l, np.dtype(dtype))
    if key not in _GRAM_CACHE:
        d = diagrams(name)
        _GRAM_CACHE[key] = d.gram(dtype) if k is None else d.gram_correlated(k, l, dtype)
    return _GRAM_CACHE[key]


def to_points(p_soa: np.ndarray) -> np.ndarray:
    """SoA p[4][n_leg][N] -> (N, n_leg, 4)."""
    return np.ascontiguousarray(np.transpose(p_soa, (2, 1, 0)))


def _chunks(N: int, name: str):
    d = diagrams(name)
    H = 2 ** d.n
    per = max(1, int(1e6 // (H * max(1, len(d.terms)))))
    for a in range(0, N, per):
        yield slice(a, min(N, a + per))


def me2(name: str, p: np.ndarray, cp: Couplings = Couplings(), grams=None,
        fixed_hel=None, override=None) -> np.ndarray:
    """Helicity- and colour-summed, averaged |M|^2 for points p (N, n_leg, 4).

    ``grams``: list of colour matrices to contract with (default: the plain Gram
    matrix); returns an array (len(grams), N) in that case, else (N,).
    """
    d = diagrams(name)
    hel = helicities(d.n, fixed_hel)
    G_list = [gram(name, dtype=ctype(p))] if grams is None else grams
    out = np.zeros((len(G_list), p.shape[0]), dtype=p.dtype)
    avg = d.proc.average()
    for sl in _chunks(p.shape[0], name):
        ov = None if override is None else {k: v[sl] for k, v in override.items()}
        A = d.amplitudes(p[sl], hel, cp.as_dict(), ov)
        for ig, G in enumerate(G_list):
            val = np.einsum("nht,ts,nhs->n", A.conj(), G, A)
            out[ig, sl] = val.real / avg
    return out[0] if grams is None else out


def coloured_legs(name: str):
    d = diagrams(name)
    return [i for i in range(d.n) if d.proc.colour_dim(i) > 1]


def colour_correlated(name: str, p: np.ndarray, cp: Couplings = Couplings()):
    """B_kl for all ordered pairs of coloured legs: dict {(k,l): (N,)}."""
    legs = coloured_legs(name)
    pairs = [(k, l) for k in legs for l in legs]
    G = [gram(name, k, l, dtype=ctype(p)) for k, l in pairs]
    vals = me2(name, p, cp, grams=G)
    return {pr: vals[i] for i, pr in enumerate(pairs)}


def spin_correlated(name: str, p: np.ndarray, leg: int, e_perp: np.ndarray,
                    cp: Couplings = Couplings()) -> np.ndarray:
    """Born with gluon ``leg`` polarised along the real vector e_perp (N,4)."""
    return me2(name, p, cp, fixed_hel={leg: 1}, override={leg: e_perp})
