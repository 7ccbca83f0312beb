"""FKS real-minus-counterterm weight (oracle, FP64).

The paper uses FKS subtraction (Sec. 2.2, refs. Frixione-Kunszt-Signer 1996 and
Frixione 1997) and notes that FKS splits phase space into sectors with their own
kinematic parametrisation (Sec. 4.2); the branch-free loop of Algorithm 2
evaluates the real, soft and collinear terms for every point and then zeroes
those whose cuts fail.  The formulas below are the standard FKS ones, restated.

Sectors.  For an FKS gluon i and partner j, S_ij = (1/d_ij) / sum_kl (1/d_kl)
with the angle-only d_ij = 1 - cos(theta_ij) (partonic centre-of-mass frame).

Variables.  xi = 2 E_i / sqrt(s);  y = cos(theta_ij) w.r.t. the partner direction
(final-state partner j) or the beam j (initial-state partner); phi = azimuth of i.

Final-state (massless) map, partner j, recoil k (the other final parton):
  Born:   kb_j = (sqrt(s)/2)(1, n_j),  kb_k = (sqrt(s)/2)(1, -n_j);
  real:   E_j = sqrt(s)(1-xi)/(2 - xi(1-y)),  k_k = P - k_j - k_i;
  dPhi_3 = dPhi_2 xi K dxi dy dphi,  K = s (1-xi) / (16 pi^3 (2 - xi(1-y))^2).
Initial-state map, beam j, heavy pair Q Qbar recoiling with mass^2 s(1-xi):
  the pair's rest-frame direction n* is kept; soft Born = pair at sqrt(s) along n*;
  collinear Born = beams (1-xi) k_j and k_other, pair boosted along the beam axis;
  K = s beta(s(1-xi)) / (64 pi^3 beta(s)),  beta(x) = sqrt(1 - 4 m^2 / x).

Subtracted weight of a sector (plus-distributions (1/xi)_c, (1/(1-y))_delta):
  G(xi,y) = xi^2 (1-y) R S_ij K,
  W = [G(xi,y) - Th(xi_c-xi) G(0,y) - Th(y-1+delta) G(xi,1)
       + Th(xi_c-xi) Th(y-1+delta) G(0,1)] / (xi^2 (1-y) K(xi,y)).
Limits (evaluated analytically with Born counter-kinematics):
  soft:      xi^2 R -> -(4 g^2/s) sum_{k,l} (pb_k.pb_l)/((pb_k.q)(pb_l.q)) B_kl,
             q = (1, n_i), k,l over all coloured Born legs including k = l;
  final-state collinear q -> q g:  xi^2 (1-y) R -> [2 xi/(s(1-xi))] 2 g^2 P_qq(1-xi) B;
  initial-state collinear (z = 1-xi):
             xi^2 (1-y) R -> (2 xi/s)(1/z) 2 g^2 <P_aa(z)> with
             P_qq B = C_F (1+z^2)/(1-z) B,
             P_gg B = 2 C_A [(z/(1-z) + z(1-z)) B + 2 ((1-z)/z) B_perp],
             B_perp the Born with the splitting gluon polarised along the
             direction of the emitted gluon's transverse momentum.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import colour
from .cuts import Cuts, passes
from .dirac import dot
from .matrix_element import (MT, Couplings, colour_correlated, coloured_legs, me2,
                             spin_correlated)


@dataclass
class FKSParams:
    xi_cut: float = 0.5
    delta: float = 1.0


REAL_PROCESSES = {
    # real process: (born process, FKS gluon leg, [(partner leg, kind)], heavy mass)
    "ee_uug": ("ee_uu", 4, [(2, "fsr"), (3, "fsr")], 0.0),
    "gg_ttg": ("gg_tt", 4, [(0, "isr"), (1, "isr")], MT),
    "uu_ttg": ("uu_tt", 4, [(0, "isr"), (1, "isr")], MT),
}


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _boost(p, b):
    """Pure boost of p (N,4) by velocity b (N,3)."""
    b2 = np.sum(b * b, axis=-1)
    g = 1.0 / np.sqrt(1.0 - b2)
    bp = np.sum(b * p[:, 1:], axis=-1)
    g2 = np.where(b2 > 0, (g - 1.0) / np.where(b2 > 0, b2, 1.0), 0.0)
    out = np.empty_like(p)
    out[:, 0] = g * (p[:, 0] + bp)
    out[:, 1:] = p[:, 1:] + ((g2 * bp + g * p[:, 0])[:, None]) * b
    return out


def sector_functions(k: np.ndarray, i_fks: int, partners) -> np.ndarray:
    """S_ij for every sector (n_sectors, N) from the real momenta k (N, n, 4)."""
    ni = _unit(k[:, i_fks, 1:])
    inv_d = []
    for j, _ in partners:
        nj = _unit(k[:, j, 1:])
        inv_d.append(1.0 / (1.0 - np.sum(ni * nj, axis=-1)))
    inv_d = np.array(inv_d)
    return inv_d / inv_d.sum(axis=0)


@dataclass
class SectorKinematics:
    xi: np.ndarray
    y: np.ndarray
    phi: np.ndarray
    born_soft: np.ndarray      # (N, n_born, 4)
    born_coll: np.ndarray      # (N, n_born, 4)
    q_dir: np.ndarray          # (N, 4) = (1, n_i)
    K: np.ndarray              # Jacobian K(xi, y) at the real point
    K_soft: np.ndarray         # K(0, y)
    K_coll: np.ndarray         # K(xi, 1)
    e_perp: np.ndarray         # (N, 4) transverse direction of the emission


def fsr_map(k: np.ndarray, i_fks: int, j: int, other: int) -> SectorKinematics:
    """Inverse final-state map of a massless 2 -> 3 point (N, 5, 4) in its c.m. frame."""
    rs = k[:, 0, 0] + k[:, 1, 0]
    s = rs * rs
    xi = 2.0 * k[:, i_fks, 0] / rs
    ni = _unit(k[:, i_fks, 1:])
    nj = _unit(k[:, j, 1:])
    y = np.sum(ni * nj, axis=-1)
    z = np.array([0.0, 0.0, 1.0])
    ea = _unit(z - np.sum(z * nj, axis=-1, keepdims=True) * nj)
    eb = np.cross(nj, ea)
    phi = np.arctan2(np.sum(ni * eb, axis=-1), np.sum(ni * ea, axis=-1))
    born = np.delete(k, i_fks, axis=1).copy()
    born[:, j, 0] = 0.5 * rs
    born[:, j, 1:] = 0.5 * rs[:, None] * nj
    born[:, other, 0] = 0.5 * rs
    born[:, other, 1:] = -0.5 * rs[:, None] * nj
    K = s * (1.0 - xi) / (16.0 * math.pi ** 3 * (2.0 - xi * (1.0 - y)) ** 2)
    K0 = s / (64.0 * math.pi ** 3) * np.ones_like(xi)
    K1 = s * (1.0 - xi) / (64.0 * math.pi ** 3)
    e_perp = np.zeros_like(k[:, 0])
    e_perp[:, 1:] = ni - y[:, None] * nj
    e_perp[:, 1:] = _unit(e_perp[:, 1:])
    q = np.concatenate([np.ones((k.shape[0], 1), dtype=k.dtype), ni], axis=1)
    return SectorKinematics(xi, y, phi, born, born, q, K, K0, K1, e_perp)


def isr_map(k: np.ndarray, i_fks: int, j: int, mass: float) -> SectorKinematics:
    """Inverse initial-state map of a 2 -> Q Qbar g point (N, 5, 4) in its c.m. frame."""
    N = k.shape[0]
    rs = k[:, 0, 0] + k[:, 1, 0]
    s = rs * rs
    xi = 2.0 * k[:, i_fks, 0] / rs
    ni = _unit(k[:, i_fks, 1:])
    beam = _unit(k[:, j, 1:])
    y = np.sum(ni * beam, axis=-1)
    phi = np.arctan2(ni[:, 1], ni[:, 0])
    Q = k[:, 0] + k[:, 1] - k[:, i_fks]
    kstar = _boost(k[:, 2], -Q[:, 1:] / Q[:, 0:1])
    nstar = _unit(kstar[:, 1:])
    beta = np.sqrt(1.0 - 4.0 * mass * mass / s)
    # soft Born: pair at sqrt(s) along n*
    soft = k[:, :4].copy()
    soft[:, 2, 0] = soft[:, 3, 0] = 0.5 * rs
    soft[:, 2, 1:] = 0.5 * (rs * beta)[:, None] * nstar
    soft[:, 3, 1:] = -soft[:, 2, 1:]
    # collinear Born: beam j scaled by (1-xi), pair boosted along the beam axis
    coll = k[:, :4].copy()
    coll[:, j] *= (1.0 - xi)[:, None]
    Qc = coll[:, 0] + coll[:, 1]
    M = np.sqrt(s * (1.0 - xi))
    betaQ = np.sqrt(np.maximum(0.0, 1.0 - 4.0 * mass * mass / (s * (1.0 - xi))))
    t_rest = np.zeros((N, 4), dtype=k.dtype)
    t_rest[:, 0] = 0.5 * M
    t_rest[:, 1:] = 0.5 * (M * betaQ)[:, None] * nstar
    tb_rest = t_rest.copy()
    tb_rest[:, 1:] *= -1.0
    bc = Qc[:, 1:] / Qc[:, 0:1]
    coll[:, 2] = _boost(t_rest, bc)
    coll[:, 3] = _boost(tb_rest, bc)
    K = s * betaQ / (64.0 * math.pi ** 3 * beta)
    K0 = s / (64.0 * math.pi ** 3) * np.ones_like(xi)
    e_perp = np.zeros((N, 4), dtype=k.dtype)
    e_perp[:, 1] = np.cos(phi)
    e_perp[:, 2] = np.sin(phi)
    q = np.concatenate([np.ones((N, 1), dtype=k.dtype), ni], axis=1)
    return SectorKinematics(xi, y, phi, soft, coll, q, K, K0, K.copy(), e_perp)


def soft_limit(born: str, pb: np.ndarray, q: np.ndarray, s: np.ndarray, cp: Couplings):
    """lim xi^2 R = -(4 g^2/s) sum_{k,l} (pb_k.pb_l)/((pb_k.q)(pb_l.q)) B_kl."""
    g2 = 4.0 * math.pi * cp.alpha_s
    Bkl = colour_correlated(born, pb, cp)
    tot = np.zeros(pb.shape[0], dtype=pb.dtype)
    for (a, b), v in Bkl.items():
        tot += dot(pb[:, a], pb[:, b]) / (dot(pb[:, a], q) * dot(pb[:, b], q)) * v
    return -(4.0 * g2 / s) * tot


def collinear_limit(real: str, born: str, kind: str, j: int, xi, pb, e_perp, s, cp):
    """lim_{y->1} xi^2 (1-y) R for partner j (final- or initial-state)."""
    g2 = 4.0 * math.pi * cp.alpha_s
    B = me2(born, pb, cp)
    z = 1.0 - xi
    if kind == "fsr":
        # q -> q g, P_qq(z) = C_F (1+z^2)/(1-z);  xi P_qq = C_F (1 + (1-xi)^2)
        return 2.0 / (s * (1.0 - xi)) * 2.0 * g2 * colour.CF * (1.0 + z * z) * B
    leg = born_leg_name(born, j)
    if leg == "g":
        Bp = spin_correlated(born, pb, j, e_perp, cp)
        xiP = 2.0 * colour.CA * ((z + xi * xi * z) * B + 2.0 * (xi * xi / z) * Bp)
    else:
        xiP = colour.CF * (1.0 + z * z) * B
    return (2.0 / s) * (1.0 / z) * 2.0 * g2 * xiP


def born_leg_name(born: str, j: int) -> str:
    from .matrix_element import PROCESSES
    return PROCESSES[born].legs[j]


def real_subtracted(real: str, k: np.ndarray, fp: FKSParams = FKSParams(),
                    cp: Couplings = Couplings(), detail: bool = False, cuts: Cuts | None = None):
    """Sum over sectors of the subtracted real weight per point (ME units; multiply by
    the phase-space weight of the generator).  ``k``: real momenta (N, n, 4).

    ``cuts`` (oracle.cuts): each term is kept only where its own kinematics pass
    (Algorithm 2): the real at k, the soft and soft-collinear terms at the sector's soft
    Born counter-event, the collinear term at the sector's collinear Born counter-event."""
    born, i_fks, partners, mass = REAL_PROCESSES[real]
    cut_on = cuts is not None and cuts.active(real)
    rs = k[:, 0, 0] + k[:, 1, 0]
    s = rs * rs
    S = sector_functions(k, i_fks, partners)
    # Algorithm 2: evaluate every term for every point, then mask
    R = me2(real, k, cp)
    total = np.zeros(k.shape[0], dtype=k.dtype)
    inside = np.ones(k.shape[0], dtype=bool)
    parts = []
    for isec, (j, kind) in enumerate(partners):
        if kind == "fsr":
            other = [x for x, _ in partners if x != j][0]
            kin = fsr_map(k, i_fks, j, other)
        else:
            kin = isr_map(k, i_fks, j, mass)
        xi, y = kin.xi, kin.y
        # sector functions in the soft limit: gluon direction vs Born directions
        ni = kin.q_dir[:, 1:]
        inv_d = []
        for jj, _ in partners:
            nj = _unit(kin.born_soft[:, jj, 1:])
            inv_d.append(1.0 / (1.0 - np.sum(ni * nj, axis=-1)))
        S_soft = inv_d[isec] / np.sum(inv_d, axis=0)
        G = xi * xi * (1.0 - y) * R * S[isec] * kin.K
        G_soft = (1.0 - y) * S_soft * kin.K_soft * soft_limit(born, kin.born_soft, kin.q_dir, s, cp)
        G_coll = kin.K_coll * collinear_limit(real, born, kind, j, xi, kin.born_coll,
                                               kin.e_perp, s, cp)
        G_sc = kin.K_soft * collinear_limit(real, born, kind, j, np.zeros_like(xi),
                                            kin.born_soft, kin.e_perp, s, cp)
        th_s = (xi < fp.xi_cut).astype(float)
        th_c = (y > 1.0 - fp.delta).astype(float)
        if cut_on:
            c_r = passes(real, k, cuts).astype(float)
            c_s = passes(born, kin.born_soft, cuts).astype(float)
            c_c = passes(born, kin.born_coll, cuts).astype(float)
            G, G_soft, G_coll, G_sc = G * c_r, G_soft * c_s, G_coll * c_c, G_sc * c_s
        W = (G - th_s * G_soft - th_c * G_coll + th_s * th_c * G_sc) / (xi * xi * (1.0 - y) * kin.K)
        total += W
        with np.errstate(invalid="ignore"):
            inside &= (xi > 0.0) & (xi < 1.0) & (1.0 - y > 0.0)
        parts.append(dict(xi=xi, y=y, G=G, G_soft=G_soft, G_coll=G_coll, G_sc=G_sc, W=W,
                          S=S[isec], K=kin.K, RS=R * S[isec]))
    # the boundary of the FKS domain (xi = 0 or 1, or the emission exactly along a
    # sector's reference direction) has measure zero, and the subtracted weight with its
    # 1 / (xi^2 (1 - y)) is not defined there: such points carry weight 0
    total = np.where(inside, total, 0.0)
    return (total, parts) if detail else total
