"""Seeded synthetic inputs: counter-based random numbers and phase-space points.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
no matrix-element, colour, FKS-mapping or counterterm arithmetic: it only turns a
seed into four-momenta (and the density with which they were drawn), so that the
CUDA path and the oracle can be fed identical points.

Layout of every momentum array: structure-of-arrays float64 ``p[comp][leg][n]``
with ``comp`` = (E, px, py, pz), legs in process order with the two incoming
partons first, ``n`` the fastest (contiguous) index.

Pieces:
  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter = (point index
    lo, point index hi, stream, draw block), key = (seed lo, seed hi).
  * uint32 pair -> double in (0,1): ((x0>>5)*2^26 + (x1>>6) + 0.5) * 2^-53.
  * RAMBO (Kleiss, Stirling, Ellis, Comput. Phys. Commun. 40 (1986) 359):
    flat massless n-body points with constant weight, plus the published
    massive rescaling with its per-point weight factor.
  * A flat 2-body generator for 2->2 with equal final masses.
  * Near-singular real-emission points (a soft or collinear gluon with a
    recoiling heavy pair), used to probe soft/collinear limits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------- Philox4x32-10
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32 with 10 rounds.  ``ctr``: uint32 array of shape (4, n).

    One round maps (c0,c1,c2,c3) with key (k0,k1) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
    the key is bumped by the Weyl constants (W0, W1) between rounds.
    """
    c = [np.asarray(ctr[i], dtype=np.uint64) for i in range(4)]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack([x.astype(np.uint32) for x in c])


def u01_from_pair(x0: np.ndarray, x1: np.ndarray) -> np.ndarray:
    """53-bit double in the open interval (0,1) from two uint32 words."""
    a = (np.asarray(x0, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (np.asarray(x1, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) * (1.0 / 9007199254740992.0)


def uniforms(seed: int, stream: int, n_points: int, n_draws: int,
             first_point: int = 0) -> np.ndarray:
    """(n_draws, n_points) uniforms in (0,1); point i, draw d uses Philox block d//2."""
    idx = np.arange(first_point, first_point + n_points, dtype=np.uint64)
    lo = (idx & _MASK32).astype(np.uint32)
    hi = (idx >> np.uint64(32)).astype(np.uint32)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = np.empty((n_draws, n_points))
    for blk in range((n_draws + 1) // 2):
        ctr = np.stack([lo, hi, np.full(n_points, stream, np.uint32),
                        np.full(n_points, blk, np.uint32)])
        x = philox4x32_10(ctr, key)
        out[2 * blk] = u01_from_pair(x[0], x[1])
        if 2 * blk + 1 < n_draws:
            out[2 * blk + 1] = u01_from_pair(x[2], x[3])
    return out


# ---------------------------------------------------------------- kinematics
def _beams(sqrt_s: float, n: int) -> np.ndarray:
    """Two massless incoming beams along +z and -z in the centre-of-mass frame."""
    p = np.zeros((4, 2, n))
    p[0, :, :] = 0.5 * sqrt_s
    p[3, 0, :] = 0.5 * sqrt_s
    p[3, 1, :] = -0.5 * sqrt_s
    return p


def rambo_massless(sqrt_s: float, n_out: int, u: np.ndarray):
    """Flat massless n-body phase space (RAMBO).  ``u``: (4*n_out, N) uniforms.

    Returns (p[4][n_out][N], weight) where the weight is the constant phase-space
    volume (2pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!).
    """
    N = u.shape[1]
    q = np.empty((4, n_out, N))
    for i in range(n_out):
        c = 2.0 * u[4 * i] - 1.0
        s = np.sqrt(1.0 - c * c)
        f = 2.0 * math.pi * u[4 * i + 1]
        q0 = -np.log(u[4 * i + 2] * u[4 * i + 3])
        q[0, i] = q0
        q[1, i] = q0 * s * np.cos(f)
        q[2, i] = q0 * s * np.sin(f)
        q[3, i] = q0 * c
    Q = q.sum(axis=1)
    M = np.sqrt(Q[0] ** 2 - Q[1] ** 2 - Q[2] ** 2 - Q[3] ** 2)
    b = -Q[1:] / M
    x = sqrt_s / M
    g = Q[0] / M
    a = 1.0 / (1.0 + g)
    p = np.empty_like(q)
    for i in range(n_out):
        bq = b[0] * q[1, i] + b[1] * q[2, i] + b[2] * q[3, i]
        p[0, i] = x * (g * q[0, i] + bq)
        for k in range(3):
            p[1 + k, i] = x * (q[1 + k, i] + b[k] * q[0, i] + a * bq * b[k])
    s = sqrt_s * sqrt_s
    w = (2.0 * math.pi) ** (4 - 3 * n_out) * (0.5 * math.pi) ** (n_out - 1) \
        * s ** (n_out - 2) / (math.factorial(n_out - 1) * math.factorial(n_out - 2))
    return p, np.full(N, w)


def rambo_massive(sqrt_s: float, masses, u: np.ndarray):
    """RAMBO with the massive rescaling step: k_i = (sqrt(m_i^2 + x^2 |p_i|^2), x p_i),
    x fixed by energy conservation (Newton iteration).  Per-point weight =
    W_massless * (sum|k|/sqrt(s))^(2n-3) * prod(|k|/E) * sqrt(s) / sum(|k|^2/E).
    """
    n = len(masses)
    p, w0 = rambo_massless(sqrt_s, n, u)
    m = np.asarray(masses, dtype=np.float64)[:, None]
    if not np.any(m):
        return p, w0
    pabs = p[0]
    x = np.full(p.shape[2], math.sqrt(max(0.0, 1.0 - (m.sum() / sqrt_s) ** 2)))
    for _ in range(60):
        e = np.sqrt(m * m + (x * pabs) ** 2)
        f = e.sum(axis=0) - sqrt_s
        df = (x * pabs * pabs / e).sum(axis=0)
        dx = f / df
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    k = np.empty_like(p)
    k[1:] = x * p[1:]
    kabs = x * pabs
    k[0] = np.sqrt(m * m + kabs * kabs)
    e = k[0]
    w = w0 * (kabs.sum(axis=0) / sqrt_s) ** (2 * n - 3) * np.prod(kabs / e, axis=0) \
        * sqrt_s / (kabs * kabs / e).sum(axis=0)
    return k, w


def two_body(sqrt_s: np.ndarray, mass: float, cos_theta: np.ndarray, phi: np.ndarray):
    """2 -> 2 with equal final masses in the centre-of-mass frame; weight beta/(8 pi)."""
    sqrt_s = np.asarray(sqrt_s, dtype=np.float64)
    N = cos_theta.shape[0]
    beta = np.sqrt(1.0 - 4.0 * mass * mass / (sqrt_s * sqrt_s))
    sin_t = np.sqrt(1.0 - cos_theta ** 2)
    p = np.zeros((4, 4, N))
    p[:, :2] = _beams(1.0, N) * sqrt_s
    e = 0.5 * sqrt_s
    k = e * beta
    p[0, 2] = e
    p[1, 2] = k * sin_t * np.cos(phi)
    p[2, 2] = k * sin_t * np.sin(phi)
    p[3, 2] = k * cos_theta
    p[0, 3] = e
    p[1:, 3] = -p[1:, 2]
    return p, beta / (8.0 * math.pi)


def with_beams(sqrt_s: float, p_out: np.ndarray) -> np.ndarray:
    """Prepend the two incoming beams to outgoing momenta p_out[4][n_out][N]."""
    N = p_out.shape[2]
    return np.ascontiguousarray(np.concatenate([_beams(sqrt_s, N), p_out], axis=1))


# ---------------------------------------------------------------- workloads
MT = 173.0


@dataclass
class Batch:
    """One batch of phase-space points: momenta p[4][n_ext][n] and generator weights."""
    process: str
    sqrt_s: float
    p: np.ndarray
    wgt: np.ndarray

    @property
    def n(self) -> int:
        return self.p.shape[2]


def flat_points(process: str, n: int, seed: int, sqrt_s: float | None = None,
                first_point: int = 0, stream: int = 0) -> Batch:
    """Flat (RAMBO) phase-space points for one of the library's processes."""
    spec = {
        "ee_uu": (100.0, [0.0, 0.0]),
        "ee_uug": (100.0, [0.0, 0.0, 0.0]),
        "gg_tt": (1000.0, [MT, MT]),
        "gg_ttg": (1000.0, [MT, MT, 0.0]),
        "gg_ttgg": (2000.0, [MT, MT, 0.0, 0.0]),
        "uu_tt": (1000.0, [MT, MT]),
        "uu_ttg": (1000.0, [MT, MT, 0.0]),
    }[process]
    rs = sqrt_s if sqrt_s is not None else spec[0]
    masses = spec[1]
    u = uniforms(seed, stream, n, 4 * len(masses), first_point)
    pout, w = rambo_massive(rs, masses, u)
    return Batch(process, rs, with_beams(rs, pout), w)


def gg_tt_scan(n: int, seed: int, first_point: int = 0, smin: float = 400.0,
               smax: float = 2000.0) -> Batch:
    """gg -> t tbar with partonic sqrt(s) ~ U[smin,smax], cos(theta) ~ U[-1,1], phi ~ U[0,2pi)."""
    u = uniforms(seed, 0, n, 3, first_point)
    rs = smin + (smax - smin) * u[0]
    p, w = two_body(rs, MT, 2.0 * u[1] - 1.0, 2.0 * math.pi * u[2])
    return Batch("gg_tt", float("nan"), np.ascontiguousarray(p), np.asarray(w))


def _boost(p: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Pure boost of four-vectors p[4][...] by velocity b[3][...] (rest frame -> lab)."""
    b2 = (b * b).sum(axis=0)
    g = 1.0 / np.sqrt(1.0 - b2)
    bp = (b * p[1:]).sum(axis=0)
    safe = np.where(b2 > 0, b2, 1.0)
    g2 = np.where(b2 > 0, (g - 1.0) / safe, 0.0)
    out = np.empty_like(p)
    out[0] = g * (p[0] + bp)
    out[1:] = p[1:] + (g2 * bp + g * p[0]) * b
    return out


def emission_points(sqrt_s: float, mass: float, e_frac: np.ndarray, cos_beam: np.ndarray,
                    phi: np.ndarray, cos_pair: np.ndarray, phi_pair: np.ndarray) -> np.ndarray:
    """2 -> Q Qbar g points with a chosen gluon: energy e_frac*sqrt(s)/2, polar angle
    cos_beam w.r.t. +z, azimuth phi; the Q Qbar pair is placed back to back in its own
    rest frame at angles (cos_pair, phi_pair) and boosted to recoil against the gluon.
    Used to place points close to the soft (e_frac -> 0) or collinear (|cos_beam| -> 1)
    regions.  Returns p[4][5][N] with the two beams first.
    """
    N = e_frac.shape[0]
    ek = 0.5 * sqrt_s * e_frac
    st = np.sqrt(np.maximum(0.0, (1.0 - cos_beam) * (1.0 + cos_beam)))
    k = np.stack([ek, ek * st * np.cos(phi), ek * st * np.sin(phi), ek * cos_beam])
    Q0 = sqrt_s - ek
    M2 = Q0 * Q0 - ek * ek
    M = np.sqrt(M2)
    pstar = np.sqrt(np.maximum(0.0, 0.25 * M2 - mass * mass))
    sp = np.sqrt(np.maximum(0.0, (1.0 - cos_pair) * (1.0 + cos_pair)))
    n = np.stack([sp * np.cos(phi_pair), sp * np.sin(phi_pair), cos_pair])
    e = 0.5 * M
    p3 = np.concatenate([e[None], pstar * n])
    p4 = np.concatenate([e[None], -pstar * n])
    bvec = -k[1:] / Q0
    out = np.zeros((4, 5, N))
    out[:, :2] = _beams(sqrt_s, N)
    out[:, 2] = _boost(p3, bvec)
    out[:, 3] = _boost(p4, bvec)
    out[:, 4] = k
    return np.ascontiguousarray(out)


def approach_points(process: str, n_bases: int, seed: int) -> tuple[Batch, dict]:
    """Points on soft/collinear approach sequences for a 2 -> Q Qbar g process.

    Each base draws (pair angles, gluon direction, gluon energy); its 16 members are
    7 points with gluon energy fraction in {1e-2..1e-8} (soft), 7 with 1-|cos| in
    {1e-2..1e-8} towards a beam (collinear), and 2 soft-collinear points
    (both = 1e-4 and 1e-8).  Returns the batch and the per-point (kind, value) labels.
    """
    rs = 1000.0
    u = uniforms(seed, 0, n_bases, 6)
    cpair = 2.0 * u[0] - 1.0
    ppair = 2.0 * math.pi * u[1]
    cbeam = 2.0 * u[2] - 1.0
    phi = 2.0 * math.pi * u[3]
    xi0 = 0.05 + 0.5 * u[4]
    side = np.where(u[5] < 0.5, 1.0, -1.0)
    vals = [10.0 ** (-k) for k in range(2, 9)]
    ef, cb, kinds, lab = [], [], [], []
    for v in vals:
        ef.append(np.full(n_bases, v)); cb.append(cbeam); kinds.append(0); lab.append(v)
    for v in vals:
        ef.append(xi0); cb.append(side * (1.0 - v)); kinds.append(1); lab.append(v)
    for v in (1e-4, 1e-8):
        ef.append(np.full(n_bases, v)); cb.append(side * (1.0 - v)); kinds.append(2); lab.append(v)
    m = len(ef)
    e_frac = np.stack(ef, axis=1).reshape(-1)
    cos_b = np.stack(cb, axis=1).reshape(-1)
    rep = lambda a: np.repeat(a, m)
    p = emission_points(rs, MT, e_frac, cos_b, rep(phi), rep(cpair), rep(ppair))
    labels = {"kind": np.tile(np.array(kinds), n_bases), "value": np.tile(np.array(lab), n_bases)}
    return Batch(process, rs, p, np.ones(p.shape[2])), labels


def mixed_stream(n_requests: int, seed: int, lo: int = 256, hi: int = 65536,
                 processes=("ee_uu", "ee_uug", "gg_tt", "gg_ttg", "gg_ttgg", "uu_ttg")):
    """Request descriptors for a served mixed stream: Poisson arrivals (unit rate,
    scaled by the caller), log-uniform sizes in [lo, hi], uniform process choice.
    Returns a list of dicts (arrival, process, n, seed)."""
    u = uniforms(seed, 7, n_requests, 3)
    gaps = -np.log(u[0])
    t = np.cumsum(gaps)
    sizes = np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u[1]).astype(np.int64)
    which = np.minimum((u[2] * len(processes)).astype(np.int64), len(processes) - 1)
    return [{"arrival": float(t[i]), "process": processes[which[i]], "n": int(sizes[i]),
             "seed": 1000 + i} for i in range(n_requests)]


def fsr_emission_points(sqrt_s: float, cos_dir: np.ndarray, phi_dir: np.ndarray,
                        e_frac: np.ndarray, cos_rel: np.ndarray, phi_rel: np.ndarray,
                        partner: int = 2) -> np.ndarray:
    """Massless 2 -> 3 points (e.g. e+e- -> q qbar g) with a gluon of energy
    e_frac*sqrt(s)/2 at angle acos(cos_rel) from the parton ``partner`` (leg 2 or 3),
    whose direction is (cos_dir, phi_dir); the partner's energy is fixed so that the
    third parton is massless.  Returns p[4][5][N], beams first (along +-z)."""
    N = e_frac.shape[0]
    sd = np.sqrt(np.maximum(0.0, (1.0 - cos_dir) * (1.0 + cos_dir)))
    nj = np.stack([sd * np.cos(phi_dir), sd * np.sin(phi_dir), cos_dir])
    zhat = np.array([0.0, 0.0, 1.0])[:, None]
    ea = zhat - (zhat * nj).sum(axis=0) * nj
    ea = ea / np.sqrt((ea * ea).sum(axis=0))
    eb = np.stack([nj[1] * ea[2] - nj[2] * ea[1], nj[2] * ea[0] - nj[0] * ea[2],
                   nj[0] * ea[1] - nj[1] * ea[0]])
    sr = np.sqrt(np.maximum(0.0, (1.0 - cos_rel) * (1.0 + cos_rel)))
    ni = cos_rel * nj + sr * (np.cos(phi_rel) * ea + np.sin(phi_rel) * eb)
    ei = 0.5 * sqrt_s * e_frac
    ej = sqrt_s * (1.0 - e_frac) / (2.0 - e_frac * (1.0 - cos_rel))
    out = np.zeros((4, 5, N))
    out[:, :2] = _beams(sqrt_s, N)
    other = 5 - partner
    out[0, partner] = ej
    out[1:, partner] = ej * nj
    out[0, 4] = ei
    out[1:, 4] = ei * ni
    out[0, other] = sqrt_s - ej - ei
    out[1:, other] = -(ej * nj + ei * ni)
    return np.ascontiguousarray(out)


FKS_ALPHA_FLAT = 0.25  # share of the flat (RAMBO) channel in fks_points
FKS_Y_CUT = 1e-6       # the FKS channels sample 1 - y_j >= FKS_Y_CUT (the flat channel covers all)


def _coll_density(y: np.ndarray) -> np.ndarray:
    """Density in y of y = 1 - 2 v^2 with v uniform in (v_min, 1), 2 v_min^2 = FKS_Y_CUT:
    1 / (4 v (1 - v_min)) for 1 - y >= FKS_Y_CUT, else 0."""
    vmin = math.sqrt(0.5 * FKS_Y_CUT)
    omy = 1.0 - y
    v = np.sqrt(np.maximum(0.0, 0.5 * omy))
    with np.errstate(divide="ignore", invalid="ignore"):
        g = 1.0 / (4.0 * v * (1.0 - vmin))
    return np.where(omy >= FKS_Y_CUT, g, 0.0)


def rambo_weight(sqrt_s: float, masses, p_out: np.ndarray) -> np.ndarray:
    """The (massive) RAMBO weight of final momenta p_out[4][n][N] (rambo_massive's weight
    as a function of the point): 1 / the density RAMBO generates it with."""
    n = len(masses)
    s = sqrt_s * sqrt_s
    w0 = (2 * math.pi) ** (4 - 3 * n) * (0.5 * math.pi) ** (n - 1) * s ** (n - 2) / (
        math.factorial(n - 1) * math.factorial(n - 2))
    if not np.any(np.asarray(masses)):
        return np.full(p_out.shape[2], w0)
    kabs = np.sqrt((p_out[1:] ** 2).sum(axis=0))
    e = p_out[0]
    return w0 * (kabs.sum(axis=0) / sqrt_s) ** (2 * n - 3) * np.prod(kabs / e, axis=0) \
        * sqrt_s / (kabs * kabs / e).sum(axis=0)


def fks_points(process: str, n: int, seed: int, first_point: int = 0, stream: int = 0,
               sqrt_s: float | None = None) -> Batch:
    """Phase-space points of a real-emission process sampled with a multichannel density
    whose channels are the variables of its FKS sectors plus flat phase space.

    Channels (u0 picks one): flat RAMBO with share FKS_ALPHA_FLAT; otherwise one of the two
    sectors, equal shares.  A sector channel is flat in the emitted gluon's energy fraction
    xi (flat three-body phase space has density ~ xi there) and samples its cosine to the
    sector's reference direction as y_j = 1 - 2 v^2, v uniform in (v_min, 1) with
    2 v_min^2 = FKS_Y_CUT (density ~ 1/sqrt(1 - y_j)), azimuth and Born direction uniform.
    The weight of a point is the phase-space measure over the summed channel densities at
    that point: 1 / (a_flat / w_RAMBO + sum_j a_j h_j), so it stays bounded by
    w_RAMBO / a_flat wherever the sector channels are thin (a hard gluon back to back
    with collinear partons), and no point closer than FKS_Y_CUT to a collinear limit
    comes from a sector channel (the flat channel still covers that region).

    Initial-state sectors (gg_ttg, uu_ttg; beams j = 0 along +z, 1 along -z; top mass
    MT): xi = xi_max u1 (xi_max = 1 - 4 m^2 / s), v from u2, phi = 2 pi u3, the heavy
    pair's rest-frame direction (2 u4 - 1, 2 pi u5); dPhi_3 = dPhi_2(s) xi K dxi dy dphi
    with dPhi_2(s) = beta(s)/(8 pi) dOmega*/(4 pi), K = s beta(s(1-xi)) / (64 pi^3 beta(s)),
    so h_j = 4 g(y_j) / (xi_max beta(s) xi K).
    Final-state sectors (ee_uug, massless): partner leg 2 or 3, its direction
    (2 u1 - 1, 2 pi u2), xi = u3, v from u4, phi = 2 pi u5 about it; each sector's
    parametrisation covers the space once, dPhi_3 = (1/(8 pi)) (dOmega/(4 pi)) xi K_j dxi dy
    dphi with K_j = s (1 - xi) / (16 pi^3 (2 - xi (1 - y_j))^2), so h_j = 4 g(y_j)/(xi K_j).
    The flat channel is RAMBO (rambo_massive) on uniforms u6..u17."""
    rs = sqrt_s if sqrt_s is not None else {"ee_uug": 100.0, "gg_ttg": 1000.0, "uu_ttg": 1000.0}[process]
    s = rs * rs
    isr = process in ("gg_ttg", "uu_ttg")
    if not isr and process != "ee_uug":
        raise ValueError(f"{process} has no FKS sectors")
    masses = [MT, MT, 0.0] if isr else [0.0, 0.0, 0.0]
    u = uniforms(seed, stream, n, 18, first_point)
    vmin = math.sqrt(0.5 * FKS_Y_CUT)
    a_f = FKS_ALPHA_FLAT
    a_s = 0.5 * (1.0 - a_f)
    flat = u[0] < a_f
    sec = np.where(u[0] < a_f + a_s, 0, 1)
    v = vmin + (1.0 - vmin) * u[2] if isr else vmin + (1.0 - vmin) * u[4]
    yj = 1.0 - 2.0 * v * v
    p = np.empty((4, 5, n))
    if isr:
        ximax = 1.0 - 4.0 * MT * MT / s
        xi = ximax * u[1]
        y = np.where(sec == 0, yj, -yj)
        p[:] = emission_points(rs, MT, xi, y, 2.0 * math.pi * u[3], 2.0 * u[4] - 1.0, 2.0 * math.pi * u[5])
    else:
        cdir, pdir, xi, phi = 2.0 * u[1] - 1.0, 2.0 * math.pi * u[2], u[3], 2.0 * math.pi * u[5]
        for partner, sel in ((2, sec == 0), (3, sec == 1)):
            if sel.any():
                p[:, :, sel] = fsr_emission_points(rs, cdir[sel], pdir[sel], xi[sel], yj[sel], phi[sel], partner)
    if flat.any():
        pf, _ = rambo_massive(rs, masses, u[6:18][:, flat])
        p[:, :, flat] = with_beams(rs, pf)
    # every channel's density at every point, from its momenta
    kg = p[1:, 4]
    ng = kg / np.sqrt((kg * kg).sum(axis=0))
    xi_pt = 2.0 * p[0, 4] / rs
    h = a_f / rambo_weight(rs, masses, p[:, 2:])
    if isr:
        ximax = 1.0 - 4.0 * MT * MT / s
        beta = math.sqrt(1.0 - 4.0 * MT * MT / s)
        K = s * np.sqrt(np.maximum(0.0, 1.0 - 4.0 * MT * MT / (s * (1.0 - xi_pt)))) / (64.0 * math.pi ** 3 * beta)
        for sign in (1.0, -1.0):
            h = h + a_s * 4.0 * _coll_density(sign * ng[2]) / (ximax * beta * xi_pt * K)
    else:
        for j in (2, 3):
            kj = p[1:, j]
            y = (ng * kj).sum(axis=0) / np.sqrt((kj * kj).sum(axis=0))
            K = s * (1.0 - xi_pt) / (16.0 * math.pi ** 3 * (2.0 - xi_pt * (1.0 - y)) ** 2)
            h = h + a_s * 4.0 * _coll_density(y) / (xi_pt * K)
    return Batch(process, rs, np.ascontiguousarray(p), 1.0 / h)
