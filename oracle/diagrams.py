"""Tree-level Feynman diagrams: enumeration, kinematic value and colour tensor (oracle).

A tree amplitude is the sum over Feynman diagrams (Sec. 2.1, Eq. (born): the
squared sum of the diagrams; Sec. 2.2, Eq. (real): one extra vertex).  Here the
diagrams are enumerated explicitly and each one is evaluated on its own:

  * all legs are treated as outgoing: an incoming particle becomes an outgoing
    antiparticle with momentum q = -p (its wavefunction still uses the physical p);
  * an off-shell "current" for a set S of legs is one sub-diagram; a diagram is a
    tree of vertices whose leaves are external legs; the last leg closes the tree;
  * each vertex of a diagram is one Feynman rule, each internal line one propagator
    (Feynman gauge), Peskin & Schroeder conventions:
        f f V   :  i c gamma^mu            (c = g_s T^a for gluons, e Q_f for photons)
        g g g   :  g_s f^abc [g^{mu nu}(k1-k2)^rho + g^{nu rho}(k2-k3)^mu + g^{rho mu}(k3-k1)^nu]
                   (momenta incoming to the vertex)
        g g g g :  -i g_s^2 [f^abe f^cde (g^{mu rho} g^{nu sig} - g^{mu sig} g^{nu rho})
                           + f^ace f^bde (g^{mu nu} g^{rho sig} - g^{mu sig} g^{nu rho})
                           + f^ade f^bce (g^{mu nu} g^{rho sig} - g^{mu rho} g^{nu sig})]
                   -- each of the three colour structures is kept as its own term;
        fermion :  i (pslash + m) / (p^2 - m^2), p along the fermion arrow;
        vector  :  -i g_{mu nu} / p^2;
  * the colour factor of each diagram is built as an explicit tensor over the colour
    indices of all external legs (T^a and f^abc from ``oracle.colour``).

A diagram "term" is one (kinematic value, colour tensor) pair; a diagram with k
four-gluon vertices contributes 3^k terms.  The colour-summed squared amplitude is
sum_colours |sum_t c_t A_t|^2 = sum_{t,t'} conj(A_t) G_{t t'} A_t' with
G_{t t'} = sum_colours conj(c_t) c_t' -- an exact rewriting of the colour sum.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

from . import colour
from .dirac import GAMMA, bar, ctype, dot, polarisation, slash, spinor_u, spinor_v

# ------------------------------------------------------------------ model
FERMIONS = {
    "e": {"charge": -1.0, "coloured": False},
    "u": {"charge": 2.0 / 3.0, "coloured": True},
    "t": {"charge": 2.0 / 3.0, "coloured": True},
}
PARTICLES = {  # name -> (kind, flavour, is_antiparticle)
    "e-": ("f", "e", False), "e+": ("f", "e", True),
    "u": ("f", "u", False), "u~": ("f", "u", True),
    "t": ("f", "t", False), "t~": ("f", "t", True),
    "g": ("v", "g", False), "a": ("v", "a", False),
}


@dataclass
class Process:
    """A 2 -> n process: leg names (two incoming first), couplings and masses."""
    name: str
    legs: tuple            # e.g. ("g", "g", "t", "t~", "g")
    couplings: frozenset   # subset of {("e","a"),("u","a"),("u","g"),("t","g"),"ggg","gggg"}
    masses: dict = field(default_factory=dict)   # flavour -> mass
    n_in: int = 2
    ident_factor: float = 1.0  # 1/(identical final-state permutations)

    def mass(self, flav: str) -> float:
        return float(self.masses.get(flav, 0.0))

    def incoming(self, i: int) -> bool:
        return i < self.n_in

    def line_type(self, i: int):
        """Type of the line an external leg opens, all-outgoing view."""
        kind, flav, anti = PARTICLES[self.legs[i]]
        if kind == "v":
            return ("vec", flav)
        crossed_anti = anti != self.incoming(i)
        # outgoing particle / incoming antiparticle -> row spinor (ubar, vbar)
        return ("col", flav) if crossed_anti else ("row", flav)

    def colour_dim(self, i: int) -> int:
        kind, flav, _ = PARTICLES[self.legs[i]]
        if kind == "v":
            return 8 if flav == "g" else 1
        return 3 if FERMIONS[flav]["coloured"] else 1

    def colour_kind(self, i: int) -> str | None:
        d = self.colour_dim(i)
        if d == 1:
            return None
        if d == 8:
            return "adj"
        return "fund" if self.line_type(i)[0] == "row" else "antifund"

    def average(self) -> float:
        """Initial spin x colour average times the identical-particle factor."""
        avg = 1.0
        for i in range(self.n_in):
            avg *= 2.0 * self.colour_dim(i)
        return avg / self.ident_factor


# ------------------------------------------------------------------ enumeration
@dataclass(eq=False)
class Node:
    kind: str          # ext | ffv_row | ffv_col | ffv_vec | vvv | vvvv
    ltype: tuple
    legs: frozenset
    kids: tuple = ()
    chan: int = 0      # four-gluon colour/Lorentz structure (0,1,2)
    boson: str = ""    # boson of an f f V vertex
    leg: int = -1      # for ext


def _couples(proc: Process, flav: str, boson: str) -> bool:
    return (flav, boson) in proc.couplings


def _subsets(S: frozenset):
    items = sorted(S)
    n = len(items)
    for mask in range(1, (1 << n) - 1):
        S1 = frozenset(items[i] for i in range(n) if mask >> i & 1)
        yield S1, S - S1


def _three_partitions(S: frozenset):
    """Unordered partitions of S into three nonempty blocks."""
    items = sorted(S)
    first = items[0]
    seen = set()
    for S1, rest in _subsets(S):
        if first not in S1:
            continue
        if len(rest) < 2:
            continue
        r0 = min(rest)
        for S2, S3 in _subsets(rest):
            if r0 not in S2:
                continue
            key = (S1, S2, S3)
            if key not in seen:
                seen.add(key)
                yield S1, S2, S3


class Diagrams:
    """All tree diagrams of a process, their colour tensors and Gram matrices."""

    def __init__(self, proc: Process):
        self.proc = proc
        self.n = len(proc.legs)
        self._cache = {}
        root = self.n - 1
        rt = proc.line_type(root)
        comp = {"row": "col", "col": "row", "vec": "vec"}[rt[0]]
        rest = frozenset(range(self.n - 1))
        self.terms = list(self._currents(rest, (comp, rt[1])))
        self.root = root
        self._ctensors = {}

    # number of Feynman diagrams (the three four-gluon structures count once)
    @property
    def n_diagrams(self) -> int:
        def base(nd):
            if nd.kind == "vvvv" and nd.chan != 0:
                return False
            return all(base(k) for k in nd.kids)
        return sum(1 for t in self.terms if base(t))

    def _currents(self, S: frozenset, lt: tuple):
        key = (S, lt)
        if key in self._cache:
            return self._cache[key]
        proc = self.proc
        out = []
        if len(S) == 1:
            (i,) = tuple(S)
            if proc.line_type(i) == lt:
                out.append(Node("ext", lt, S, leg=i))
            self._cache[key] = out
            return out
        kind, flav = lt
        if kind == "row":
            for boson in ("g", "a"):
                if not _couples(proc, flav, boson):
                    continue
                for S1, S2 in _subsets(S):
                    for a in self._currents(S1, ("row", flav)):
                        for b in self._currents(S2, ("vec", boson)):
                            out.append(Node("ffv_row", lt, S, (a, b), boson=boson))
        elif kind == "col":
            for boson in ("g", "a"):
                if not _couples(proc, flav, boson):
                    continue
                for S1, S2 in _subsets(S):
                    for a in self._currents(S1, ("vec", boson)):
                        for b in self._currents(S2, ("col", flav)):
                            out.append(Node("ffv_col", lt, S, (a, b), boson=boson))
        else:  # vector boson current
            boson = flav
            for f in FERMIONS:
                if not _couples(proc, f, boson):
                    continue
                for S1, S2 in _subsets(S):
                    for a in self._currents(S1, ("row", f)):
                        for b in self._currents(S2, ("col", f)):
                            out.append(Node("ffv_vec", lt, S, (a, b), boson=boson))
            if boson == "g" and "ggg" in proc.couplings:
                first = min(S)
                for S1, S2 in _subsets(S):
                    if first not in S1:
                        continue
                    for a in self._currents(S1, ("vec", "g")):
                        for b in self._currents(S2, ("vec", "g")):
                            out.append(Node("vvv", lt, S, (a, b)))
            if boson == "g" and "gggg" in proc.couplings and len(S) >= 3:
                for S1, S2, S3 in _three_partitions(S):
                    for a in self._currents(S1, ("vec", "g")):
                        for b in self._currents(S2, ("vec", "g")):
                            for c in self._currents(S3, ("vec", "g")):
                                for ch in range(3):
                                    out.append(Node("vvvv", lt, S, (a, b, c), chan=ch))
        self._cache[key] = out
        return out

    # -------------------------------------------------------------- colour
    def _colour_vertex(self, nd: Node, dtype) -> np.ndarray:
        T, f, _ = colour.generators(dtype)
        proc = self.proc
        if nd.kind in ("ffv_row", "ffv_col", "ffv_vec"):
            flav = nd.ltype[1] if nd.kind != "ffv_vec" else nd.kids[0].ltype[1]
            qc = FERMIONS[flav]["coloured"]
            if nd.boson == "g":
                X = T  # [a, l, l']
            else:
                d = 3 if qc else 1
                X = np.eye(d, dtype=dtype)[None]  # [0, l, l']
            if nd.kind == "ffv_row":      # out[l'] = R[l] X[a,l,l'] V[a]
                return np.transpose(X, (1, 0, 2))       # [l, a, l']
            if nd.kind == "ffv_col":      # out[l] = X[a,l,l'] V[a] C[l']
                return np.transpose(X, (0, 2, 1))       # [a, l', l]
            return np.transpose(X, (1, 2, 0))           # [l, l', a]
        if nd.kind == "vvv":
            return f.astype(dtype)                      # [a, b, c]
        if nd.kind == "vvvv":
            if nd.chan == 0:
                X = np.einsum("abe,cde->abcd", f, f)
            elif nd.chan == 1:
                X = np.einsum("ace,bde->abcd", f, f)
            else:
                X = np.einsum("ade,bce->abcd", f, f)
            return X.astype(dtype)
        raise ValueError(nd.kind)

    def _colour(self, nd: Node, memo: dict, dtype=complex):
        """Colour tensor of a current: axes (line, *legs in increasing order)."""
        if id(nd) in memo:
            return memo[id(nd)]
        if nd.kind == "ext":
            d = self.proc.colour_dim(nd.leg)
            t = np.eye(d, dtype=dtype)
            memo[id(nd)] = t
            return t
        kids = [self._colour(k, memo, dtype) for k in nd.kids]
        X = self._colour_vertex(nd, dtype)
        letters = iter("ABCDEFGH")
        kid_lines = [next(letters) for _ in kids]
        new_line = "Z"
        leg_letter = lambda i: "abcdefghijklmnopqrstuvwxy"[i]
        subs = []
        for k, nd_k, ln in zip(kids, nd.kids, kid_lines):
            subs.append(ln + "".join(leg_letter(i) for i in sorted(nd_k.legs)))
        subs.append("".join(kid_lines) + new_line)
        out_legs = "".join(leg_letter(i) for i in sorted(nd.legs))
        expr = ",".join(subs) + "->" + new_line + out_legs
        t = np.einsum(expr, *kids, X)
        memo[id(nd)] = t
        return t

    def colour_tensors(self, dtype=complex) -> np.ndarray:
        """(n_terms, prod of leg colour dims): full colour tensor of every term, in the
        given complex type (complex128, or that of np.longdouble)."""
        key = np.dtype(dtype)
        if key not in self._ctensors:
            memo = {}
            rows = []
            for t in self.terms:
                c = self._colour(t, memo, key)  # axes: line(=root leg), legs 0..n-2
                c = np.moveaxis(c, 0, -1)  # root leg is the last leg
                rows.append(c.reshape(-1))
            self._ctensors[key] = np.array(rows)
        return self._ctensors[key]

    def colour_shape(self):
        return tuple(self.proc.colour_dim(i) for i in range(self.n))

    def gram(self, dtype=complex) -> np.ndarray:
        C = self.colour_tensors(dtype)
        return C.conj() @ C.T

    def charge_on_leg(self, leg: int, dtype=complex) -> np.ndarray:
        """(8, n_terms, D): T_leg^a applied to every term's colour tensor."""
        kind = self.proc.colour_kind(leg)
        M = colour.charge_matrices(kind, dtype)
        C = self.colour_tensors(dtype).reshape((-1,) + self.colour_shape())
        Cm = np.moveaxis(C, leg + 1, -1)              # (t, ..., d)
        res = np.einsum("aij,t...j->at...i", M, Cm)   # (a, t, ..., d)
        res = np.moveaxis(res, -1, leg + 2)
        return res.reshape(8, C.shape[0], -1)

    def gram_correlated(self, k: int, l: int, dtype=complex) -> np.ndarray:
        """G^{kl}_{t t'} = sum_a sum_colours conj(T_k^a c_t) (T_l^a c_t')."""
        Tk = self.charge_on_leg(k, dtype)
        Tl = Tk if k == l else self.charge_on_leg(l, dtype)
        return np.einsum("atd,asd->ts", Tk.conj(), Tl)

    # -------------------------------------------------------------- kinematics
    def wavefunctions(self, p: np.ndarray, hel: np.ndarray, override=None):
        """External wavefunctions, shape (n_legs) of (N, H, 4).

        ``p``: (N, n_legs, 4) physical momenta; ``hel``: (H, n_legs) in {-1,+1};
        ``override``: {leg: (N,4) vector} replaces that leg's wavefunction.
        """
        proc = self.proc
        wfs = []
        for i in range(self.n):
            if override and i in override:
                w = np.asarray(override[i], dtype=ctype(p))[:, None, :]
                wfs.append(np.broadcast_to(w, (p.shape[0], hel.shape[0], 4)))
                continue
            kind, flav, anti = PARTICLES[proc.legs[i]]
            pi = p[:, i, :]
            per = {}
            for lam in (-1, 1):
                if kind == "v":
                    e = polarisation(pi, lam)
                    per[lam] = e if proc.incoming(i) else e.conj()
                else:
                    m = proc.mass(flav)
                    if proc.incoming(i):
                        per[lam] = bar(spinor_v(pi, m, lam)) if anti else spinor_u(pi, m, lam)
                    else:
                        per[lam] = spinor_v(pi, m, lam) if anti else bar(spinor_u(pi, m, lam))
            both = np.stack([per[-1], per[1]], axis=1)     # (N, 2, 4)
            idx = (hel[:, i] > 0).astype(int)
            wfs.append(both[:, idx, :])
        return wfs

    def amplitudes(self, p: np.ndarray, hel: np.ndarray, couplings: dict, override=None):
        """Kinematic value of every diagram term: (N, H, n_terms) complex."""
        proc = self.proc
        N = p.shape[0]
        q = p.copy()
        q[:, : proc.n_in, :] *= -1.0  # all-outgoing momenta
        wfs = self.wavefunctions(p, hel, override)
        memo = {}

        def Q(nd):
            return q[:, sorted(nd.legs), :].sum(axis=1)[:, None, :]  # (N,1,4)

        def coup(nd):
            flav = nd.ltype[1] if nd.kind != "ffv_vec" else nd.kids[0].ltype[1]
            if nd.boson == "g":
                return couplings["gs"]
            return couplings["e"] * FERMIONS[flav]["charge"]

        def ev(nd, amputate=False):
            key = (id(nd), amputate)
            if key in memo:
                return memo[key]
            if nd.kind == "ext":
                val = wfs[nd.leg]
            elif nd.kind == "ffv_row":
                R = ev(nd.kids[0]); V = ev(nd.kids[1])
                val = 1j * coup(nd) * np.einsum("...i,...ij->...j", R, slash(V))
                if not amputate:
                    P = Q(nd); m = proc.mass(nd.ltype[1])
                    prop = 1j * (slash(P) + m * np.eye(4)) / (dot(P, P) - m * m)[..., None, None]
                    val = np.einsum("...i,...ij->...j", val, prop)
            elif nd.kind == "ffv_col":
                V = ev(nd.kids[0]); C = ev(nd.kids[1])
                val = 1j * coup(nd) * np.einsum("...ij,...j->...i", slash(V), C)
                if not amputate:
                    P = Q(nd); m = proc.mass(nd.ltype[1])
                    prop = 1j * (-slash(P) + m * np.eye(4)) / (dot(P, P) - m * m)[..., None, None]
                    val = np.einsum("...ij,...j->...i", prop, val)
            elif nd.kind == "ffv_vec":
                R = ev(nd.kids[0]); C = ev(nd.kids[1])
                J = np.einsum("...i,nij,...j->...n", R, GAMMA, C)
                c = coup(nd)
                if amputate:
                    val = 1j * c * J
                else:
                    P = Q(nd)
                    val = (c / dot(P, P))[..., None] * J
            elif nd.kind == "vvv":
                J1 = ev(nd.kids[0]); J2 = ev(nd.kids[1])
                k1 = -Q(nd.kids[0]); k2 = -Q(nd.kids[1]); k3 = -(k1 + k2)
                W = (dot(J1, J2)[..., None] * (k1 - k2)
                     + J2 * dot(k2 - k3, J1)[..., None]
                     + J1 * dot(k3 - k1, J2)[..., None])
                g = couplings["gs"]
                if amputate:
                    val = g * W
                else:
                    P = Q(nd)
                    val = (-1j * g / dot(P, P))[..., None] * W
            elif nd.kind == "vvvv":
                J1, J2, J3 = (ev(k) for k in nd.kids)
                if nd.chan == 0:
                    L = dot(J1, J3)[..., None] * J2 - dot(J2, J3)[..., None] * J1
                elif nd.chan == 1:
                    L = dot(J1, J2)[..., None] * J3 - dot(J2, J3)[..., None] * J1
                else:
                    L = dot(J1, J2)[..., None] * J3 - dot(J1, J3)[..., None] * J2
                g2 = couplings["gs"] ** 2
                if amputate:
                    val = -1j * g2 * L
                else:
                    P = Q(nd)
                    val = (-g2 / dot(P, P))[..., None] * L
            else:
                raise ValueError(nd.kind)
            memo[key] = val
            return val

        root_wf = wfs[self.root]
        rt = proc.line_type(self.root)[0]
        out = np.empty((N, hel.shape[0], len(self.terms)), dtype=ctype(p))
        for it, t in enumerate(self.terms):
            X = ev(t, amputate=True)
            if rt == "row":      # root ubar / vbar on the left of a column current
                out[..., it] = np.einsum("...i,...i->...", root_wf, X)
            elif rt == "col":    # row current on the left of root u / v
                out[..., it] = np.einsum("...i,...i->...", X, root_wf)
            else:
                out[..., it] = dot(X, root_wf)
        return out


def helicities(n_legs: int, fixed: dict | None = None) -> np.ndarray:
    """All helicity assignments (H, n_legs); legs in ``fixed`` take the given value."""
    rows = []
    for h in itertools.product((-1, 1), repeat=n_legs):
        if fixed and any(h[i] != v for i, v in fixed.items()):
            continue
        rows.append(h)
    return np.array(rows, dtype=int)
