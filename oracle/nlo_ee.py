"""n-body NLO piece for e+e- -> q qbar: Born + virtual + integrated FKS counterterms.

Standard physics (the paper gives no formulas; FKS is its subtraction scheme,
Sec. 2.2).  With a_s = alpha_s C_F / (2 pi) and N(eps) = (4 pi mu^2/s)^eps / Gamma(1-eps):

  virtual (CDR, massless quark form factor, real part):
      2 Re(M_B^* M_V) = a_s N(eps) B (-2/eps^2 - 3/eps - 8 + pi^2)

  integrated FKS counterterms of the two final-state sectors (q,g) and (qbar,g)
  in the parametrisation of ``oracle.fks.fsr_map`` (d-dimensional measure
  dPhi_3 = dPhi_2 (2pi)^(1-d) (s/4)^(1-eps) xi^(1-2eps) e_j^(1-2eps) (1-y^2)^(-eps)
  / (2 - xi(1-y)) dxi dy dOmega_phi), expanding xi^(-1-2eps) and (1-y)^(-1-eps)
  in plus-distributions with cut-offs xi_c and delta:
      soft, per sector:       a_s N B (1 - pi^2 eps^2/6) xi_c^(-2eps) / eps^2
      collinear, per sector:  -(1/eps)(delta/2)^(-eps) a_s N B
                                * [(-3/2 - 2 ln xi_c) + eps (2pi^2/3 - 13/2 + 2 ln^2 xi_c)]
      both sectors together:  a_s N B [2/eps^2 + 3/eps + 13 - 5 pi^2/3
                                       - (3 + 4 ln xi_c) ln(delta/2)]

so the poles cancel and the n-body weight per Born point is
      B [1 + a_s (5 - 2 pi^2/3 - (3 + 4 ln xi_c) ln(delta/2))].
Adding the subtracted real (``oracle.fks.real_subtracted``) gives
sigma_NLO = sigma_LO (1 + alpha_s/pi) independently of xi_c and delta.
"""
from __future__ import annotations

import math

import numpy as np

from . import colour
from .matrix_element import Couplings, me2


def nbody_coefficient(xi_cut: float, delta: float) -> float:
    """Finite part of (virtual + integrated counterterms) / (a_s B)."""
    return 5.0 - 2.0 * math.pi ** 2 / 3.0 - (3.0 + 4.0 * math.log(xi_cut)) * math.log(0.5 * delta)


def nbody_nlo(p: np.ndarray, xi_cut: float = 0.5, delta: float = 1.0,
              cp: Couplings = Couplings(), cuts=None) -> np.ndarray:
    """B (1 + a_s c(xi_c, delta)) for e+e- -> u ubar Born points p (N, 4, 4); with
    ``cuts`` (oracle.cuts), 0 where the Born point fails them (Algorithm 2's n-body term)."""
    from .cuts import passes
    a_s = cp.alpha_s * colour.CF / (2.0 * math.pi)
    w = me2("ee_uu", p, cp) * (1.0 + a_s * nbody_coefficient(xi_cut, delta))
    return np.where(passes("ee_uu", p, cuts), w, 0.0) if cuts is not None else w
