"""Float64 parity rule between the CUDA float64 path and the oracle (test infrastructure).

Two float64 evaluations of the same point can disagree beyond 1e-12 for a reason that
is not a mistake in either: the value is ill conditioned in its float64 inputs (a
subtracted weight W = R S - CT with |R S| >> |W|, or a matrix element at a nearly
collinear configuration whose small invariants are differences of large momentum
components).  Then every float64 evaluation carries an error of about
cond x 2^-53 relative, whatever its formulation.  The rule below decides each point:

  1. |got - oracle_f64| <= 1e-12 |oracle_f64|: the two independent evaluations agree;
  2. otherwise the oracle is re-evaluated at the same float64 inputs in extended
     precision (np.longdouble: 64-bit significand on x86-64, 113-bit on aarch64), and
     the input condition number is estimated there,
        cond = max over K random sign vectors s of |f(p + s h) - f(p)| / (u |f(p)|),
     u = 2^-53, h_i = half a float64 ulp of p_i (between u/2 and u relative, exactly
     representable in extended precision), i.e. the relative change of the value when
     every float64 input moves by about one rounding error.  The point passes when
        |got - f(p)| <= max(1e-12, C cond u) |f(p)|,   C = 64;
  3. a point with C cond u >= 1 (or no finite extended value) is not determined by its
     float64 inputs at all; there the CUDA result must only be finite.

C = 64: on the seeded parity points (about 4000 flat and approach points of all seven
processes) the CUDA float64 path stays within 11 cond u, the float64 oracle within 63.
"""
from __future__ import annotations

import numpy as np

U = 2.0 ** -53
RTOL = 1e-12
C_COND = 64.0


def extended_precision_available() -> bool:
    return np.finfo(np.longdouble).eps < 1e-18


def extended(f, k: np.ndarray, n_perturb: int = 8, seed: int = 0):
    """f at the float64 points k in extended precision, and the estimated condition
    number of f in its float64 inputs (see the module docstring)."""
    L = np.longdouble
    k64 = np.asarray(k, dtype=np.float64)
    kx = k64.astype(L)
    # half a float64 ulp of every input (zero inputs carry no rounding error): p + h is
    # exact in extended precision, so the perturbation applied is exactly h
    h = np.where(k64 != 0.0, np.ldexp(np.ones_like(kx), np.frexp(k64)[1] - 54), L(0))
    with np.errstate(all="ignore"):
        f0 = np.asarray(f(kx))
        rng = np.random.default_rng(seed)
        cond = np.zeros(kx.shape[0])
        for _ in range(n_perturb):
            s = rng.choice(np.array([-1.0, 1.0]), size=kx.shape).astype(L)
            f1 = np.asarray(f(kx + s * h))
            c = np.abs((f1 - f0) / f0).astype(np.float64) / U
            cond = np.maximum(cond, np.where(np.isfinite(c), c, np.inf))
    return f0, cond


def check_fp64(got: np.ndarray, f, k: np.ndarray, scale=None, n_perturb: int = 8):
    """Apply the rule to float64 results `got` of f at points k (N, n_leg, 4); `scale`
    (N,) multiplies f (a phase-space weight) on both sides.  Returns a summary dict;
    raises AssertionError naming the worst point otherwise."""
    got = np.asarray(got, dtype=np.float64)
    w = np.ones(got.shape) if scale is None else np.asarray(scale, dtype=np.float64)
    with np.errstate(all="ignore"):
        r64 = np.asarray(f(k), dtype=np.float64) * w
        agree = np.isfinite(r64) & (np.abs(got - r64) <= RTOL * np.abs(r64))
    assert np.all(np.isfinite(got)), "non-finite float64 result"
    out = {"n": int(got.size), "agree_1e-12": int(agree.sum()), "arbitrated": 0, "unresolved": 0,
           "max_err_over_cond_u": 0.0, "max_rel_err": 0.0}
    rest = np.flatnonzero(~agree)
    if rest.size == 0:
        return out
    fx, cond = extended(f, k[rest], n_perturb)
    with np.errstate(all="ignore"):
        fx = fx * w[rest].astype(np.longdouble)
        err = (np.abs(got[rest] - fx) / np.abs(fx)).astype(np.float64)
    resolved = np.isfinite(err) & np.isfinite(cond) & (C_COND * cond * U < 1.0)
    bound = np.maximum(RTOL, C_COND * cond * U)
    bad = resolved & ~(err <= bound)
    out["arbitrated"] = int(resolved.sum())
    out["unresolved"] = int((~resolved).sum())
    if resolved.any():
        out["max_err_over_cond_u"] = float(np.max(err[resolved] / np.maximum(cond[resolved] * U, 1e-300)))
        out["max_rel_err"] = float(np.max(err[resolved]))
    if bad.any():
        i = int(np.argmax(np.where(bad, err / bound, 0.0)))
        raise AssertionError(f"point {int(rest[i])}: rel. error {err[i]:.3e} against the extended-precision "
                             f"oracle, bound {bound[i]:.3e} (cond {cond[i]:.3e}); {int(bad.sum())} point(s) fail")
    return out
