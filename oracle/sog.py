"""Sum-of-Gaussians (SOG) decomposition of the Yukawa kernel, FP64 (Algorithm 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Formulas, in the paper's notation:
  f(t, r) = pi^{-1/2} exp(-r^2 e^t - 1/(4 lambda^2 e^t) + t/2)                  Eq. (1)
  h*      = pi^2 / (log(eps + 6 sqrt(2 pi) e^{1/6} / delta) + log(1/eps))        Eq. (27)
  M1 >= (1/h)[t0 - log(pi eps^2/36) - W(18/(pi lambda^2 eps^2))]               Eq. (29)
  M2 >= (1/h) max{-t0 - 2 log delta + log log(3/(eps delta)),
                  -t0 - h - 2 log(sqrt(2) R)}                                    Eq. (30)
  F(r)    = h [ w f(t_M2, r) + sum_{m=-M1}^{M2-1} f(t_m, r) ],  t_m = t0 + m h   Eq. (37)
  w       = [Y(r_c) - h sum_{m<M2} f(t_m, r_c)] / (h f(t_M2, r_c))   (C0)       Eq. (38)
  d/dr [Y - F](r_c) = 0                                               (C1)       Eq. (36)
  C0 roots of the untruncated rule: alpha_{1,2} = C h + {1,3} h/4 - log(2 lambda r_c)  Eq. (35)

Algorithm 1 takes delta = r_c and R = 33 lambda.  Three ways to pick (M1, M2):
  * "table":   (M1, M2) given (reproduces Table 1).
  * "bound":   the ceilings of Eqs. (29)-(30) evaluated at t0 = alpha_1 (Algorithm 1 step 4).
  * "minimal": the fewest Gaussians whose C1 decomposition has max |Y - F| <= eps on a
               2000-point log grid over [r_c, 33 lambda]; ties broken by the smaller error.
In every mode t0 is the smallest root in [0, h) of the C1 condition with w from C0
(Algorithm 1 step 6); roots are bracketed on a 200-interval grid and refined by bisection to the last bit.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import lambertw

SQRT_PI = math.sqrt(math.pi)
R_FACTOR = 33.0          # R = 33 lambda (Sec. 3.2)
GRID_POINTS = 2000       # error grid of the "minimal" mode
ROOT_GRID = 200          # bracketing grid for t0 on [0, h)


@dataclasses.dataclass(frozen=True)
class SOG:
    lam: float
    rc: float
    eps: float
    h: float
    t0: float
    M1: int
    M2: int
    w: float

    @property
    def m(self) -> np.ndarray:
        return np.arange(-self.M1, self.M2 + 1)

    @property
    def t(self) -> np.ndarray:
        return self.t0 + self.m * self.h

    @property
    def weights(self) -> np.ndarray:
        wt = np.ones(self.M1 + self.M2 + 1)
        wt[-1] = self.w
        return wt

    @property
    def M_tot(self) -> int:
        return self.M1 + self.M2 + 1

    def as_array(self) -> np.ndarray:
        """{h, t0, M1, M2, w, lambda}: the layout the C oracle takes."""
        return np.array([self.h, self.t0, float(self.M1), float(self.M2), self.w, self.lam], dtype=np.float64)

    # -- kernel pieces (vectorised over r) --
    def F(self, r):
        r = np.asarray(r, dtype=np.float64)
        return self.h * np.sum(self.weights[:, None] * f_tr(self.t[:, None], r.ravel()[None, :], self.lam),
                               axis=0).reshape(r.shape)

    def dF(self, r):
        r = np.asarray(r, dtype=np.float64)
        rr = r.ravel()[None, :]
        terms = self.weights[:, None] * (-2.0 * rr * np.exp(self.t[:, None])) * f_tr(self.t[:, None], rr, self.lam)
        return self.h * np.sum(terms, axis=0).reshape(r.shape)

    def max_error(self, R: float | None = None) -> float:
        R = R_FACTOR * self.lam if R is None else R
        rg = np.geomspace(self.rc, R, GRID_POINTS)
        return float(np.max(np.abs(yukawa(rg, self.lam) - self.F(rg))))


def f_tr(t, r, lam):
    """Eq. (1)."""
    et = np.exp(t)
    return np.exp(-r * r * et - 1.0 / (4.0 * lam * lam * et) + 0.5 * t) / SQRT_PI


def yukawa(r, lam):
    return np.exp(-r / lam) / r


def dyukawa(r, lam):
    return -np.exp(-r / lam) * (1.0 / (lam * r) + 1.0 / (r * r))


def step_h(eps: float, delta: float) -> float:
    """Eq. (27) with equality."""
    return math.pi ** 2 / (math.log(eps + 6.0 * math.sqrt(2.0 * math.pi) * math.exp(1.0 / 6.0) / delta)
                           + math.log(1.0 / eps))


def c0_roots(h: float, lam: float, rc: float) -> tuple:
    """Eq. (35): the two C0 roots in [0, h) of the untruncated trapezoid rule."""
    base = -math.log(2.0 * lam * rc)
    return tuple(sorted(((base + h / 4.0) % h, (base + 3.0 * h / 4.0) % h)))


def m1_bound(t0: float, h: float, lam: float, eps: float) -> float:
    """Eq. (29) right-hand side."""
    W = float(np.real(lambertw(18.0 / (math.pi * lam * lam * eps * eps))))
    return (t0 - math.log(math.pi * eps * eps / 36.0) - W) / h


def m2_bound(t0: float, h: float, eps: float, delta: float, R: float) -> float:
    """Eq. (30) right-hand side."""
    a = -t0 - 2.0 * math.log(delta) + math.log(math.log(3.0 / (eps * delta)))
    b = -t0 - h - 2.0 * math.log(math.sqrt(2.0) * R)
    return max(a, b) / h


INV_SQRT_PI = 0.5641895835477563     # 1/sqrt(pi) as the nearest double


def f_scalar(t: float, r: float, lam: float) -> float:
    """Eq. (1) for one (t, r), evaluated with the C library's exp."""
    et = math.exp(t)
    return math.exp(-r * r * et - 1.0 / (4.0 * lam * lam * et) + 0.5 * t) * INV_SQRT_PI


def w_c0(t0: float, h: float, M1: int, M2: int, lam: float, rc: float) -> float:
    """Eq. (38), a sequential sum over m = -M1 .. M2-1."""
    partial = 0.0
    for m in range(-M1, M2):
        partial += f_scalar(t0 + m * h, rc, lam)
    partial *= h
    den = h * f_scalar(t0 + M2 * h, rc, lam)
    if not den > 0.0:          # the narrowest Gaussian underflows at r_c: no C0 weight exists
        return math.nan
    return (math.exp(-rc / lam) / rc - partial) / den


def c1_residual(t0: float, h: float, M1: int, M2: int, lam: float, rc: float) -> float:
    """Eq. (36) with w of Eq. (38): d/dr [Y - F](r_c), d/dr f(t, r) = -2 r e^t f(t, r).

    Near its root this residual is a difference of nearly equal terms and its slope in t0
    is small, so t0 is only defined to a band set by rounding.  It is evaluated as plain
    sequential FP64 sums with the C library's exp; any FP64 evaluation in the same
    operation order lands on the same root."""
    w = w_c0(t0, h, M1, M2, lam, rc)
    if not math.isfinite(w):
        return math.nan
    dF = 0.0
    for m in range(-M1, M2 + 1):
        t = t0 + m * h
        wt = w if m == M2 else 1.0
        dF += wt * (-2.0 * rc * math.exp(t)) * f_scalar(t, rc, lam)
    dy = -math.exp(-rc / lam) * (1.0 / (lam * rc) + 1.0 / (rc * rc))
    return dy - h * dF


def bisect(fun, a: float, b: float, fa: float) -> float:
    """Bisection on a sign change of fun in [a, b] until the midpoint is no longer
    strictly inside the bracket (the last representable bit)."""
    for _ in range(400):
        mid = 0.5 * (a + b)
        if not (a < mid < b):
            break
        fm = fun(mid)
        if not math.isfinite(fm) or fm == 0.0:
            return mid
        if (fm < 0.0) == (fa < 0.0):
            a, fa = mid, fm
        else:
            b = mid
    return 0.5 * (a + b)


def smallest_root(fun, h: float):
    """Smallest root of fun on [0, h): the first sign change on a ROOT_GRID-interval grid,
    refined by bisection."""
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        prev_x, prev_v = 0.0, fun(0.0)
        for k in range(1, ROOT_GRID + 1):
            x = h * k / ROOT_GRID
            v = fun(x)
            if math.isfinite(prev_v) and math.isfinite(v):
                if prev_v == 0.0:
                    return prev_x
                if (prev_v < 0.0) != (v < 0.0) and v != 0.0:
                    root = bisect(fun, prev_x, x, prev_v)
                    if root < h:
                        return root
            prev_x, prev_v = x, v
    return None


def build_table(lam: float, rc: float, eps: float, M1: int, M2: int) -> SOG | None:
    h = step_h(eps, rc)
    t0 = smallest_root(lambda x: c1_residual(x, h, M1, M2, lam, rc), h)
    if t0 is None:
        return None
    return SOG(lam, rc, eps, h, t0, M1, M2, w_c0(t0, h, M1, M2, lam, rc))


def build_bound(lam: float, rc: float, eps: float) -> SOG | None:
    h = step_h(eps, rc)
    a1 = c0_roots(h, lam, rc)[0]
    M1 = math.ceil(m1_bound(a1, h, lam, eps))
    M2 = math.ceil(m2_bound(a1, h, eps, rc, R_FACTOR * lam))
    return build_table(lam, rc, eps, M1, M2)


def build_minimal(lam: float, rc: float, eps: float, max_terms: int = 40) -> SOG:
    h = step_h(eps, rc)
    a1 = c0_roots(h, lam, rc)[0]
    M2c = math.ceil(m2_bound(a1, h, eps, rc, R_FACTOR * lam))
    for mtot in range(1, max_terms + 1):
        best = None
        for M2 in range(M2c - mtot - 3, M2c + 4):
            M1 = mtot - 1 - M2
            s = build_table(lam, rc, eps, M1, M2)
            if s is None or not np.isfinite(s.w):
                continue
            err = s.max_error()
            if err <= eps and (best is None or err < best[0]):
                best = (err, s)
        if best is not None:
            return best[1]
    raise RuntimeError("no SOG decomposition within max_terms")


def build(lam: float, rc: float, eps: float, mode: str = "minimal", M1: int | None = None,
          M2: int | None = None) -> SOG:
    if mode == "table":
        s = build_table(lam, rc, eps, M1, M2)
    elif mode == "bound":
        s = build_bound(lam, rc, eps)
    elif mode == "minimal":
        s = build_minimal(lam, rc, eps)
    else:
        raise ValueError(mode)
    if s is None:
        raise RuntimeError("C1 condition has no root in [0, h)")
    return s
