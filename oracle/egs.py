"""EGS screening: the kernel of eps_EGS(k) as two Yukawa kernels, and the random-batch
estimator on it, composed from the single-Yukawa oracle by linearity.  FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 1 gives the gradient-corrected screening form
    eps_EGS(k) = 1 + (lambda k)^{-2} (1 + nu lambda^2 k^2 / 4)^{-1}
and notes that its potential 4 pi / (k^2 eps_EGS(k)) splits by partial fractions into two
Yukawa kernels.  With a = nu lambda^2 / 4 the denominator k^2 eps_EGS(k) (1 + a k^2) is
a k^4 + k^2 + 1/lambda^2 = a (k^2 + alpha)(k^2 + beta); for 0 < nu < 1, with
s = sqrt(1 - nu),
    alpha = 2 (1 + s) / (nu lambda^2),   beta = 2 (1 - s) / (nu lambda^2),
    4 pi / (k^2 eps_EGS) = 4 pi [ B / (k^2 + beta) + A / (k^2 + alpha) ],
    B = (1 + s) / (2 s),   A = -(1 - s) / (2 s),   A + B = 1,
so phi(r) = B Y_{lambda_B}(r) + A Y_{lambda_A}(r) with lambda_B = beta^{-1/2} (-> lambda as
nu -> 0) and lambda_A = alpha^{-1/2} (a short-ranged negative term).

Each term gets its own SOG decomposition (Algorithm 1) at the same r_c and eps.  Near
field, full far field, self energy and the brute-force lattice sum are the coefficient-
weighted sums of the single-Yukawa quantities.  The far part's transform
Fhat(k) = sum_i c_i Fhat_i(k) may change sign, so the modes are drawn from the envelope
Fhat_env(k) = sum_i |c_i| Fhat_i(k) with P(k) = calF(k) Fhat_env(k) / S_env, and the
estimator carries Fhat(k) / Fhat_env(k):
    coef_l = S_env Fhat(k_l) / (P V calF(k_l) Fhat_env(k_l)),
which is unbiased for the same reason as Eq. (60).  The adaptive correction of Eq. (62)
takes the EGS kernel in place of the Yukawa one:
    calF(k) = kT V / (kT V / Q2 + psi(k)),  psi(k) = sum_i c_i / (k^2 + lambda_i^{-2}) > 0,
with 4 pi psi for the Debye-unit variant; calF = 1 and calF = k^2 are unchanged.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import core
from . import sog as sog_mod
from .sog import SOG

NU_MAX = 0.96    # B and |A| stay below 3 (they grow like 1/sqrt(1 - nu))


def terms(lam: float, nu: float):
    """[(B, lambda_B), (A, lambda_A)] of the partial-fraction split (module docstring)."""
    if not (0.0 < nu <= NU_MAX):
        raise ValueError("need 0 < nu <= %g" % NU_MAX)
    s = math.sqrt(1.0 - nu)
    beta = 2.0 * (1.0 - s) / (nu * lam * lam)
    alpha = 2.0 * (1.0 + s) / (nu * lam * lam)
    return [((1.0 + s) / (2.0 * s), 1.0 / math.sqrt(beta)), (-(1.0 - s) / (2.0 * s), 1.0 / math.sqrt(alpha))]


def phi_hat(k2, lam: float, nu: float):
    """4 pi / (k^2 eps_EGS(k)) straight from eps_EGS (k > 0)."""
    k2 = np.asarray(k2, dtype=np.float64)
    eps = 1.0 + 1.0 / (lam * lam * k2 * (1.0 + nu * lam * lam * k2 / 4.0))
    return 4.0 * math.pi / (k2 * eps)


@dataclasses.dataclass(frozen=True)
class EGS:
    lam: float
    nu: float
    rc: float
    eps: float
    coef: tuple        # (B, A)
    lams: tuple        # (lambda_B, lambda_A)
    sogs: tuple        # one SOG per term

    def psi(self, k2):
        k2 = np.asarray(k2, dtype=np.float64)
        return sum(c / (k2 + 1.0 / (l * l)) for c, l in zip(self.coef, self.lams))

    def fhat(self, k2):
        return sum(c * _fhat_vec(s, k2) for c, s in zip(self.coef, self.sogs))

    def fhat_env(self, k2):
        return sum(abs(c) * _fhat_vec(s, k2) for c, s in zip(self.coef, self.sogs))

    def F0(self) -> float:
        """F(0) = sum_i c_i F_i(0), for the self energy of Eq. (52)."""
        return sum(c * core.sog_F(s, 0.0) for c, s in zip(self.coef, self.sogs))

    def kmax2(self) -> float:
        return max(core.kmax2_of(s) for s in self.sogs)


def build(lam: float, nu: float, rc: float, eps: float, mode: str = "minimal") -> EGS:
    tt = terms(lam, nu)
    sogs = tuple(sog_mod.build(l, rc, eps, mode) for _, l in tt)
    return EGS(lam, nu, rc, eps, tuple(c for c, _ in tt), tuple(l for _, l in tt), sogs)


def measure(kind: int, k2, kT: float, V: float, Q2: float, e: EGS):
    k2 = np.asarray(k2, dtype=np.float64)
    if kind == core.UNIFORM:
        return np.ones_like(k2)
    if kind == core.K2:
        return k2
    psi = e.psi(k2) * (4.0 * math.pi if kind == core.DEBYE else 1.0)
    return kT * V / (kT * V / Q2 + psi)


def all_modes(L, kmax2: float) -> np.ndarray:
    """Every m != 0 with |k|^2 <= kmax2, k = 2 pi m / L."""
    L = [float(x) for x in L]
    n = [int(math.floor(math.sqrt(kmax2) * La / (2.0 * math.pi))) for La in L]
    g = np.meshgrid(*[np.arange(-na, na + 1) for na in n], indexing="ij")
    m = np.stack([x.ravel() for x in g], axis=1)
    k2 = np.sum((m * (2.0 * math.pi / np.asarray(L))) ** 2, axis=1)
    keep = (k2 <= kmax2) & np.any(m != 0, axis=1)
    return m[keep]


def k2_of(m, L) -> np.ndarray:
    m = np.asarray(m, dtype=np.float64).reshape(-1, 3)
    return np.sum((m * (2.0 * math.pi / np.asarray([float(x) for x in L]))) ** 2, axis=1)


def S_sum(L, e: EGS, kT: float, Q2: float, kind: int = core.ADAPTIVE, kmax2=None) -> float:
    """S_env = sum_{k != 0} calF(k) Fhat_env(k) (Eq. 59 with the envelope)."""
    kmax2 = e.kmax2() if kmax2 is None else float(kmax2)
    k2 = k2_of(all_modes(L, kmax2), L)
    V = (float(L[0]) * float(L[1])) * float(L[2])
    fe = sum(abs(c) * _fhat_vec(s, k2) for c, s in zip(e.coef, e.sogs))
    return float(np.sum(measure(kind, k2, kT, V, Q2, e) * fe))


def _fhat_vec(s: SOG, k2):
    """Fhat of one SOG at many k^2 (the C oracle's formula, evaluated one by one)."""
    return np.array([core.fhat(s, float(x)) for x in np.ravel(k2)])


def rb_coef(m, L, e: EGS, kT: float, Q2: float, S: float, P=None, kind: int = core.ADAPTIVE) -> np.ndarray:
    m = np.asarray(m, dtype=np.float64).reshape(-1, 3)
    P = m.shape[0] if P is None else P
    V = (float(L[0]) * float(L[1])) * float(L[2])
    k2 = k2_of(m, L)
    f = sum(c * _fhat_vec(s, k2) for c, s in zip(e.coef, e.sogs))
    fe = sum(abs(c) * _fhat_vec(s, k2) for c, s in zip(e.coef, e.sogs))
    return S * f / (P * V * measure(kind, k2, kT, V, Q2, e) * fe)


def near(r, q, L, e: EGS, idx=None, cells: bool = True):
    F, U = None, 0.0
    for c, s in zip(e.coef, e.sogs):
        Fi, Ui = (core.near_cells if cells else core.near_images)(r, q, L, e.rc, s, idx=idx)
        F = c * Fi if F is None else F + c * Fi
        U += c * Ui
    return F, U


def far_full(r, q, L, e: EGS):
    F, U = None, 0.0
    for c, s in zip(e.coef, e.sogs):
        Fi, Ui = core.far_full(r, q, L, s, kmax2=e.kmax2())
        F = c * Fi if F is None else F + c * Fi
        U += c * Ui
    return F, U


def brute(r, q, L, e: EGS, rcut: float):
    F, U = None, 0.0
    for c, l in zip(e.coef, e.lams):
        Fi, Ui = core.brute_yukawa(r, q, L, l, rcut)
        F = c * Fi if F is None else F + c * Fi
        U += c * Ui
    return F, U


def self_energy(q, e: EGS) -> float:
    q = np.asarray(q, dtype=np.float64)
    return -0.5 * float(np.sum(q * q)) * e.F0()


def rb_forces(r, q, L, e: EGS, m, kT: float, S=None, idx=None, kind: int = core.ADAPTIVE, cells: bool = True):
    """Total force (near + random-batch far) on the k-set m and the energy terms, as
    core.rb_forces for a single Yukawa kernel."""
    q = np.asarray(q, dtype=np.float64)
    Q2 = float(np.sum(q * q))
    if S is None:
        S = S_sum(L, e, kT, Q2, kind=kind)
    coef = rb_coef(m, L, e, kT, Q2, S, kind=kind)
    rho_ = core.rho(r, q, L, m)
    Ff = core.far_rb(r, q, L, m, coef, rho_, idx=idx)
    Fn, UN = near(r, q, L, e, idx=idx, cells=cells)
    V = (float(L[0]) * float(L[1])) * float(L[2])
    qs = float(np.sum(q))
    f0 = sum(c * core.fhat(s, 0.0) for c, s in zip(e.coef, e.sogs))
    UF = float(np.sum(0.5 * coef * (rho_[:, 0] ** 2 + rho_[:, 1] ** 2))) + f0 * qs * qs / (2.0 * V)
    return Fn + Ff, Fn, Ff, dict(U_N=UN, U_F=UF, U_self=self_energy(q, e)), S
