"""Exact fluctuations of the random-batch estimators for one configuration, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 5 (Fig. 9) compares the sampling corrections calF of Eq. (59) by
  E_fluc = <(E* - E)^2>  and  F_fluc = <(1/N) sum_i |F*_i - F_i|^2>,
ensemble averages over configurations of a run.  For one configuration the
variance over k-draws is known in closed form (P i.i.d. draws from P(k) = calF Fhat / S):
  single draw, force:  X_i(k) = -(q_i S / (V calF(k))) k Im(exp(-i k.r_i) rho(k))
     E|X_i|^2 = (q_i^2 S / V^2) sum_k k^2 Fhat Im_i(k)^2 / calF(k)          (Eq. 66)
     E X_i    = F_i = -(q_i / V) sum_k k Fhat Im_i(k)                       (Lemma 4.1)
  single draw, energy: Y(k) = S |rho(k)|^2 / (2 V calF(k))
     E Y^2 = (S / (4 V^2)) sum_k Fhat |rho|^4 / calF,   E Y = sum_k Fhat |rho|^2 / (2V)
and the mean of P draws has 1/P of the single-draw variance.  The k = 0 energy term is
deterministic and drops out.  Sums run over every mode the sampler can draw (k^2 <=
4 b_max ln 1e17).
"""
from __future__ import annotations

import numpy as np

from . import core
from .sampler import ModeSampler


def fluctuations(r, q, L, sog, kT, P, kinds=(core.ADAPTIVE, core.UNIFORM, core.K2, core.DEBYE), chunk=4096,
                 with_force=False):
    """{kind: (F_fluc, E_fluc)} for the configuration (r, q) and batch size P; with
    with_force also the exact far force [N, 3] (the estimators' mean)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    N = r.shape[0]
    Q2 = float(np.sum(q * q))
    base = ModeSampler(sog, L, kT, Q2)
    modes = base.all_modes()
    V = (float(L[0]) * float(L[1])) * float(L[2])
    tpl = np.array([2.0 * np.pi / float(x) for x in L])
    k = modes * tpl[None, :]
    k2 = np.sum(k * k, axis=1)
    fh = base.fhat(k2)
    rho = core.rho(r, q, L, modes)
    rho2 = rho[:, 0] ** 2 + rho[:, 1] ** 2
    cal = {}
    for kind in kinds:
        cal[kind] = ModeSampler(sog, L, kT, Q2, kind=kind).calF(k2)
    S = {kind: float(np.sum(cal[kind] * fh)) for kind in kinds}
    # per particle: sum_k w(k) Im_i(k)^2 for each measure, and the exact force
    acc = {kind: np.zeros(N) for kind in kinds}
    Fexact = np.zeros((N, 3))
    for c0 in range(0, modes.shape[0], chunk):
        sl = slice(c0, c0 + chunk)
        th = r @ k[sl].T
        im = np.cos(th) * rho[sl, 1][None, :] - np.sin(th) * rho[sl, 0][None, :]
        Fexact += -(im * fh[sl][None, :]) @ k[sl]
        im2 = im * im
        for kind in kinds:
            acc[kind] += im2 @ (k2[sl] * fh[sl] / cal[kind][sl])
    Fexact *= q[:, None] / V
    F2 = np.sum(Fexact * Fexact, axis=1)
    EY = float(np.sum(fh * rho2)) / (2.0 * V)
    out = {}
    for kind in kinds:
        EX2 = q * q * S[kind] / (V * V) * acc[kind]
        F_fluc = float(np.mean(EX2 - F2)) / P
        EY2 = S[kind] / (4.0 * V * V) * float(np.sum(fh * rho2 * rho2 / cal[kind]))
        E_fluc = (EY2 - EY * EY) / P
        out[kind] = (F_fluc, E_fluc)
    return (out, Fexact) if with_force else out
