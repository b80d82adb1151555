"""Pins of the EGS oracle (oracle/egs.py): the two-Yukawa split against eps_EGS itself,
its limits, the composed decomposition against the brute-force periodic lattice sum of
the EGS potential, and the unbiasedness of the envelope estimator over the whole mode
support."""
import math

import numpy as np
import pytest

from oracle import core, egs

LAM = 0.6


def small_system(N=20, seed=11):
    rng = np.random.default_rng(seed)
    L = np.array([4.0, 4.5, 5.0])
    r = rng.random((N, 3)) * L
    q = rng.choice([-1.0, 1.0], size=N)
    return r, q, L


@pytest.mark.parametrize("nu", [1e-3, 0.2, 0.5, 0.9])
@pytest.mark.parametrize("lam", [0.3, 0.6, 2.0])
def test_two_yukawa_split_reproduces_eps_egs(lam, nu):
    """4 pi sum_i c_i / (k^2 + lambda_i^-2) equals 4 pi / (k^2 eps_EGS(k)) computed from
    eps_EGS itself, over six decades of k."""
    tt = egs.terms(lam, nu)
    k2 = np.logspace(-4, 4, 200) / (lam * lam)
    split = 4.0 * math.pi * sum(c / (k2 + 1.0 / (l * l)) for c, l in tt)
    direct = egs.phi_hat(k2, lam, nu)
    assert np.max(np.abs(split - direct) / direct) <= 1e-12
    B, A = tt[0][0], tt[1][0]
    assert abs(A + B - 1.0) <= 1e-14 and B > 1.0 and A < 0.0


def test_small_nu_is_the_yukawa_kernel():
    (B, lB), (A, lA) = egs.terms(LAM, 1e-8)
    assert abs(B - 1.0) <= 1e-8 and abs(lB - LAM) <= 1e-8 * LAM and abs(A) <= 1e-8
    assert lA <= 1e-3 * LAM


@pytest.mark.parametrize("nu", [0.3, 0.8])
def test_egs_decomposition_matches_brute_force_lattice_sum(nu):
    """Near (image sum) + full far + self of both terms against the brute-force periodic
    sum of B Y_{lambda_B} + A Y_{lambda_A}."""
    r, q, L = small_system()
    e = egs.build(LAM, nu, 2.0, 1e-9)
    Fn, Un = egs.near(r, q, L, e, cells=False)
    Ff, Uf = egs.far_full(r, q, L, e)
    Us = egs.self_energy(q, e)
    Fb, Ub = egs.brute(r, q, L, e, 40 * LAM)
    assert core.rel_l2(Fn + Ff, Fb) <= 1e-6
    assert abs(Un + Uf + Us - Ub) <= 1e-6 * abs(Ub)


def test_envelope_estimator_is_unbiased_over_the_support():
    """Summing P(k) times the one-draw estimator over every mode of the support gives the
    full k-space far force and energy: P(k) coef_1(k) = Fhat(k) / V for the envelope
    measure, whatever sign Fhat takes."""
    r, q, L = small_system(N=12)
    e = egs.build(LAM, 0.7, 2.0, 1e-6)
    Q2 = float(np.sum(q * q))
    kT = 1.3
    V = float(L[0] * L[1] * L[2])
    kmax2 = e.kmax2()
    m = egs.all_modes(L, kmax2)
    k2 = egs.k2_of(m, L)
    S = egs.S_sum(L, e, kT, Q2, kmax2=kmax2)
    prob = egs.measure(core.ADAPTIVE, k2, kT, V, Q2, e) * e.fhat_env(k2) / S
    assert abs(np.sum(prob) - 1.0) <= 1e-12
    one_draw = egs.rb_coef(m, L, e, kT, Q2, S, P=1)
    rho = core.rho(r, q, L, m)
    F_expect = core.far_rb(r, q, L, m, prob * one_draw, rho)
    Ff, Uf = egs.far_full(r, q, L, e)
    assert core.rel_l2(F_expect, Ff) <= 1e-10
    qs = float(np.sum(q))
    f0 = float(e.fhat(0.0)[0])
    U_expect = float(np.sum(0.5 * prob * one_draw * (rho[:, 0] ** 2 + rho[:, 1] ** 2))) + f0 * qs * qs / (2 * V)
    assert abs(U_expect - Uf) <= 1e-10 * abs(Uf)
