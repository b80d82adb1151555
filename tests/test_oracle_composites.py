"""Pins of the oracle's composite quantities: the random-batch energy U*_F (Eq. 60 plus the
k = 0 term) and the composite total force, for the Yukawa kernel and the EGS screening.

Each is pinned by an identity it must satisfy and that does not go through its own code:
  * with every mode of the support and coef_l = Fhat(k_l)/V, the estimator's energy is
    the deterministic far energy of Eq. (53), which the Poisson identity and the
    brute-force lattice sum pin elsewhere;
  * the exact expectation over one-mode draws, sum_k P(k) X(k), of the composite force and
    energy is the near field plus the full far field (Lemma 4.1, E Xi = 0).
The systems are not neutral, so the k = 0 energy term F^(0)(sum q)^2/(2V) is non-zero and
a dropped term fails; a dropped 1/2 or a wrong volume fails the first identity."""
import math

import numpy as np
import pytest

from oracle import core, egs
from oracle import sog as S
from oracle.sampler import ModeSampler

LAM = 0.6


def system(N=8, L=4.0, seed=21, charges=(1.0, 1.0, -1.0, 2.0)):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.0, L, size=(N, 3))
    q = rng.choice(np.asarray(charges), size=N)
    return r, q, [L, L, L]


def support(L, kmax2):
    n = int(math.sqrt(kmax2) * max(L) / (2 * math.pi)) + 1
    g = np.arange(-n, n + 1)
    m = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k2 = np.sum((2 * math.pi * m / np.asarray(L)) ** 2, axis=1)
    return m[k2 <= kmax2].astype(np.int32), k2[k2 <= kmax2]


@pytest.mark.parametrize("seed", [21, 22])
def test_rb_energy_with_the_whole_support_is_the_far_energy(seed):
    """rb_energy on every mode with coef = Fhat/V equals U_F of Eq. (53) (k = 0 included)."""
    r, q, L = system(seed=seed)
    sg = S.build(LAM, 1.9, 1e-7)
    m, k2 = support(L, core.kmax2_of(sg))
    V = L[0] * L[1] * L[2]
    coef = np.array([core.fhat(sg, float(x)) / V for x in k2])
    rho = core.rho(r, q, L, m)
    U = core.rb_energy(rho, coef, q, L, sg)
    _, Ufull = core.far_full(r, q, L, sg)
    assert abs(float(np.sum(q))) > 0.5           # the k = 0 term matters here
    assert abs(U - Ufull) <= 1e-12 * abs(Ufull), (U, Ufull)


def test_rb_energy_of_a_single_mode_closed_form():
    """One particle of charge q at r, one mode, coef c: U = c q^2 / 2 + Fhat(0) q^2 / (2V)."""
    sg = S.build(LAM, 1.9, 1e-7)
    L = [3.0, 4.0, 5.0]
    V = 60.0
    r = np.array([[0.4, 1.3, 2.2]])
    q = np.array([1.5])
    rho = core.rho(r, q, L, np.array([[1, -2, 3]], dtype=np.int32))
    U = core.rb_energy(rho, [0.7], q, L, sg)
    ref = 0.7 * 1.5 ** 2 / 2 + core.fhat(sg, 0.0) * 1.5 ** 2 / (2 * V)
    assert abs(U - ref) <= 1e-14 * abs(ref)


@pytest.mark.parametrize("kind", [core.ADAPTIVE, core.UNIFORM, core.K2])
def test_rb_forces_expectation_is_near_plus_full_far(kind):
    """sum over the support of P(k) rb_forces([k]) (one-mode draws, P = 1) equals the near
    field of the explicit image loop plus the full far field, forces and energies; the
    near part and the self energy come back unchanged in every draw."""
    r, q, L = system()
    sg = S.build(LAM, 1.9, 1e-5)
    kT = 1.0
    Q2 = float(np.sum(q * q))
    ms = ModeSampler(sg, L, kT, Q2, kind=kind)
    modes = ms.all_modes()
    k2 = ms.k2_of(modes)
    V = L[0] * L[1] * L[2]
    S_ = core.S_sum(L, sg, kT, Q2, kind=kind)
    p = np.array([core.measure(kind, x, kT, V, Q2, LAM) * core.fhat(sg, x) for x in k2]) / S_
    assert abs(np.sum(p) - 1.0) <= 1e-12
    Fsum = np.zeros_like(r)
    Usum = 0.0
    Fn0, Un0 = core.near_images(r, q, L, 1.9, sg)
    for j in range(len(modes)):
        Ft, Fn, Ff, e = core.rb_forces(r, q, L, 1.9, sg, modes[j:j + 1], kT, S=S_, kind=kind)
        Fsum += p[j] * Ft
        Usum += p[j] * e["U_F"]
        if j % 997 == 0:
            assert core.rel_l2(Fn, Fn0) <= 1e-14 and abs(e["U_N"] - Un0) <= 1e-13 * abs(Un0)
            assert np.array_equal(Ft, Fn + Ff)
            assert e["U_self"] == core.self_energy(q, sg)
    Ffull, Ufull = core.far_full(r, q, L, sg)
    assert core.rel_l2(Fsum, Fn0 + Ffull) <= 1e-11
    assert abs(Usum - Ufull) <= 1e-11 * abs(Ufull)


def test_rb_forces_rows_follow_idx():
    """rb_forces with idx returns those particles' rows of the whole-system evaluation."""
    r, q, L = system(N=30, L=6.0, seed=4)
    sg = S.build(LAM, 2.0, 1e-6)
    m = np.array([[1, 0, 0], [0, 2, -1], [3, 1, 1], [-1, -1, 2]], dtype=np.int32)
    Ft, Fn, Ff, _ = core.rb_forces(r, q, L, 2.0, sg, m, 0.8)
    idx = np.array([0, 7, 29])
    Ft3, Fn3, Ff3, _ = core.rb_forces(r, q, L, 2.0, sg, m, 0.8, idx=idx)
    scale = np.abs(Ft).max()
    assert np.allclose(Ft3, Ft[idx], rtol=0, atol=1e-13 * scale)
    assert np.allclose(Ff3, Ff[idx], rtol=0, atol=1e-13 * scale)


def test_egs_rb_forces_expectation_is_near_plus_full_far():
    """The EGS composite force over one-mode draws from the envelope measure: its exact
    mean is the EGS near field plus the EGS full far field, forces and energies."""
    r, q, L = system(N=6, seed=9)
    L = np.asarray(L)
    e = egs.build(LAM, 0.6, 1.9, 1e-5)
    kT = 1.1
    Q2 = float(np.sum(q * q))
    V = float(np.prod(L))
    kmax2 = e.kmax2()
    m = egs.all_modes(L, kmax2)
    k2 = egs.k2_of(m, L)
    S_ = egs.S_sum(L, e, kT, Q2, kmax2=kmax2)
    prob = egs.measure(core.ADAPTIVE, k2, kT, V, Q2, e) * e.fhat_env(k2) / S_
    Fsum = np.zeros_like(r)
    Usum = 0.0
    Fn0, Un0 = egs.near(r, q, L, e, cells=False)
    for j in range(len(m)):
        Ft, Fn, Ff, en, _ = egs.rb_forces(r, q, L, e, m[j:j + 1], kT, S=S_, cells=False)
        Fsum += prob[j] * Ft
        Usum += prob[j] * en["U_F"]
    Ffull, Ufull = egs.far_full(r, q, L, e)
    assert core.rel_l2(Fsum, Fn0 + Ffull) <= 1e-10
    assert abs(Usum - Ufull) <= 1e-10 * abs(Ufull)
