"""Pins of the random-batch estimator and the sampler: exact mean and variance
(Lemma 4.1), chi-square of draws against P(k) (Eq. 59), Philox known answers."""
import math
import os

import numpy as np
import pytest

from oracle import core, philox
from oracle import sog as S
from oracle.sampler import ModeSampler, vose_alias
from paper_2501_10946_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = philox.philox4x32_10(*v[:6])
        assert [int(x) for x in out] == v[6:]


def test_vose_alias_tables_encode_the_distribution():
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 100):
        w = rng.uniform(0.01, 1.0, n) ** 3
        prob, alias = vose_alias(w)
        implied = np.zeros(n)
        for j in range(n):
            implied[j] += prob[j] / n
            implied[alias[j]] += (1.0 - prob[j]) / n
        assert np.allclose(implied, w / w.sum(), rtol=1e-12, atol=1e-15)


def test_index_below_is_floor_of_u_times_n():
    a = np.array([0, 0xFFFFFFFF, 0x80000000, 0x12345678], dtype=np.uint64)
    b = np.array([0, 0xFFFFFFFF, 0, 0x9ABCDEF0], dtype=np.uint64)
    for n in (1, 3, 1000, 2 ** 30 + 7):
        got = philox.index_below(a, b, n)
        exp = [((int(x) << 32 | int(y)) * n) >> 64 for x, y in zip(a, b)]
        assert got.tolist() == exp


class Fixture:
    def __init__(self, mix, kT, kind=0):
        self.kind = kind
        self.N, self.L = 8, [4.0, 4.0, 4.0]
        self.lam, self.rc = 0.6, 1.9
        self.r, self.q = W.small_system(self.N, 4.0, 21, charge_mix=mix)
        self.sog = S.build(self.lam, self.rc, 1e-5)
        self.kT = kT
        self.Q2 = float(np.sum(self.q ** 2))
        self.ms = ModeSampler(self.sog, self.L, kT, self.Q2, kind=kind)
        self.S = core.S_sum(self.L, self.sog, kT, self.Q2, kind=kind)
        self.V = 64.0
        self.modes = self.ms.all_modes()
        k2 = self.ms.k2_of(self.modes)
        self.p = np.array([core.measure(kind, x, kT, self.V, self.Q2, self.lam) * core.fhat(self.sog, x)
                           for x in k2]) / self.S
        # single-draw estimator X_i(k) (P = 1) through the oracle's own estimator functions
        self.X = np.zeros((len(self.modes), self.N, 3))
        self.Ue = np.zeros(len(self.modes))
        rho = core.rho(self.r, self.q, self.L, self.modes)
        coef = core.rb_coef(self.modes, self.L, self.sog, kT, self.Q2, self.S, P=1, kind=kind)
        for j in range(len(self.modes)):
            self.X[j] = core.far_rb(self.r, self.q, self.L, self.modes[j:j + 1], coef[j:j + 1], rho[j:j + 1])
            self.Ue[j] = 0.5 * coef[j] * (rho[j, 0] ** 2 + rho[j, 1] ** 2)
        self.index = {tuple(m): j for j, m in enumerate(self.modes)}


@pytest.fixture(scope="module", params=[(False, 1.0, 0), (True, 0.05, 0), (False, 40.0, 0), (False, 1.0, 1),
                                        (True, 0.05, 1), (False, 1.0, 2), (True, 0.05, 2), (False, 1.0, 3),
                                        (True, 0.05, 3)],
                ids=["ocp", "mix-cold", "hot", "ocp-F1", "mix-cold-F1", "ocp-k2", "mix-cold-k2", "ocp-debye",
                     "mix-cold-debye"])
def fx(request):
    return Fixture(*request.param)


def test_S_matches_the_sampler_support(fx):
    k2 = fx.ms.k2_of(fx.modes)
    S_py = float(np.sum(fx.ms.calF(k2) * fx.ms.fhat(k2)))
    assert abs(S_py - fx.S) <= 1e-12 * fx.S
    assert abs(np.sum(fx.p) - 1.0) <= 1e-12


def test_exact_mean_is_the_full_far_field(fx):
    """Lemma 4.1 (E Xi = 0): sum_k P(k) X_i(k) equals the deterministic far force of Eq. (55)."""
    mean = np.tensordot(fx.p, fx.X, axes=1)
    Ff, Uf = core.far_full(fx.r, fx.q, fx.L, fx.sog)
    assert core.rel_l2(mean, Ff) <= 1e-11
    qs = float(np.sum(fx.q))
    U0 = core.fhat(fx.sog, 0.0) * qs * qs / (2 * fx.V)
    assert abs(float(fx.p @ fx.Ue) + U0 - Uf) <= 1e-11 * abs(Uf)


def test_exact_variance_formula(fx):
    """Eq. (66) with S = sum calF Fhat: E|X_i|^2 = (q_i^2 S / V^2) sum_k k^2 Fhat Im^2 / calF
    (any measure)."""
    EX2 = np.tensordot(fx.p, np.sum(fx.X ** 2, axis=2), axes=1)
    rho = core.rho(fx.r, fx.q, fx.L, fx.modes)
    k = 2 * math.pi * fx.modes / 4.0
    k2 = np.sum(k * k, axis=1)
    cal = np.array([core.measure(fx.kind, x, fx.kT, fx.V, fx.Q2, fx.lam) for x in k2])
    fh = np.array([core.fhat(fx.sog, x) for x in k2])
    for i in range(fx.N):
        th = k @ fx.r[i]
        im = np.cos(th) * rho[:, 1] - np.sin(th) * rho[:, 0]
        ref = fx.q[i] ** 2 * fx.S / fx.V ** 2 * float(np.sum(k2 * fh * im * im / cal))
        assert abs(EX2[i] - ref) <= 1e-11 * ref


def test_monte_carlo_mean_and_variance(fx):
    """Draws from the oracle sampler: z-test of the mean (P = 4) and variance test of single draws."""
    P, sets = 4, 20000
    m, _ = fx.ms.draw(seed=99, draw_index=5, P=P * sets)
    j = np.array([fx.index[tuple(x)] for x in m])
    Fstar = fx.X[j].reshape(sets, P, fx.N, 3).mean(axis=1)
    mean_exact = np.tensordot(fx.p, fx.X, axes=1)
    var1 = np.tensordot(fx.p, fx.X ** 2, axes=1) - mean_exact ** 2
    z = (Fstar.mean(axis=0) - mean_exact) / np.sqrt(var1 / P / sets)
    assert np.max(np.abs(z)) < 5.0
    # single-draw variance with a tolerance from the exact fourth central moment
    Xs = fx.X[j]
    n = Xs.shape[0]
    mu4 = np.tensordot(fx.p, (fx.X - mean_exact) ** 4, axes=1)
    s2 = Xs.var(axis=0, ddof=1)
    sd = np.sqrt(np.maximum(mu4 - var1 ** 2, 0) / n)
    assert np.all(np.abs(s2 - var1) <= 5 * sd + 1e-300)
    # energy estimator is unbiased too
    Ustar = fx.Ue[j].reshape(sets, P).mean(axis=1)
    Uvar = float(fx.p @ fx.Ue ** 2) - float(fx.p @ fx.Ue) ** 2
    assert abs(Ustar.mean() - float(fx.p @ fx.Ue)) <= 5 * math.sqrt(Uvar / P / sets)


def test_sampler_chi_square(fx):
    """T5 on the oracle sampler: 2e5 draws against P(k) on the 100 most probable modes + tail."""
    m, att = fx.ms.draw(seed=1234, draw_index=0, P=200000)
    j = np.array([fx.index[tuple(x)] for x in m])
    cnt = np.bincount(j, minlength=len(fx.modes)).astype(float)
    order = np.argsort(-fx.p)
    top = order[:100]
    e = np.append(fx.p[top], fx.p[order[100:]].sum()) * len(j)
    o = np.append(cnt[top], cnt[order[100:]].sum())
    keep = e > 5
    chi2 = float(np.sum((o[keep] - e[keep]) ** 2 / e[keep]))
    dof = int(keep.sum()) - 1
    # 5-sigma bound of the chi-square distribution
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)
    assert np.all(att >= 1)


def test_replay_is_deterministic():
    f = Fixture(False, 1.0)
    a, _ = f.ms.draw(7, 3, 64)
    b, _ = f.ms.draw(7, 3, 64)
    c, _ = f.ms.draw(7, 4, 64)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(np.any(a != 0, axis=1))


def _image_sum(L, fn, rmax):
    """sum over lattice vectors n L (n in Z^3, |n L| <= rmax) of fn(|n L|)."""
    nm = [int(math.ceil(rmax / L[a])) for a in range(3)]
    tot = 0.0
    for i in range(-nm[0], nm[0] + 1):
        for j in range(-nm[1], nm[1] + 1):
            for k in range(-nm[2], nm[2] + 1):
                d = math.sqrt((i * L[0]) ** 2 + (j * L[1]) ** 2 + (k * L[2]) ** 2)
                if d <= rmax:
                    tot += fn(d)
    return tot


@pytest.mark.parametrize("L", [(4.0, 4.0, 4.0), (3.0, 4.0, 5.5)])
def test_S_of_the_other_measures_by_poisson_summation(L):
    """The k-space normalisations against real space (Poisson summation of the Gaussian
    sum F = sum_m a_m exp(-b_m r^2)): sum_k Fhat(k) = V sum_n F(|n L|) and
    sum_k k^2 Fhat(k) = -V sum_n (Laplacian F)(|n L|), the k = 0 terms being Fhat(0) and 0."""
    sog = S.build(0.6, 1.9, 1e-5)
    V = L[0] * L[1] * L[2]
    t = np.asarray(sog.t, dtype=np.float64)
    b = np.exp(t)
    a = np.array([sog.h * float(w) * float(S.f_tr(float(x), 0.0, sog.lam)) for x, w in zip(t, sog.weights)])
    rmax = math.sqrt(45.0 / float(np.min(b)))

    def F(r):
        return float(np.sum(a * np.exp(-b * r * r)))

    def lapF(r):
        return float(np.sum(a * np.exp(-b * r * r) * (4.0 * b * b * r * r - 6.0 * b)))

    # the Gaussian sum reproduces the library-independent kernel evaluation
    assert abs(F(0.7) - core.sog_F(sog, 0.7)) <= 1e-13 * abs(F(0.7))
    S1 = core.S_sum(L, sog, 1.0, 1.0, kind=core.UNIFORM)
    S2 = core.S_sum(L, sog, 1.0, 1.0, kind=core.K2)
    ref1 = V * _image_sum(L, F, rmax) - core.fhat(sog, 0.0)
    ref2 = -V * _image_sum(L, lapF, rmax)
    assert abs(S1 - ref1) <= 1e-11 * abs(ref1)
    assert abs(S2 - ref2) <= 1e-11 * abs(ref2)


def test_closed_form_fluctuations_match_the_single_draw_moments(fx):
    """oracle.variance against the per-mode estimator table of the fixture:
    F_fluc = (1/N) sum_i Var X_i / P and E_fluc = Var Y / P for every measure."""
    from oracle import variance
    P = 3
    out = variance.fluctuations(fx.r, fx.q, fx.L, fx.sog, fx.kT, P, kinds=(fx.kind,))
    mean = np.tensordot(fx.p, fx.X, axes=1)
    var = np.tensordot(fx.p, np.sum(fx.X ** 2, axis=2), axes=1) - np.sum(mean ** 2, axis=1)
    F_ref = float(np.mean(var)) / P
    E_ref = (float(fx.p @ fx.Ue ** 2) - float(fx.p @ fx.Ue) ** 2) / P
    F_fluc, E_fluc = out[fx.kind]
    assert abs(F_fluc - F_ref) <= 1e-9 * F_ref
    assert abs(E_fluc - E_ref) <= 1e-9 * E_ref
