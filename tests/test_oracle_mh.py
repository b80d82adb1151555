"""Pins of the oracle's Metropolis-Hastings chains (oracle.sampler.MHChains), the sampler
that Sec. 4.3 names for drawing the batch from P(k) of Eq. (59):
  * the acceptance test is the Metropolis-Hastings ratio min(1, P(k')Q(k) / (P(k)Q(k')))
    of the exact measure P and the exact proposal Q (computed here from calF and Fhat,
    not from the chain's code);
  * independent chains sampled at one evaluation after burn-in pass a chi-square test
    against P(k);
  * the lag-1 autocorrelation of k^2 along the chains equals the value of the exact
    transition kernel K(k, k') = Q(k') alpha(k, k') (+ rejection mass on the diagonal);
    the integrated autocorrelation time is printed."""
import json
import math

import numpy as np
import pytest

from oracle import sog as S
from oracle.sampler import ADAPTIVE, DEBYE, K2, UNIFORM, MHChains, ModeSampler


def fixture(kind, kT=0.01):
    sg = S.build(0.6, 1.9, 1e-5)
    L = [4.0, 4.0, 4.0]
    ms = ModeSampler(sg, L, kT, 8.0, kind=kind)
    modes = ms.all_modes()
    k2 = ms.k2_of(modes)
    p = ms.calF(k2) * ms.fhat(k2)
    p = p / p.sum()
    # proposal: the mixture of steps 1-2 over the whole table box, k = 0 included
    q = ms.fhat(k2) * (k2 if kind == K2 else 1.0)
    z = q.sum() + (0.0 if kind == K2 else float(ms.fhat(0.0)))
    return ms, modes, k2, p, q / z


@pytest.mark.parametrize("kind", [ADAPTIVE, DEBYE, UNIFORM, K2])
def test_acceptance_is_the_metropolis_hastings_ratio(kind):
    ms, modes, k2, p, q = fixture(kind)
    ch = MHChains(ms, 1)
    rng = np.random.default_rng(3)
    i = rng.integers(0, len(modes), 20000)
    j = rng.integers(0, len(modes), 20000)
    u = rng.random(20000)
    ratio = np.minimum(1.0, (p[j] * q[i]) / (p[i] * q[j]))
    got = ch.accepts(u, k2[i], k2[j])
    clear = np.abs(u - ratio) > 1e-12 * np.maximum(1.0, ratio)
    assert np.array_equal(got[clear], (u < ratio)[clear])
    if kind in (UNIFORM, K2):
        assert np.all(got)
    else:
        assert 0.001 < float(np.mean(~got)) < 0.5      # the test does reject here


def chi_square(draws, modes, p):
    index = {tuple(x): j for j, x in enumerate(modes)}
    js = np.array([index[tuple(x)] for x in draws])
    counts = np.bincount(js, minlength=len(modes))
    n = len(js)
    order = np.argsort(-p)
    top = order[:200]
    e = np.append(p[top], p[order[200:]].sum()) * n
    o = np.append(counts[top], counts[order[200:]].sum())
    keep = e > 5
    chi2 = float(np.sum((o[keep] - e[keep]) ** 2 / e[keep]))
    return chi2, int(keep.sum()) - 1


@pytest.mark.parametrize("kind", [ADAPTIVE, DEBYE, K2])
def test_independent_chains_after_burn_in_follow_P(kind):
    ms, modes, k2, p, q = fixture(kind)
    ch = MHChains(ms, 20000, sweeps=1, burnin=64)
    ch.draw(11)
    draws = ch.draw(11)
    chi2, dof = chi_square(draws, modes, p)
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def test_a_chain_without_burn_in_starts_from_the_proposal():
    """Zero burn-in: the first batch is the proposal's law Q, not P, when they differ
    (the chain needs its burn-in)."""
    ms, modes, k2, p, q = fixture(ADAPTIVE)
    ch = MHChains(ms, 20000, burnin=0)
    chi2_p, dof = chi_square(ch.draw(5), modes, p)
    assert chi2_p > dof + 10 * math.sqrt(2 * dof)


def exact_lag1(ms, modes, k2, p, q, kind):
    """Lag-1 autocorrelation of f = k^2 under the exact independence-sampler kernel."""
    A = ms.kT * ms.V
    Q2 = (4.0 * math.pi) * ms.Q2 if kind == DEBYE else ms.Q2
    a = (A * (k2 + ms.inv_lam2)) / (A * (k2 + ms.inv_lam2) + Q2)      # a(k) = calF / Q2
    f = k2
    Ef = float(p @ f)
    Vf = float(p @ (f * f)) - Ef * Ef
    E01 = 0.0
    for s in range(0, len(modes), 512):
        ai = a[s:s + 512, None]
        alpha = np.minimum(1.0, a[None, :] / ai)                      # alpha(k_i -> k_j)
        move = q[None, :] * alpha
        stay = 1.0 - move.sum(axis=1)                                 # rejections, proposals of 0 included
        E01 += float(np.sum(p[s:s + 512] * f[s:s + 512] * (move @ f + stay * f[s:s + 512])))
    return (E01 - Ef * Ef) / Vf


@pytest.mark.parametrize("kind", [ADAPTIVE, DEBYE])
def test_lag1_autocorrelation_matches_the_exact_kernel(kind):
    ms, modes, k2, p, q = fixture(kind)
    rho_exact = exact_lag1(ms, modes, k2, p, q, kind)
    P, T = 8192, 24
    ch = MHChains(ms, P, sweeps=1, burnin=64)
    xs = np.stack([ms.k2_of(ch.draw(9)) for _ in range(T)])           # [T, P]
    mu, var = float(np.mean(xs)), float(np.var(xs))
    lag = [float(np.mean((xs[:-t] - mu) * (xs[t:] - mu)) / var) for t in range(1, 8)]
    # standard error of a lag-1 estimate from P (T - 1) correlated pairs: about
    # sqrt((1 + 2 tau) / (P (T - 1)))
    tau = 1.0 + 2.0 * sum(max(x, 0.0) for x in lag)
    se = math.sqrt(tau / (P * (T - 1)))
    print(json.dumps({"kind": kind, "lag1_exact": rho_exact, "lag1_chain": lag[0], "lags": lag,
                      "integrated_autocorrelation_time": tau,
                      "acceptance": ch.accepted / ch.proposed}))
    assert abs(lag[0] - rho_exact) <= 5 * se + 1e-3, (lag[0], rho_exact, se)
    assert 0.0 < rho_exact < 1.0
