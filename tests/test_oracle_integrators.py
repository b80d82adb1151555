"""Pins of the oracle integrators: harmonic special case, time reversibility, BAOAB
stationary variance, and the dt^2 energy drift of velocity Verlet with the
deterministic (all-modes) RBSOG force."""
import math

import numpy as np

from oracle import core, integrate
from oracle import sog as S
from paper_2501_10946_gb300 import workloads as W


def test_wrap():
    L = [10.0, 10.0, 10.0]
    r = np.array([[0.0, 9.999, 10.0], [-1e-300, -2.5, 25.0], [np.nextafter(10.0, 0), 3.0, -10.0]])
    w = integrate.wrap(r, L)
    assert np.all(w >= 0) and np.all(w < 10.0)
    assert w[0].tolist() == [0.0, 9.999, 0.0]
    assert w[1, 1] == 7.5 and w[1, 2] == 5.0 and w[2, 2] == 0.0


def test_velocity_verlet_harmonic():
    """VV on x'' = -x obeys the closed-form recurrence x_{n+1} = (2 - dt^2) x_n - x_{n-1}."""
    L = [1e6] * 3
    dt = 0.05
    r = np.array([[5e5 + 1.0, 5e5, 5e5]])
    v = np.zeros((1, 3))
    centre = np.array([5e5, 5e5, 5e5])
    f = lambda x: -(x - centre)
    F = f(r)
    xs = [r[0, 0] - centre[0]]
    for _ in range(200):
        r, v, F = integrate.vv_step(r, v, F, np.ones(1), L, dt, f)
        xs.append(r[0, 0] - centre[0])
    xs = np.array(xs)
    pred = (2 - dt * dt) * xs[1:-1] - xs[:-2]
    assert np.max(np.abs(pred - xs[2:])) < 1e-9


def rbsog_system():
    N, L = 12, 5.0
    r, q = W.small_system(N, L, 8, charge_mix=True)
    # push apart any very close pair so the force stays moderate
    sg = S.build(0.6, 2.4, 1e-8)
    def force(x):
        Fn, _ = core.near_images(x, q, [L] * 3, 2.4, sg)
        Ff, _ = core.far_full(x, q, [L] * 3, sg)
        return Fn + Ff
    def energy(x, v):
        _, Un = core.near_images(x, q, [L] * 3, 2.4, sg)
        _, Uf = core.far_full(x, q, [L] * 3, sg)
        return Un + Uf + core.self_energy(q, sg) + integrate.kinetic(v, np.ones(N))
    rng = np.random.default_rng(3)
    v = rng.normal(0, 0.3, (N, 3))
    return r, v, q, force, energy, [L] * 3


def test_time_reversibility():
    r0, v0, q, force, energy, L = rbsog_system()
    r, v = r0.copy(), v0.copy()
    F = force(r)
    for _ in range(20):
        r, v, F = integrate.vv_step(r, v, F, np.ones(len(q)), L, 0.01, force)
    v = -v
    for _ in range(20):
        r, v, F = integrate.vv_step(r, v, F, np.ones(len(q)), L, 0.01, force)
    d = r - r0
    d -= 5.0 * np.round(d / 5.0)
    assert np.max(np.abs(d)) < 1e-11 and np.max(np.abs(-v - v0)) < 1e-11


def test_vv_energy_error_scales_as_dt_squared():
    r0, v0, q, force, energy, L = rbsog_system()
    dev = []
    for dt in (0.02, 0.01):
        r, v = r0.copy(), v0.copy()
        F = force(r)
        E0 = energy(r, v)
        worst = 0.0
        for _ in range(int(round(0.6 / dt))):
            r, v, F = integrate.vv_step(r, v, F, np.ones(len(q)), L, dt, force)
            worst = max(worst, abs(energy(r, v) - E0))
        dev.append(worst)
    ratio = dev[0] / dev[1]
    assert 2.5 < ratio < 6.0, ratio


def test_baoab_stationary_velocity_variance():
    """With zero force the O-step is an exact Ornstein-Uhlenbeck update: Var v -> kT/m."""
    N = 20000
    L = [100.0] * 3
    mass = np.full(N, 2.0)
    kT = 1.7
    r = np.zeros((N, 3))
    v = np.zeros((N, 3))
    F = np.zeros((N, 3))
    zero = lambda x: np.zeros_like(x)
    for step in range(60):
        r, v, F = integrate.baoab_step(r, v, F, mass, L, 0.05, 2.0, kT, seed=9, step=step, force_fn=zero)
    target = kT / 2.0 * (1 - math.exp(-2 * 2.0 * 0.05 * 60))
    assert abs(v.var() - target) < 0.03 * target
    assert abs(v.mean()) < 5 * math.sqrt(target / (3 * N))


def test_langevin_noise_is_standard_normal():
    z = integrate.langevin_noise(5, 17, np.arange(100000))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert abs(np.mean(z ** 4) - 3) < 0.1
