"""Time integration for the oracle: velocity Verlet (NVE) and BAOAB Langevin, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Algorithm 2 integrates Newton's equations after each force evaluation; the paper
names velocity Verlet for NVE runs (Sec. 5.1) and cites Langevin dynamics for the
convergence theory (Sec. 4.4) without giving a scheme.  Readings used here:
  NVE:      v <- v + F dt/(2m);  r <- wrap(r + v dt);  F <- force(r);  v <- v + F dt/(2m)
  Langevin: BAOAB (Leimkuhler & Matthews 2013) with c1 = exp(-gamma dt):
            B: v += F dt/(2m);  A: r += v dt/2;  O: v = c1 v + sqrt((1-c1^2) kT/m) xi;
            A: r += v dt/2;  wrap;  F <- force(r);  B: v += F dt/(2m)
  xi: standard normals from Philox4x32-10, key = seed, counter = (particle id,
  0x40000000 + j, step lo, step hi); j = 0 gives (xi_x, xi_y) by Box-Muller of its
  four words, j = 1 gives xi_z (cosine branch).
  wrap(r) = r - L floor(r (1/L)), then + L if negative, then - L if >= L.
With the instantaneous temperature of Sec. 4.3 (NVT), the force evaluation also takes the
velocities it sees (after B A O A, or after the half kick of velocity Verlet), whose
kinetic temperature 2K/(3N) enters calF of Eq. (62).
"""
from __future__ import annotations

import math

import numpy as np

from . import philox


def wrap(r, L):
    L = np.asarray(L, dtype=np.float64)
    w = r - L * np.floor(r * (1.0 / L))
    w = np.where(w < 0.0, w + L, w)
    return np.where(w >= L, w - L, w)


def langevin_noise(seed: int, step: int, ids) -> np.ndarray:
    ids = np.asarray(ids, dtype=np.uint64)
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
    s0 = np.uint64(step & 0xFFFFFFFF)
    s1 = np.uint64((step >> 32) & 0xFFFFFFFF)
    a = philox.philox4x32_10(ids, np.uint64(0x40000000), s0, s1, k0, k1)
    b = philox.philox4x32_10(ids, np.uint64(0x40000001), s0, s1, k0, k1)
    x, y = philox.normal_pair(*a)
    z, _ = philox.normal_pair(*b)
    return np.stack([x, y, z], axis=1)


def vv_step(r, v, F, mass, L, dt, force_fn, with_v=False):
    """One velocity-Verlet step; force_fn(r) -> F, or force_fn(r, v) with the half-kicked
    velocities when with_v.  Returns (r, v, F)."""
    hm = (0.5 * dt / np.asarray(mass, dtype=np.float64))[:, None]
    v = v + hm * F
    r = wrap(r + dt * v, L)
    F = force_fn(r, v) if with_v else force_fn(r)
    v = v + hm * F
    return r, v, F


def kinetic_temperature(v, mass) -> float:
    """Instantaneous k_B T = 2 K / (3 N) (three degrees of freedom per particle)."""
    return 2.0 * kinetic(v, mass) / (3.0 * np.asarray(v).shape[0])


def baoab_step(r, v, F, mass, L, dt, gamma, kT, seed, step, force_fn, ids=None, with_v=False):
    mass = np.asarray(mass, dtype=np.float64)
    ids = np.arange(r.shape[0]) if ids is None else ids
    hm = (0.5 * dt / mass)[:, None]
    c1 = math.exp(-gamma * dt)
    c2 = np.sqrt((1.0 - c1 * c1) * kT / mass)[:, None]
    v = v + hm * F
    r = r + (0.5 * dt) * v
    v = c1 * v + c2 * langevin_noise(seed, step, ids)
    r = wrap(r + (0.5 * dt) * v, L)
    F = force_fn(r, v) if with_v else force_fn(r)
    v = v + hm * F
    return r, v, F


def kinetic(v, mass) -> float:
    return 0.5 * float(np.sum(np.asarray(mass)[:, None] * v * v))
