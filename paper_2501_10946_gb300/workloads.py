"""Seeded synthetic inputs for Yukawa one-component-plasma (YOCP) runs.

This module produces inputs only: particle positions, velocities, charges and
masses, and the physical parameters of a run in absolute units.  It contains
none of the force-field arithmetic (no kernel, no sum-of-Gaussians, no
sampling measure), so both the CUDA path and the CPU oracle can draw their
inputs from it without sharing any of the method.

Reduced OCP units (Sec. 5.1 of the paper defines Gamma~ = Q^2/(a k_B T) and
kappa = a/lambda): every particle has charge Q = 1 and mass 1, a is the
Wigner-Seitz radius a = (3/(4 pi n))^(1/3) with n = N/V, and lengths given
"in units of a" are multiplied by a here.  The paper prints a = (4 pi n)^(-1/3),
which lacks the factor 3 of the Wigner-Seitz radius; the Wigner-Seitz radius is
used here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One YOCP run in absolute units (box lengths, a, r_c are absolute)."""

    name: str
    N: int
    box: tuple          # (L_x, L_y, L_z)
    a_ws: float         # Wigner-Seitz radius
    kappa: float        # a / lambda
    Gamma: float        # bare coupling Q^2 / (a k_B T)
    r_c: float          # near-field cutoff (absolute)
    sog_eps: float      # SOG tolerance on [r_c, 33 lambda]
    P: int              # random-batch size
    dt: float
    steps: int
    ensemble: str       # "nve" or "langevin"
    langevin_gamma: float
    placement: str      # "uniform" or "bcc"
    seed_pos: int
    seed_vel: int
    seed_k: int
    bcc_cells: int = 0
    bcc_sigma: float = 0.0   # displacement std in units of a
    min_sep: float = 0.0     # uniform placement: minimum pair separation in units of a (0: none)

    @property
    def volume(self) -> float:
        return float(self.box[0] * self.box[1] * self.box[2])

    @property
    def kT(self) -> float:
        """k_B T implied by Gamma~ = Q^2/(a k_B T) with Q = 1 (input parameter)."""
        return 1.0 / (self.a_ws * self.Gamma)


def wigner_seitz(N: int, volume: float) -> float:
    return (3.0 * volume / (4.0 * math.pi * N)) ** (1.0 / 3.0)


def box_for_unit_a(N: int) -> float:
    """Cubic box side for N particles when lengths are measured in a (n = 3/(4 pi))."""
    return (4.0 * math.pi * N / 3.0) ** (1.0 / 3.0)


def cfg_small_fp64() -> Workload:
    """N=1000 at reduced density 1 (L=10), Gamma=1, kappa=1, r_c=3.5a, P=100, dt=0.01, 10 NVE steps."""
    N, L = 1000, 10.0
    a = wigner_seitz(N, L ** 3)
    return Workload("yocp_n1000_fp64", N, (L, L, L), a, 1.0, 1.0, 3.5 * a, 1e-6, 100, 0.01, 10,
                    "nve", 1.0, "uniform", 101, 102, 103)


def cfg_bcc_fp32() -> Workload:
    """bcc 37^3 (N=101306), sigma=0.05a, Gamma=100, kappa=0.5, r_c=4a, P=200, dt=0.005, 1000 NVE steps."""
    nc = 37
    N = 2 * nc ** 3
    L = box_for_unit_a(N)
    return Workload("yocp_bcc_n101306_fp32", N, (L, L, L), 1.0, 0.5, 100.0, 4.0, 1e-6, 200, 0.005, 1000,
                    "nve", 1.0, "bcc", 201, 202, 203, bcc_cells=nc, bcc_sigma=0.05)


def cfg_large(N: int = 1_000_000) -> Workload:
    """Weak coupling at scale: N=1e6 uniform, Gamma=0.1, kappa=2, r_c=3a, P=500, dt=0.01, 200 Langevin steps."""
    L = box_for_unit_a(N)
    return Workload(f"yocp_uniform_n{N}", N, (L, L, L), 1.0, 2.0, 0.1, 3.0, 1e-6, 500, 0.01, 200,
                    "langevin", 1.0, "uniform", 301, 302, 303)


def scaled(w: Workload, N: int, name: str | None = None) -> Workload:
    """Same physical state point with a different N (box rescaled to keep n)."""
    L = w.box[0] * (N / w.N) ** (1.0 / 3.0)
    return dataclasses.replace(w, name=name or f"{w.name}_N{N}", N=N, box=(L, L, L),
                               bcc_cells=0, placement="uniform" if w.placement == "bcc" else w.placement)


def positions(w: Workload) -> np.ndarray:
    """Particle positions [N,3] float64 in [0, L)."""
    rng = np.random.Generator(np.random.PCG64(w.seed_pos))
    L = np.asarray(w.box, dtype=np.float64)
    if w.placement == "uniform":
        r = rng.uniform(0.0, 1.0, size=(w.N, 3)) * L
        if w.min_sep > 0.0:
            r = _separate(r, L, w.min_sep * w.a_ws, rng)
        return r
    if w.placement == "bcc":
        nc = w.bcc_cells
        g = np.arange(nc, dtype=np.float64)
        cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
        base = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
        lat = np.concatenate([base, base + 0.5], axis=0) * (L / nc)
        lat = lat + rng.normal(0.0, w.bcc_sigma * w.a_ws, size=lat.shape)
        return np.mod(lat, L)
    raise ValueError(w.placement)


def _separate(r: np.ndarray, L: np.ndarray, dmin: float, rng) -> np.ndarray:
    """Uniform positions with no pair (minimum image) closer than dmin: every pair closer
    than dmin gives up its higher-indexed particle, which is drawn again uniformly, until
    no such pair is left.  At the densities used here (hard-sphere packing fraction below
    2%) a few rounds suffice."""
    from scipy.spatial import cKDTree
    r = np.mod(r, L)
    pairs = cKDTree(r, boxsize=L).query_pairs(dmin, output_type="ndarray")
    for _ in range(200):
        if len(pairs) == 0:
            return r
        redo = np.unique(np.max(pairs, axis=1))
        r[redo] = np.mod(rng.uniform(0.0, 1.0, size=(len(redo), 3)) * L, L)
        # only pairs with a redrawn particle can be new
        near = cKDTree(r, boxsize=L).query_ball_point(r[redo], dmin)
        pairs = np.asarray([(min(i, j), max(i, j)) for i, js in zip(redo.tolist(), near) for j in js if j != i],
                           dtype=np.int64).reshape(-1, 2)
    raise RuntimeError("minimum-separation placement did not converge")


def velocities(w: Workload) -> np.ndarray:
    """Maxwell-Boltzmann velocities at k_B T (mass 1), centre-of-mass velocity removed."""
    rng = np.random.Generator(np.random.PCG64(w.seed_vel))
    v = rng.normal(0.0, math.sqrt(w.kT), size=(w.N, 3))
    return v - v.mean(axis=0, keepdims=True)


def charges(w: Workload) -> np.ndarray:
    return np.ones(w.N, dtype=np.float64)


def masses(w: Workload) -> np.ndarray:
    return np.ones(w.N, dtype=np.float64)


def random_modes(P: int, nmax: int, seed: int) -> np.ndarray:
    """A seeded set of P nonzero integer mode triples with |m_a| <= nmax (for parity tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < P:
        m = rng.integers(-nmax, nmax + 1, size=3)
        if np.any(m != 0):
            out.append(m)
    return np.asarray(out, dtype=np.int32)


def small_system(N: int, L: float, seed: int, charge_mix: bool = False):
    """Tiny random system for pins: positions [N,3], charges [N] (+-1 mix if requested)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(0.0, L, size=(N, 3))
    q = np.ones(N) if not charge_mix else rng.choice([-1.0, 1.0], size=N)
    return r, q


def cfg_replicas(R: int = 256, seed: int = 401, steps: int = 500) -> list:
    """Batched replica sweep: R independent YOCP systems at reduced density 1 (lengths in a),
    N log-uniform in [500, 5e4], kappa uniform in [0.1, 3], Gamma log-uniform in [0.1, 200],
    P in {64, 128, 256}, r_c = 3a, SOG tolerance 1e-6, dt = 0.01, NVE, FP32 forces; uniform
    positions with a minimum separation of 0.5a."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(R):
        N = int(round(math.exp(rng.uniform(math.log(500.0), math.log(5e4)))))
        kappa = float(rng.uniform(0.1, 3.0))
        Gamma = float(math.exp(rng.uniform(math.log(0.1), math.log(200.0))))
        P = int(rng.choice([64, 128, 256]))
        L = box_for_unit_a(N)
        s = seed * 1000 + 4 * i
        out.append(Workload(f"replica{i}_n{N}", N, (L, L, L), 1.0, kappa, Gamma, 3.0, 1e-6, P, 0.01, steps,
                            "nve", 1.0, "uniform", s + 1, s + 2, s + 3, min_sep=0.5))
    return out


def cfg_stream(n_jobs: int = 64, rate: float = 50.0, seed: int = 501) -> list:
    """Served request stream: n_jobs YOCP jobs with Poisson arrivals (mean `rate` per s),
    N log-uniform in [1e3, 2e5], kappa uniform in [0.2, 3], Gamma log-uniform in
    [0.5, 150], steps uniform in [100, 2000], P = 128, r_c = 3a, reduced density 1, NVE,
    FP32 forces, uniform positions with a minimum separation of 0.5a.  Returns
    [(Workload, nsteps, t_arrival_s)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    t = 0.0
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        N = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
        kappa = float(rng.uniform(0.2, 3.0))
        Gamma = float(math.exp(rng.uniform(math.log(0.5), math.log(150.0))))
        nsteps = int(rng.integers(100, 2001))
        P = 128
        L = box_for_unit_a(N)
        s = seed * 1000 + 4 * i
        w = Workload(f"job{i}_n{N}", N, (L, L, L), 1.0, kappa, Gamma, 3.0, 1e-6, P, 0.01, nsteps, "nve", 1.0,
                     "uniform", s + 1, s + 2, s + 3, min_sep=0.5)
        out.append((w, nsteps, t))
    return out


def job_inputs(w: Workload) -> tuple:
    """(charges, masses, positions, velocities) of one workload: the inputs a job submits."""
    return charges(w), masses(w), positions(w), velocities(w)

