"""GPU dynamics through rbsog_step (CUDA-graph replay): velocity Verlet and BAOAB
trajectories against the oracle's integrators with the GPU's k-sets, determinism, and
energy behaviour."""
import numpy as np
import pytest

from gpu_common import FP32_TOL, FP64_TOL, Ctx, oracle_forces, oracle_sog, require_gpu, workload
from oracle import core, integrate
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def gpu_trajectory(w, prec, r0, v0, nsteps, q=None, m=None):
    """Positions, velocities and the k-set of every force evaluation, one step at a time."""
    ks, rs, vs, es = [], [], [], []
    with Ctx(w, prec, q=q, m=m) as c:
        R.rbsog_set_state(c.h, r0, v0)
        R.rbsog_forces(c.h)
        ks.append(R.rbsog_get_ksample(c.h, c.P)[0])
        for _ in range(nsteps):
            es.append(R.rbsog_step(c.h, 1, energy=True))
            ks.append(R.rbsog_get_ksample(c.h, c.P)[0])
            r = np.zeros((w.N, 3))
            v = np.zeros((w.N, 3))
            R.rbsog_get_state(c.h, r, v)
            rs.append(r)
            vs.append(v)
    return ks, rs, vs, es


def oracle_trajectory(w, r0, v0, ks, nsteps, q=None, m=None):
    q = W.charges(w) if q is None else q
    m = W.masses(w) if m is None else m
    sog = oracle_sog(w)
    S_ = core.S_sum(w.box, sog, w.kT, float(np.sum(q * q)))
    state = {"i": 0}

    def force(x):
        Ft, _, _, _, _ = oracle_forces(w, x, q, ks[state["i"]], sog=sog, S_=S_)
        state["i"] += 1
        return Ft

    r, v = integrate.wrap(r0, w.box), v0.copy()
    F = force(r)
    rs, vs = [], []
    for n in range(nsteps):
        if w.ensemble == "langevin":
            # the GPU keys step n's noise by the force evaluations before it: n + 1
            r, v, F = integrate.baoab_step(r, v, F, m, w.box, w.dt, w.langevin_gamma, w.kT, w.seed_k, n + 1, force)
        else:
            r, v, F = integrate.vv_step(r, v, F, m, w.box, w.dt, force)
        rs.append(r)
        vs.append(v)
    return rs, vs


def box_diff(a, b, L):
    d = a - b
    L = np.asarray(L)
    return d - L * np.round(d / L)


@pytest.mark.parametrize("ensemble", ["nve", "langevin"])
@pytest.mark.parametrize("prec", [R.RBSOG_FP64, R.RBSOG_FP32], ids=["fp64", "fp32"])
def test_trajectory_parity(prec, ensemble):
    w = workload(500, 8.0, kappa=1.0, Gamma=1.0, P=64, seed=41, dt=0.002, ensemble=ensemble)
    r0 = W.positions(w)
    v0 = W.velocities(w)
    n = 5
    ks, rg, vg, _ = gpu_trajectory(w, prec, r0, v0, n)
    ro, vo = oracle_trajectory(w, r0, v0, ks, n)
    tol = FP64_TOL if prec == R.RBSOG_FP64 else FP32_TOL
    for s in range(n):
        dr = box_diff(rg[s], ro[s], w.box)
        assert np.max(np.abs(dr)) <= tol * w.box[0], (s, np.max(np.abs(dr)))
        assert core.rel_l2(vg[s], vo[s]) <= tol, (s, core.rel_l2(vg[s], vo[s]))


@pytest.mark.parametrize("prec", [R.RBSOG_FP64, R.RBSOG_FP32], ids=["fp64", "fp32"])
def test_two_species_trajectory_parity(prec):
    """A two-species plasma (like the D-alpha mixture of Sec. 5: charges 1 and 2, masses 2
    and 4, half of each), BAOAB: the per-particle charges enter the forces and the
    adaptive measure through sum q^2, the masses the kick and the noise amplitude."""
    w = workload(600, 8.0, kappa=1.0, Gamma=1.0, P=64, seed=43, dt=0.002, ensemble="langevin")
    alpha = np.arange(w.N) % 2 == 1
    q = np.where(alpha, 2.0, 1.0)
    m = np.where(alpha, 4.0, 2.0)
    r0 = W.positions(w)
    v0 = W.velocities(w) / np.sqrt(m)[:, None]
    n = 5
    ks, rg, vg, _ = gpu_trajectory(w, prec, r0, v0, n, q=q, m=m)
    ro, vo = oracle_trajectory(w, r0, v0, ks, n, q=q, m=m)
    tol = FP64_TOL if prec == R.RBSOG_FP64 else FP32_TOL
    for s in range(n):
        dr = box_diff(rg[s], ro[s], w.box)
        assert np.max(np.abs(dr)) <= tol * w.box[0], (s, np.max(np.abs(dr)))
        assert core.rel_l2(vg[s], vo[s]) <= tol, (s, core.rel_l2(vg[s], vo[s]))


def test_graph_replay_is_deterministic():
    w = workload(800, 9.0, P=48, seed=3)
    outs = []
    for _ in range(2):
        with Ctx(w, R.RBSOG_FP32) as c:
            R.rbsog_set_state(c.h, W.positions(w), W.velocities(w))
            e = R.rbsog_step(c.h, 7, energy=True)
            r = np.zeros((w.N, 3))
            step = R.rbsog_get_state(c.h, r)
            outs.append((r, e["total"], step))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    assert outs[0][2] == 7


@pytest.mark.parametrize("ensemble", ["nve", "langevin"])
@pytest.mark.parametrize("prec", [R.RBSOG_FP64, R.RBSOG_FP32], ids=["fp64", "fp32"])
def test_host_round_trip_with_forces_follows_the_device_trajectory(prec, ensemble):
    """Reading r, v and F back after every step and uploading them with
    rbsog_set_state_forces gives the device-resident trajectory bit for bit: one force
    evaluation per step, the same draws, and forces that do not depend on the particle
    layout the upload resets."""
    w = workload(700, 8.5, kappa=1.0, Gamma=1.0, P=48, seed=47, dt=0.002, ensemble=ensemble)
    r0, v0 = W.positions(w), W.velocities(w)
    n = 4
    dev = []
    with Ctx(w, prec) as c:
        R.rbsog_set_state(c.h, r0, v0)
        for _ in range(n):
            R.rbsog_step(c.h, 1)
            r, v = np.zeros((w.N, 3)), np.zeros((w.N, 3))
            R.rbsog_get_state(c.h, r, v)
            dev.append((r, v))
    with Ctx(w, prec) as c:
        R.rbsog_set_state(c.h, r0, v0)
        F = np.zeros((w.N, 3))
        with pytest.raises(R.RbsogError):
            R.rbsog_get_forces(c.h, F)              # no forces at an uploaded state yet
        R.rbsog_forces(c.h)
        R.rbsog_get_forces(c.h, F)
        r, v = r0.copy(), v0.copy()
        for s in range(n):
            R.rbsog_set_state_forces(c.h, r, v, F)
            R.rbsog_step(c.h, 1)
            R.rbsog_get_state(c.h, r, v)
            R.rbsog_get_forces(c.h, F)
            assert np.array_equal(r, dev[s][0]), s
            assert np.array_equal(v, dev[s][1]), s


@pytest.mark.parametrize("ensemble", ["nve", "langevin"])
def test_fp32_forces_round_trip_follows_the_device_trajectory(ensemble):
    """The FP32 build's forces are FP32 values: rbsog_get_forces_f32 returns exactly what
    rbsog_get_forces does, and a host loop that moves F as FP32 follows the
    device-resident trajectory bit for bit."""
    w = workload(700, 8.5, kappa=1.0, Gamma=1.0, P=48, seed=53, dt=0.002, ensemble=ensemble)
    r0, v0 = W.positions(w), W.velocities(w)
    n = 4
    dev = []
    with Ctx(w, R.RBSOG_FP32) as c:
        R.rbsog_set_state(c.h, r0, v0)
        for _ in range(n):
            R.rbsog_step(c.h, 1)
            r, v = np.zeros((w.N, 3)), np.zeros((w.N, 3))
            R.rbsog_get_state(c.h, r, v)
            dev.append((r, v))
    with Ctx(w, R.RBSOG_FP32) as c:
        R.rbsog_set_state(c.h, r0, v0)
        F = np.zeros((w.N, 3), dtype=np.float32)
        with pytest.raises(R.RbsogError):
            R.rbsog_get_forces_f32(c.h, F)          # no forces at an uploaded state yet
        R.rbsog_forces(c.h)
        R.rbsog_get_forces_f32(c.h, F)
        F64 = np.zeros((w.N, 3))
        R.rbsog_get_forces(c.h, F64)
        assert np.array_equal(F.astype(np.float64), F64)
        r, v = r0.copy(), v0.copy()
        for s in range(n):
            R.rbsog_set_state_forces_f32(c.h, r, v, F)
            R.rbsog_step(c.h, 1)
            R.rbsog_get_state(c.h, r, v)
            R.rbsog_get_forces_f32(c.h, F)
            assert np.array_equal(r, dev[s][0]), s
            assert np.array_equal(v, dev[s][1]), s


def test_fp32_force_calls_refuse_the_fp64_build():
    w = workload(300, 6.5, P=16, seed=55)
    F = np.zeros((w.N, 3), dtype=np.float32)
    with Ctx(w, R.RBSOG_FP64) as c:
        R.rbsog_set_state(c.h, W.positions(w), W.velocities(w))
        R.rbsog_forces(c.h)
        for call in (lambda: R.rbsog_get_forces_f32(c.h, F),
                     lambda: R.rbsog_set_state_forces_f32(c.h, W.positions(w), W.velocities(w), F)):
            with pytest.raises(R.RbsogError, match="EINVAL"):
                call()


@pytest.mark.parametrize("prec", [R.RBSOG_FP64, R.RBSOG_FP32], ids=["fp64", "fp32"])
def test_get_forces_returns_the_last_evaluation(prec):
    """rbsog_get_forces gives, in the caller's order, the forces that rbsog_forces returned."""
    w = workload(600, 8.0, P=32, seed=51)
    with Ctx(w, prec) as c:
        R.rbsog_set_state(c.h, W.positions(w), W.velocities(w))
        F = np.zeros((w.N, 3))
        R.rbsog_forces(c.h, F)
        G = np.zeros((w.N, 3))
        R.rbsog_get_forces(c.h, G)
        assert np.array_equal(F, G)


def test_set_state_forces_without_forces_is_set_state():
    w = workload(500, 8.0, P=32, seed=49)
    outs = []
    for with_forces in (False, True):
        with Ctx(w, R.RBSOG_FP32) as c:
            if with_forces:
                R.rbsog_set_state_forces(c.h, W.positions(w), W.velocities(w), None)
            else:
                R.rbsog_set_state(c.h, W.positions(w), W.velocities(w))
            R.rbsog_step(c.h, 2)
            r = np.zeros((w.N, 3))
            R.rbsog_get_state(c.h, r)
            outs.append(r)
    assert np.array_equal(outs[0], outs[1])


def test_energy_components_after_steps_match_oracle():
    """After steps, the GPU energies at the final state equal the oracle's on the GPU's k-set."""
    w = W.cfg_small_fp64()
    with Ctx(w, R.RBSOG_FP64) as c:
        R.rbsog_set_state(c.h, W.positions(w), W.velocities(w))
        e = R.rbsog_step(c.h, 3, energy=True)
        m, _ = R.rbsog_get_ksample(c.h, c.P)
        r = np.zeros((w.N, 3))
        v = np.zeros((w.N, 3))
        R.rbsog_get_state(c.h, r, v)
    Ft, Fn, Ff, eo, _ = oracle_forces(w, r, W.charges(w), m)
    assert abs(e["U_near"] - eo["U_N"]) <= 1e-11 * abs(eo["U_N"])
    assert abs(e["U_far"] - eo["U_F"]) <= 1e-11 * abs(eo["U_F"])
    assert abs(e["kinetic"] - integrate.kinetic(v, W.masses(w))) <= 1e-12 * e["kinetic"]
    assert e["step"] == 3


def test_each_upload_draws_fresh_langevin_noise():
    """A host loop that uploads the state before every step (set_state, step, get_state)
    must not reuse the Langevin noise: the same state uploaded twice and stepped once
    gives velocities that differ by about sqrt(2) times the noise amplitude c2 sigma,
    far more than the random far force makes them differ."""
    w = workload(500, 8.0, kappa=1.0, Gamma=1.0, P=64, seed=47, dt=0.002, ensemble="langevin")
    r0, v0 = W.positions(w), W.velocities(w)
    vs = []
    with Ctx(w, R.RBSOG_FP32) as c:
        for _ in range(2):
            R.rbsog_set_state(c.h, r0, v0)
            R.rbsog_step(c.h, 1)
            v = np.zeros((w.N, 3))
            R.rbsog_get_state(c.h, None, v)
            vs.append(v)
    c1 = np.exp(-w.langevin_gamma * w.dt)
    c2 = np.sqrt((1.0 - c1 * c1) * w.kT)          # unit masses
    rms = float(np.sqrt(np.mean((vs[0] - vs[1]) ** 2)))
    assert 0.8 * np.sqrt(2.0) * c2 <= rms <= 1.2 * np.sqrt(2.0) * c2, (rms, c2)
