"""Strong-coupling OCP in the FP32 build (37^3 bcc, N = 101,306, Gamma = 100, kappa = 0.5,
r_c = 4a, P = 200, dt = 0.005): 1000 NVE steps through the CUDA graph.  Every 100 steps
the total force of the current state on 256 sampled particles is checked against the
FP64 oracle on the same k-set (a second context evaluates it, so the trajectory is not
touched), and the total energy is tracked; the same run with ten times the modes shows
that the energy change comes from the random-batch variance, and the FP64 build's run
from the same seed (the same k-draws) shows the same change, so the FP32 arithmetic adds
no drift of its own.  The figures are printed."""
import json

import numpy as np
import pytest

from gpu_common import FP32_TOL, Ctx, force_errors, modes_for, oracle_forces, require_gpu
from oracle import core
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def run_nve(w, P, nsteps, checks=None, precision=R.RBSOG_FP32):
    """Energies every 100 steps of an NVE run with P modes; with `checks`, the force
    error of each checkpoint state against the oracle."""
    q = W.charges(w)
    rng = np.random.default_rng(5)
    errs, energies = [], []
    S_ = None
    with Ctx(w, precision, P=P) as run, Ctx(w, R.RBSOG_FP32) as probe:
        R.rbsog_set_state(run.h, W.positions(w), W.velocities(w))
        for block in range(nsteps // 100):
            e = R.rbsog_step(run.h, 100, energy=True)
            energies.append(e["total"])
            if checks:
                r = np.zeros((w.N, 3))
                R.rbsog_get_state(run.h, r)
                modes = modes_for(w, w.P, 1000 + block)
                R.rbsog_set_state(probe.h, r)
                R.rbsog_set_ksample(probe.h, modes)
                F = np.zeros((w.N, 3))
                R.rbsog_forces(probe.h, F)
                idx = rng.choice(w.N, checks, replace=False)
                Ft, _, _, _, S_ = oracle_forces(w, r, q, modes, idx=idx, S_=S_)
                errs.append(max(force_errors(F[idx], Ft)))
        kin = e["kinetic"]
    return np.asarray(energies), errs, kin


@pytest.fixture(scope="module")
def fp32_run():
    w = W.cfg_bcc_fp32()
    return w, run_nve(w, w.P, 1000, checks=256)


def test_strong_coupling_force_error_and_energy_drift(fp32_run):
    w, (E, errs, kin) = fp32_run
    K0 = 1.5 * w.N * w.kT
    # the random-batch force is unbiased with variance ~ 1/P; plain velocity Verlet turns
    # that variance into a slow heating, so the same run with 10x the modes heats less
    E10, _, kin10 = run_nve(w, 10 * w.P, 1000)
    dE, dE10 = float(E[-1] - E[0]), float(E10[-1] - E10[0])
    print(json.dumps({"workload": w.name, "steps": 1000, "P": w.P, "force_rel_l2_every_100": errs,
                      "energy_total_every_100": E.tolist(), "energy_change_100_to_1000": dE,
                      "rel_energy_change": dE / abs(E[0]), "kinetic_initial_expected": K0,
                      "kinetic_end": kin, "P10x": {"energy_change_100_to_1000": dE10, "kinetic_end": kin10}}))
    assert max(errs) <= FP32_TOL
    assert np.all(np.isfinite(E)) and np.all(np.isfinite(E10))
    assert abs(dE) <= 1e-2 * abs(E[0])
    assert abs(dE10) <= 0.5 * abs(dE)


def test_strong_coupling_fp32_drift_tracks_the_fp64_build(fp32_run):
    """The FP64 build, whose forces match the FP64 oracle to 1e-12, run from the same state
    and seed: its energy change over steps 100-1000 and the FP32 build's agree within a
    factor of 2 (both come from the random-batch variance, not from rounding)."""
    w, (E, _, _) = fp32_run
    E64, _, _ = run_nve(w, w.P, 1000, precision=R.RBSOG_FP64)
    dE, dE64 = float(E[-1] - E[0]), float(E64[-1] - E64[0])
    print(json.dumps({"workload": w.name, "energy_change_fp32": dE, "energy_change_fp64": dE64,
                      "energy_total_every_100_fp64": E64.tolist()}))
    assert np.all(np.isfinite(E64))
    assert 0.5 * abs(dE64) <= abs(dE) <= 2.0 * abs(dE64), (dE, dE64)
