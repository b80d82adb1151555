"""The persistent form of the batched step (rbsog_batch_set_persistent): one cooperative
launch per step over every system, replayed from a CUDA graph.  Against the graph of
batched kernels it gives the same forces and trajectories bit for bit (the same per-block
arithmetic, with the near-field tiles and structure-factor blocks taken from work lists);
against the FP64 oracle it holds the FP32 tolerance; and a grid-barrier wait that runs out
(a wait limit of one poll) ends the call with RBSOG_ETIMEOUT instead of hanging, after
which the batch recovers."""
import numpy as np
import pytest

from gpu_common import FP32_TOL, check_energy, check_forces, modes_for, oracle_forces, require_gpu
from oracle import core
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W
from test_gpu_batch import Batch, state, systems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def run(ws, persistent, nsteps, r, v):
    with Batch(ws) as b:
        if persistent:
            R.rbsog_batch_set_persistent(b.h, True)
        R.rbsog_batch_set_state(b.h, r, v)
        e = R.rbsog_batch_step(b.h, b.R, nsteps, energy=True)
        rb = np.zeros((b.Ntot, 3))
        vb = np.zeros((b.Ntot, 3))
        step = R.rbsog_batch_get_state(b.h, rb, vb)
        m, coef = R.rbsog_batch_get_ksample(b.h, b.Ptot)
    return rb, vb, e, step, m, coef


def test_persistent_steps_equal_the_graph_form():
    ws = systems()
    r, v = state(ws)
    rg, vg, eg, sg, mg, cg = run(ws, False, 6, r, v)
    rp, vp, ep, sp, mp, cp = run(ws, True, 6, r, v)
    assert sg == sp == 6
    assert np.array_equal(mg, mp) and np.array_equal(cg, cp)
    assert np.array_equal(rg, rp)
    assert np.array_equal(vg, vp)
    for a, b in zip(eg, ep):
        for k in ("U_far", "U_self", "kinetic"):
            assert a[k] == b[k], k
        assert abs(a["U_near"] - b["U_near"]) <= 1e-12 * abs(a["U_near"])


def test_persistent_forces_match_the_oracle():
    ws = systems()
    r, _ = state(ws)
    modes = [modes_for(w, w.P, 500 + i) for i, w in enumerate(ws)]
    with Batch(ws) as b:
        R.rbsog_batch_set_persistent(b.h, True)
        R.rbsog_batch_set_state(b.h, r)
        R.rbsog_batch_set_ksample(b.h, np.concatenate(modes))
        F = np.zeros((b.Ntot, 3))
        e = R.rbsog_batch_forces(b.h, b.R, F, energy=True)
        split_F, split_r = b.split(F), b.split(r)
    for i, w in enumerate(ws):
        Ft, _, _, eo, _ = oracle_forces(w, split_r[i], W.charges(w), modes[i])
        check_forces(split_F[i], Ft, FP32_TOL, ("system", i))
        check_energy(e[i]["U_near"], eo["U_N"], FP32_TOL, ("U_near", i))
        check_energy(e[i]["U_far"], eo["U_F"], FP32_TOL, ("U_far", i))


def test_switching_forms_mid_run_keeps_the_trajectory():
    ws = systems()
    r, v = state(ws)
    rg, vg, _, _, _, _ = run(ws, False, 4, r, v)
    with Batch(ws) as b:
        R.rbsog_batch_set_state(b.h, r, v)
        R.rbsog_batch_step(b.h, b.R, 2)
        R.rbsog_batch_set_persistent(b.h, True)
        with pytest.raises(R.RbsogError, match="EINVAL"):
            R.rbsog_batch_step(b.h, b.R, 0, energy=True)   # partials of the other form
        R.rbsog_batch_step(b.h, b.R, 2)
        rb = np.zeros((b.Ntot, 3))
        vb = np.zeros((b.Ntot, 3))
        R.rbsog_batch_get_state(b.h, rb, vb)
    assert np.array_equal(rg, rb) and np.array_equal(vg, vb)


def test_a_barrier_wait_that_runs_out_returns_etimeout():
    """One poll per barrier wait: CTAs that arrive before the last give up at once, set the
    status and return; the call reports RBSOG_ETIMEOUT.  With the default limit again the
    batch steps normally."""
    ws = systems()
    r, v = state(ws)
    with Batch(ws) as b:
        R.rbsog_batch_set_persistent(b.h, True)
        R.rbsog_batch_set_state(b.h, r, v)
        R.rbsog_batch_set_wait_limit(b.h, 1)
        R.rbsog_batch_step(b.h, b.R, 1)
        with pytest.raises(R.RbsogError, match="ETIMEOUT"):
            R.rbsog_batch_get_state(b.h, np.zeros((b.Ntot, 3)))
        R.rbsog_batch_set_wait_limit(b.h, 20_000_000)
        R.rbsog_batch_set_state(b.h, r, v)
        R.rbsog_batch_step(b.h, b.R, 2)
        rb = np.zeros((b.Ntot, 3))
        assert R.rbsog_batch_get_state(b.h, rb) == 2
    rg, _, _, _, _, _ = run(ws, False, 2, r, v)
    assert np.array_equal(rb, rg)
