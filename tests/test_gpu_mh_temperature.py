"""GPU sampling variants of Sec. 4.3 through the C ABI:
  * the Metropolis-Hastings chains (RBSOG_SAMPLER_MH): the GPU's chain states replay the
    oracle's chains (oracle.sampler.MHChains) bit for bit from the same seed, their
    coefficients match the oracle's, and independent chains after burn-in pass a
    chi-square test against P(k) of Eq. (59);
  * the instantaneous temperature (RBSOG_KT_INSTANT): k_B T = 2K/(3N) of the velocities
    at the evaluation, S of Eq. (59) re-summed at it against the oracle's lattice sum, the
    draws and coefficients at that temperature, and a BAOAB trajectory against the oracle's
    integrator with calF at the instantaneous temperature of each evaluation."""
import math

import numpy as np
import pytest

from gpu_common import FP32_TOL, FP64_TOL, Ctx, oracle_sog, require_gpu, workload
from oracle import core, integrate
from oracle.sampler import MHChains, ModeSampler
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


MEASURES = [pytest.param(0, id="adaptive"), pytest.param(3, id="debye"), pytest.param(2, id="k2")]


@pytest.mark.parametrize("kind", MEASURES)
@pytest.mark.parametrize("Gamma", [1.0, 100.0])
def test_gpu_chains_replay_the_oracle_chains(kind, Gamma):
    w = workload(400, 9.0, kappa=0.7, Gamma=Gamma, P=256, seed=31)
    q = W.charges(w)
    Q2 = float(np.sum(q * q))
    sog = oracle_sog(w)
    ms = ModeSampler(sog, w.box, w.kT, Q2, kind=kind)
    chains = MHChains(ms, w.P, sweeps=2, burnin=16)
    S_ = core.S_sum(w.box, sog, w.kT, Q2, kind=kind)
    with Ctx(w, R.RBSOG_FP32, sampling=kind, sampler=R.RBSOG_SAMPLER_MH, mh_sweeps=2, mh_burnin=16) as c:
        R.rbsog_set_state(c.h, W.positions(w))
        for d in range(4):
            R.rbsog_forces(c.h)
            m_gpu, coef = R.rbsog_get_ksample(c.h, c.P)
            m_or = chains.draw(w.seed_k)
            assert np.array_equal(m_gpu, m_or), f"evaluation {d}"
            ref = core.rb_coef(m_or, w.box, sog, w.kT, Q2, S_, kind=kind)
            assert np.max(np.abs(coef - ref) / ref) <= 1e-11
    if kind != 2:
        assert chains.accepted < chains.proposed          # the chains do reject here


@pytest.mark.parametrize("kind", [pytest.param(0, id="adaptive"), pytest.param(3, id="debye")])
def test_gpu_chain_states_follow_P(kind):
    """4096 chains after burn-in, five evaluations ten proposals apart: chi-square of the
    20480 states against the exact P(k)."""
    w = workload(2, 6.0, kappa=1.0, Gamma=20.0, rc=2.5, P=4096, seed=77)
    q = W.charges(w)
    ms = ModeSampler(oracle_sog(w), w.box, w.kT, float(np.sum(q * q)), kind=kind)
    modes = ms.all_modes()
    k2 = ms.k2_of(modes)
    p = ms.calF(k2) * ms.fhat(k2)
    p = p / p.sum()
    index = {tuple(x): j for j, x in enumerate(modes)}
    counts = np.zeros(len(modes))
    with Ctx(w, R.RBSOG_FP32, sampling=kind, sampler=R.RBSOG_SAMPLER_MH, mh_sweeps=10, mh_burnin=64) as c:
        R.rbsog_set_state(c.h, W.positions(w))
        for _ in range(5):
            R.rbsog_forces(c.h)
            m, _ = R.rbsog_get_ksample(c.h, c.P)
            counts += np.bincount([index[tuple(x)] for x in m], minlength=len(modes))
    n = counts.sum()
    order = np.argsort(-p)
    top = order[:200]
    e = np.append(p[top], p[order[200:]].sum()) * n
    o = np.append(counts[top], counts[order[200:]].sum())
    keep = e > 5
    chi2 = float(np.sum((o[keep] - e[keep]) ** 2 / e[keep]))
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def test_mh_sampler_is_refused_where_it_is_not_built():
    w = workload(400, 9.0, P=64, seed=3)
    with pytest.raises(R.RbsogError, match="EUNSUPPORTED"):
        Ctx(w, R.RBSOG_FP32, sampler=R.RBSOG_SAMPLER_MH, egs_nu=0.5)
    p = R.make_params(w, precision=R.RBSOG_FP32, sampler=R.RBSOG_SAMPLER_MH)
    with pytest.raises(R.RbsogError, match="EUNSUPPORTED"):
        R.rbsog_batch_init([p], [w.N], W.charges(w), W.masses(w))


@pytest.mark.parametrize("prec,tol", [(R.RBSOG_FP64, FP64_TOL), (R.RBSOG_FP32, FP32_TOL)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("scale", [0.5, 1.0, 3.0])
def test_instantaneous_temperature_draws_and_coefficients(prec, tol, scale):
    w = workload(800, 9.0, kappa=1.0, Gamma=5.0, P=128, seed=61)
    r, q, m = W.positions(w), W.charges(w), W.masses(w)
    v = W.velocities(w) * scale
    Q2 = float(np.sum(q * q))
    sog = oracle_sog(w)
    with Ctx(w, prec, temperature=R.RBSOG_KT_INSTANT) as c:
        kT0, S0 = R.rbsog_get_temperature(c.h)
        assert kT0 == pytest.approx(w.kT, rel=1e-15)
        R.rbsog_set_state(c.h, r, v)
        F = np.zeros((w.N, 3))
        e = R.rbsog_forces(c.h, F, energy=True)
        kT_g, S_g = R.rbsog_get_temperature(c.h)
        m_g, coef = R.rbsog_get_ksample(c.h, c.P)
    kT_o = integrate.kinetic_temperature(v, m)
    assert abs(kT_g - kT_o) <= 1e-12 * kT_o
    S_o = core.S_sum(w.box, sog, kT_o, Q2)
    assert abs(S_g - S_o) <= 1e-11 * S_o
    m_o, _ = ModeSampler(sog, w.box, kT_o, Q2).draw(w.seed_k, 0, w.P)
    assert np.array_equal(m_g, m_o)
    ref = core.rb_coef(m_o, w.box, sog, kT_o, Q2, S_o)
    assert np.max(np.abs(coef - ref) / ref) <= 1e-11
    Ft, _, _, eo = core.rb_forces(r, q, w.box, w.r_c, sog, m_o, kT_o, S=S_o)
    assert core.rel_l2(F, Ft) <= tol
    assert abs(e["U_far"] - eo["U_F"]) <= tol * abs(eo["U_F"])


@pytest.mark.parametrize("ensemble", ["langevin", "nve"])
def test_instantaneous_temperature_trajectory(ensemble):
    """Five steps in the FP64 build with calF at the kinetic temperature of each evaluation,
    against the oracle's integrator given the same k-sets."""
    w = workload(500, 8.0, kappa=1.0, Gamma=1.0, P=64, seed=47, dt=0.002, ensemble=ensemble)
    r0, v0, q, m = W.positions(w), W.velocities(w), W.charges(w), W.masses(w)
    n = 5
    ks, kTs, rg, vg = [], [], [], []
    with Ctx(w, R.RBSOG_FP64, temperature=R.RBSOG_KT_INSTANT) as c:
        R.rbsog_set_state(c.h, r0, v0)
        R.rbsog_forces(c.h)
        ks.append(R.rbsog_get_ksample(c.h, c.P)[0])
        kTs.append(R.rbsog_get_temperature(c.h)[0])
        for _ in range(n):
            R.rbsog_step(c.h, 1)
            ks.append(R.rbsog_get_ksample(c.h, c.P)[0])
            kTs.append(R.rbsog_get_temperature(c.h)[0])
            r = np.zeros((w.N, 3))
            v = np.zeros((w.N, 3))
            R.rbsog_get_state(c.h, r, v)
            rg.append(r)
            vg.append(v)
    sog = oracle_sog(w)
    Q2 = float(np.sum(q * q))
    st = {"i": 0}

    def force(x, vel):
        kT = integrate.kinetic_temperature(vel, m)
        assert abs(kT - kTs[st["i"]]) <= 1e-12 * kT, st["i"]
        S_ = core.S_sum(w.box, sog, kT, Q2)
        Ft, _, _, _ = core.rb_forces(x, q, w.box, w.r_c, sog, ks[st["i"]], kT, S=S_)
        st["i"] += 1
        return Ft

    r, v = integrate.wrap(r0, w.box), v0.copy()
    F = force(r, v)
    for s in range(n):
        if ensemble == "langevin":
            r, v, F = integrate.baoab_step(r, v, F, m, w.box, w.dt, w.langevin_gamma, w.kT, w.seed_k, s + 1, force,
                                           with_v=True)
        else:
            r, v, F = integrate.vv_step(r, v, F, m, w.box, w.dt, force, with_v=True)
        d = rg[s] - r
        d -= np.asarray(w.box) * np.round(d / np.asarray(w.box))
        assert np.max(np.abs(d)) <= FP64_TOL * w.box[0], s
        assert core.rel_l2(vg[s], v) <= FP64_TOL, s
    assert len(set(kTs)) == len(kTs)          # the temperature does change from step to step
