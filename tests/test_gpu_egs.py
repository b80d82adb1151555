"""GPU parity for the EGS screening (params.egs_nu > 0): the kernel of
eps(k) = 1 + (lambda k)^-2 (1 + nu lambda^2 k^2/4)^-1 as two Yukawa kernels, each with its
own SOG decomposition, against the FP64 oracle (oracle/egs.py) on the same k-set; the
sampler's coefficients with the envelope ratio Fhat/Fhat_env; the mean of many random
batches against the full far field; and an EGS system inside a batch."""
import numpy as np
import pytest

from gpu_common import FP32_TOL, FP64_TOL, Ctx, check_energy, check_forces, modes_for, require_gpu, workload
from oracle import core, egs
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NU = 0.5


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def oracle_egs(w, nu=NU):
    return egs.build(w.a_ws / w.kappa, nu, w.r_c, w.sog_eps)


@pytest.mark.parametrize("prec,tol", [(R.RBSOG_FP64, FP64_TOL), (R.RBSOG_FP32, FP32_TOL)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("kind", [core.ADAPTIVE, core.K2])
def test_egs_forces_and_energies_match_the_oracle(prec, tol, kind):
    w = workload(1500, 11.0, kappa=1.0, Gamma=2.0, P=96, seed=81)
    r, q = W.positions(w), W.charges(w)
    modes = modes_for(w, w.P, 82)
    e = oracle_egs(w)
    with Ctx(w, prec, egs_nu=NU, sampling=kind) as c:
        R.rbsog_set_state(c.h, r)
        R.rbsog_set_ksample(c.h, modes)
        Fn = np.zeros((w.N, 3)); Ff = np.zeros((w.N, 3))
        eg = R.rbsog_forces_split(c.h, Fn, Ff, energy=True)
        m_used, coef = R.rbsog_get_ksample(c.h, c.P)
    Ft, Fno, Ffo, eo, S = egs.rb_forces(r, q, w.box, e, modes, w.kT, kind=kind)
    assert np.array_equal(m_used, modes)
    assert core.rel_l2(coef, egs.rb_coef(modes, w.box, e, w.kT, float(np.sum(q * q)), S, kind=kind)) <= 1e-12
    check_forces(Fn, Fno, tol, "near")
    check_forces(Ff, Ffo, tol, "far")
    check_forces(Fn + Ff, Ft, tol, "total")
    for key, ref in (("U_near", eo["U_N"]), ("U_far", eo["U_F"]), ("U_self", eo["U_self"])):
        check_energy(eg[key], ref, tol, key)


@pytest.mark.parametrize("prec,tol", [(R.RBSOG_FP64, FP64_TOL), (R.RBSOG_FP32, FP32_TOL)], ids=["fp64", "fp32"])
def test_egs_small_box_per_particle_path(prec, tol):
    """Fewer than 3 cells per axis: the per-particle near path with both Yukawa terms."""
    w = workload(200, 4.0, kappa=1.0, Gamma=1.0, rc=1.9, P=64, seed=91)
    r, q = W.positions(w), W.charges(w)
    modes = modes_for(w, w.P, 92)
    e = oracle_egs(w, nu=0.8)
    with Ctx(w, prec, egs_nu=0.8) as c:
        assert R.rbsog_get_cells(c.h, w.N)[0].tolist() == [1, 1, 1]
        R.rbsog_set_state(c.h, r)
        R.rbsog_set_ksample(c.h, modes)
        F = np.zeros((w.N, 3))
        eg = R.rbsog_forces(c.h, F, energy=True)
    Ft, _, _, eo, _ = egs.rb_forces(r, q, w.box, e, modes, w.kT, cells=False)
    check_forces(F, Ft, tol, "total")
    check_energy(eg["U_near"], eo["U_N"], tol, "U_near")


def test_egs_sampled_coefficients_match_the_oracle():
    """Modes drawn by the GPU sampler from the envelope: their coefficients are the oracle's
    S_env Fhat / (P V calF Fhat_env), including modes where Fhat < 0."""
    w = workload(800, 9.0, kappa=1.0, Gamma=1.0, P=512, seed=83)
    e = oracle_egs(w)
    with Ctx(w, R.RBSOG_FP64, egs_nu=NU) as c:
        R.rbsog_set_state(c.h, W.positions(w))
        R.rbsog_forces(c.h)
        m, coef = R.rbsog_get_ksample(c.h, c.P)
    Q2 = float(np.sum(W.charges(w) ** 2))
    S = egs.S_sum(w.box, e, w.kT, Q2)
    ref = egs.rb_coef(m, w.box, e, w.kT, Q2, S)
    assert core.rel_l2(coef, ref) <= 1e-12


def test_egs_random_batches_average_to_the_full_far_field():
    """Lemma 4.1 with the envelope measure: the mean of many independent random-batch far
    forces approaches the full k-space far force of the two-term SOG."""
    w = workload(300, 7.0, kappa=1.0, Gamma=1.0, P=256, seed=85)
    r, q = W.positions(w), W.charges(w)
    e = oracle_egs(w)
    draws = 300
    acc = np.zeros((w.N, 3))
    with Ctx(w, R.RBSOG_FP64, egs_nu=NU) as c:
        R.rbsog_set_state(c.h, r)
        Ff = np.zeros((w.N, 3))
        for _ in range(draws):
            R.rbsog_forces_split(c.h, None, Ff)
            acc += Ff
    Ffull, _ = egs.far_full(r, q, w.box, e)
    one = core.rel_l2(Ff, Ffull)
    mean = core.rel_l2(acc / draws, Ffull)
    print({"one_draw_rel_l2": one, "mean_rel_l2": mean, "draws": draws})
    assert mean <= 3.0 * one / np.sqrt(draws) + 1e-3


def test_egs_system_in_a_batch_matches_a_single_context():
    ws = [workload(1000, 10.0, kappa=1.0, Gamma=1.0, P=100, seed=87),
          workload(900, 9.5, kappa=0.8, Gamma=3.0, P=80, seed=89)]
    nus = [NU, 0.0]
    params = [R.make_params(w, precision=R.RBSOG_FP32, egs_nu=nu) for w, nu in zip(ws, nus)]
    q = np.concatenate([W.charges(w) for w in ws])
    m = np.concatenate([W.masses(w) for w in ws])
    r = np.concatenate([W.positions(w) for w in ws])
    modes = [modes_for(w, w.P, 90 + i) for i, w in enumerate(ws)]
    b = R.rbsog_batch_init(params, [w.N for w in ws], q, m)
    try:
        p_off, _, _ = R.rbsog_batch_layout(b, len(ws))
        R.rbsog_batch_set_state(b, r)
        R.rbsog_batch_set_ksample(b, np.concatenate(modes))
        F = np.zeros((int(p_off[-1]), 3))
        eb = R.rbsog_batch_forces(b, len(ws), F, energy=True)
    finally:
        R.rbsog_batch_free(b)
    for i, (w, nu) in enumerate(zip(ws, nus)):
        with Ctx(w, R.RBSOG_FP32, egs_nu=nu) as c:
            R.rbsog_set_state(c.h, W.positions(w))
            R.rbsog_set_ksample(c.h, modes[i])
            Fs = np.zeros((w.N, 3))
            es = R.rbsog_forces(c.h, Fs, energy=True)
        # different tile shapes, the same pairs per particle: FP32 rounding of the pass sums
        assert abs(eb[i]["U_near"] - es["U_near"]) <= 1e-7 * abs(es["U_near"]), i
        assert core.rel_l2(F[p_off[i]:p_off[i + 1]], Fs) <= FP32_TOL, i
