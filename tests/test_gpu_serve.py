"""GPU job server (rbsog_server_*): continuous batching of MD jobs.  Each job's result is
bit-identical alone and in a mix where jobs join while others are mid-run, agrees with the
FP64 oracle's trajectory of that job and with a single context within the FP32 tolerance,
waits for memory when the arenas are full, and fails alone when its own cells overflow."""
import numpy as np
import pytest

from gpu_common import FP32_TOL, Ctx, oracle_sog, require_gpu, workload
from oracle import core, integrate
from oracle.sampler import ModeSampler
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def jobs():
    """(workload, nsteps): uneven N, box shapes, screening, coupling, P and ensembles."""
    return [
        (workload(1500, 11.0, kappa=1.0, Gamma=2.0, P=96, seed=51, ensemble="langevin"), 50),
        (workload(600, 8.0, kappa=2.5, Gamma=20.0, P=300, seed=53), 20),
        (workload(800, 9.0, kappa=0.5, Gamma=1.0, P=128, seed=55, ensemble="langevin"), 37),
        (workload(200, 4.0, kappa=1.0, Gamma=1.0, rc=1.9, P=64, seed=57), 10),
        (workload(2500, None, kappa=1.5, Gamma=5.0, P=200, seed=59, box=(15.0, 12.0, 12.0)), 13),
    ]


def server(max_jobs=8, max_particles=20000, steps_per_round=8):
    cfg = R.make_server_config(max_particles, max_particles, 4096, max_jobs, steps_per_round=steps_per_round)
    return R.rbsog_server_create(cfg)


def submit(s, w, nsteps, t=0.0, r=None):
    p = R.make_params(w, precision=R.RBSOG_FP32)
    r = W.positions(w) if r is None else r
    return R.rbsog_server_submit(s, p, W.charges(w), W.masses(w), r, W.velocities(w), nsteps, t)


def run_jobs(js, **kw):
    s = server(**kw)
    try:
        ids = [submit(s, w, n) for w, n in js]
        R.rbsog_server_run(s)
        out = [R.rbsog_server_job(s, i, w.N, state=True) for i, (w, _) in zip(ids, js)]
        stats = R.rbsog_server_stats(s)
    finally:
        R.rbsog_server_free(s)
    return out, stats


def test_each_job_is_the_same_alone_and_in_the_mix():
    js = jobs()
    # two job slots: jobs 3.. are admitted only as earlier ones retire, so they join
    # while others are mid-run
    mix, stats = run_jobs(js, max_jobs=2)
    assert stats["admissions"] == len(js) and stats["retirements"] == len(js)
    assert stats["peak_jobs"] == 2
    infos = [m[0] for m in mix]
    # at least one job was admitted while another was resident and mid-run
    joined = [i for i in range(len(js)) for k in range(len(js))
              if k != i and infos[k]["t_admit"] < infos[i]["t_admit"] < infos[k]["t_done"]]
    assert joined
    for i, (w, n) in enumerate(js):
        alone, _ = run_jobs([(w, n)])
        info_a, r_a, v_a = alone[0]
        info_m, r_m, v_m = mix[i]
        assert info_m["status"] == R.RBSOG_JOB_DONE and info_m["steps_done"] == n
        assert info_m["energy"]["step"] == n
        assert np.array_equal(r_a, r_m), i
        assert np.array_equal(v_a, v_m), i
        assert info_a["energy"]["total"] == info_m["energy"]["total"], i


def oracle_job(w, nsteps):
    """The oracle's run of one job (Algorithm 2): evaluation d uses the oracle sampler's
    draw d from the job's seed, the integrator is the oracle's velocity Verlet or BAOAB
    (step n keyed by the n + 1 evaluations before it).  Returns the final positions,
    velocities and the energy terms of the last evaluation."""
    r0, v0, q, m = W.positions(w), W.velocities(w), W.charges(w), W.masses(w)
    sog = oracle_sog(w)
    Q2 = float(np.sum(q * q))
    S_ = core.S_sum(w.box, sog, w.kT, Q2)
    ms = ModeSampler(sog, w.box, w.kT, Q2)
    near = "cells" if min(core.n_cells(w.box, w.r_c)) >= 3 else "images"
    st = {"d": 0, "e": None}

    def force(x):
        ks, _ = ms.draw(w.seed_k, st["d"], w.P)
        st["d"] += 1
        Ft, _, _, e = core.rb_forces(x, q, w.box, w.r_c, sog, ks, w.kT, S=S_, near=near)
        st["e"] = e
        return Ft

    r, v = integrate.wrap(r0, w.box), v0.copy()
    F = force(r)
    for n in range(nsteps):
        if w.ensemble == "langevin":
            r, v, F = integrate.baoab_step(r, v, F, m, w.box, w.dt, w.langevin_gamma, w.kT, w.seed_k, n + 1, force)
        else:
            r, v, F = integrate.vv_step(r, v, F, m, w.box, w.dt, force)
    e = dict(st["e"])
    e["kinetic"] = integrate.kinetic(v, m)
    return r, v, e


def test_served_jobs_match_the_oracle():
    """Three jobs of different N, kappa, Gamma, P and ensemble, with two job slots and
    two-step rounds, so the third is admitted while the others are mid-run: each job's
    final positions, velocities and energies against the oracle's run of that job alone."""
    js = [
        (workload(1200, 10.5, kappa=1.2, Gamma=3.0, P=96, seed=151, dt=0.004, ensemble="langevin"), 5),
        (workload(700, 8.5, kappa=2.2, Gamma=30.0, P=160, seed=153, dt=0.004), 3),
        (workload(900, 9.5, kappa=0.6, Gamma=0.8, P=64, seed=155, dt=0.004), 4),
    ]
    out, stats = run_jobs(js, max_jobs=2, steps_per_round=2)
    infos = [o[0] for o in out]
    assert any(infos[k]["t_admit"] < infos[2]["t_admit"] < infos[k]["t_done"] for k in (0, 1))
    for i, (w, n) in enumerate(js):
        info, r, v = out[i]
        assert info["status"] == R.RBSOG_JOB_DONE and info["steps_done"] == n
        ro, vo, eo = oracle_job(w, n)
        d = r - ro
        L = np.asarray(w.box)
        d -= L * np.round(d / L)
        assert np.max(np.abs(d)) <= FP32_TOL * np.max(L), (i, np.max(np.abs(d)))
        assert core.rel_l2(v, vo) <= FP32_TOL, (i, core.rel_l2(v, vo))
        for k_gpu, k_or in (("U_near", "U_N"), ("U_far", "U_F"), ("U_self", "U_self"), ("kinetic", "kinetic")):
            err = abs(info["energy"][k_gpu] - eo[k_or]) / abs(eo[k_or])
            assert err <= FP32_TOL, (i, k_gpu, info["energy"][k_gpu], eo[k_or])


def test_served_job_follows_a_single_context():
    w, n = jobs()[2]
    out, _ = run_jobs([(w, n)])
    info, r, v = out[0]
    with Ctx(w, R.RBSOG_FP32) as c:
        R.rbsog_set_state(c.h, W.positions(w), W.velocities(w))
        e = R.rbsog_step(c.h, n, energy=True)
        rs = np.zeros((w.N, 3))
        vs = np.zeros((w.N, 3))
        R.rbsog_get_state(c.h, rs, vs)
    d = r - rs
    L = np.asarray(w.box)
    d -= L * np.round(d / L)
    assert np.max(np.abs(d)) <= 1e-6 * np.max(L)
    assert core.rel_l2(v, vs) <= FP32_TOL
    assert info["energy"]["step"] == e["step"] == n


def test_admission_waits_for_memory():
    """Arenas for 2000 particles: a 1500- and an 800-particle job cannot be resident
    together, so the second is admitted only after the first retires."""
    js = [jobs()[0], jobs()[2]]
    out, stats = run_jobs(js, max_particles=2000)
    first, second = out[0][0], out[1][0]
    assert first["status"] == second["status"] == R.RBSOG_JOB_DONE
    assert second["t_admit"] >= first["t_done"]
    assert stats["peak_jobs"] == 1
    assert first["footprint_bytes"] > 1500 * 200


def test_a_failing_job_fails_alone():
    """A job whose particles all sit in one cell overflows the cell list: it fails with
    EOVERFLOW and the job beside it completes unchanged."""
    good, n_good = jobs()[0]
    bad = workload(5000, 20.0, kappa=1.0, Gamma=1.0, P=64, seed=61)
    s = server(max_particles=20000)
    try:
        i_bad = submit(s, bad, 5, r=np.full((bad.N, 3), 3.0))
        i_good = submit(s, good, n_good)
        R.rbsog_server_run(s)
        info_bad, _, _ = R.rbsog_server_job(s, i_bad)
        info_good, r_g, v_g = R.rbsog_server_job(s, i_good, good.N, state=True)
    finally:
        R.rbsog_server_free(s)
    assert info_bad["status"] == R.RBSOG_JOB_FAILED and R.STATUS[info_bad["error"]] == "EOVERFLOW"
    alone, _ = run_jobs([(good, n_good)])
    assert info_good["status"] == R.RBSOG_JOB_DONE
    assert np.array_equal(alone[0][1], r_g) and np.array_equal(alone[0][2], v_g)


def test_arrivals_in_the_future_wait_and_stats_add_up():
    js = jobs()[:3]
    s = server()
    try:
        ids = [submit(s, w, n, t=0.05 * k) for k, (w, n) in enumerate(js)]
        R.rbsog_server_run(s)
        infos = [R.rbsog_server_job(s, i)[0] for i in ids]
        stats = R.rbsog_server_stats(s)
    finally:
        R.rbsog_server_free(s)
    for k, info in enumerate(infos):
        assert info["status"] == R.RBSOG_JOB_DONE
        assert info["t_admit"] >= info["t_arrival"] == pytest.approx(0.05 * k)
        assert info["t_done"] >= info["t_admit"]
    assert stats["particle_steps"] == sum(w.N * n for w, n in js)


def test_edge_jobs_are_handled_and_do_not_block_the_queue():
    """Zero steps (only the initial evaluation), two particles, a job larger than the
    arenas and a job with invalid parameters, mixed with a normal job: the impossible ones
    fail at admission, the rest complete."""
    normal, n_normal = jobs()[2]
    s = server(max_particles=5000)
    try:
        ids = {}
        ids["zero"] = submit(s, normal, 0)
        two = workload(2, 4.0, rc=1.9, P=8, seed=71)
        ids["two"] = submit(s, two, 7)
        big = workload(6000, 18.0, P=64, seed=73)
        ids["big"] = submit(s, big, 3)
        bad = R.make_params(normal, precision=R.RBSOG_FP32)
        bad.kappa = -1.0
        ids["bad"] = R.rbsog_server_submit(s, bad, W.charges(normal), W.masses(normal), W.positions(normal), None, 5)
        ids["normal"] = submit(s, normal, n_normal)
        R.rbsog_server_run(s)
        info = {k: R.rbsog_server_job(s, v)[0] for k, v in ids.items()}
        _, r0, v0 = R.rbsog_server_job(s, ids["zero"], normal.N, state=True)
    finally:
        R.rbsog_server_free(s)
    assert info["zero"]["status"] == R.RBSOG_JOB_DONE and info["zero"]["steps_done"] == 0
    assert np.array_equal(r0, W.positions(normal))         # no step taken
    assert info["zero"]["energy"]["step"] == 0 and np.isfinite(info["zero"]["energy"]["total"])
    assert info["two"]["status"] == R.RBSOG_JOB_DONE and info["two"]["steps_done"] == 7
    assert info["big"]["status"] == R.RBSOG_JOB_FAILED and R.STATUS[info["big"]["error"]] == "ENOMEM"
    assert info["bad"]["status"] == R.RBSOG_JOB_FAILED and R.STATUS[info["bad"]["error"]] == "EINVAL"
    assert info["normal"]["status"] == R.RBSOG_JOB_DONE and info["normal"]["steps_done"] == n_normal
