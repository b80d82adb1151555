"""GPU batches of independent systems (rbsog_batch_*): every system of a batch against its
own single context and against the FP64 oracle, on systems that differ in size, box
shape, screening, coupling, P (one above 256, so the structure factor takes two mode
passes), ensemble, and near-field path (one box too small for the tiled kernel)."""
import numpy as np
import pytest

from gpu_common import FP32_TOL, Ctx, check_energy, check_forces, modes_for, oracle_forces, require_gpu, workload
from oracle import core
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def systems():
    ws = [
        workload(1000, 10.0, kappa=1.0, Gamma=1.0, P=100, seed=31),
        workload(600, 8.0, kappa=2.0, Gamma=10.0, P=300, seed=37, ensemble="langevin"),
        workload(200, 4.0, kappa=1.0, Gamma=1.0, rc=1.9, P=64, seed=41),                    # n_c = 1: per-particle path
        workload(2000, None, kappa=0.5, Gamma=3.0, P=128, seed=43, box=(12.0, 10.0, 9.0), ensemble="langevin"),
    ]
    return ws


class Batch:
    def __init__(self, ws, chunk=None):
        self.ws = ws
        self.R = len(ws)
        self.params = [R.make_params(w, precision=R.RBSOG_FP32) for w in ws]
        self.q = np.concatenate([W.charges(w) for w in ws])
        self.m = np.concatenate([W.masses(w) for w in ws])
        self.N = [w.N for w in ws]
        self.h = R.rbsog_batch_init(self.params, self.N, self.q, self.m)
        self.p_off, self.m_off, self.chunk = R.rbsog_batch_layout(self.h, self.R)
        if chunk is not None:
            R.rbsog_batch_set_rho_chunk(self.h, [chunk] * self.R)
        self.Ntot = int(self.p_off[-1])
        self.Ptot = int(self.m_off[-1])

    def split(self, x):
        return [x[self.p_off[i]:self.p_off[i + 1]] for i in range(self.R)]

    def close(self):
        R.rbsog_batch_free(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def state(ws):
    r = np.concatenate([W.positions(w) for w in ws])
    v = np.concatenate([W.velocities(w) for w in ws])
    return r, v


def test_layout_is_the_concatenation():
    ws = systems()
    with Batch(ws) as b:
        assert list(b.p_off) == list(np.concatenate([[0], np.cumsum([w.N for w in ws])]))
        assert list(b.m_off) == list(np.concatenate([[0], np.cumsum([w.P for w in ws])]))
        assert all(c >= 64 for c in b.chunk)


def test_batch_forces_match_single_contexts_and_the_oracle():
    ws = systems()
    r, _ = state(ws)
    modes = [modes_for(w, w.P, 100 + i) for i, w in enumerate(ws)]
    with Batch(ws) as b:
        R.rbsog_batch_set_state(b.h, r)
        R.rbsog_batch_set_ksample(b.h, np.concatenate(modes))
        F = np.zeros((b.Ntot, 3))
        e = R.rbsog_batch_forces(b.h, b.R, F, energy=True)
        m_used, _ = R.rbsog_batch_get_ksample(b.h, b.Ptot)
    assert np.array_equal(m_used, np.concatenate(modes))
    for i, (w, Fi, ri) in enumerate(zip(ws, b.split(F), b.split(r))):
        with Ctx(w, R.RBSOG_FP32) as c:
            R.rbsog_set_state(c.h, ri)
            R.rbsog_set_ksample(c.h, modes[i])
            Fs = np.zeros((w.N, 3))
            es = R.rbsog_forces(c.h, Fs, energy=True)
        # same cells and the same pairs in the same order per particle; the tile shapes of
        # the two near kernels differ, and with them which two pairs share a pass, so the
        # near energies agree to FP32 rounding
        assert abs(e[i]["U_near"] - es["U_near"]) <= 1e-7 * abs(es["U_near"]), i
        assert e[i]["U_self"] == es["U_self"], i
        assert core.rel_l2(Fi, Fs) <= FP32_TOL, i
        assert abs(e[i]["U_far"] - es["U_far"]) <= FP32_TOL * abs(es["U_far"]), i
        Ft, _, _, eo, _ = oracle_forces(w, ri, W.charges(w), modes[i])
        check_forces(Fi, Ft, FP32_TOL, ("system", i))
        check_energy(e[i]["U_near"], eo["U_N"], FP32_TOL, ("U_near", i))
        check_energy(e[i]["U_far"], eo["U_F"], FP32_TOL, ("U_far", i))


def test_batch_draws_the_modes_of_single_contexts():
    """Shared draw counter, per-system seed: system i draws what a single context draws."""
    ws = systems()
    r, _ = state(ws)
    with Batch(ws) as b:
        R.rbsog_batch_set_state(b.h, r)
        R.rbsog_batch_forces(b.h, b.R)
        R.rbsog_batch_forces(b.h, b.R)
        m_b, coef_b = R.rbsog_batch_get_ksample(b.h, b.Ptot)
    for i, w in enumerate(ws):
        with Ctx(w, R.RBSOG_FP32) as c:
            R.rbsog_set_state(c.h, b.split(r)[i])
            R.rbsog_forces(c.h)
            R.rbsog_forces(c.h)
            m_s, coef_s = R.rbsog_get_ksample(c.h, c.P)
        sl = slice(b.m_off[i], b.m_off[i + 1])
        assert np.array_equal(m_b[sl], m_s), i
        assert np.array_equal(coef_b[sl], coef_s), i


def test_batch_trajectories_follow_single_contexts():
    ws = systems()
    r, v = state(ws)
    nsteps = 5
    with Batch(ws) as b:
        R.rbsog_batch_set_state(b.h, r, v)
        e = R.rbsog_batch_step(b.h, b.R, nsteps, energy=True)
        rb = np.zeros((b.Ntot, 3))
        vb = np.zeros((b.Ntot, 3))
        step = R.rbsog_batch_get_state(b.h, rb, vb)
    assert step == nsteps
    for i, w in enumerate(ws):
        with Ctx(w, R.RBSOG_FP32) as c:
            R.rbsog_set_state(c.h, b.split(r)[i], b.split(v)[i])
            es = R.rbsog_step(c.h, nsteps, energy=True)
            rs = np.zeros((w.N, 3))
            vs = np.zeros((w.N, 3))
            R.rbsog_get_state(c.h, rs, vs)
        d = b.split(rb)[i] - rs
        L = np.asarray(w.box)
        d -= L * np.round(d / L)
        assert np.max(np.abs(d)) <= 1e-6 * np.max(L), i
        assert core.rel_l2(b.split(vb)[i], vs) <= 1e-5, i
        assert e[i]["step"] == es["step"] == nsteps
        assert abs(e[i]["total"] - es["total"]) <= 1e-5 * abs(es["U_near"]) + 1e-5 * abs(es["kinetic"]), i


def test_batch_is_deterministic():
    ws = systems()
    r, v = state(ws)
    outs = []
    for _ in range(2):
        with Batch(ws) as b:
            R.rbsog_batch_set_state(b.h, r, v)
            R.rbsog_batch_step(b.h, b.R, 3)
            rb = np.zeros((b.Ntot, 3))
            vb = np.zeros((b.Ntot, 3))
            R.rbsog_batch_get_state(b.h, rb, vb)
            outs.append((rb, vb))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_rho_chunk_changes_only_the_rounding():
    ws = systems()
    r, _ = state(ws)
    modes = np.concatenate([modes_for(w, w.P, 200 + i) for i, w in enumerate(ws)])
    Fs = []
    for chunk in (None, 64, 4096):
        with Batch(ws, chunk=chunk) as b:
            R.rbsog_batch_set_state(b.h, r)
            R.rbsog_batch_set_ksample(b.h, modes)
            F = np.zeros((b.Ntot, 3))
            R.rbsog_batch_forces(b.h, b.R, F)
            Fs.append(F)
    assert core.rel_l2(Fs[1], Fs[0]) <= FP32_TOL
    assert core.rel_l2(Fs[2], Fs[0]) <= FP32_TOL


def test_device_pointers_and_repeated_batches():
    torch = require_gpu()
    ws = systems()[:2]
    r, v = state(ws)
    with Batch(ws) as b:
        rd = torch.tensor(r, device="cuda", dtype=torch.float64)
        vd = torch.tensor(v, device="cuda", dtype=torch.float64)
        R.rbsog_batch_set_state(b.h, rd, vd)
        modes = np.concatenate([modes_for(w, w.P, 300 + i) for i, w in enumerate(ws)])
        R.rbsog_batch_set_ksample(b.h, modes)
        Fd = torch.zeros((b.Ntot, 3), device="cuda", dtype=torch.float64)
        R.rbsog_batch_forces(b.h, b.R, Fd)
        R.rbsog_batch_set_state(b.h, r, v)
        R.rbsog_batch_set_ksample(b.h, modes)
        Fh = np.zeros((b.Ntot, 3))
        R.rbsog_batch_forces(b.h, b.R, Fh)
        assert np.array_equal(Fd.cpu().numpy(), Fh)
        out = torch.zeros((b.Ntot, 3), device="cuda", dtype=torch.float64)
        R.rbsog_batch_get_state(b.h, out)
        assert np.array_equal(out.cpu().numpy(), r)


def test_tuner_leaves_no_trace_in_the_trajectory():
    """A batch tuned right after set_state follows the trajectory of one given the tuned
    shapes directly (the tuner restores the step and draw counters)."""
    ws = systems()
    r, v = state(ws)
    with Batch(ws) as b:
        R.rbsog_batch_set_state(b.h, r, v)
        near_t, rho_t = R.rbsog_batch_tune(b.h, reps=2)
        R.rbsog_batch_step(b.h, b.R, 3)
        ra = np.zeros((b.Ntot, 3))
        R.rbsog_batch_get_state(b.h, ra)
        m_a, _ = R.rbsog_batch_get_ksample(b.h, b.Ptot)
    assert near_t in (128.0, 160.0, 192.0, 230.0) and rho_t in (256, 512, 1024, 2048)
    with Batch(ws) as b:
        R.rbsog_batch_set_shapes(b.h, near_t, rho_t)
        R.rbsog_batch_set_state(b.h, r, v)
        R.rbsog_batch_step(b.h, b.R, 3)
        rb = np.zeros((b.Ntot, 3))
        R.rbsog_batch_get_state(b.h, rb)
        m_b, _ = R.rbsog_batch_get_ksample(b.h, b.Ptot)
    assert np.array_equal(m_a, m_b)
    assert np.array_equal(ra, rb)


def test_near_shape_changes_no_force():
    """The near tile width changes which CTA handles a particle, not its pairs."""
    ws = systems()
    r, _ = state(ws)
    modes = np.concatenate([modes_for(w, w.P, 400 + i) for i, w in enumerate(ws)])
    Fs, Us = [], []
    for near_t in (64.0, 230.0):
        with Batch(ws) as b:
            R.rbsog_batch_set_shapes(b.h, near_t, 512)
            R.rbsog_batch_set_state(b.h, r)
            R.rbsog_batch_set_ksample(b.h, modes)
            F = np.zeros((b.Ntot, 3))
            e = R.rbsog_batch_forces(b.h, b.R, F, energy=True)
            Fs.append(F)
            Us.append([x["U_near"] for x in e])
    # same pairs in the same order per particle; a tile whose staged region overflows takes
    # the per-particle path, which may round differently
    assert core.rel_l2(Fs[0], Fs[1]) <= 1e-7
    assert np.allclose(Us[0], Us[1], rtol=1e-6, atol=0)


def test_batch_profile_reports_every_group():
    ws = systems()
    r, v = state(ws)
    with Batch(ws) as b:
        R.rbsog_batch_set_state(b.h, r, v)
        prof = R.rbsog_batch_profile(b.h, 2)
        assert set(prof) == {R.rbsog_profile_name(g) for g in range(R.RBSOG_NPROF)}
        assert all(t > 0 for t in prof.values())
        assert R.rbsog_batch_get_state(b.h) == 2
