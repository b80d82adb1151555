"""GPU k-sampler: bit-exact replay against the oracle's sampler from the same seed, and
chi-square of GPU draws against the exact measure P(k) of Eq. (59), for the three
corrections calF (Eq. 62, 1, k^2); coefficients against the oracle for each."""
import math

import numpy as np
import pytest

from gpu_common import Ctx, oracle_sog, require_gpu, workload
from oracle import core
from oracle.sampler import ModeSampler
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


MEASURES = [pytest.param(0, id="adaptive"), pytest.param(1, id="F1"), pytest.param(2, id="k2"),
            pytest.param(3, id="debye")]


@pytest.mark.parametrize("kind", MEASURES)
@pytest.mark.parametrize("Gamma,kappa", [(1.0, 1.0), (100.0, 0.5), (0.1, 2.0)])
def test_gpu_draws_replay_the_oracle_sampler(Gamma, kappa, kind):
    w = workload(400, 9.0, kappa=kappa, Gamma=Gamma, P=256, seed=31)
    r = W.positions(w)
    q = W.charges(w)
    Q2 = float(np.sum(q * q))
    sog = oracle_sog(w)
    ms = ModeSampler(sog, w.box, w.kT, Q2, kind=kind)
    S_ = core.S_sum(w.box, sog, w.kT, Q2, kind=kind)
    with Ctx(w, R.RBSOG_FP32, sampling=kind) as c:
        R.rbsog_set_state(c.h, r)
        assert abs(R.rbsog_get_sog(c.h)["S"] - S_) <= 1e-11 * S_
        for d in range(3):
            R.rbsog_forces(c.h)
            m_gpu, coef = R.rbsog_get_ksample(c.h, c.P)
            m_or, _ = ms.draw(w.seed_k, d, c.P)
            assert np.array_equal(m_gpu, m_or), f"draw {d}"
            ref = core.rb_coef(m_or, w.box, sog, w.kT, Q2, S_, kind=kind)
            assert np.max(np.abs(coef - ref) / ref) <= 1e-11


@pytest.mark.parametrize("kind", MEASURES)
def test_gpu_sampler_chi_square(kind):
    """2e6 GPU draws (P = 4096 per force evaluation) against the exact P(k)."""
    w = workload(2, 6.0, kappa=1.0, Gamma=1.0, rc=2.5, P=4096, seed=77)
    q = W.charges(w)
    ms = ModeSampler(oracle_sog(w), w.box, w.kT, float(np.sum(q * q)), kind=kind)
    modes = ms.all_modes()
    k2 = ms.k2_of(modes)
    p = ms.calF(k2) * ms.fhat(k2)
    p = p / p.sum()
    index = {tuple(x): j for j, x in enumerate(modes)}
    counts = np.zeros(len(modes))
    n = 0
    with Ctx(w, R.RBSOG_FP32, sampling=kind) as c:
        R.rbsog_set_state(c.h, W.positions(w))
        for _ in range(500):
            R.rbsog_forces(c.h)
            m, _ = R.rbsog_get_ksample(c.h, c.P)
            js = np.array([index[tuple(x)] for x in m])
            counts += np.bincount(js, minlength=len(modes))
            n += len(js)
    order = np.argsort(-p)
    top = order[:200]
    e = np.append(p[top], p[order[200:]].sum()) * n
    o = np.append(counts[top], counts[order[200:]].sum())
    keep = e > 5
    chi2 = float(np.sum((o[keep] - e[keep]) ** 2 / e[keep]))
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)
