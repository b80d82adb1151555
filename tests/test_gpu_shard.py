"""Domain decomposition through the C ABI (Sec. 4.3: local structure factors, a global
reduction of rho, a broadcast): a system split into slabs, one context per slab holding
its owned particles and their halo, partial rho from each (rbsog_forces_partial), the sum
over slabs, and the far force from the summed rho (rbsog_forces_complete).  The owned rows
of the slabs together are the whole system's forces: against the FP64 oracle on the same
k-set (1e-12 in FP64, 1e-5 in FP32), in one process with a host sum, and across two gloo
processes on one GPU with the sum as an all-reduce (each process's kernels run on their
own; the exchange is on the host)."""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from gpu_common import FP32_TOL, FP64_TOL, Ctx, check_forces, modes_for, oracle_forces, require_gpu, workload
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def shard_forces(w, prec, r, q, modes, nslabs, axis=0):
    """Whole-system forces assembled from the owned rows of nslabs slab contexts."""
    Q2, qs = float(np.sum(q * q)), float(np.sum(q))
    ctxs, splits, parts = [], [], []
    try:
        for s in range(nslabs):
            idx, n_owned = R.rbsog_slab_split(r, w.box, axis, nslabs, s, w.r_c)
            c = Ctx(w, prec, q=q[idx], m=W.masses(w)[idx], q2_total=Q2, qsum_total=qs)
            ctxs.append(c)
            splits.append((idx, n_owned))
            R.rbsog_set_owned(c.h, n_owned)
            R.rbsog_set_state(c.h, r[idx])
            R.rbsog_set_ksample(c.h, modes)
            part = np.zeros((w.P, 2))
            R.rbsog_forces_partial(c.h, part)
            parts.append(part)
        rho = np.sum(parts, axis=0)
        F = np.full((w.N, 3), np.nan)
        draws = []
        for c, (idx, n_owned) in zip(ctxs, splits):
            Fl = np.zeros((len(idx), 3))
            R.rbsog_forces_complete(c.h, rho, Fl)
            F[idx[:n_owned]] = Fl[:n_owned]
            draws.append(R.rbsog_get_ksample(c.h, c.P))
    finally:
        for c in ctxs:
            c.close()
    return F, rho, draws


@pytest.mark.parametrize("prec,tol", [(R.RBSOG_FP64, FP64_TOL), (R.RBSOG_FP32, FP32_TOL)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("nslabs,axis", [(2, 0), (3, 1)])
def test_slab_forces_equal_the_whole_system(prec, tol, nslabs, axis):
    w = workload(4000, 16.0, kappa=1.0, Gamma=2.0, P=96, seed=171)
    r, q = W.positions(w), W.charges(w)
    q = np.where(np.arange(w.N) % 5 == 0, 2.0, 1.0)
    modes = modes_for(w, w.P, 172)
    F, rho, draws = shard_forces(w, prec, r, q, modes, nslabs, axis)
    assert np.all(np.isfinite(F))
    Ft, _, _, _, _ = oracle_forces(w, r, q, modes)
    check_forces(F, Ft, tol, ("slabs", nslabs))
    from oracle import core
    rho_o = core.rho(r, q, w.box, modes)
    assert np.max(np.abs(rho - rho_o)) <= tol * np.sqrt(np.sum(q * q))
    # every slab drew (here: took) the same modes with the whole system's coefficients
    for m, coef in draws[1:]:
        assert np.array_equal(m, draws[0][0]) and np.array_equal(coef, draws[0][1])


def test_slab_contexts_draw_the_whole_systems_modes():
    """Without injection each slab context draws the modes and coefficients of a context
    of the whole system (same seed, same draw counter, q2_total)."""
    w = workload(3000, 14.0, kappa=1.0, Gamma=10.0, P=128, seed=173)
    r, q = W.positions(w), W.charges(w)
    with Ctx(w, R.RBSOG_FP32) as c:
        R.rbsog_set_state(c.h, r)
        R.rbsog_forces(c.h)
        m0, coef0 = R.rbsog_get_ksample(c.h, c.P)
    idx, n_owned = R.rbsog_slab_split(r, w.box, 2, 2, 1, w.r_c)
    with Ctx(w, R.RBSOG_FP32, q=q[idx], m=W.masses(w)[idx], q2_total=float(np.sum(q * q)),
             qsum_total=float(np.sum(q))) as c:
        R.rbsog_set_owned(c.h, n_owned)
        R.rbsog_set_state(c.h, r[idx])
        part = np.zeros((w.P, 2))
        R.rbsog_forces_partial(c.h, part)
        m1, coef1 = R.rbsog_get_ksample(c.h, c.P)
        with pytest.raises(R.RbsogError, match="EINVAL"):
            R.rbsog_step(c.h, 0, energy=True)                 # no energies of a domain evaluation
    assert np.array_equal(m0, m1)
    assert np.max(np.abs(coef1 - coef0) / coef0) <= 1e-14


WORKER = textwrap.dedent("""
    import json, os, sys
    import numpy as np
    import torch, torch.distributed as dist
    sys.path.insert(0, {root!r}); sys.path.insert(0, os.path.join({root!r}, "tests"))
    from gpu_common import Ctx, modes_for, workload
    from paper_2501_10946_gb300 import rbsog as R
    from paper_2501_10946_gb300 import workloads as W
    rank, ws = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    w = workload(4000, 16.0, kappa=1.0, Gamma=2.0, P=96, seed=171)
    r, q = W.positions(w), W.charges(w)
    modes = modes_for(w, w.P, 172)
    idx, n_owned = R.rbsog_slab_split(r, w.box, 0, ws, rank, w.r_c)
    with Ctx(w, {prec}, q=q[idx], m=W.masses(w)[idx], q2_total=float(np.sum(q * q)),
             qsum_total=float(np.sum(q))) as c:
        R.rbsog_set_owned(c.h, n_owned)
        R.rbsog_set_state(c.h, r[idx])
        R.rbsog_set_ksample(c.h, modes)
        part = np.zeros((w.P, 2))
        R.rbsog_forces_partial(c.h, part)
        t = torch.from_numpy(part)
        dist.all_reduce(t)                      # the global reduction of rho (2P numbers)
        F = np.zeros((len(idx), 3))
        R.rbsog_forces_complete(c.h, t.numpy(), F)
    out = [None] * ws
    dist.all_gather_object(out, (idx[:n_owned].tolist(), F[:n_owned].tolist()))
    if rank == 0:
        json.dump(out, open(sys.argv[1], "w"))
    dist.destroy_process_group()
""")


@pytest.mark.parametrize("prec,tol", [(R.RBSOG_FP64, FP64_TOL), (R.RBSOG_FP32, FP32_TOL)], ids=["fp64", "fp32"])
def test_two_gloo_ranks_reduce_rho_and_match_the_oracle(tmp_path, prec, tol):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT, prec=prec))
    out = tmp_path / "out.json"
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT="29731")
        procs.append(subprocess.Popen([sys.executable, str(script), str(out)], env=env))
    for p in procs:
        assert p.wait(timeout=300) == 0
    parts = json.load(open(out))
    w = workload(4000, 16.0, kappa=1.0, Gamma=2.0, P=96, seed=171)
    F = np.full((w.N, 3), np.nan)
    for idx, Fo in parts:
        F[np.asarray(idx)] = np.asarray(Fo)
    assert np.all(np.isfinite(F))
    r, q = W.positions(w), W.charges(w)
    Ft, _, _, _, _ = oracle_forces(w, r, q, modes_for(w, w.P, 172))
    check_forces(F, Ft, tol, "two ranks")
