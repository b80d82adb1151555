"""The exchange step of a spatially partitioned RBSOG force (the multi-GPU design, run
here as two gloo processes on CPU with the FP64 oracle): each rank owns the particles of
one slab along x.  The random-batch far field needs one all-reduce of the partial
structure factors rho(k_l) (2P numbers; every rank draws the same k-set), after which
each rank gathers the far force of its own particles; the near field needs the
particles within r_c of the slab faces from the other rank (a halo).  Every rank's
forces must equal the unpartitioned evaluation."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import core
from oracle import sog as S
from paper_2501_10946_gb300 import workloads as W


def _system():
    N, L = 1200, 12.0
    V = L ** 3
    a = W.wigner_seitz(N, V)
    w = W.Workload("slabs", N, (L, L, L), a, 1.0, 3.0, 2.5 * a, 1e-6, 64, 0.01, 1, "nve", 1.0, "uniform",
                   901, 902, 903)
    r = W.positions(w)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -0.5)
    modes = W.random_modes(w.P, 4, 904)
    return w, r, q, modes


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, q, modes = _system()
        L = w.box[0]
        sog = S.build(w.a_ws / w.kappa, w.r_c, w.sog_eps)
        Q2 = float(np.sum(q * q))
        S_ = core.S_sum(w.box, sog, w.kT, Q2)
        coef = core.rb_coef(modes, w.box, sog, w.kT, Q2, S_)
        lo, hi = rank * L / world, (rank + 1) * L / world
        own = np.nonzero((r[:, 0] >= lo) & (r[:, 0] < hi))[0]
        # far field: partial rho over the slab, all-reduced
        part = torch.tensor(core.rho(r[own], q[own], w.box, modes))
        dist.all_reduce(part)
        rho = part.numpy()
        Ff = core.far_rb(r[own], q[own], w.box, modes, coef, rho)
        # near field: own particles plus the other ranks' particles within r_c of the slab
        # (periodic distance along x to the slab interval)
        def halo_of(lo_, hi_):
            x = r[:, 0]
            dx = np.minimum(np.minimum(np.abs(x - lo_), np.abs(x - hi_)),
                            np.minimum(np.abs(x - L - lo_), np.abs(x + L - hi_)))
            inside = (x >= lo_) & (x < hi_)
            return np.nonzero(~inside & (dx < w.r_c))[0]
        # every rank publishes the particles it owns; each takes what lies in its halo
        gathered = [None] * world
        dist.all_gather_object(gathered, (own, r[own], q[own]))
        ids = np.concatenate([g[0] for g in gathered])
        pos = np.concatenate([g[1] for g in gathered])
        chg = np.concatenate([g[2] for g in gathered])
        want = set(halo_of(lo, hi).tolist())
        take = np.array([k for k in range(ids.size) if ids[k] in want], dtype=np.int64)
        loc_r = np.concatenate([r[own], pos[take]])
        loc_q = np.concatenate([q[own], chg[take]])
        Fn, _ = core.near_cells(loc_r, loc_q, w.box, w.r_c, sog, idx=np.arange(own.size))
        out[rank] = (own, rho, Ff, Fn)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_slab_partition_matches_the_whole_system():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(k, world, port, out)) for k in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=240)
            assert p.exitcode == 0
        res = dict(out)
    w, r, q, modes = _system()
    sog = S.build(w.a_ws / w.kappa, w.r_c, w.sog_eps)
    Q2 = float(np.sum(q * q))
    S_ = core.S_sum(w.box, sog, w.kT, Q2)
    Ft, Fn, Ff, _ = core.rb_forces(r, q, w.box, w.r_c, sog, modes, w.kT, S=S_)
    rho = core.rho(r, q, w.box, modes)
    seen = np.concatenate([res[k][0] for k in range(world)])
    assert np.array_equal(np.sort(seen), np.arange(w.N))
    for k in range(world):
        own, rho_k, Ff_k, Fn_k = res[k]
        assert np.max(np.abs(rho_k - rho)) <= 1e-12 * np.max(np.abs(rho))
        assert core.rel_l2(Ff_k, Ff[own]) <= 1e-12
        assert core.rel_l2(Fn_k, Fn[own]) <= 1e-12
