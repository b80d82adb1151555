"""Shared helpers of the GPU parity tests: contexts through the C ABI and the oracle's
reference values on the same seeded inputs."""
import dataclasses
import math

import numpy as np

from oracle import core
from oracle import sog as S
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

FP64_TOL = 1e-12
FP32_TOL = 1e-5
# Floor of the per-particle relative force error, as a fraction of the RMS force.  A
# particle's force is a sum of pair terms (and of mode terms); where they nearly cancel,
# as on a bcc lattice, the rounding error scales with the terms, not with their small
# total, so the relative error of such a particle says nothing about the arithmetic.
PP_FLOOR = 0.1


def force_errors(got, ref):
    """The force-error metrics of the parity tests: the relative L2 error over all
    particles, sqrt(sum |dF|^2 / sum |F|^2), and the largest per-particle relative error
    max_i |dF_i| / (|F_i| + PP_FLOOR rms|F|)."""
    got = np.asarray(got, dtype=np.float64).reshape(-1, 3)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1, 3)
    d = np.linalg.norm(got - ref, axis=1)
    n = np.linalg.norm(ref, axis=1)
    rms = float(np.sqrt(np.mean(n * n))) if n.size else 0.0
    rel = core.rel_l2(got, ref)
    pp = float(np.max(d / (n + PP_FLOOR * rms))) if rms > 0 else float(np.max(d, initial=0.0))
    return rel, pp


def check_forces(got, ref, tol, what=""):
    """Relative L2 and per-particle relative error (with the floor above) both <= tol."""
    rel, pp = force_errors(got, ref)
    assert rel <= tol and pp <= tol, (what, {"rel_l2": rel, "per_particle_max": pp, "tol": tol})
    return rel, pp


def check_rho(got, ref, q, tol, what="rho"):
    """Every mode: |rho_gpu - rho_ref| <= tol (|rho_ref| + sqrt(sum q^2)); sqrt(sum q^2) is
    the size of rho for uncorrelated phases, the scale of a rounding error that grows
    like a random walk over the particles."""
    got = np.asarray(got, dtype=np.float64).reshape(-1, 2)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1, 2)
    scale = np.hypot(ref[:, 0], ref[:, 1]) + float(np.sqrt(np.sum(np.asarray(q, dtype=np.float64) ** 2)))
    err = float(np.max(np.hypot(got[:, 0] - ref[:, 0], got[:, 1] - ref[:, 1]) / scale))
    assert err <= tol, (what, err, tol)
    return err


def check_energy(got, ref, tol, what=""):
    err = abs(got - ref) / abs(ref)
    assert err <= tol, (what, got, ref, err, tol)
    return err


def require_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


class Ctx:
    def __init__(self, w, precision, q=None, m=None, **kw):
        self.w = w
        self.q = W.charges(w) if q is None else np.asarray(q, dtype=np.float64)
        self.m = W.masses(w) if m is None else np.asarray(m, dtype=np.float64)
        self.params = R.make_params(w, precision=precision, **kw)
        self.P = self.params.P
        # N of the context: the charges given (a domain of the workload), else the workload's
        self.h = R.rbsog_init(self.params, len(self.q), self.q, self.m)

    def close(self):
        R.rbsog_free(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def oracle_sog(w):
    return S.build(w.a_ws / w.kappa, w.r_c, w.sog_eps)


def oracle_forces(w, r, q, modes, near="cells", idx=None, rho=None, sog=None, S_=None):
    sog = oracle_sog(w) if sog is None else sog
    Q2 = float(np.sum(np.asarray(q) ** 2))
    S_ = core.S_sum(w.box, sog, w.kT, Q2) if S_ is None else S_
    Ft, Fn, Ff, e = core.rb_forces(r, q, w.box, w.r_c, sog, modes, w.kT, S=S_, near=near, idx=idx, rho_=rho)
    return Ft, Fn, Ff, e, S_


def workload(N, L, kappa=1.0, Gamma=1.0, rc=None, P=64, eps=1e-6, seed=7, box=None, dt=0.01, ensemble="nve"):
    """A small uniform YOCP workload of the requested shape."""
    box = (L, L, L) if box is None else tuple(box)
    V = box[0] * box[1] * box[2]
    a = W.wigner_seitz(N, V)
    rc = 2.5 * a if rc is None else rc
    return W.Workload(f"test_N{N}", N, box, a, kappa, Gamma, rc, eps, P, dt, 10, ensemble, 1.0, "uniform", seed,
                      seed + 1, seed + 2)


def modes_for(w, P, seed):
    nmax = max(2, int(math.ceil(4.0 * max(w.box) / (2 * math.pi))))
    return W.random_modes(P, nmax, seed)
