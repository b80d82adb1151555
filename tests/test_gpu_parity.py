"""GPU parity through the C ABI: every step of the force path against the FP64 oracle on
the same seeded inputs and the same injected k-set.  FP64 build: 1e-12; FP32 build: 1e-5,
applied to the relative L2 error of the forces, to every particle's relative force error
(with a floor of 0.1 of the RMS force), to every mode of rho (relative to |rho_l| +
sqrt(sum q^2)) and to each energy; cell lists bit-exact."""
import math

import numpy as np
import pytest

from gpu_common import (FP32_TOL, FP64_TOL, Ctx, check_energy, check_forces, check_rho, modes_for, oracle_forces,
                        oracle_sog, require_gpu, workload)
from oracle import core
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {R.RBSOG_FP64: FP64_TOL, R.RBSOG_FP32: FP32_TOL}
PRECS = [pytest.param(R.RBSOG_FP64, id="fp64"), pytest.param(R.RBSOG_FP32, id="fp32")]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    return require_gpu()


def run_forces(w, prec, r, modes, q=None, split=True):
    with Ctx(w, prec, q=q) as c:
        R.rbsog_set_state(c.h, r)
        R.rbsog_set_ksample(c.h, modes)
        Fn = np.zeros((w.N, 3))
        Ff = np.zeros((w.N, 3))
        e = R.rbsog_forces_split(c.h, Fn, Ff, energy=True)
        rho = R.rbsog_get_rho(c.h, c.P)
        m_used, coef = R.rbsog_get_ksample(c.h, c.P)
        sog = R.rbsog_get_sog(c.h)
        cells = R.rbsog_get_cells(c.h, w.N)
    return dict(Fn=Fn, Ff=Ff, e=e, rho=rho, m=m_used, coef=coef, sog=sog, cells=cells)


@pytest.mark.parametrize("prec", PRECS)
def test_small_workload_parity(prec):
    """N=1000, L=10, Gamma=1, kappa=1, r_c=3.5a, P=100: near, far, total, rho, coef, energies."""
    w = W.cfg_small_fp64()
    r = W.positions(w)
    q = W.charges(w)
    modes = modes_for(w, w.P, 11)
    g = run_forces(w, prec, r, modes)
    assert np.array_equal(g["m"], modes)
    Ft, Fn, Ff, e, S_ = oracle_forces(w, r, q, modes)
    tol = TOL[prec]
    # S sums ~1e5 lattice terms in a different order on each side
    assert abs(g["sog"]["S"] - S_) <= 1e-11 * S_
    check_forces(g["Fn"], Fn, tol, "near")
    check_forces(g["Ff"], Ff, tol, "far")
    check_forces(g["Fn"] + g["Ff"], Ft, tol, "total")
    rho = core.rho(r, q, w.box, modes)
    check_rho(g["rho"], rho, q, tol)
    coef = core.rb_coef(modes, w.box, oracle_sog(w), w.kT, float(np.sum(q * q)), S_)
    assert np.max(np.abs(g["coef"] - coef) / coef) <= 1e-11
    for k_gpu, k_or in (("U_near", "U_N"), ("U_far", "U_F"), ("U_self", "U_self")):
        check_energy(g["e"][k_gpu], e[k_or], tol, k_gpu)


@pytest.mark.parametrize("prec", PRECS)
def test_cell_list_is_bit_exact(prec):
    w = W.cfg_small_fp64()
    r = W.positions(w)
    # edge cases: origin, cell faces (exact in binary for L=10, n=4), L - ulp, negative, beyond L
    r[0] = [0.0, 0.0, 0.0]
    r[1] = [2.5, 5.0, 7.5]
    r[2] = [np.nextafter(10.0, 0.0)] * 3
    r[3] = [-2.5, 12.5, 10.0]
    g = run_forces(w, prec, r, modes_for(w, w.P, 3))
    nc, start, perm = g["cells"]
    nco = core.n_cells(w.box, w.r_c)
    assert list(nc) == list(nco)
    _, start_o, perm_o = core.cell_list(r, w.box, nco)
    assert np.array_equal(start, start_o)
    assert np.array_equal(perm, perm_o)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["tiny", "ragged", "one_cell", "noncubic", "mixed", "P1", "Pmany", "dense"])
def test_edge_cases(prec, case):
    kw = {}
    q = None
    if case == "tiny":
        w = workload(2, 4.0, rc=1.9, P=8)
    elif case == "ragged":
        w = workload(1237, 11.0, P=37)
    elif case == "one_cell":       # fewer than 3 cells per axis: one cell spans the box
        w = workload(300, 4.0, rc=1.9, P=50)
    elif case == "noncubic":
        w = workload(900, 0, box=(8.0, 11.0, 13.5), P=70, rc=2.0)
    elif case == "mixed":
        w = workload(800, 9.0, P=64)
        q = np.random.default_rng(5).choice([-1.0, 1.0, 2.0], size=800)
    elif case == "P1":
        w = workload(500, 8.0, P=1)
    elif case == "Pmany":          # several passes of the structure-factor kernel
        w = workload(700, 9.0, P=1500)
    else:                          # dense cells (strong overlap of neighbour lists)
        w = workload(3000, 6.0, rc=2.0, P=40)
    r = W.positions(w)
    qq = W.charges(w) if q is None else q
    modes = modes_for(w, w.P, 21)
    g = run_forces(w, prec, r, modes, q=q)
    Ft, Fn, Ff, e, S_ = oracle_forces(w, r, qq, modes, near="images" if case == "one_cell" else "cells")
    tol = TOL[prec]
    check_forces(g["Fn"] + g["Ff"], Ft, tol, "total")
    check_forces(g["Ff"], Ff, tol, "far")
    if np.any(Fn != 0):
        check_forces(g["Fn"], Fn, tol, "near")
    check_rho(g["rho"], core.rho(r, qq, w.box, modes), qq, tol)
    for k_gpu, k_or in (("U_near", "U_N"), ("U_far", "U_F")):
        if e[k_or] != 0:
            check_energy(g["e"][k_gpu], e[k_or], tol, k_gpu)


@pytest.mark.parametrize("nc", [3, 4, 5, 6, 7, 9, 12])
def test_near_field_all_tile_geometries(nc):
    """FP32 near field (shared-memory tiles) for 3..12 cells per axis, which makes the staged
    neighbourhood span the whole periodic row for small counts, against the oracle."""
    rc = 1.5
    L = nc * rc * 1.05
    w = workload(int(0.5 * L ** 3), L, rc=rc, P=16, seed=nc)
    r = W.positions(w)
    g = run_forces(w, R.RBSOG_FP32, r, modes_for(w, w.P, 1))
    assert list(g["cells"][0]) == [nc] * 3
    Ft, Fn, Ff, e, S_ = oracle_forces(w, r, W.charges(w), modes_for(w, w.P, 1))
    check_forces(g["Fn"], Fn, FP32_TOL, "near")
    # a missing or extra pair shows up as an error of the order of that pair's force; FP32
    # rounding stays orders of magnitude below 1e-3 of the force scale
    rms = float(np.sqrt(np.mean(np.sum(Fn * Fn, axis=1))))
    worst = np.max(np.linalg.norm(g["Fn"] - Fn, axis=1) / (np.linalg.norm(Fn, axis=1) + 0.1 * rms))
    assert worst <= 1e-3, worst


@pytest.mark.parametrize("ncells,occ", [((12, 3, 3), 2.0), ((5, 4, 7), 6.5), ((20, 6, 5), 3.0), ((3, 12, 4), 6.5),
                                         ((9, 9, 3), 1.0), ((7, 5, 13), 9.0), ((6, 6, 6), 24.0)],
                         ids=["x12y3z3", "x5y4z7", "x20y6z5", "x3y12z4", "x9y9z3", "x7y5z13", "dense6"])
def test_near_field_brick_geometries(ncells, occ):
    """FP32 near field of one system in bricks of up to 2 x 4 rows: boxes of 3 to 20 cells
    per axis (bricks with fewer rows, seams along every axis, one brick spanning a whole
    axis) and a dense one whose neighbourhood exceeds the staging buffer (the per-particle
    fallback), against the oracle, with the missing-pair check."""
    rc = 1.5
    box = tuple(n * rc * 1.03 for n in ncells)
    N = int(occ * ncells[0] * ncells[1] * ncells[2])
    w = workload(N, None, rc=rc, P=16, seed=sum(ncells), box=box)
    r = W.positions(w)
    g = run_forces(w, R.RBSOG_FP32, r, modes_for(w, w.P, 2))
    assert list(g["cells"][0]) == list(ncells)
    Ft, Fn, Ff, e, S_ = oracle_forces(w, r, W.charges(w), modes_for(w, w.P, 2))
    check_forces(g["Fn"], Fn, FP32_TOL, ("near", ncells))
    check_energy(g["e"]["U_near"], e["U_N"], FP32_TOL, ("U_near", ncells))
    rms = float(np.sqrt(np.mean(np.sum(Fn * Fn, axis=1))))
    worst = np.max(np.linalg.norm(g["Fn"] - Fn, axis=1) / (np.linalg.norm(Fn, axis=1) + 0.1 * rms))
    assert worst <= 1e-3, worst


def test_host_and_device_pointers_agree(gpu):
    torch = gpu
    w = workload(600, 8.0, P=32)
    r = W.positions(w)
    modes = modes_for(w, w.P, 2)
    with Ctx(w, R.RBSOG_FP64) as c:
        R.rbsog_set_state(c.h, r)
        R.rbsog_set_ksample(c.h, modes)
        F_host = np.zeros((w.N, 3))
        R.rbsog_forces(c.h, F_host)
        rd = torch.tensor(r, device="cuda", dtype=torch.float64)
        R.rbsog_set_state(c.h, rd)
        R.rbsog_set_ksample(c.h, modes)
        Fd = torch.zeros((w.N, 3), device="cuda", dtype=torch.float64)
        R.rbsog_forces(c.h, Fd, energy=True)
        assert np.array_equal(Fd.cpu().numpy(), F_host)


@pytest.mark.parametrize("prec", PRECS)
def test_scaled_strong_coupling_bcc(prec):
    """bcc lattice, Gamma=100, kappa=0.5, r_c=4a, P=200 at 8^3 cells (N=1024)."""
    base = W.cfg_bcc_fp32()
    nc = 8
    N = 2 * nc ** 3
    L = W.box_for_unit_a(N)
    import dataclasses
    w = dataclasses.replace(base, N=N, box=(L, L, L), bcc_cells=nc, name="bcc8")
    r = W.positions(w)
    modes = modes_for(w, w.P, 5)
    g = run_forces(w, prec, r, modes)
    Ft, Fn, Ff, e, S_ = oracle_forces(w, r, W.charges(w), modes)
    check_forces(g["Fn"] + g["Ff"], Ft, TOL[prec], "total")
    check_forces(g["Fn"], Fn, TOL[prec], "near")
    check_energy(g["e"]["U_near"], e["U_N"], TOL[prec], "U_near")


def cell_rows(r, box, r_c, rows):
    """Particles of whole rows of the cell list: (c_y, c_z) fixed, every c_x."""
    nc = core.n_cells(box, r_c)
    cell_of, _, _ = core.cell_list(r, box, nc)
    cy = (cell_of // nc[0]) % nc[1]
    cz = cell_of // (nc[0] * nc[1])
    sel = np.zeros(len(r), dtype=bool)
    for y, z in rows:
        sel |= (cy == y) & (cz == z)
    return np.nonzero(sel)[0]


def test_full_size_uniform_fp32_sampled():
    """N=1e6 uniform, Gamma=0.1, kappa=2, r_c=3a, P=500 in the FP32 build: rho over all
    particles (every mode), and the total, near and far forces on three whole rows of the
    cell list (one through the periodic corner, one through the middle, one on a face)
    plus 256 sampled particles against the oracle."""
    w = W.cfg_large()
    r = W.positions(w)
    q = W.charges(w)
    modes = modes_for(w, w.P, 17)
    with Ctx(w, R.RBSOG_FP32) as c:
        R.rbsog_set_state(c.h, r)
        R.rbsog_set_ksample(c.h, modes)
        Fn = np.zeros((w.N, 3))
        Ff = np.zeros((w.N, 3))
        R.rbsog_forces_split(c.h, Fn, Ff)
        rho_g = R.rbsog_get_rho(c.h, c.P)
        S_g = R.rbsog_get_sog(c.h)["S"]
    rho = core.rho(r, q, w.box, modes)
    check_rho(rho_g, rho, q, FP32_TOL)
    nc = int(core.n_cells(w.box, w.r_c)[1])
    rows = cell_rows(r, w.box, w.r_c, [(0, 0), (nc // 2, nc // 2), (nc - 1, nc // 3)])
    assert len(rows) > 900
    idx = np.unique(np.concatenate([rows, np.random.default_rng(0).choice(w.N, 256, replace=False)]))
    Ft, Fno, Ffo, e, S_ = oracle_forces(w, r, q, modes, idx=idx, rho=rho)
    # ~1e8 lattice terms summed in a different order on each side
    assert abs(S_g - S_) <= 1e-11 * S_
    check_forces(Fn[idx] + Ff[idx], Ft, FP32_TOL, "total")
    check_forces(Fn[idx], Fno, FP32_TOL, "near")
    check_forces(Ff[idx], Ffo, FP32_TOL, "far")
