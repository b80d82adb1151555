"""Pins of the oracle's kernel pieces, far/near fields and cell list against closed forms,
brute-force sums and identities that do not use the code under test."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import core
from oracle import sog as S
from paper_2501_10946_gb300 import workloads as W

LAM = 0.6


@pytest.fixture(scope="module")
def sog7():
    return S.build(LAM, 2.4, 1e-7)


def test_fhat_is_the_3d_fourier_transform_of_F(sog7):
    """Eq. (54) against Lemma 3.6: Fhat(k) = 4 pi int_0^inf sin(kr)/k F(r) r dr."""
    for k in (0.0, 0.7, 2.0, 5.0):
        if k == 0.0:
            integrand = lambda r: 4.0 * math.pi * float(sog7.F(r)) * r * r
        else:
            integrand = lambda r: 4.0 * math.pi * math.sin(k * r) / k * float(sog7.F(r)) * r
        val, _ = quad(integrand, 0.0, 80.0, limit=800, epsabs=1e-14, epsrel=1e-12)
        assert abs(core.fhat(sog7, k * k) - val) <= 1e-9 * abs(core.fhat(sog7, 0.0))


def test_near_force_pieces_are_minus_gradient_of_near_kernel(sog7):
    """Eqs. (56)-(57): F_N1 + F_N2 = -(1/r) d/dr [Y - F] (central differences)."""
    for r in (0.2, 0.9, 1.7, 2.3):
        hstep = 1e-5
        def N(x):
            return float(S.yukawa(x, LAM)) - core.sog_F(sog7, x)
        dN = (N(r + hstep) - N(r - hstep)) / (2 * hstep)
        fn1 = math.exp(-r / LAM) * (1 + r / LAM) / r ** 3
        got = fn1 + core.force_n2(sog7, r)
        # near r_c the force itself is ~0 (C1), so scale the tolerance by F_N1's size
        assert abs(got - (-dN / r)) <= 1e-7 * abs(fn1)


def test_sog_F_c_equals_python(sog7):
    for r in (0.0, 0.5, 2.4, 7.0):
        assert abs(core.sog_F(sog7, r) - float(sog7.F(r))) <= 1e-15 * max(1.0, abs(float(sog7.F(r))))


def test_calF_limits():
    """Eq. (62): calF -> sum q^2 as k -> inf; Coulomb limit (lambda -> inf) gives kT V k^2 + O(k^4)."""
    kT, V, Q2 = 0.7, 100.0, 50.0
    assert abs(core.calF(1e12, kT, V, Q2, 0.5) - Q2) <= 1e-9 * Q2
    for k in (1e-3, 3e-3):
        got = core.calF(k * k, kT, V, Q2, 1e9)
        assert abs(got - kT * V * k * k) <= 1e-3 * kT * V * k * k
    ks = np.linspace(0.01, 20, 200)
    vals = [core.calF(k * k, kT, V, Q2, 0.5) for k in ks]
    assert all(np.diff(vals) > 0) and max(vals) <= Q2


def small_system(N=24, L=5.0, seed=5, mix=False):
    r, q = W.small_system(N, L, seed, charge_mix=mix)
    return r, q, [L, L, L]


@pytest.mark.parametrize("mix", [False, True])
def test_poisson_identity_far_field(sog7, mix):
    """Eq. (53): the k-space far energy and force equal the real-space image sum of F."""
    r, q, L = small_system(mix=mix)
    Fk, Uk = core.far_full(r, q, L, sog7)
    Fr, Ur = core.real_far(r, q, L, sog7, nimg=6)
    assert abs(Uk - Ur) <= 1e-12 * abs(Ur)
    assert core.rel_l2(Fk, Fr) <= 1e-11


def test_far_rb_with_all_modes_equals_full(sog7):
    """With every mode and coef = Fhat/V the estimator of Eq. (60) is the sum of Eq. (55)."""
    r, q, L = small_system(N=12)
    kmax2 = core.kmax2_of(sog7)
    nm = int(math.sqrt(kmax2) * L[0] / (2 * math.pi)) + 1
    g = np.arange(-nm, nm + 1)
    m = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k2 = np.sum((2 * math.pi * m / L[0]) ** 2, axis=1)
    m = m[k2 <= kmax2]
    V = L[0] ** 3
    coef = np.array([core.fhat(sog7, float(x)) / V for x in np.sum((2 * math.pi * m / L[0]) ** 2, axis=1)])
    rho = core.rho(r, q, L, m)
    Frb = core.far_rb(r, q, L, m, coef, rho)
    Ffull, Ufull = core.far_full(r, q, L, sog7)
    assert core.rel_l2(Frb, Ffull) <= 1e-12
    qs = float(np.sum(q))
    U = float(np.sum(0.5 * coef * (rho[:, 0] ** 2 + rho[:, 1] ** 2))) + core.fhat(sog7, 0.0) * qs * qs / (2 * V)
    assert abs(U - Ufull) <= 1e-12 * abs(Ufull)


def test_rho_of_a_single_particle():
    """rho(k) of one unit charge at r is exp(i k.r)."""
    L = [3.0, 4.0, 5.0]
    r = np.array([[0.3, 1.1, 4.2]])
    m = np.array([[1, 0, 0], [0, -2, 1], [3, 1, -1]], dtype=np.int32)
    rho = core.rho(r, [2.0], L, m)
    for l in range(3):
        th = sum(2 * math.pi * m[l, a] / L[a] * r[0, a] for a in range(3))
        assert abs(rho[l, 0] - 2 * math.cos(th)) < 1e-14 and abs(rho[l, 1] - 2 * math.sin(th)) < 1e-14


@pytest.mark.parametrize("eps", [1e-4, 1e-7, 1e-10, 1e-13])
@pytest.mark.parametrize("mix", [False, True])
def test_decomposition_matches_brute_force_lattice_sum(eps, mix):
    """T2: U_N + U_F + U_self and F_N + F_F against the brute-force periodic Yukawa sum;
    the error tracks the SOG tolerance eps (Thm 3.7)."""
    r, q, L = small_system(N=20, seed=11, mix=mix)
    rc = 2.4
    sg = S.build(LAM, rc, eps)
    Fn, Un = core.near_images(r, q, L, rc, sg)
    Ff, Uf = core.far_full(r, q, L, sg)
    Us = core.self_energy(q, sg)
    Fb, Ub = core.brute_yukawa(r, q, L, LAM, 40 * LAM)
    ferr = core.rel_l2(Fn + Ff, Fb)
    uerr = abs(Un + Uf + Us - Ub) / abs(Ub)
    assert ferr <= 300 * eps and uerr <= 300 * eps, (ferr, uerr)
    if eps <= 1e-13:
        assert ferr <= 1e-10


def test_S_closed_form_in_the_hot_limit(sog7):
    """kT -> inf gives calF = sum q^2, so S = Q2 (V sum_n F(|n L|) - Fhat(0)) by Poisson summation."""
    L = [5.0, 5.0, 5.0]
    Q2 = 7.0
    S_num = core.S_sum(L, sog7, 1e18, Q2)
    nimg = 6
    acc = 0.0
    for nx in range(-nimg, nimg + 1):
        for ny in range(-nimg, nimg + 1):
            for nz in range(-nimg, nimg + 1):
                acc += core.sog_F(sog7, 5.0 * math.sqrt(nx * nx + ny * ny + nz * nz))
    S_ref = Q2 * (125.0 * acc - core.fhat(sog7, 0.0))
    assert abs(S_num - S_ref) <= 1e-12 * abs(S_ref)


def test_near_cells_equals_near_images(sog7):
    r, q, L = small_system(N=200, L=8.0, seed=3, mix=True)
    F1, U1 = core.near_images(r, q, L, 2.4, sog7)
    F2, U2 = core.near_cells(r, q, L, 2.4, sog7)
    assert core.rel_l2(F2, F1) <= 1e-14 and abs(U1 - U2) <= 1e-13 * abs(U1)
    idx = np.array([0, 17, 199])
    F3, _ = core.near_cells(r, q, L, 2.4, sog7, idx=idx)
    assert np.allclose(F3, F1[idx], rtol=0, atol=1e-13 * np.abs(F1).max())


def test_cell_list_is_a_stable_counting_sort():
    L = [8.0, 8.0, 8.0]
    nc = np.array([4, 4, 4], dtype=np.intc)
    r = np.random.default_rng(1).uniform(0, 8.0, size=(500, 3))
    # edge cases: the origin, a point on cell faces, L - ulp, a tiny negative value, exactly L
    r[0] = [0.0, 0.0, 0.0]
    r[1] = [2.0, 4.0, 6.0]
    r[2] = [np.nextafter(8.0, 0.0)] * 3
    r[3] = [-1e-300, 8.0, 1.9999999999999998]
    cell_of, start, perm = core.cell_list(r, L, nc)
    assert sorted(perm.tolist()) == list(range(500))
    assert start[0] == 0 and start[-1] == 500 and np.all(np.diff(start.astype(np.int64)) >= 0)
    for c in range(64):
        seg = perm[start[c]:start[c + 1]]
        assert np.all(np.diff(seg.astype(np.int64)) > 0)
        assert np.all(cell_of[seg] == c)
    # exact rational cell of the edge cases: floor(frac(r/L) * n)
    assert cell_of[0] == 0
    assert cell_of[1] == 1 + 4 * (2 + 4 * 3)
    assert cell_of[2] == 3 + 4 * (3 + 4 * 3)
    assert cell_of[3] == 0 + 4 * (0 + 4 * 0)
    # every particle: cell = floor(r/L * n) for interior points (exact in binary for this L)
    inner = np.arange(4, 500)
    c3 = np.floor(r[inner] / 8.0 * 4).astype(np.int64)
    assert np.all(cell_of[inner] == c3[:, 0] + 4 * (c3[:, 1] + 4 * c3[:, 2]))


def test_fixed_point_definition():
    L = [10.0, 10.0, 10.0]
    r = np.array([[0.0, 5.0, 2.5], [-2.5, 12.5, 10.0]])
    s32, s64 = core.fixed_point(r, L)
    assert s32[0].tolist() == [0, 1 << 31, 1 << 30]
    assert s32[1].tolist() == [3 << 30, 1 << 30, 0]
    assert s64[0].tolist() == [0, 1 << 63, 1 << 62]
