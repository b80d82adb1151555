"""ctypes bindings to the oracle's C core plus the composite oracle quantities.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Composite quantities (all FP64, paper notation):
  U_self  = -1/2 sum_i q_i^2 F(0)                                     Eq. (52)
  coef_l  = S / (P V calF(k_l))          so that F*_i = -q_i sum_l coef_l k_l Im(e^{-ik_l.r_i} rho_l)
  U*_F    = sum_l coef_l |rho_l|^2 / 2 + Fhat(0) (sum q)^2 / (2V)     Eq. (60) + the k = 0 term
  kmax2   = 4 b_max ln(1e17), b_max = max_m e^{t_m}: the k-space sums drop terms below
            1e-17 of Fhat's scale.
The k = 0 mode carries no force; its energy term is added deterministically and it
is excluded from the sampled support.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build
from .sog import SOG

_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.intc, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        i64, d, vp = C.c_int64, C.c_double, C.c_void_p
        L.orc_sog_F.argtypes = [_dp, d]; L.orc_sog_F.restype = d
        L.orc_force_n2.argtypes = [_dp, d]; L.orc_force_n2.restype = d
        L.orc_fhat.argtypes = [_dp, d]; L.orc_fhat.restype = d
        L.orc_calF.argtypes = [d, d, d, d, d]; L.orc_calF.restype = d
        L.orc_fixed_point.argtypes = [i64, _dp, _dp, vp, vp]
        L.orc_cell_list.argtypes = [i64, _dp, _dp, _ip, _u32p, _u32p, _u32p]
        L.orc_near_images.argtypes = [i64, _dp, _dp, _dp, d, _dp, i64, vp, _dp, C.POINTER(d)]
        L.orc_near_cells.argtypes = [i64, _dp, _dp, _dp, d, _dp, _ip, _u32p, _u32p, _u32p, i64, vp, _dp,
                                     C.POINTER(d)]
        L.orc_rho.argtypes = [i64, _dp, _dp, _dp, C.c_int, _i32p, _dp]
        L.orc_far_rb.argtypes = [i64, _dp, _dp, _dp, C.c_int, _i32p, _dp, _dp, i64, vp, _dp]
        L.orc_far_full.argtypes = [i64, _dp, _dp, _dp, _dp, d, _dp, C.POINTER(d)]
        L.orc_S_sum.argtypes = [_dp, _dp, d, d, d, C.c_int]; L.orc_S_sum.restype = d
        L.orc_measure.argtypes = [C.c_int, d, d, d, d, d]; L.orc_measure.restype = d
        L.orc_real_far.argtypes = [i64, _dp, _dp, _dp, _dp, C.c_int, _dp, C.POINTER(d)]
        L.orc_brute_yukawa.argtypes = [i64, _dp, _dp, _dp, d, d, _dp, C.POINTER(d)]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = None
        _lib = L
    return _lib


def _f64(x, shape=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _idx(idx):
    if idx is None:
        return None, None
    arr = np.ascontiguousarray(idx, dtype=np.int64)
    return arr, arr.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """Thread count of the C core's parallel loops (used by timing legs)."""
    lib().orc_set_threads(int(n))


# ---- scalar kernel pieces (C) ----
def sog_F(sog: SOG, r: float) -> float:
    return lib().orc_sog_F(sog.as_array(), float(r))


def force_n2(sog: SOG, r: float) -> float:
    return lib().orc_force_n2(sog.as_array(), float(r))


def fhat(sog: SOG, k2: float) -> float:
    return lib().orc_fhat(sog.as_array(), float(k2))


def calF(k2: float, kT: float, V: float, Q2: float, lam: float) -> float:
    return lib().orc_calF(float(k2), float(kT), float(V), float(Q2), float(lam))


# sampling measures of Eq. (59): adaptive calF of Eq. (62), calF = 1, calF = k^2, and Eq. (62)
# with the Debye wavenumber of Gaussian units (4 pi sum q^2 / (kT V))
ADAPTIVE, UNIFORM, K2, DEBYE = 0, 1, 2, 3


def measure(kind: int, k2: float, kT: float, V: float, Q2: float, lam: float) -> float:
    return lib().orc_measure(int(kind), float(k2), float(kT), float(V), float(Q2), float(lam))


def kmax2_of(sog: SOG) -> float:
    return 4.0 * float(np.max(np.exp(sog.t))) * math.log(1e17)


# ---- cell list ----
def n_cells(L, rc) -> np.ndarray:
    """Cells per axis: floor(L_a / r_c) when that is at least 3, else a single cell."""
    out = []
    for La in L:
        n = int(math.floor(float(La) / float(rc)))
        out.append(n if n >= 3 else 1)
    return np.asarray(out, dtype=np.intc)


def fixed_point(r, L):
    r = _f64(r, (-1, 3))
    N = r.shape[0]
    s32 = np.zeros((N, 3), dtype=np.uint32)
    s64 = np.zeros((N, 3), dtype=np.uint64)
    lib().orc_fixed_point(N, r, _f64(L), s32.ctypes.data_as(C.c_void_p), s64.ctypes.data_as(C.c_void_p))
    return s32, s64


def cell_list(r, L, nc):
    r = _f64(r, (-1, 3))
    N = r.shape[0]
    nc = np.ascontiguousarray(nc, dtype=np.intc)
    ncell = int(nc[0]) * int(nc[1]) * int(nc[2])
    cell_of = np.zeros(N, dtype=np.uint32)
    start = np.zeros(ncell + 1, dtype=np.uint32)
    perm = np.zeros(N, dtype=np.uint32)
    lib().orc_cell_list(N, r, _f64(L), nc, cell_of, start, perm)
    return cell_of, start, perm


# ---- forces and energies ----
def near_images(r, q, L, rc, sog: SOG, idx=None):
    r = _f64(r, (-1, 3)); q = _f64(q)
    ia, ip = _idx(idx)
    n_out = r.shape[0] if ia is None else ia.size
    F = np.zeros((n_out, 3)); U = C.c_double(0.0)
    lib().orc_near_images(r.shape[0], r, q, _f64(L), float(rc), sog.as_array(), n_out, ip, F, C.byref(U))
    return F, U.value


def near_cells(r, q, L, rc, sog: SOG, idx=None):
    r = _f64(r, (-1, 3)); q = _f64(q)
    nc = n_cells(L, rc)
    cell_of, start, perm = cell_list(r, L, nc)
    ia, ip = _idx(idx)
    n_out = r.shape[0] if ia is None else ia.size
    F = np.zeros((n_out, 3)); U = C.c_double(0.0)
    lib().orc_near_cells(r.shape[0], r, q, _f64(L), float(rc), sog.as_array(), nc, cell_of, start, perm,
                         n_out, ip, F, C.byref(U))
    return F, U.value


def rho(r, q, L, m):
    r = _f64(r, (-1, 3)); q = _f64(q)
    m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((m.shape[0], 2))
    lib().orc_rho(r.shape[0], r, q, _f64(L), m.shape[0], m, out)
    return out


def far_rb(r, q, L, m, coef, rho_, idx=None):
    r = _f64(r, (-1, 3)); q = _f64(q)
    m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
    ia, ip = _idx(idx)
    n_out = r.shape[0] if ia is None else ia.size
    F = np.zeros((n_out, 3))
    lib().orc_far_rb(r.shape[0], r, q, _f64(L), m.shape[0], m, _f64(coef), _f64(rho_, (-1, 2)), n_out, ip, F)
    return F


def far_full(r, q, L, sog: SOG, kmax2=None):
    r = _f64(r, (-1, 3)); q = _f64(q)
    kmax2 = kmax2_of(sog) if kmax2 is None else float(kmax2)
    F = np.zeros_like(r); U = C.c_double(0.0)
    lib().orc_far_full(r.shape[0], r, q, _f64(L), sog.as_array(), kmax2, F, C.byref(U))
    return F, U.value


def S_sum(L, sog: SOG, kT, Q2, kmax2=None, kind: int = ADAPTIVE):
    """S = sum_{k != 0} calF(k) Fhat(k) for the measure `kind` (Eq. 59)."""
    kmax2 = kmax2_of(sog) if kmax2 is None else float(kmax2)
    return lib().orc_S_sum(_f64(L), sog.as_array(), float(kT), float(Q2), kmax2, int(kind))


def real_far(r, q, L, sog: SOG, nimg: int):
    r = _f64(r, (-1, 3)); q = _f64(q)
    F = np.zeros_like(r); U = C.c_double(0.0)
    lib().orc_real_far(r.shape[0], r, q, _f64(L), sog.as_array(), int(nimg), F, C.byref(U))
    return F, U.value


def brute_yukawa(r, q, L, lam, rcut):
    r = _f64(r, (-1, 3)); q = _f64(q)
    F = np.zeros_like(r); U = C.c_double(0.0)
    lib().orc_brute_yukawa(r.shape[0], r, q, _f64(L), float(lam), float(rcut), F, C.byref(U))
    return F, U.value


def self_energy(q, sog: SOG) -> float:
    """Eq. (52)."""
    q = _f64(q)
    return -0.5 * float(np.sum(q * q)) * sog_F(sog, 0.0)


def rb_coef(m, L, sog: SOG, kT, Q2, S, P=None, kind: int = ADAPTIVE):
    """coef_l = S / (P V calF(k_l)) for the modes m (Eq. 60 with P(k) of Eq. 59), calF of
    the measure `kind`."""
    m = np.asarray(m, dtype=np.float64).reshape(-1, 3)
    P = m.shape[0] if P is None else P
    V = (float(L[0]) * float(L[1])) * float(L[2])
    out = np.empty(m.shape[0])
    for l in range(m.shape[0]):
        k = [2.0 * math.pi * m[l, a] / float(L[a]) for a in range(3)]
        k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2]
        out[l] = S / (P * V * measure(kind, k2, kT, V, Q2, sog.lam))
    return out


def rb_energy(rho_, coef, q, L, sog: SOG) -> float:
    """U*_F = sum_l coef_l |rho_l|^2 / 2 + Fhat(0) (sum q)^2 / (2V)."""
    rho_ = _f64(rho_, (-1, 2))
    V = (float(L[0]) * float(L[1])) * float(L[2])
    qs = float(np.sum(q))
    return float(np.sum(0.5 * _f64(coef) * (rho_[:, 0] ** 2 + rho_[:, 1] ** 2))) + fhat(sog, 0.0) * qs * qs / (2.0 * V)


def rb_forces(r, q, L, rc, sog: SOG, m, kT, S=None, near="cells", idx=None, rho_=None, kind: int = ADAPTIVE):
    """Total force (near + random-batch far) on the k-set m and the energy terms.

    Returns (F_total, F_near, F_far, energies) with energies = dict(U_N, U_F, U_self).
    U_N is the full near energy only when idx is None.
    """
    q = _f64(q)
    Q2 = float(np.sum(q * q))
    if S is None:
        S = S_sum(L, sog, kT, Q2, kind=kind)
    coef = rb_coef(m, L, sog, kT, Q2, S, kind=kind)
    if rho_ is None:
        rho_ = rho(r, q, L, m)
    Ff = far_rb(r, q, L, m, coef, rho_, idx=idx)
    Fn, UN = (near_cells if near == "cells" else near_images)(r, q, L, rc, sog, idx=idx)
    e = dict(U_N=UN, U_F=rb_energy(rho_, coef, q, L, sog), U_self=self_energy(q, sog))
    return Fn + Ff, Fn, Ff, e


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = float(np.sqrt(np.sum(b * b)))
    return float(np.sqrt(np.sum((a - b) ** 2))) / den if den > 0 else float(np.sqrt(np.sum(a * a)))
