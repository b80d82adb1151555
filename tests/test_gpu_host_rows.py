"""Caller rows [N][3] in and out of a context through the three kinds of buffer the C ABI
takes: pageable host memory (staged through a device buffer and a copy), pinned host
memory (read and written by the kernels through its mapped address) and device memory.
All three give the same bits, for a particle count whose last block of 256 rows is
ragged; uploaded states and forces come back in the caller's order (positions wrapped
into the box)."""
import numpy as np
import pytest

from gpu_common import Ctx, require_gpu, workload
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KINDS = ("pageable", "pinned", "device")
L = 16.0


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def put(torch, kind, a):
    """The array a in a buffer of the given kind."""
    a = np.ascontiguousarray(a)
    if kind == "pageable":
        return a.copy()
    t = torch.from_numpy(a.copy())
    return t.pin_memory() if kind == "pinned" else t.to("cuda")


def empty(torch, kind, shape, dtype):
    return put(torch, kind, np.zeros(shape, dtype=dtype))


def host(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else x


def case(ensemble="nve"):
    # 3001 particles: 11 full blocks of 256 rows and one of 185
    w = workload(3001, L, P=32, dt=0.005, ensemble=ensemble)
    r0 = W.positions(w).copy()
    # positions outside [0, L): within one box length, and one beyond
    r0[::7] -= L
    r0[::11] += L
    r0[5] += 3 * L
    return w, r0, W.velocities(w)


def read_all(torch, c, prec, kind, N):
    r = empty(torch, kind, (N, 3), np.float64)
    v = empty(torch, kind, (N, 3), np.float64)
    F = empty(torch, kind, (N, 3), np.float64)
    R.rbsog_get_state(c.h, r, v)
    R.rbsog_get_forces(c.h, F)
    out = [host(r), host(v), host(F)]
    if prec == R.RBSOG_FP32:
        F32 = empty(torch, kind, (N, 3), np.float32)
        R.rbsog_get_forces_f32(c.h, F32)
        out.append(host(F32))
    return out


@pytest.mark.parametrize("prec", [R.RBSOG_FP32, R.RBSOG_FP64])
def test_state_rows_every_buffer_kind(torch, prec):
    w, r0, v0 = case()
    N = w.N
    after = {}
    for kin in KINDS:
        with Ctx(w, prec) as c:
            R.rbsog_set_state(c.h, put(torch, kin, r0), put(torch, kin, v0))
            # before any step the rest order is the caller's: r wrapped, v as given
            for kout in KINDS:
                r = empty(torch, kout, (N, 3), np.float64)
                v = empty(torch, kout, (N, 3), np.float64)
                R.rbsog_get_state(c.h, r, v)
                r, v = host(r), host(v)
                assert np.all((r >= 0.0) & (r < L))
                d = np.abs(r - np.mod(r0, L))
                assert np.all(np.minimum(d, L - d) <= 1e-12 * L), (kin, kout)
                np.testing.assert_array_equal(v, v0)
            R.rbsog_step(c.h, 3)
            got = {k: read_all(torch, c, prec, k, N) for k in KINDS}
            for k in KINDS:
                for a, b in zip(got[k], got["pageable"]):
                    np.testing.assert_array_equal(a, b, err_msg=f"{kin} in, {k} out")
            after[kin] = got["pageable"]
    for k in KINDS:
        for a, b in zip(after[k], after["pageable"]):
            np.testing.assert_array_equal(a, b, err_msg=f"{k} in")


@pytest.mark.parametrize("prec", [R.RBSOG_FP32, R.RBSOG_FP64])
def test_force_rows_round_trip(torch, prec):
    """Forces uploaded with a state come back unchanged before any step (FP64 values into
    the FP32 build: rounded to FP32 once)."""
    w, r0, v0 = case()
    N = w.N
    F0 = np.random.default_rng(3).standard_normal((N, 3))
    for kin in KINDS:
        with Ctx(w, prec) as c:
            R.rbsog_set_state_forces(c.h, put(torch, kin, r0), put(torch, kin, v0), put(torch, kin, F0))
            want = F0.astype(np.float32).astype(np.float64) if prec == R.RBSOG_FP32 else F0
            for kout in KINDS:
                F = empty(torch, kout, (N, 3), np.float64)
                R.rbsog_get_forces(c.h, F)
                np.testing.assert_array_equal(host(F), want, err_msg=f"{kin} in, {kout} out")
            if prec == R.RBSOG_FP32:
                F32in = F0.astype(np.float32)
                R.rbsog_set_state_forces_f32(c.h, put(torch, kin, r0), put(torch, kin, v0), put(torch, kin, F32in))
                for kout in KINDS:
                    F = empty(torch, kout, (N, 3), np.float32)
                    R.rbsog_get_forces_f32(c.h, F)
                    np.testing.assert_array_equal(host(F), F32in, err_msg=f"{kin} in, {kout} out")


@pytest.mark.parametrize("prec,nsteps,ensemble", [(R.RBSOG_FP32, 1, "nve"), (R.RBSOG_FP32, 3, "nve"),
                                                   (R.RBSOG_FP64, 2, "nve"), (R.RBSOG_FP32, 2, "langevin")])
def test_step_get_equals_step_then_reads(torch, prec, nsteps, ensemble):
    """rbsog_step_get (positions read back beside the last step's force kernels) returns
    the bits of rbsog_step followed by rbsog_get_state and rbsog_get_forces(_f32), energies
    included, for every kind of buffer (velocity Verlet and BAOAB); the context continues
    from the same state."""
    w, r0, v0 = case(ensemble)
    N = w.N
    fdt = np.float32 if prec == R.RBSOG_FP32 else np.float64
    with Ctx(w, prec) as ref:
        R.rbsog_set_state(ref.h, r0, v0)
        e_ref = R.rbsog_step(ref.h, nsteps, energy=True)
        r_ref, v_ref = np.zeros((N, 3)), np.zeros((N, 3))
        R.rbsog_get_state(ref.h, r_ref, v_ref)
        F_ref = np.zeros((N, 3), dtype=fdt)
        (R.rbsog_get_forces_f32 if fdt == np.float32 else R.rbsog_get_forces)(ref.h, F_ref)
        e2_ref = R.rbsog_step(ref.h, 1, energy=True)
        for kind in KINDS:
            with Ctx(w, prec) as c:
                R.rbsog_set_state(c.h, r0, v0)
                r = empty(torch, kind, (N, 3), np.float64)
                v = empty(torch, kind, (N, 3), np.float64)
                F = empty(torch, kind, (N, 3), fdt)
                e = R.rbsog_step_get(c.h, nsteps, r, v, F, energy=True)
                np.testing.assert_array_equal(host(r), r_ref, err_msg=kind)
                np.testing.assert_array_equal(host(v), v_ref, err_msg=kind)
                np.testing.assert_array_equal(host(F), F_ref, err_msg=kind)
                assert e == e_ref, (kind, e, e_ref)
                assert R.rbsog_step(c.h, 1, energy=True) == e2_ref, kind


def test_step_get_refuses_zero_steps(torch):
    w, r0, v0 = case()
    with Ctx(w, R.RBSOG_FP32) as c:
        R.rbsog_set_state(c.h, r0, v0)
        with pytest.raises(R.RbsogError, match="EINVAL"):
            R.rbsog_step_get(c.h, 0, np.zeros((w.N, 3)))
