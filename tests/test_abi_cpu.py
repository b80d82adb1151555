"""Host-side checks of the C-ABI library that need no GPU: it builds and loads, exports
every entry point include/rbsog.h declares, rejects invalid parameters before touching a
device, and its host-side SOG construction (Algorithm 1) agrees with the oracle's."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import sog as S
from paper_2501_10946_gb300 import rbsog as R
from paper_2501_10946_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rbsog.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rbsog_\w+)\s*\(", txt)))


def test_library_exports_every_declared_function():
    lib = R.load()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(R.EXPORTS) == names


@pytest.mark.parametrize("struct", [R.rbsog_params, R.rbsog_energy, R.rbsog_server_config, R.rbsog_job_info])
def test_struct_layouts_match_the_c_header(tmp_path, struct):
    """ctypes mirrors of the ABI structs against the C compiler's own layout."""
    name = struct.__name__
    src = tmp_path / "layout.c"
    fields = [f for f, _ in struct._fields_]
    body = [f'printf("%zu\\n", sizeof({name}));']
    body += [f'printf("%zu\\n", offsetof({name}, {f}));' for f in fields]
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rbsog.h"\nint main(void){' +
                   "".join(body) + "return 0;}\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    vals = [int(x) for x in out]
    assert vals[0] == C.sizeof(struct)
    assert vals[1:] == [getattr(struct, f).offset for f in fields]


def base_params():
    w = W.cfg_small_fp64()
    return w, R.make_params(w, precision=R.RBSOG_FP64)


@pytest.mark.parametrize("field,value", [("r_c", 6.0), ("P", 0), ("P", 5000), ("kappa", 0.0), ("precision", 7),
                                         ("ensemble", 3), ("sog_mode", 9), ("sampling", 4), ("sampling", -1),
                                         ("dt", -1.0), ("egs_nu", -0.1), ("egs_nu", 0.97)])
def test_invalid_parameters_are_rejected_on_the_host(field, value):
    w, p = base_params()
    setattr(p, field, value)
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_init(p, w.N, W.charges(w), W.masses(w))
    assert R.rbsog_last_error(None)


def test_state_entry_points_reject_a_null_context():
    """The state and force entry points check their context and pointers on the host."""
    F = np.zeros((4, 3))
    calls = [lambda: R.rbsog_set_state(None, F, F), lambda: R.rbsog_set_state_forces(None, F, F, F),
             lambda: R.rbsog_get_state(None, F, F), lambda: R.rbsog_get_forces(None, F),
             lambda: R.rbsog_set_state_forces_f32(None, F, F, F.astype(np.float32)),
             lambda: R.rbsog_get_forces_f32(None, F.astype(np.float32))]
    for call in calls:
        with pytest.raises(R.RbsogError, match="EINVAL"):
            call()


def test_egs_screening_rejects_a_table_of_one_kernel():
    """The EGS screening builds one SOG per Yukawa term, so a given (M1, M2) is refused."""
    w, p = base_params()
    p.egs_nu = 0.5
    p.sog_mode = R.RBSOG_SOG_TABLE
    p.sog_M1, p.sog_M2 = 4, 0
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_init(p, w.N, W.charges(w), W.masses(w))


def test_invalid_sizes_are_rejected():
    w, p = base_params()
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_init(p, 1, np.ones(1), np.ones(1))
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_init(p, 4, np.ones(4), np.array([1.0, 0.0, 1.0, 1.0]))
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_init(p, 4, np.zeros(4), np.ones(4))


def test_sog_table_mode_reproduces_table1_through_the_abi():
    gold = os.path.join(os.path.dirname(__file__), "golden", "table1_c1_sog.txt")
    for line in open(gold):
        if line.startswith("#") or not line.strip():
            continue
        e, h, t0, m1, m2, mt, w = line.split()
        a = R.rbsog_build_sog(0.5773, 5 * 0.5773, float(e), R.RBSOG_SOG_TABLE, int(m1), int(m2))
        assert abs(a["h"] - float(h)) <= 1e-15
        assert abs(a["t0"] - float(t0)) <= (1e-13 if float(e) >= 1e-5 else 1e-6)
        assert abs(a["w"] - float(w)) <= 1e-8 * float(w)
        assert a["max_error"] <= float(e)


@pytest.mark.parametrize("mode,name", [(R.RBSOG_SOG_MINIMAL, "minimal"), (R.RBSOG_SOG_BOUND, "bound")])
@pytest.mark.parametrize("eps", [1e-3, 1e-5, 1e-7, 1e-9, 1e-11, 1e-13])
def test_library_sog_equals_oracle_sog(mode, name, eps):
    """Same (M1, M2) and the same C1 root.  The residual of Eq. 36 is flat near its root for
    tight eps, so t0 is defined only up to rounding; both sides evaluate Eqs. 36 and 38 as
    plain FP64 sums in the same operation order and land on the same bits."""
    lam, rc = 0.5773, 5 * 0.5773
    a = R.rbsog_build_sog(lam, rc, eps, mode)
    o = S.build(lam, rc, eps, name)
    assert (a["M1"], a["M2"]) == (o.M1, o.M2)
    assert abs(a["h"] - o.h) <= 1e-15
    assert abs(a["t0"] - o.t0) <= 1e-15 and abs(a["w"] - o.w) <= 1e-14 * abs(o.w)
    lib = S.SOG(lam, rc, eps, a["h"], a["t0"], a["M1"], a["M2"], a["w"])
    assert lib.max_error() <= eps
    dy = float(S.dyukawa(rc, lam))
    assert abs(float(lib.dF(rc)) - dy) <= 1e-12 * abs(dy)


@pytest.mark.parametrize("wl", [W.cfg_small_fp64, W.cfg_bcc_fp32, W.cfg_large], ids=lambda f: f.__name__)
def test_library_sog_equals_oracle_on_workloads(wl):
    w = wl()
    lam = w.a_ws / w.kappa
    a = R.rbsog_build_sog(lam, w.r_c, w.sog_eps)
    o = S.build(lam, w.r_c, w.sog_eps)
    assert (a["M1"], a["M2"]) == (o.M1, o.M2)
    assert abs(a["t0"] - o.t0) <= 1e-13 and abs(a["w"] - o.w) <= 1e-13


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(R, "_lib", None)
    monkeypatch.setattr(R._build, "LIB", str(tmp_path / "nope.so"))
    with pytest.raises(R.RbsogError):
        R.load(build_if_missing=False)


def test_batch_rejects_fp64_and_names_the_bad_system():
    """Host-side checks of rbsog_batch_init (no device call is reached)."""
    w, p = base_params()
    q, m = W.charges(w), W.masses(w)
    with pytest.raises(R.RbsogError, match="EUNSUPPORTED"):
        R.rbsog_batch_init([p], [w.N], q, m)
    good = R.make_params(w, precision=R.RBSOG_FP32)
    bad = R.make_params(w, precision=R.RBSOG_FP32)
    bad.kappa = 0.0
    with pytest.raises(R.RbsogError, match="EINVAL: system 1: kappa"):
        R.rbsog_batch_init([good, bad], [w.N, w.N], np.concatenate([q, q]), np.concatenate([m, m]))
    other_dev = R.make_params(w, precision=R.RBSOG_FP32, device=1)
    with pytest.raises(R.RbsogError, match="same device"):
        R.rbsog_batch_init([good, other_dev], [w.N, w.N], np.concatenate([q, q]), np.concatenate([m, m]))
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_batch_init([], [], q, m)
    assert R.rbsog_batch_last_error(None)


def test_server_config_is_checked_on_the_host():
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_server_create(R.make_server_config(1, 10, 10, 1))
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_server_create(R.make_server_config(1000, 10, 10, 0))
    cfg = R.make_server_config(1000, 10, 10, 1)
    cfg.reserved[1] = 3
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_server_create(cfg)
    assert "configuration" in R.rbsog_server_last_error(None)


def test_slab_split_owns_every_particle_once_and_finds_the_halo():
    """rbsog_slab_split (host only): the slabs' owned lists partition the particles; each
    slab's halo is exactly the particles of other slabs whose periodic distance to the slab
    along the axis is below the halo width."""
    from paper_2501_10946_gb300 import rbsog as R
    rng = np.random.default_rng(3)
    L = np.array([12.0, 9.0, 10.0])
    r = rng.uniform(-5.0, 20.0, size=(2000, 3))          # not wrapped: the split wraps
    for axis, nslabs, halo in ((0, 2, 2.5), (1, 3, 1.2), (2, 4, 2.0), (0, 1, 3.0)):
        w = L[axis] / nslabs
        x = np.mod(r[:, axis], L[axis])
        seen = np.zeros(len(r), dtype=int)
        for slab in range(nslabs):
            idx, n_owned = R.rbsog_slab_split(r, L, axis, nslabs, slab, halo)
            own, hal = idx[:n_owned], idx[n_owned:]
            assert np.all(np.diff(own) > 0) and np.all(np.diff(hal) > 0)
            seen[own] += 1
            lo, hi = slab * w, (slab + 1) * w
            inside = np.minimum(np.floor(x / w), nslabs - 1) == slab
            assert np.array_equal(np.sort(own), np.nonzero(inside)[0])
            d = np.minimum(np.mod(lo - x, L[axis]), np.mod(x - hi, L[axis]))
            expect = np.nonzero(~inside & (d < halo))[0] if nslabs > 1 else np.array([], dtype=int)
            assert np.array_equal(hal, expect), (axis, nslabs, slab)
        assert np.all(seen == 1)
    with pytest.raises(R.RbsogError, match="EINVAL"):
        R.rbsog_slab_split(r, L, 0, 2, 2, 1.0)
