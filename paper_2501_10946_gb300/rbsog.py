"""Thin ctypes binding of librbsog (include/rbsog.h): argument marshalling only.

Every function has the C name and signature; device arrays are passed as raw pointers
(``torch.Tensor.data_ptr()``), host arrays as numpy buffers.  All computation happens in
the CUDA library.  There is no fallback: if the shared library or a CUDA device is
missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RBSOG_OK = 0
RBSOG_FP64, RBSOG_FP32 = 0, 1
RBSOG_NVE, RBSOG_LANGEVIN = 0, 1
RBSOG_SOG_MINIMAL, RBSOG_SOG_BOUND, RBSOG_SOG_TABLE = 0, 1, 2
RBSOG_SAMPLING_ADAPTIVE, RBSOG_SAMPLING_UNIFORM, RBSOG_SAMPLING_K2, RBSOG_SAMPLING_DEBYE = 0, 1, 2, 3
RBSOG_SAMPLER_IID, RBSOG_SAMPLER_MH = 0, 1
RBSOG_KT_TARGET, RBSOG_KT_INSTANT = 0, 1
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOCONV", 6: "EUNSUPPORTED",
          7: "EOVERFLOW"}


class rbsog_params(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("kappa", C.c_double), ("a_ws", C.c_double), ("Gamma", C.c_double),
                ("kT", C.c_double), ("r_c", C.c_double), ("sog_eps", C.c_double), ("dt", C.c_double),
                ("langevin_gamma", C.c_double), ("seed", C.c_uint64), ("P", C.c_int32),
                ("precision", C.c_int32), ("ensemble", C.c_int32), ("sog_mode", C.c_int32),
                ("sog_M1", C.c_int32), ("sog_M2", C.c_int32), ("device", C.c_int32), ("sampling", C.c_int32),
                ("egs_nu", C.c_double), ("sampler", C.c_int32), ("mh_sweeps", C.c_int32), ("mh_burnin", C.c_int32),
                ("temperature", C.c_int32), ("q2_total", C.c_double), ("qsum_total", C.c_double)]


class rbsog_energy(C.Structure):
    _fields_ = [("U_near", C.c_double), ("U_far", C.c_double), ("U_self", C.c_double), ("kinetic", C.c_double),
                ("total", C.c_double), ("step", C.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class rbsog_server_config(C.Structure):
    _fields_ = [("max_particles", C.c_int64), ("max_cells", C.c_int64), ("max_modes", C.c_int64),
                ("near_target", C.c_double), ("max_jobs", C.c_int32), ("steps_per_round", C.c_int32),
                ("rho_target", C.c_int32), ("device", C.c_int32), ("reserved", C.c_int32 * 2)]


class rbsog_job_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("error", C.c_int32), ("N", C.c_int64), ("nsteps", C.c_int32),
                ("steps_done", C.c_int32), ("t_arrival", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("footprint_bytes", C.c_uint64), ("energy", rbsog_energy)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "energy"}
        d["energy"] = self.energy.as_dict()
        return d


RBSOG_JOB_QUEUED, RBSOG_JOB_RESIDENT, RBSOG_JOB_DONE, RBSOG_JOB_FAILED = 0, 1, 2, 3


class RbsogError(RuntimeError):
    pass


_lib = None
EXPORTS = ["rbsog_init", "rbsog_set_state", "rbsog_get_state", "rbsog_set_state_forces", "rbsog_get_forces", "rbsog_set_state_forces_f32", "rbsog_get_forces_f32", "rbsog_forces", "rbsog_forces_split", "rbsog_step", "rbsog_step_get",
           "rbsog_set_ksample", "rbsog_get_ksample", "rbsog_get_rho", "rbsog_get_cells", "rbsog_get_sog", "rbsog_get_temperature", "rbsog_set_owned", "rbsog_forces_partial", "rbsog_forces_complete", "rbsog_slab_split",
           "rbsog_build_sog", "rbsog_profile", "rbsog_profile_read", "rbsog_profile_name", "rbsog_rho_noalloc",
           "rbsog_last_error", "rbsog_free", "rbsog_batch_init", "rbsog_batch_set_state", "rbsog_batch_get_state",
           "rbsog_batch_forces", "rbsog_batch_step", "rbsog_batch_set_ksample", "rbsog_batch_get_ksample",
           "rbsog_batch_layout", "rbsog_batch_set_rho_chunk", "rbsog_batch_set_shapes", "rbsog_batch_tune",
           "rbsog_batch_profile", "rbsog_batch_set_persistent", "rbsog_batch_set_wait_limit", "rbsog_batch_last_error", "rbsog_batch_free", "rbsog_server_create",
           "rbsog_server_submit", "rbsog_server_run", "rbsog_server_job", "rbsog_server_stats", "rbsog_server_clock",
           "rbsog_server_last_error", "rbsog_server_free"]
RBSOG_NPROF = 10


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librbsog.so (building it first when asked).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RbsogError(f"librbsog not built: {path}")
        _build.build()
    L = C.CDLL(path)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    L.rbsog_init.argtypes = [C.POINTER(rbsog_params), i64, vp, vp, C.POINTER(vp)]
    L.rbsog_set_state.argtypes = [vp, vp, vp, vp]
    L.rbsog_get_state.argtypes = [vp, vp, vp, C.POINTER(C.c_uint64), vp]
    L.rbsog_set_state_forces.argtypes = [vp, vp, vp, vp, vp]
    L.rbsog_get_forces.argtypes = [vp, vp, vp]
    L.rbsog_set_state_forces_f32.argtypes = [vp, vp, vp, vp, vp]
    L.rbsog_get_forces_f32.argtypes = [vp, vp, vp]
    L.rbsog_forces.argtypes = [vp, vp, C.POINTER(rbsog_energy), vp]
    L.rbsog_forces_split.argtypes = [vp, vp, vp, C.POINTER(rbsog_energy), vp]
    L.rbsog_step.argtypes = [vp, i32, C.POINTER(rbsog_energy), vp]
    L.rbsog_step_get.argtypes = [vp, i32, vp, vp, vp, i32, C.POINTER(rbsog_energy), vp]
    L.rbsog_set_ksample.argtypes = [vp, vp, i32]
    L.rbsog_get_ksample.argtypes = [vp, vp, vp]
    L.rbsog_get_rho.argtypes = [vp, vp]
    L.rbsog_get_cells.argtypes = [vp, vp, vp, vp]
    L.rbsog_get_sog.argtypes = [vp, dp, dp, C.POINTER(i32), C.POINTER(i32), dp, dp, dp]
    L.rbsog_get_temperature.argtypes = [vp, dp, dp]
    L.rbsog_set_owned.argtypes = [vp, i64]
    L.rbsog_forces_partial.argtypes = [vp, vp, vp]
    L.rbsog_forces_complete.argtypes = [vp, vp, vp, vp]
    L.rbsog_slab_split.argtypes = [i64, vp, vp, i32, i32, i32, C.c_double, vp, C.POINTER(i64), C.POINTER(i64)]
    L.rbsog_build_sog.argtypes = [C.c_double, C.c_double, C.c_double, i32, i32, i32, vp]
    L.rbsog_profile.argtypes = [vp, i32]
    L.rbsog_profile_read.argtypes = [vp, vp, vp]
    L.rbsog_profile_name.argtypes = [i32]
    L.rbsog_profile_name.restype = C.c_char_p
    L.rbsog_rho_noalloc.argtypes = [vp, vp, i64, vp, vp, i32, vp, vp]
    L.rbsog_last_error.argtypes = [vp]
    L.rbsog_last_error.restype = C.c_char_p
    L.rbsog_free.argtypes = [vp]
    L.rbsog_free.restype = None
    L.rbsog_batch_init.argtypes = [vp, i32, vp, vp, vp, C.POINTER(vp)]
    L.rbsog_batch_set_state.argtypes = [vp, vp, vp, vp]
    L.rbsog_batch_get_state.argtypes = [vp, vp, vp, C.POINTER(C.c_uint64), vp]
    L.rbsog_batch_forces.argtypes = [vp, vp, vp, vp]
    L.rbsog_batch_step.argtypes = [vp, i32, vp, vp]
    L.rbsog_batch_set_ksample.argtypes = [vp, vp]
    L.rbsog_batch_get_ksample.argtypes = [vp, vp, vp]
    L.rbsog_batch_layout.argtypes = [vp, vp, vp, vp]
    L.rbsog_batch_set_rho_chunk.argtypes = [vp, vp]
    L.rbsog_batch_set_shapes.argtypes = [vp, C.c_double, i32]
    L.rbsog_batch_tune.argtypes = [vp, i32, dp, C.POINTER(i32), vp]
    L.rbsog_batch_profile.argtypes = [vp, i32, vp, vp]
    L.rbsog_batch_set_persistent.argtypes = [vp, i32]
    L.rbsog_batch_set_wait_limit.argtypes = [vp, i64]
    L.rbsog_batch_last_error.argtypes = [vp]
    L.rbsog_batch_last_error.restype = C.c_char_p
    L.rbsog_batch_free.argtypes = [vp]
    L.rbsog_batch_free.restype = None
    L.rbsog_server_create.argtypes = [C.POINTER(rbsog_server_config), C.POINTER(vp)]
    L.rbsog_server_submit.argtypes = [vp, C.POINTER(rbsog_params), i64, vp, vp, vp, vp, i32, C.c_double,
                                      C.POINTER(i64)]
    L.rbsog_server_run.argtypes = [vp, C.c_double]
    L.rbsog_server_job.argtypes = [vp, i64, C.POINTER(rbsog_job_info), vp, vp]
    L.rbsog_server_stats.argtypes = [vp, vp]
    L.rbsog_server_clock.argtypes = [vp]
    L.rbsog_server_clock.restype = C.c_double
    L.rbsog_server_last_error.argtypes = [vp]
    L.rbsog_server_last_error.restype = C.c_char_p
    L.rbsog_server_free.argtypes = [vp]
    L.rbsog_server_free.restype = None
    for name in EXPORTS:
        if name not in ("rbsog_profile_name", "rbsog_last_error", "rbsog_free", "rbsog_batch_last_error",
                        "rbsog_batch_free", "rbsog_server_clock", "rbsog_server_last_error", "rbsog_server_free"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(x):
    """Raw address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def _check(ctx, code):
    if code != RBSOG_OK:
        msg = load().rbsog_last_error(ctx)
        raise RbsogError(f"{STATUS.get(code, code)}: {msg.decode() if msg else ''}")


def rbsog_init(params: rbsog_params, N: int, q, m):
    q = np.ascontiguousarray(q, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    out = C.c_void_p()
    _check(None, load().rbsog_init(C.byref(params), int(N), q.ctypes.data, m.ctypes.data, C.byref(out)))
    return out.value


def rbsog_set_state(ctx, r, v=None, stream=None):
    _check(ctx, load().rbsog_set_state(ctx, _ptr(r), _ptr(v), _stream(stream)))


def rbsog_get_state(ctx, r=None, v=None, stream=None) -> int:
    step = C.c_uint64(0)
    _check(ctx, load().rbsog_get_state(ctx, _ptr(r), _ptr(v), C.byref(step), _stream(stream)))
    return step.value


def rbsog_set_state_forces(ctx, r, v=None, F=None, stream=None):
    _check(ctx, load().rbsog_set_state_forces(ctx, _ptr(r), _ptr(v), _ptr(F), _stream(stream)))


def rbsog_get_forces(ctx, F, stream=None):
    _check(ctx, load().rbsog_get_forces(ctx, _ptr(F), _stream(stream)))


def rbsog_set_state_forces_f32(ctx, r, v=None, F=None, stream=None):
    """F: [N][3] float32 (FP32 build only)."""
    _check(ctx, load().rbsog_set_state_forces_f32(ctx, _ptr(r), _ptr(v), _ptr(F), _stream(stream)))


def rbsog_get_forces_f32(ctx, F, stream=None):
    """F: [N][3] float32 (FP32 build only)."""
    _check(ctx, load().rbsog_get_forces_f32(ctx, _ptr(F), _stream(stream)))


def rbsog_forces(ctx, F=None, energy: bool = False, stream=None):
    e = rbsog_energy()
    _check(ctx, load().rbsog_forces(ctx, _ptr(F), C.byref(e) if energy else None, _stream(stream)))
    return e.as_dict() if energy else None


def rbsog_forces_split(ctx, F_near=None, F_far=None, energy: bool = False, stream=None):
    e = rbsog_energy()
    _check(ctx, load().rbsog_forces_split(ctx, _ptr(F_near), _ptr(F_far), C.byref(e) if energy else None,
                                          _stream(stream)))
    return e.as_dict() if energy else None


def rbsog_step(ctx, nsteps: int, energy: bool = False, stream=None):
    e = rbsog_energy()
    _check(ctx, load().rbsog_step(ctx, int(nsteps), C.byref(e) if energy else None, _stream(stream)))
    return e.as_dict() if energy else None


def rbsog_step_get(ctx, nsteps: int, r=None, v=None, F=None, energy: bool = False, stream=None):
    """nsteps steps, then r, v ([N][3] float64) and F ([N][3], float32 for the FP32 form,
    else float64) in the caller's order; any may be None.  Returns the energies when asked."""
    f32 = 0
    if F is not None:
        dt = getattr(F, "dtype", None)
        f32 = 1 if str(dt) in ("float32", "torch.float32") else 0
    e = rbsog_energy()
    _check(ctx, load().rbsog_step_get(ctx, int(nsteps), _ptr(r), _ptr(v), _ptr(F), f32,
                                      C.byref(e) if energy else None, _stream(stream)))
    return e.as_dict() if energy else None


def rbsog_set_ksample(ctx, m):
    m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
    _check(ctx, load().rbsog_set_ksample(ctx, m.ctypes.data, m.shape[0]))


def rbsog_get_ksample(ctx, P: int):
    m = np.zeros((P, 3), dtype=np.int32)
    coef = np.zeros(P, dtype=np.float64)
    _check(ctx, load().rbsog_get_ksample(ctx, m.ctypes.data, coef.ctypes.data))
    return m, coef


def rbsog_get_rho(ctx, P: int):
    rho = np.zeros((P, 2), dtype=np.float64)
    _check(ctx, load().rbsog_get_rho(ctx, rho.ctypes.data))
    return rho


def rbsog_get_cells(ctx, N: int):
    nc = np.zeros(3, dtype=np.int32)
    _check(ctx, load().rbsog_get_cells(ctx, nc.ctypes.data, None, None))
    start = np.zeros(int(nc[0]) * int(nc[1]) * int(nc[2]) + 1, dtype=np.uint32)
    perm = np.zeros(N, dtype=np.uint32)
    _check(ctx, load().rbsog_get_cells(ctx, None, start.ctypes.data, perm.ctypes.data))
    return nc, start, perm


def rbsog_get_sog(ctx) -> dict:
    h, t0, w, lam, S = (C.c_double() for _ in range(5))
    M1, M2 = C.c_int32(), C.c_int32()
    _check(ctx, load().rbsog_get_sog(ctx, C.byref(h), C.byref(t0), C.byref(M1), C.byref(M2), C.byref(w),
                                     C.byref(lam), C.byref(S)))
    return dict(h=h.value, t0=t0.value, M1=M1.value, M2=M2.value, w=w.value, lam=lam.value, S=S.value)


def rbsog_get_temperature(ctx) -> tuple:
    """(k_B T, S) of the last force evaluation."""
    kT, S = C.c_double(), C.c_double()
    _check(ctx, load().rbsog_get_temperature(ctx, C.byref(kT), C.byref(S)))
    return kT.value, S.value


def rbsog_set_owned(ctx, n_owned: int):
    _check(ctx, load().rbsog_set_owned(ctx, int(n_owned)))


def rbsog_forces_partial(ctx, rho_out, stream=None):
    """Partial rho over the owned particles into rho_out ([P][2], host numpy or device tensor)."""
    _check(ctx, load().rbsog_forces_partial(ctx, _ptr(rho_out), _stream(stream)))


def rbsog_forces_complete(ctx, rho, F=None, stream=None):
    """Far force from the summed rho ([P][2], host or device) plus the near force into F."""
    if isinstance(rho, np.ndarray):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
    _check(ctx, load().rbsog_forces_complete(ctx, _ptr(rho), _ptr(F), _stream(stream)))


def rbsog_slab_split(r, box, axis: int, nslabs: int, slab: int, halo: float):
    """(idx, n_owned): the slab's owned particles, then its halo copies (host arrays)."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, dtype=np.float64)
    idx = np.zeros(r.shape[0], dtype=np.int64)
    no, nl = C.c_int64(), C.c_int64()
    _check(None, load().rbsog_slab_split(r.shape[0], r.ctypes.data, box.ctypes.data, int(axis), int(nslabs),
                                         int(slab), float(halo), idx.ctypes.data, C.byref(no), C.byref(nl)))
    return idx[:nl.value].copy(), int(no.value)


def rbsog_build_sog(lam: float, r_c: float, eps: float, mode: int = RBSOG_SOG_MINIMAL, M1: int = 0,
                    M2: int = 0) -> dict:
    out = np.zeros(6, dtype=np.float64)
    _check(None, load().rbsog_build_sog(float(lam), float(r_c), float(eps), int(mode), int(M1), int(M2),
                                        out.ctypes.data))
    return dict(h=out[0], t0=out[1], M1=int(out[2]), M2=int(out[3]), w=out[4], max_error=out[5])


def rbsog_profile(ctx, enable: bool):
    _check(ctx, load().rbsog_profile(ctx, 1 if enable else 0))


def rbsog_profile_read(ctx) -> dict:
    ms = np.zeros(RBSOG_NPROF, dtype=np.float64)
    n = np.zeros(RBSOG_NPROF, dtype=np.int64)
    _check(ctx, load().rbsog_profile_read(ctx, ms.ctypes.data, n.ctypes.data))
    return {rbsog_profile_name(g): (float(ms[g]), int(n[g])) for g in range(RBSOG_NPROF)}


def rbsog_profile_name(group: int) -> str:
    return load().rbsog_profile_name(int(group)).decode()


def rbsog_rho_noalloc(r_dev, q_dev, N: int, box, m_dev, P: int, rho_dev, stream=None):
    """Structure factor of device arrays into rho_dev ([P][2] float64) without any device
    allocation by the library (for callers that cannot allocate; see include/rbsog.h)."""
    box = np.ascontiguousarray(box, dtype=np.float64)
    _check(None, load().rbsog_rho_noalloc(_ptr(r_dev), _ptr(q_dev), int(N), box.ctypes.data, _ptr(m_dev), int(P),
                                          _ptr(rho_dev), _stream(stream)))


def rbsog_last_error(ctx=None) -> str:
    msg = load().rbsog_last_error(ctx)
    return msg.decode() if msg else ""


def rbsog_free(ctx):
    if ctx:
        load().rbsog_free(ctx)


# ---- batches of independent systems ----------------------------------------------------

def _bcheck(b, code):
    if code != RBSOG_OK:
        msg = load().rbsog_batch_last_error(b)
        raise RbsogError(f"{STATUS.get(code, code)}: {msg.decode() if msg else ''}")


def rbsog_batch_init(params, N, q, m):
    """params: sequence of rbsog_params; N: particle counts; q, m: concatenated host arrays."""
    R = len(params)
    arr = (rbsog_params * R)(*params)
    n = np.ascontiguousarray(N, dtype=np.int64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    out = C.c_void_p()
    _bcheck(None, load().rbsog_batch_init(C.cast(arr, C.c_void_p), R, n.ctypes.data, q.ctypes.data,
                                          m.ctypes.data, C.byref(out)))
    return out.value


def rbsog_batch_set_state(b, r, v=None, stream=None):
    _bcheck(b, load().rbsog_batch_set_state(b, _ptr(r), _ptr(v), _stream(stream)))


def rbsog_batch_get_state(b, r=None, v=None, stream=None) -> int:
    step = C.c_uint64(0)
    _bcheck(b, load().rbsog_batch_get_state(b, _ptr(r), _ptr(v), C.byref(step), _stream(stream)))
    return step.value


def _energies(e) -> list:
    return [x.as_dict() for x in e]


def rbsog_batch_forces(b, R: int, F=None, energy: bool = False, stream=None):
    e = (rbsog_energy * R)()
    _bcheck(b, load().rbsog_batch_forces(b, _ptr(F), C.cast(e, C.c_void_p) if energy else None, _stream(stream)))
    return _energies(e) if energy else None


def rbsog_batch_step(b, R: int, nsteps: int, energy: bool = False, stream=None):
    e = (rbsog_energy * R)()
    _bcheck(b, load().rbsog_batch_step(b, int(nsteps), C.cast(e, C.c_void_p) if energy else None,
                                       _stream(stream)))
    return _energies(e) if energy else None


def rbsog_batch_set_ksample(b, m):
    m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
    _bcheck(b, load().rbsog_batch_set_ksample(b, m.ctypes.data))


def rbsog_batch_get_ksample(b, Ptot: int):
    m = np.zeros((Ptot, 3), dtype=np.int32)
    coef = np.zeros(Ptot, dtype=np.float64)
    _bcheck(b, load().rbsog_batch_get_ksample(b, m.ctypes.data, coef.ctypes.data))
    return m, coef


def rbsog_batch_layout(b, R: int):
    p_off = np.zeros(R + 1, dtype=np.int64)
    m_off = np.zeros(R + 1, dtype=np.int64)
    chunk = np.zeros(R, dtype=np.int32)
    _bcheck(b, load().rbsog_batch_layout(b, p_off.ctypes.data, m_off.ctypes.data, chunk.ctypes.data))
    return p_off, m_off, chunk


def rbsog_batch_set_rho_chunk(b, chunk):
    chunk = np.ascontiguousarray(chunk, dtype=np.int32)
    _bcheck(b, load().rbsog_batch_set_rho_chunk(b, chunk.ctypes.data))


def rbsog_batch_set_shapes(b, near_target: float, rho_target: int):
    _bcheck(b, load().rbsog_batch_set_shapes(b, float(near_target), int(rho_target)))


def rbsog_batch_tune(b, reps: int = 3, stream=None):
    nt = C.c_double(0.0)
    rt = C.c_int32(0)
    _bcheck(b, load().rbsog_batch_tune(b, int(reps), C.byref(nt), C.byref(rt), _stream(stream)))
    return nt.value, rt.value


def rbsog_batch_set_persistent(b, enable: bool = True):
    _bcheck(b, load().rbsog_batch_set_persistent(b, 1 if enable else 0))


def rbsog_batch_set_wait_limit(b, polls: int):
    _bcheck(b, load().rbsog_batch_set_wait_limit(b, int(polls)))


def rbsog_batch_profile(b, nsteps: int, stream=None) -> dict:
    ms = np.zeros(RBSOG_NPROF, dtype=np.float64)
    _bcheck(b, load().rbsog_batch_profile(b, int(nsteps), ms.ctypes.data, _stream(stream)))
    return {rbsog_profile_name(g): float(ms[g]) for g in range(RBSOG_NPROF)}


def rbsog_batch_last_error(b=None) -> str:
    msg = load().rbsog_batch_last_error(b)
    return msg.decode() if msg else ""


def rbsog_batch_free(b):
    if b:
        load().rbsog_batch_free(b)


# ---- job server ------------------------------------------------------------------------

def _scheck(s, code):
    if code != RBSOG_OK:
        msg = load().rbsog_server_last_error(s)
        raise RbsogError(f"{STATUS.get(code, code)}: {msg.decode() if msg else ''}")


def make_server_config(max_particles: int, max_cells: int, max_modes: int, max_jobs: int,
                       steps_per_round: int = 32, near_target: float = 0.0, rho_target: int = 0,
                       device: int = 0) -> rbsog_server_config:
    c = rbsog_server_config()
    c.max_particles, c.max_cells, c.max_modes = int(max_particles), int(max_cells), int(max_modes)
    c.near_target, c.max_jobs, c.steps_per_round = float(near_target), int(max_jobs), int(steps_per_round)
    c.rho_target, c.device = int(rho_target), int(device)
    c.reserved[0] = c.reserved[1] = 0
    return c


def rbsog_server_create(cfg: rbsog_server_config):
    out = C.c_void_p()
    _scheck(None, load().rbsog_server_create(C.byref(cfg), C.byref(out)))
    return out.value


def rbsog_server_submit(s, params: rbsog_params, q, m, r, v=None, nsteps: int = 0, t_arrival: float = -1.0) -> int:
    q = np.ascontiguousarray(q, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    jid = C.c_int64(-1)
    _scheck(s, load().rbsog_server_submit(s, C.byref(params), int(q.shape[0]), q.ctypes.data, m.ctypes.data,
                                          r.ctypes.data, None if v is None else v.ctypes.data, int(nsteps),
                                          float(t_arrival), C.byref(jid)))
    return jid.value


def rbsog_server_run(s, t_until: float = -1.0):
    _scheck(s, load().rbsog_server_run(s, float(t_until)))


def rbsog_server_job(s, job_id: int, N: int | None = None, state: bool = False):
    """(info dict, r, v); r and v only for a done job when state is True.  A failed job's
    info is returned with its error code (no exception)."""
    info = rbsog_job_info()
    r = v = None
    if state:
        r = np.zeros((N, 3))
        v = np.zeros((N, 3))
    code = load().rbsog_server_job(s, int(job_id), C.byref(info), None if r is None else r.ctypes.data,
                                   None if v is None else v.ctypes.data)
    if code != RBSOG_OK and not (info.status == RBSOG_JOB_FAILED and code == info.error):
        _scheck(s, code)
    return info.as_dict(), r, v


def rbsog_server_stats(s) -> dict:
    out = np.zeros(8, dtype=np.float64)
    _scheck(s, load().rbsog_server_stats(s, out.ctypes.data))
    keys = ["rounds", "admissions", "retirements", "busy_s", "particle_steps", "peak_particles", "peak_jobs",
            "setup_s"]
    return dict(zip(keys, out.tolist()))


def rbsog_server_clock(s) -> float:
    return float(load().rbsog_server_clock(s))


def rbsog_server_last_error(s=None) -> str:
    msg = load().rbsog_server_last_error(s)
    return msg.decode() if msg else ""


def rbsog_server_free(s):
    if s:
        load().rbsog_server_free(s)


def make_params(w, precision: int = RBSOG_FP32, P: int | None = None, seed: int | None = None,
                sog_mode: int = RBSOG_SOG_MINIMAL, M1: int = 0, M2: int = 0, device: int = 0,
                ensemble: int | None = None, dt: float | None = None,
                sampling: int = RBSOG_SAMPLING_ADAPTIVE, egs_nu: float = 0.0, sampler: int = RBSOG_SAMPLER_IID,
                mh_sweeps: int = 0, mh_burnin: int = 0, temperature: int = RBSOG_KT_TARGET, q2_total: float = 0.0,
                qsum_total: float = 0.0) -> rbsog_params:
    """rbsog_params from a workloads.Workload (plain field copy)."""
    p = rbsog_params()
    for d in range(3):
        p.box[d] = float(w.box[d])
    p.kappa = float(w.kappa)
    p.a_ws = float(w.a_ws)
    p.Gamma = float(w.Gamma)
    p.kT = 0.0
    p.r_c = float(w.r_c)
    p.sog_eps = float(w.sog_eps)
    p.dt = float(w.dt if dt is None else dt)
    p.langevin_gamma = float(w.langevin_gamma)
    p.seed = int(w.seed_k if seed is None else seed)
    p.P = int(w.P if P is None else P)
    p.precision = int(precision)
    if ensemble is None:
        ensemble = RBSOG_LANGEVIN if w.ensemble == "langevin" else RBSOG_NVE
    p.ensemble = int(ensemble)
    p.sog_mode = int(sog_mode)
    p.sog_M1, p.sog_M2 = int(M1), int(M2)
    p.device = int(device)
    p.sampling = int(sampling)
    p.egs_nu = float(egs_nu)
    p.sampler = int(sampler)
    p.mh_sweeps = int(mh_sweeps)
    p.mh_burnin = int(mh_burnin)
    p.temperature = int(temperature)
    p.q2_total = float(q2_total)
    p.qsum_total = float(qsum_total)
    return p
