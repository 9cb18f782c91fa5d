"""Python binding of the C ABI in include/lbmdem.h (argument marshalling only).

Every step of the coupled LBM-DEM update runs in the CUDA library
(_liblbmdem.so, built for sm_103a by paper_1808_08921_gb300.build).  There is
no CPU path: if the library cannot be loaded, or no sm_103-class GPU is
present, the constructor raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SINE, COSINE, STEP, RICKER = 0, 1, 2, 3
INLET_PRESSURE, X_WALL, X_PERIODIC = 0, 1, 2
OUT_ZERO_GRAD, OUT_RHO_F, OUT_WALL = 0, 1, 2
F32, BF16_DEV, F16_DEV = 0, 1, 2  # population storage (arithmetic is FP32)

ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "UNSTABLE", -5: "TIMEOUT",
          -6: "STATE", -7: "CAPACITY", -8: "SKIN", -9: "NO_DEVICE"}

# every symbol include/lbmdem.h declares
SYMBOLS = ("lbm_dem_default_params", "lbm_dem_init", "lbm_dem_set_packing",
           "lbm_dem_set_pressure_source", "lbm_dem_step", "lbm_dem_relayout", "lbm_dem_status",
           "lbm_dem_read_fields", "lbm_dem_read_particles", "lbm_dem_read_particles_noalloc",
           "lbm_dem_read_probe",
           "lbm_dem_read_monitors", "lbm_dem_read_counters", "lbm_dem_set_timing",
           "lbm_dem_read_timing", "lbm_dem_last_error", "lbm_dem_destroy",
           "lbm_dem_batch_create", "lbm_dem_batch_set_time_limit", "lbm_dem_batch_step", "lbm_dem_batch_sync",
           "lbm_dem_batch_graph_launches", "lbm_dem_batch_last_error", "lbm_dem_batch_destroy",
           "lbm_dem_adjoint", "lbm_dem_adjoint_psm", "lbm_dem_read_plane_means")


class Params(C.Structure):
    """Mirror of lbmdem_params."""
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("tau", C.c_double), ("rho_f", C.c_double),
                ("storage", C.c_int32), ("inlet", C.c_int32), ("outlet", C.c_int32),
                ("dem_substeps", C.c_int32),
                ("E_p", C.c_double), ("nu_p", C.c_double), ("mu", C.c_double),
                ("rho_p", C.c_double), ("body_force", C.c_double * 3),
                ("probe_x", C.c_int32), ("lbm_on", C.c_int32),
                ("skin", C.c_double), ("dem_skin", C.c_double),
                ("monitor_every", C.c_int32), ("graph_steps", C.c_int32),
                ("max_flips", C.c_int32), ("tile", C.c_int32), ("device", C.c_int32),
                ("link_mode", C.c_int32), ("cuda_stream", C.c_void_p)]


class LbmDemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library not built: {_build.LIB}")
    lib = C.CDLL(_build.LIB)
    P, d, i32, i64, vp = C.POINTER, C.c_double, C.c_int32, C.c_int64, C.c_void_p
    lib.lbm_dem_default_params.argtypes = [P(Params)]
    lib.lbm_dem_default_params.restype = None
    lib.lbm_dem_init.argtypes = [P(Params), P(vp)]
    lib.lbm_dem_set_packing.argtypes = [vp, i32, P(d), P(d), P(d), P(d), P(C.c_uint8)]
    lib.lbm_dem_set_pressure_source.argtypes = [vp, i32, d, d, i64, d]
    lib.lbm_dem_step.argtypes = [vp, i64]
    lib.lbm_dem_status.argtypes = [vp]
    lib.lbm_dem_relayout.argtypes = [vp]
    lib.lbm_dem_read_fields.argtypes = [vp, P(d), P(d), P(C.c_uint8)]
    lib.lbm_dem_read_particles.argtypes = [vp, P(d), P(d), P(d), P(d), P(d), P(d)]
    lib.lbm_dem_read_particles_noalloc.argtypes = [vp, P(d), P(d), P(d), P(d), P(d), P(d)]
    lib.lbm_dem_read_probe.argtypes = [vp, P(d), i64, P(i64)]
    lib.lbm_dem_read_monitors.argtypes = [vp, P(d)]
    lib.lbm_dem_read_counters.argtypes = [vp, P(i64)]
    lib.lbm_dem_set_timing.argtypes = [vp, i32]
    lib.lbm_dem_read_timing.argtypes = [vp, P(d), P(i64)]
    lib.lbm_dem_last_error.argtypes = [vp]
    lib.lbm_dem_last_error.restype = C.c_char_p
    lib.lbm_dem_destroy.argtypes = [vp]
    lib.lbm_dem_destroy.restype = None
    lib.lbm_dem_adjoint.argtypes = [vp, i64, i32, P(d), P(d), P(d), P(d), P(d)]
    lib.lbm_dem_adjoint_psm.argtypes = [vp, i64, i32, P(d), P(d), P(d), P(d), P(d), P(d)]
    lib.lbm_dem_read_plane_means.argtypes = [vp, P(d), P(d)]
    lib.lbm_dem_batch_create.argtypes = [P(vp), i32, P(vp)]
    lib.lbm_dem_batch_set_time_limit.argtypes = [vp, d]
    lib.lbm_dem_batch_step.argtypes = [vp, P(i64)]
    lib.lbm_dem_batch_sync.argtypes = [vp]
    lib.lbm_dem_batch_graph_launches.argtypes = [vp]
    lib.lbm_dem_batch_graph_launches.restype = i64
    lib.lbm_dem_batch_last_error.argtypes = [vp]
    lib.lbm_dem_batch_last_error.restype = C.c_char_p
    lib.lbm_dem_batch_destroy.argtypes = [vp]
    lib.lbm_dem_batch_destroy.restype = None
    _lib = lib
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def default_params() -> Params:
    p = Params()
    load().lbm_dem_default_params(C.byref(p))
    return p


def params_from_workload(w, **over) -> Params:
    """lbmdem_params for a workloads.Workload (same field names)."""
    p = default_params()
    p.nx, p.ny, p.nz = w.nx, w.ny, w.nz
    p.tau, p.rho_f = w.tau, w.rho_f
    p.inlet, p.outlet = w.inlet, w.outlet
    p.dem_substeps = w.dem_substeps
    p.E_p, p.nu_p, p.mu, p.rho_p = w.E_p, w.nu_p, w.mu, w.rho_p
    p.body_force = (C.c_double * 3)(*w.body_force)
    p.probe_x = w.probe_x
    for k, v in over.items():
        if k == "cuda_stream":
            v = C.c_void_p(v) if v is not None else None
        setattr(p, k, v)
    return p


class Sim:
    """One coupled LBM-DEM simulation on the GPU (wraps an lbmdem_ctx)."""

    def __init__(self, params: Params):
        lib = load()
        self._p = params
        h = C.c_void_p()
        rc = lib.lbm_dem_init(C.byref(params), C.byref(h))
        if rc != 0:
            raise LbmDemError(rc, "lbm_dem_init failed")
        self._h = h
        self.N = params.nx * params.ny * params.nz
        self.shape = (params.nx, params.ny, params.nz)
        self.np = 0

    @classmethod
    def from_workload(cls, w, set_source=True, **over):
        s = cls(params_from_workload(w, **over))
        if set_source:
            s.set_pressure_source(w.waveform, w.amplitude, w.omega, w.t_n, w.t0)
        s.set_packing(w.X, w.R, w.V, w.W, w.fixed)
        return s

    def _check(self, rc):
        if rc != 0:
            msg = load().lbm_dem_last_error(self._h)
            raise LbmDemError(rc, msg.decode() if msg else "")
        return rc

    def set_packing(self, X, R, V=None, W=None, fixed=None):
        n = 0 if X is None else int(np.asarray(X).shape[0])
        Xa = np.ascontiguousarray(X, np.float64).reshape(n, 3) if n else np.zeros((1, 3))
        Ra = np.ascontiguousarray(R, np.float64).reshape(n) if n else np.zeros(1)
        Va = None if V is None or not n else np.ascontiguousarray(V, np.float64).reshape(n, 3)
        Wa = None if W is None or not n else np.ascontiguousarray(W, np.float64).reshape(n, 3)
        fx = None if fixed is None or not n else np.ascontiguousarray(fixed, np.uint8)
        self._check(load().lbm_dem_set_packing(
            self._h, n, _dp(Xa), _dp(Ra), _dp(Va), _dp(Wa),
            None if fx is None else fx.ctypes.data_as(C.POINTER(C.c_uint8))))
        self.np = n

    def set_pressure_source(self, waveform, amplitude, omega, t_n=-1, t0=0.0):
        self._check(load().lbm_dem_set_pressure_source(self._h, int(waveform), float(amplitude),
                                                       float(omega), int(t_n), float(t0)))

    def step(self, n=1):
        self._check(load().lbm_dem_step(self._h, int(n)))

    def relayout(self):
        self._check(load().lbm_dem_relayout(self._h))

    def status(self):
        return load().lbm_dem_status(self._h)

    def fields(self):
        rho = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        sol = np.zeros(self.N, np.uint8)
        self._check(load().lbm_dem_read_fields(self._h, _dp(rho), _dp(u),
                                               sol.ctypes.data_as(C.POINTER(C.c_uint8))))
        return rho.reshape(self.shape), u.reshape((3,) + self.shape), sol.reshape(self.shape)

    def particles(self):
        n = max(self.np, 1)
        out = {k: np.zeros((n, 3)) for k in ("X", "V", "W", "Fh", "Th")}
        out["q"] = np.zeros((n, 4))
        self._check(load().lbm_dem_read_particles(
            self._h, *[_dp(out[k]) for k in ("X", "V", "W", "q", "Fh", "Th")]))
        return {k: v[:self.np] for k, v in out.items()}

    def particles_noalloc(self):
        """particles() through lbm_dem_read_particles_noalloc: no device memory
        is allocated; at most 65536 spheres."""
        n = max(self.np, 1)
        out = {k: np.zeros((n, 3)) for k in ("X", "V", "W", "Fh", "Th")}
        out["q"] = np.zeros((n, 4))
        self._check(load().lbm_dem_read_particles_noalloc(
            self._h, *[_dp(out[k]) for k in ("X", "V", "W", "q", "Fh", "Th")]))
        return {k: v[:self.np] for k, v in out.items()}

    def probe(self):
        ln = C.c_int64()
        load().lbm_dem_read_probe(self._h, None, 0, C.byref(ln))
        out = np.zeros(max(ln.value, 1))
        self._check(load().lbm_dem_read_probe(self._h, _dp(out), ln.value, C.byref(ln)))
        return out[:ln.value]

    def monitors(self):
        out = np.zeros(6)
        self._check(load().lbm_dem_read_monitors(self._h, _dp(out)))
        return out

    def counters(self):
        out = np.zeros(10, np.int64)
        self._check(load().lbm_dem_read_counters(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        keys = ("nodes", "stored", "fluid", "band", "links", "neighbour_entries", "t",
                "relayouts", "conversions", "launches")
        return dict(zip(keys, (int(v) for v in out)))

    def set_timing(self, on=True):
        self._check(load().lbm_dem_set_timing(self._h, 1 if on else 0))

    def timing(self):
        ms = np.zeros(6)
        n = np.zeros(6, np.int64)
        self._check(load().lbm_dem_read_timing(self._h, _dp(ms), n.ctypes.data_as(C.POINTER(C.c_int64))))
        names = ("collide_odd", "links", "map_update", "inlet_outlet", "dem", "collide_even")
        return {k: (float(a), int(b)) for k, a, b in zip(names, ms, n)}

    def plane_means(self):
        """(rho[nx], rho u_x[nx]): averages over the fluid nodes of each x plane."""
        rho, jx = np.zeros(self.shape[0]), np.zeros(self.shape[0])
        self._check(load().lbm_dem_read_plane_means(self._h, _dp(rho), _dp(jx)))
        return rho, jx

    def adjoint(self, steps, every, target):
        """lbm_dem_adjoint: (loss, dL/dtau, dL/damplitude, pressure trace)."""
        tgt = np.ascontiguousarray(target, np.float64)
        assert tgt.shape == (steps,)
        L, dt, da = C.c_double(), C.c_double(), C.c_double()
        tr = np.zeros(steps)
        self._check(load().lbm_dem_adjoint(self._h, int(steps), int(every), _dp(tgt), C.byref(L), C.byref(dt),
                                           C.byref(da), _dp(tr)))
        return L.value, dt.value, da.value, tr

    def adjoint_psm(self, steps, every, target):
        """lbm_dem_adjoint_psm: (loss, dL/dtau, dL/damplitude, dL/dX[n, 3],
        pressure trace) of the smooth coupling surrogate, from rest."""
        tgt = np.ascontiguousarray(target, np.float64)
        assert tgt.shape == (steps,)
        L, dt, da = C.c_double(), C.c_double(), C.c_double()
        dX = np.zeros((max(self.np, 1), 3))
        tr = np.zeros(steps)
        self._check(load().lbm_dem_adjoint_psm(self._h, int(steps), int(every), _dp(tgt), C.byref(L), C.byref(dt),
                                               C.byref(da), _dp(dX), _dp(tr)))
        return L.value, dt.value, da.value, dX[:self.np], tr

    def surrogate_loss(self, steps, target):
        """The smooth surrogate's forward loss and pressure trace alone."""
        tgt = np.ascontiguousarray(target, np.float64)
        L = C.c_double()
        tr = np.zeros(steps)
        self._check(load().lbm_dem_adjoint_psm(self._h, int(steps), 1, _dp(tgt), C.byref(L), None, None, None,
                                               _dp(tr)))
        return L.value, tr

    def close(self):
        if getattr(self, "_h", None):
            load().lbm_dem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several Sim columns advanced together (lbm_dem_batch_*): one launch of
    one CUDA graph runs every column's steps (a device-side loop per column)."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s._h for s in self.sims])
        h = C.c_void_p()
        rc = load().lbm_dem_batch_create(arr, len(self.sims), C.byref(h))
        if rc != 0:
            raise LbmDemError(rc, "lbm_dem_batch_create")
        self._h = h

    def _check(self, rc):
        if rc != 0:
            msg = load().lbm_dem_batch_last_error(self._h)
            raise LbmDemError(rc, msg.decode() if msg else "")
        return rc

    def step(self, steps):
        """Advance column i by steps[i] steps (an int applies to every column)."""
        if np.isscalar(steps):
            steps = [int(steps)] * len(self.sims)
        arr = np.ascontiguousarray(steps, np.int64)
        assert arr.shape == (len(self.sims),)
        self._check(load().lbm_dem_batch_step(self._h, arr.ctypes.data_as(C.POINTER(C.c_int64))))

    def set_time_limit(self, seconds):
        """GPU-clock limit of each following step() launch (0 = none)."""
        self._check(load().lbm_dem_batch_set_time_limit(self._h, float(seconds)))

    def sync(self):
        self._check(load().lbm_dem_batch_sync(self._h))

    @property
    def graph_launches(self):
        return int(load().lbm_dem_batch_graph_launches(self._h))

    def close(self):
        if self._h:
            load().lbm_dem_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
