"""ctypes binding of the FP64 CPU oracle (lbmdem_oracle.c).

Test infrastructure only: see the package docstring.  Every routine here
marshals arrays to the C reference and back; the arithmetic is in C.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmdem_oracle.c")
_LIB = os.path.join(_HERE, "_liblbmdem_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 19


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("rho_f", C.c_double),
                ("inlet", C.c_int), ("outlet", C.c_int),
                ("dem_substeps", C.c_int),
                ("E_p", C.c_double), ("nu_p", C.c_double), ("mu", C.c_double),
                ("rho_p", C.c_double), ("body_force", C.c_double * 3),
                ("probe_x", C.c_int), ("lbm_on", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_liblbmdem_oracle.so."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
                os.path.getmtime(_SRC), os.path.getmtime(_SRC[:-2] + ".h")):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fopenmp",
                                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.POINTER
        d, i, ll = C.c_double, C.c_int, C.c_longlong
        lib.orc_create.restype = C.c_void_p
        lib.orc_create.argtypes = [P(_Params)]
        lib.orc_set_packing.argtypes = [C.c_void_p, i, P(d), P(d), P(d), P(d), P(C.c_ubyte)]
        lib.orc_set_source.argtypes = [C.c_void_p, i, d, d, ll, d]
        lib.orc_step.argtypes = [C.c_void_p, ll]
        lib.orc_time.restype = ll
        lib.orc_time.argtypes = [C.c_void_p]
        lib.orc_fields.argtypes = [C.c_void_p, P(d), P(d), P(C.c_ubyte)]
        lib.orc_populations.argtypes = [C.c_void_p, P(d)]
        lib.orc_set_populations.argtypes = [C.c_void_p, P(d)]
        lib.orc_owner.argtypes = [C.c_void_p, P(i)]
        lib.orc_particles.argtypes = [C.c_void_p] + [P(d)] * 6
        lib.orc_contact_forces.argtypes = [C.c_void_p, P(d), P(d)]
        lib.orc_probe.restype = ll
        lib.orc_probe.argtypes = [C.c_void_p, P(d), ll]
        lib.orc_destroy.argtypes = [C.c_void_p]
        lib.orc_lattice.argtypes = [P(i), P(i), P(i), P(d), P(i)]
        lib.orc_equilibrium.argtypes = [d, d, d, d, P(d)]
        lib.orc_collide_node.argtypes = [P(d), d]
        lib.orc_pressure_face.argtypes = [P(d), d, i]
        lib.orc_source_density.restype = d
        lib.orc_source_density.argtypes = [C.c_void_p, ll]
        lib.orc_pair_force.argtypes = [P(_Params), d, d, P(d), P(d), d, P(d), P(d), P(d)]
        lib.orc_set_link_form.argtypes = [C.c_void_p, i]
        lib.orc_set_coupling.argtypes = [C.c_void_p, i]
        lib.orc_psm_fraction.argtypes = [C.c_void_p, P(d)]
        lib.orc_psm_set_fraction.argtypes = [C.c_void_p, P(d)]
        lib.orc_set_threads.argtypes = [i]
        lib.orc_get_threads.restype = i
        _lib = lib
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle (its results do not depend on the count)."""
    _load().orc_set_threads(int(n))


def threads() -> int:
    return int(_load().orc_get_threads())


def lattice():
    """(c[19,3] int, w[19], opp[19]) of the oracle's D3Q19 tables."""
    lib = _load()
    cx, cy, cz, opp = (C.c_int * Q)(), (C.c_int * Q)(), (C.c_int * Q)(), (C.c_int * Q)()
    w = (C.c_double * Q)()
    lib.orc_lattice(cx, cy, cz, w, opp)
    c = np.array([list(cx), list(cy), list(cz)]).T
    return c, np.array(list(w)), np.array(list(opp))


def equilibrium(rho, u):
    lib = _load()
    out = np.zeros(Q)
    lib.orc_equilibrium(float(rho), float(u[0]), float(u[1]), float(u[2]), _dp(out))
    return out


def collide_node(f, tau):
    lib = _load()
    f = _f64(f).copy()
    lib.orc_collide_node(_dp(f), float(tau))
    return f


def pressure_face(f, rho_b, side):
    lib = _load()
    f = _f64(f).copy()
    lib.orc_pressure_face(_dp(f), float(rho_b), int(side))
    return f


def _params(w, lbm_on=True):
    p = _Params()
    p.nx, p.ny, p.nz = w.nx, w.ny, w.nz
    p.tau, p.rho_f = w.tau, w.rho_f
    p.inlet, p.outlet = w.inlet, w.outlet
    p.dem_substeps = w.dem_substeps
    p.E_p, p.nu_p, p.mu, p.rho_p = w.E_p, w.nu_p, w.mu, w.rho_p
    p.body_force = (C.c_double * 3)(*w.body_force)
    p.probe_x = w.probe_x
    p.lbm_on = 1 if lbm_on else 0
    return p


def pair_force(params_like, Ri, Rj, d_ij, vrel, dt, ft_hist):
    """Eqs. 11-12 for one pair; returns (F_on_i[3], new_hist[3], overlap)."""
    lib = _load()
    p = _params(params_like)
    d = _f64(d_ij)
    v = _f64(vrel)
    h = _f64(ft_hist).copy()
    F = np.zeros(3)
    ov = np.zeros(1)
    lib.orc_pair_force(C.byref(p), float(Ri), float(Rj), _dp(d), _dp(v), float(dt),
                       _dp(h), _dp(F), _dp(ov))
    return F, h, float(ov[0])


class Oracle:
    """FP64 reference simulation of one workload (workloads.Workload)."""

    def __init__(self, w, lbm_on=True):
        lib = _load()
        self.w = w
        self._p = _params(w, lbm_on)
        self._s = lib.orc_create(C.byref(self._p))
        if not self._s:
            raise ValueError("oracle: invalid parameters")
        self.N = w.nx * w.ny * w.nz
        self.np = 0
        lib.orc_set_source(self._s, int(w.waveform), float(w.amplitude), float(w.omega),
                           int(w.t_n), float(w.t0))
        if w.X is not None:
            self.set_packing(w.X, w.R, w.V, w.W, w.fixed)

    def set_packing(self, X, R, V=None, W=None, fixed=None):
        lib = _load()
        n = 0 if X is None else int(np.asarray(X).shape[0])
        X = _f64(X, (n, 3)) if n else np.zeros((0, 3))
        R = _f64(R, (n,)) if n else np.zeros(0)
        V = _f64(V, (n, 3)) if V is not None else None
        W = _f64(W, (n, 3)) if W is not None else None
        fx = None
        if fixed is not None and n:
            fx = np.ascontiguousarray(fixed, dtype=np.uint8)
        rc = lib.orc_set_packing(self._s, n, _dp(X), _dp(R), _dp(V), _dp(W),
                                 None if fx is None else fx.ctypes.data_as(C.POINTER(C.c_ubyte)))
        if rc != 0:
            raise ValueError("oracle: invalid packing")
        self.np = n

    def step(self, n=1):
        _load().orc_step(self._s, int(n))

    def set_link_form(self, literal: bool):
        """True: the link momentum as printed in Eq. 15, c_d (f~_d + f_d*);
        False (default): about the rest state (the reading both sides use)."""
        _load().orc_set_link_form(self._s, 1 if literal else 0)

    def set_coupling(self, psm: bool):
        """True: the smooth partially-saturated surrogate (fixed spheres, every
        node fluid-carrying, solid-fraction-weighted collision); False: the
        momentum-exchange coupling of the paper (default)."""
        _load().orc_set_coupling(self._s, 1 if psm else 0)

    def psm_fraction(self):
        """The surrogate's solid fraction per node, [nx, ny, nz]."""
        e = np.zeros(self.N)
        _load().orc_psm_fraction(self._s, _dp(e))
        return e.reshape(self.w.nx, self.w.ny, self.w.nz)

    def psm_set_fraction(self, eps):
        """Replace the surrogate's solid fraction (None: back to the spheres')."""
        e = None if eps is None else _f64(eps, (self.N,))
        _load().orc_psm_set_fraction(self._s, _dp(e))

    @property
    def t(self):
        return int(_load().orc_time(self._s))

    def fields(self):
        """rho[nx,ny,nz], u[3,nx,ny,nz], solid[nx,ny,nz] (rho = u = 0 on solid)."""
        lib = _load()
        w = self.w
        rho = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        sol = np.zeros(self.N, np.uint8)
        lib.orc_fields(self._s, _dp(rho), _dp(u), sol.ctypes.data_as(C.POINTER(C.c_ubyte)))
        sh = (w.nx, w.ny, w.nz)
        return rho.reshape(sh), u.reshape((3,) + sh), sol.reshape(sh)

    def populations(self):
        f = np.zeros(Q * self.N)
        _load().orc_populations(self._s, _dp(f))
        return f.reshape(Q, self.w.nx, self.w.ny, self.w.nz)

    def set_populations(self, f):
        f = _f64(f, (Q * self.N,))
        _load().orc_set_populations(self._s, _dp(f))

    def owner(self):
        o = np.zeros(self.N, np.int32)
        _load().orc_owner(self._s, o.ctypes.data_as(C.POINTER(C.c_int)))
        return o.reshape(self.w.nx, self.w.ny, self.w.nz)

    def particles(self):
        """dict of X, V, W, q, Fh, Th (the last step's hydrodynamic load)."""
        n = max(self.np, 1)
        out = {k: np.zeros((n, 3)) for k in ("X", "V", "W", "Fh", "Th")}
        out["q"] = np.zeros((n, 4))
        _load().orc_particles(self._s, *[_dp(out[k]) for k in ("X", "V", "W", "q", "Fh", "Th")])
        return {k: v[:self.np] for k, v in out.items()}

    def contact_forces(self):
        n = max(self.np, 1)
        Fc, Tc = np.zeros((n, 3)), np.zeros((n, 3))
        _load().orc_contact_forces(self._s, _dp(Fc), _dp(Tc))
        return Fc[:self.np], Tc[:self.np]

    def probe(self):
        lib = _load()
        n = lib.orc_probe(self._s, None, 0)
        out = np.zeros(max(n, 1))
        lib.orc_probe(self._s, _dp(out), n)
        return out[:n]

    def source_density(self, t):
        return float(_load().orc_source_density(self._s, int(t)))

    def close(self):
        if self._s:
            _load().orc_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
