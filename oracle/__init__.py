"""CPU oracle for the e-ph collision integral (TEST INFRASTRUCTURE ONLY).

Plain FP64 implementations of what the GPU library computes, written from the
paper (arXiv:2511.03683): Eq. 2 (collision integral), the scattering rates it
implies, classic RK4 time stepping of the rt-BTE (Eq. 1 with no field) and the
linearised iterative transport solve.  ``oracle.c`` holds the channel loops;
``dense.py`` is an independent numpy brute force over all window-state pairs for
tiny grids.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_2511_03683_gb300``) and imports nothing from it; both consume the seeded
inputs of the ``synth`` package.

Parity status: every function here is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or library solvers; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

HBAR_EVFS = 0.6582119569
KB_EVK = 8.617333262e-5

G2FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p)


class OrModel(ctypes.Structure):
    _fields_ = [
        ("nk", ctypes.c_int32 * 3),
        ("nbands", ctypes.c_int32),
        ("nmodes", ctypes.c_int32),
        ("nthreads", ctypes.c_int32),
        ("eps", ctypes.c_void_p),
        ("omega", ctypes.c_void_p),
        ("win", ctypes.c_void_p),
        ("T", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("g2", ctypes.c_void_p),
        ("g2_user", ctypes.c_void_p),
        ("g2_min", ctypes.c_double),
        ("delta_nsigma", ctypes.c_double),
    ]


def build(force: bool = False, plant: int = 0) -> str:
    """Compile oracle.c (gcc -O2 -fopenmp, portable flags) into liboracle.so.  ``plant`` > 0
    builds a deliberately wrong variant (liboracle_plant<k>.so) for the mutant tests."""
    src = os.path.join(_HERE, "oracle.c")
    path = _LIB_PATH if plant == 0 else os.path.join(_HERE, f"liboracle_plant{plant}.so")
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(src):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fopenmp", f"-DORACLE_PLANT={plant}",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, path)
    return path


_libs = {}


def lib(plant: int = 0) -> ctypes.CDLL:
    if plant not in _libs:
        L = ctypes.CDLL(build(plant=plant))
        P = ctypes.POINTER(OrModel)
        vp = ctypes.c_void_p
        L.oracle_window.restype = ctypes.c_int64
        L.oracle_window.argtypes = [P, vp]
        L.oracle_collision.restype = ctypes.c_int
        L.oracle_collision.argtypes = [P, vp, vp, ctypes.c_int64, vp, vp]
        L.oracle_rates.restype = ctypes.c_int
        L.oracle_rates.argtypes = [P, vp, vp, ctypes.c_int64, vp]
        L.oracle_rk4.restype = ctypes.c_int
        L.oracle_rk4.argtypes = [P, vp, ctypes.c_double, ctypes.c_int32]
        L.oracle_transport_map.restype = ctypes.c_int
        L.oracle_transport_map.argtypes = [P, vp, vp, vp, vp, ctypes.c_int64, vp, vp]
        L.oracle_transport.restype = ctypes.c_int
        L.oracle_transport.argtypes = [P, vp, vp, ctypes.c_double, ctypes.c_int32, vp,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        L.oracle_count_channels.restype = ctypes.c_int64
        L.oracle_count_channels.argtypes = [P]
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_collision_vjp.restype = ctypes.c_int
        L.oracle_collision_vjp.argtypes = [P, vp, vp, vp]
        L.oracle_g2_grad.restype = ctypes.c_int
        L.oracle_g2_grad.argtypes = [P, vp, vp, ctypes.c_int64, vp, vp, vp, vp]
        L.oracle_rk4_vjp.restype = ctypes.c_int
        L.oracle_rk4_vjp.argtypes = [P, vp, ctypes.c_double, ctypes.c_int32, vp]
        _libs[plant] = L
    return _libs[plant]


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """Bind one synth.Model to the C oracle.  Arrays passed in and out are over the
    window states in ascending full-grid id order (see ``window_ids``)."""

    def __init__(self, model, nthreads: int = 0, plant: int = 0, g2_min: float = 0.0, delta_nsigma: float = 0.0):
        self.model = model
        self._L = lib(plant)
        self._eps = _f64(model.eps)
        self._omega = _f64(model.omega)
        self._win = None if model.win is None else _f64(model.win)
        m = OrModel()
        for i in range(3):
            m.nk[i] = int(model.nk[i])
        m.nbands = model.nbands
        m.nmodes = model.nmodes
        m.nthreads = int(nthreads)
        m.eps = self._eps.ctypes.data
        m.omega = self._omega.ctypes.data
        m.win = None if self._win is None else self._win.ctypes.data
        m.T = float(model.T)
        m.sigma = float(model.sigma)
        m.g2 = model.g2_fn_ptr()
        m.g2_user = model.g2_user_ptr()
        m.g2_min = float(g2_min)
        m.delta_nsigma = float(delta_nsigma)
        self._m = m
        n = self._L.oracle_window(ctypes.byref(m), None)
        ids = np.empty(max(n, 1), dtype=np.int32)
        self._L.oracle_window(ctypes.byref(m), ids.ctypes.data)
        self.ids = ids[:n]

    @property
    def nstate(self) -> int:
        return len(self.ids)

    def window_values(self, full: np.ndarray) -> np.ndarray:
        """Pick window-state values out of a full-grid [Nk, nb] (or [Nk, nb, ...]) array."""
        nb = self.model.nbands
        flat = full.reshape((full.shape[0] * nb,) + full.shape[2:])
        return np.ascontiguousarray(flat[self.ids])

    def count_channels(self) -> int:
        return int(self._L.oracle_count_channels(ctypes.byref(self._m)))

    def _rows(self, rows):
        if rows is None:
            return None, 0, self.nstate
        r = np.ascontiguousarray(rows, dtype=np.int32)
        return r, len(r), len(r)

    def collision(self, f, rows=None, with_abs: bool = False):
        """I_s of the rows (all by default); with_abs also returns each row's gross
        scattering sum (the in- and out-scattering products that Eq. 2 differences)."""
        f = _f64(f)
        assert f.shape == (self.nstate,)
        r, nr, nout = self._rows(rows)
        out = np.empty(nout)
        ab = np.empty(nout) if with_abs else None
        rc = self._L.oracle_collision(ctypes.byref(self._m), f.ctypes.data, None if r is None else r.ctypes.data, nr,
                                    out.ctypes.data, None if ab is None else ab.ctypes.data)
        if rc:
            raise MemoryError("oracle_collision failed")
        return (out, ab) if with_abs else out

    def rates(self, f, rows=None):
        f = _f64(f)
        r, nr, nout = self._rows(rows)
        out = np.empty(nout)
        rc = self._L.oracle_rates(ctypes.byref(self._m), f.ctypes.data, None if r is None else r.ctypes.data, nr,
                                out.ctypes.data)
        if rc:
            raise MemoryError("oracle_rates failed")
        return out

    def rk4(self, f, dt: float, nsteps: int):
        y = _f64(f).copy()
        rc = self._L.oracle_rk4(ctypes.byref(self._m), y.ctypes.data, float(dt), int(nsteps))
        if rc:
            raise MemoryError("oracle_rk4 failed")
        return y

    def transport_map(self, f0, vel3, F3, rows=None):
        f0, vel3, F3 = _f64(f0), _f64(vel3), _f64(F3)
        r, nr, nout = self._rows(rows)
        out = np.empty((nout, 3))
        tau = np.empty(nout)
        rc = self._L.oracle_transport_map(ctypes.byref(self._m), f0.ctypes.data, vel3.ctypes.data, F3.ctypes.data,
                                        None if r is None else r.ctypes.data, nr, out.ctypes.data, tau.ctypes.data)
        if rc:
            raise MemoryError("oracle_transport_map failed")
        return out, tau

    def transport(self, f0, vel3, tol: float = 1e-10, maxit: int = 1000):
        f0, vel3 = _f64(f0), _f64(vel3)
        F = np.empty((self.nstate, 3))
        it = ctypes.c_int32(0)
        res = ctypes.c_double(0.0)
        rc = self._L.oracle_transport(ctypes.byref(self._m), f0.ctypes.data, vel3.ctypes.data, float(tol), int(maxit),
                                    F.ctypes.data, ctypes.byref(it), ctypes.byref(res))
        if rc < 0:
            raise MemoryError("oracle_transport failed")
        return F, int(it.value), float(res.value), rc == 0


    # ---------------------------------------------------------------- adjoint

    def collision_vjp(self, f, lam):
        """(J^T lam)_x = sum_s lam_s dI_s/df_x."""
        f, lam = _f64(f), _f64(lam)
        out = np.empty(self.nstate)
        if self._L.oracle_collision_vjp(ctypes.byref(self._m), f.ctypes.data, lam.ctypes.data, out.ctypes.data):
            raise MemoryError("oracle_collision_vjp failed")
        return out

    def g2_grad(self, f, lam, s, p, nu):
        """dL/dg2 of the ordered channels (s[i] -> p[i], nu[i]) for L = sum_s lam_s I_s."""
        f, lam = _f64(f), _f64(lam)
        s = np.ascontiguousarray(s, np.int32)
        p = np.ascontiguousarray(p, np.int32)
        nu = np.ascontiguousarray(nu, np.int32)
        out = np.empty(len(s))
        rc = self._L.oracle_g2_grad(ctypes.byref(self._m), f.ctypes.data, lam.ctypes.data, len(s), s.ctypes.data,
                                    p.ctypes.data, nu.ctypes.data, out.ctypes.data)
        if rc == -1:
            raise MemoryError("oracle_g2_grad failed")
        if rc == -2:
            raise ValueError("a listed channel does not exist (phonon energy <= 0)")
        return out

    def rk4_vjp(self, f0, dt, nsteps, lam):
        """dL/df0 for L depending on f(T) after nsteps RK4 steps, given lam = dL/df(T)."""
        f0 = _f64(f0)
        lam = _f64(lam).copy()
        if self._L.oracle_rk4_vjp(ctypes.byref(self._m), f0.ctypes.data, float(dt), int(nsteps), lam.ctypes.data):
            raise MemoryError("oracle_rk4_vjp failed")
        return lam


def max_threads() -> int:
    return int(lib().oracle_max_threads())
