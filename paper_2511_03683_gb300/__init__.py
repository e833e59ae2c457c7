"""GB300 (sm_103a) electron-phonon collision integrals: Python binding of libpb.so.

Argument marshalling only: every step of the computation runs in the C ABI of
``include/pb.h`` (host channel builder in C++, device work in hand-written CUDA).
PyTorch supplies device memory (one arena tensor per device handle) and streams.
There is no CPU fallback: importing this package raises if libpb.so is missing,
and every device call raises if the GPU library reports an error.

What is computed follows arXiv:2511.03683 (Eq. 2: the e-ph collision integral;
the rt-BTE it drives; the iterative transport solve with three field directions).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Channels", "Device", "Batch", "PBError", "lib", "VARIANTS", "G2_BATCH_FN"]

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libpb.so")

PB_OK, PB_EINVAL, PB_ENOMEM, PB_ECUDA, PB_ENOTCLOSED, PB_ENOCONV, PB_ETIMEOUT, PB_ECALLBACK, PB_EDEVICE = range(9)
_CODES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCLOSED", 5: "ENOCONV", 6: "ETIMEOUT", 7: "ECALLBACK",
          8: "EDEVICE"}
VARIANTS = {"ff": 0, "f64": 1, "literal": 2, "g32": 3, "g16": 4, "paper": 5, "h16": 6, "c32": 7}


class PBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pb error {_CODES.get(code, code)}: {msg}")
        self.code = code


class _Model(ctypes.Structure):
    _fields_ = [("nk", ctypes.c_int32 * 3), ("nbands", ctypes.c_int32), ("nmodes", ctypes.c_int32),
                ("eps", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("omega", ctypes.c_void_p),
                ("win", ctypes.c_void_p), ("T", ctypes.c_double), ("sigma", ctypes.c_double)]


class _BuildOpts(ctypes.Structure):
    _fields_ = [("nthreads", ctypes.c_int32), ("callback_threadsafe", ctypes.c_int32),
                ("check_closure", ctypes.c_int32), ("reserved", ctypes.c_int32), ("g2_min", ctypes.c_double),
                ("delta_nsigma", ctypes.c_double)]


class _ChInfo(ctypes.Structure):
    _fields_ = [("nstate", ctypes.c_int64), ("nchannels", ctypes.c_int64), ("nq", ctypes.c_int64),
                ("nk", ctypes.c_int32 * 3), ("nbands", ctypes.c_int32), ("nmodes", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("T", ctypes.c_double), ("sigma", ctypes.c_double),
                ("max_row", ctypes.c_int64)]


class _DevOpts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("item_channels", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("transport", ctypes.c_int32), ("transport_gather", ctypes.c_int32),
                ("transport_ctas", ctypes.c_int32), ("channel_per_lane", ctypes.c_int32),
                ("stream_mode", ctypes.c_int32), ("merge_branches", ctypes.c_int32), ("dense_rows", ctypes.c_int32),
                ("tile_sweep", ctypes.c_int32), ("adjoint", ctypes.c_int32)]


class _DevInfo(ctypes.Structure):
    _fields_ = [("nstate", ctypes.c_int64), ("nchannels", ctypes.c_int64), ("nchannels_padded", ctypes.c_int64),
                ("nitems", ctypes.c_int64), ("variant", ctypes.c_int32), ("sm_count", ctypes.c_int32),
                ("bytes_per_channel", ctypes.c_double), ("c", ctypes.c_double)]


G2_BATCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)

_lib = None


def builder():
    """The in-tree build script (``_build.py``), loaded by path so that building never
    needs the (possibly stale) library this package loads."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("_pb_build", os.path.join(_PKG, "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def lib() -> ctypes.CDLL:
    """Load libpb.so, rebuilding it in-tree first when its sources are newer and nvcc is
    present.  Raises ImportError when the library is missing and cannot be built."""
    global _lib
    if _lib is not None:
        return _lib
    b = builder()
    if not b.up_to_date():
        try:
            b.build()
        except Exception as e:  # noqa: BLE001
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing and could not be built: {e}") from e
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "pb_build_channels": [ctypes.POINTER(_Model), vp, vp, ctypes.POINTER(_BuildOpts), ctypes.POINTER(vp)],
        "pb_channels_get_info": [vp, ctypes.POINTER(_ChInfo)],
        "pb_channels_export": [vp, vp, vp, vp, vp, vp],
        "pb_dev_arena_bytes": [vp, ctypes.POINTER(_DevOpts), ctypes.POINTER(ctypes.c_size_t)],
        "pb_dev_create": [vp, ctypes.POINTER(_DevOpts), vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "pb_dev_get_info": [vp, ctypes.POINTER(_DevInfo)],
        "pb_dev_check": [vp, vp],
        "pb_dev_selftest_wait": [vp, i32, vp],
        "pb_dev_time_sweep": [vp, vp, i32, i32, ctypes.POINTER(ctypes.c_float), vp],
        "pb_collision": [vp, vp, vp, vp],
        "pb_collision_static": [vp, vp, vp, vp],
        "pb_scatter_rates": [vp, vp, vp, vp],
        "pb_rtbte_rk4_step": [vp, vp, dbl, i32, vp],
        "pb_rtbte_rk4_host": [vp, vp, vp, dbl, i32, vp],
        "pb_iter_transport": [vp, vp, vp, dbl, i32, vp, ctypes.POINTER(i32), ctypes.POINTER(dbl), vp],
        "pb_transport_map": [vp, vp, vp, vp, vp, vp],
        "pb_transport_setup": [vp, vp, vp],
        "pb_transport_iterate": [vp, vp, vp, vp, vp, vp],
        "pb_transport_iterate_host": [vp, vp, vp, vp, vp, vp],
        "pb_observables": [vp, vp, vp, vp],
        "pb_collision_vjp": [vp, vp, vp, vp, vp, vp],
        "pb_batch_arena_bytes": [vp, i32, vp, ctypes.POINTER(ctypes.c_size_t)],
        "pb_batch_create": [vp, i32, vp, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        "pb_batch_get_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), vp, ctypes.POINTER(i32),
                              ctypes.POINTER(i32)],
        "pb_batch_collision": [vp, vp, vp, vp],
        "pb_batch_rk4_step": [vp, vp, dbl, i32, vp],
        "pb_batch_autotune": [vp, vp, vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(dbl)],
        "pb_batch_check": [vp, vp],
        "pb_rtbte_rk4_vjp": [vp, vp, vp, dbl, vp, vp],
        "pb_rtbte_rk4_vjp_defer": [vp, vp, vp, dbl, vp],
        "pb_dev_g2grad_flush": [vp, vp, vp],
        "pb_dev_set_g2": [vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.pb_channels_free.argtypes = [vp]
    L.pb_channels_free.restype = None
    L.pb_dev_destroy.argtypes = [vp]
    L.pb_dev_destroy.restype = None
    L.pb_batch_destroy.argtypes = [vp]
    L.pb_batch_destroy.restype = None
    L.pb_last_error.restype = ctypes.c_char_p
    L.pb_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int):
    if rc != PB_OK:
        raise PBError(rc, lib().pb_last_error().decode(errors="replace"))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Channels:
    """Host CSR of every scattering channel inside the energy window (pb_build_channels)."""

    def __init__(self, handle: int, keep=()):
        self._h = ctypes.c_void_p(handle)
        self._keep = keep
        info = _ChInfo()
        _check(lib().pb_channels_get_info(self._h, ctypes.byref(info)))
        self.nstate = int(info.nstate)
        self.nchannels = int(info.nchannels)
        self.nq = int(info.nq)
        self.nk = tuple(info.nk)
        self.nbands = int(info.nbands)
        self.nmodes = int(info.nmodes)
        self.T = float(info.T)
        self.sigma = float(info.sigma)
        self.max_row = int(info.max_row)

    @classmethod
    def build(cls, nk, nbands, nmodes, eps, omega, T, sigma, g2, g2_user=None, vel=None, win=None,
              nthreads=0, threadsafe=True, check_closure=True, g2_min=0.0, delta_nsigma=0.0) -> "Channels":
        """``g2`` is either the address of a C function with the pb_g2_fn signature (then
        ``g2_user`` is its user pointer) or a Python callable g2(s, p, nu) -> array on
        numpy int32 id arrays (full-grid ids), called one row at a time."""
        m = _Model()
        for i in range(3):
            m.nk[i] = int(nk[i])
        m.nbands, m.nmodes = int(nbands), int(nmodes)
        eps_a, omega_a = _f64(eps), _f64(omega)
        vel_a = None if vel is None else _f64(vel)
        win_a = None if win is None else _f64(win)
        m.eps, m.omega = eps_a.ctypes.data, omega_a.ctypes.data
        m.vel = None if vel_a is None else vel_a.ctypes.data
        m.win = None if win_a is None else win_a.ctypes.data
        m.T, m.sigma = float(T), float(sigma)
        o = _BuildOpts(int(nthreads), 1 if threadsafe else 0, 1 if check_closure else 0, 0, float(g2_min),
                       float(delta_nsigma))
        keep = []
        if callable(g2):
            pyfn = g2

            def tramp(n, s, p, nu, out, user):
                try:
                    n = int(n)
                    res = pyfn(np.ctypeslib.as_array(s, (n,)).copy(), np.ctypeslib.as_array(p, (n,)).copy(),
                               np.ctypeslib.as_array(nu, (n,)).copy())
                    np.ctypeslib.as_array(out, (n,))[:] = np.asarray(res, dtype=np.float64)
                    return 0
                except Exception:  # noqa: BLE001 - reported through the status code
                    return 1

            cb = G2_BATCH_FN(tramp)
            keep.append(cb)
            fn_ptr = ctypes.cast(cb, ctypes.c_void_p)
            o.callback_threadsafe = 0
            user = None
        else:
            fn_ptr = ctypes.c_void_p(int(g2))
            user = None if g2_user is None else ctypes.c_void_p(int(g2_user))
        h = ctypes.c_void_p()
        _check(lib().pb_build_channels(ctypes.byref(m), fn_ptr, user, ctypes.byref(o), ctypes.byref(h)))
        return cls(h.value, keep=tuple(keep))

    @classmethod
    def from_model(cls, model, **kw) -> "Channels":
        """Build from any object with nk, nbands, nmodes, eps, vel, omega, win, T, sigma and
        g2_batch_ptr()/g2_user_ptr() (the seeded generator's model has these)."""
        return cls.build(model.nk, model.nbands, model.nmodes, model.eps, model.omega, model.T, model.sigma,
                         model.g2_batch_ptr(), model.g2_user_ptr(), vel=model.vel, win=model.win, **kw)

    def export(self) -> dict:
        ns, nc = self.nstate, self.nchannels
        out = {"row_ptr": np.empty(ns + 1, np.int64), "col": np.empty(nc, np.int32), "nu": np.empty(nc, np.int32),
               "g2": np.empty(nc, np.float64), "state_ids": np.empty(ns, np.int32)}
        _check(lib().pb_channels_export(self._h, *(out[k].ctypes.data for k in
                                                   ("row_ptr", "col", "nu", "g2", "state_ids"))))
        return out

    def state_ids(self) -> np.ndarray:
        """Full-grid id of every window state, in state order."""
        ids = np.empty(self.nstate, np.int32)
        _check(lib().pb_channels_export(self._h, None, None, None, None, ids.ctypes.data))
        return ids

    def close(self):
        if self._h:
            lib().pb_channels_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def _stream_ptr(stream=None):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_vec(t, n, name, cols=None):
    import torch

    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    shape = (n,) if cols is None else (n, cols)
    if tuple(t.shape) != shape:
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Device:
    """Device-resident channel list and tables (pb_dev_create) in one torch arena.

    ``variant``: "ff" (default, FP64-accurate float-float), "f64", "literal", "g32", "g16"
    (BF16 |g|^2), "h16" (FP16 |g|^2 times a power of two), "c32" (the FF coefficients in FP32
    symmetric tiles) or "paper"; the other keywords are
    the fields of pb_dev_opts.  ``adjoint=True`` reserves the accumulators of the deferred
    |g|^2 gradient (``rk4_vjp_defer`` / ``g2grad_flush``); ``deferred`` tells whether this
    device has them (FF with branch merging, G32, G16, H16)."""

    def __init__(self, channels: Channels, variant: str = "ff", item_channels: int = 0, ctas_per_sm: int = 0,
                 transport: bool = False, transport_gather: int = 0, transport_ctas: int = 0,
                 channel_per_lane: int = 0, stream_mode: int = 0, merge_branches: int = 0, dense_rows: int = 0,
                 tile_sweep: int = 0, adjoint: bool = False, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise PBError(PB_EDEVICE, "no CUDA device is visible")
        self.channels = channels
        self.variant = variant
        # FF/F64 stream one entry per state pair unless merge_branches == 2
        self.merged = variant in ("ff", "f64") and int(merge_branches) != 2
        # per-pair accumulators of the deferred |g|^2 gradient (rk4_vjp_defer / g2grad_flush)
        self.deferred = bool(adjoint) and ((variant == "ff" and self.merged) or variant in ("g32", "g16", "h16"))
        o = _DevOpts(VARIANTS[variant], int(item_channels), int(ctas_per_sm), 1 if transport else 0,
                     int(transport_gather), int(transport_ctas), int(channel_per_lane), int(stream_mode),
                     int(merge_branches), int(dense_rows), int(tile_sweep), 1 if adjoint else 0)
        nbytes = ctypes.c_size_t(0)
        _check(lib().pb_dev_arena_bytes(channels._h, ctypes.byref(o), ctypes.byref(nbytes)))
        self.arena = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        _check(lib().pb_dev_create(channels._h, ctypes.byref(o), ctypes.c_void_p(self.arena.data_ptr()),
                                   ctypes.c_size_t(int(nbytes.value)), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        info = _DevInfo()
        _check(lib().pb_dev_get_info(self._h, ctypes.byref(info)))
        self.nstate = int(info.nstate)
        self.nchannels = int(info.nchannels)
        self.nchannels_padded = int(info.nchannels_padded)
        self.nitems = int(info.nitems)
        self.bytes_per_channel = float(info.bytes_per_channel)
        self.sm_count = int(info.sm_count)
        self.c = float(info.c)
        self._g2 = None  # the device's |g|^2 when set through set_g2 (None: the channel list's)

    def _new(self, *shape):
        import torch

        return torch.empty(shape, dtype=torch.float64, device="cuda")

    def collision(self, f, out=None, stream=None):
        """dfdt = I[f] (Eq. 2) for every window state."""
        fp = _dev_vec(f, self.nstate, "f")
        out = self._new(self.nstate) if out is None else out
        _check(lib().pb_collision(self._h, fp, _dev_vec(out, self.nstate, "out"), _stream_ptr(stream)))
        return out

    def check(self, stream=None):
        """Synchronise and raise PBError(PB_ETIMEOUT) if a bounded device wait gave up, or
        PBError(PB_EINVAL) if a |g|^2 value overflowed the scaled FP16 storage (h16)."""
        _check(lib().pb_dev_check(self._h, _stream_ptr(stream)))

    def collision_static(self, f, out, stream=None):
        """pb_collision_static: the same integral with scratch in the library's fixed
        device array (no allocation anywhere, so ``out`` must be given)."""
        _check(lib().pb_collision_static(self._h, _dev_vec(f, self.nstate, "f"), _dev_vec(out, self.nstate, "out"),
                                         _stream_ptr(stream)))
        return out

    def selftest_wait(self, wait_us: int = 1000, stream=None):
        """Launch the bounded-wait self-test (a wait that nothing completes gives up after
        wait_us microseconds); the next check() raises PBError(PB_ETIMEOUT) and clears it."""
        _check(lib().pb_dev_selftest_wait(self._h, int(wait_us), _stream_ptr(stream)))

    def time_sweep(self, f, nlaunch: int = 20, order: int = 0, stream=None) -> float:
        """Average device milliseconds of the collision sweep kernel alone (CUDA events on
        the stream around nlaunch back-to-back launches); order 1 alternates the tile order of
        the launches as the RK4 stages do."""
        ms = ctypes.c_float(0.0)
        _check(lib().pb_dev_time_sweep(self._h, _dev_vec(f, self.nstate, "f"), int(nlaunch), int(order),
                                       ctypes.byref(ms), _stream_ptr(stream)))
        return float(ms.value)

    def rates(self, f, out=None, stream=None):
        """Scattering rates 1/tau_s (1/fs)."""
        fp = _dev_vec(f, self.nstate, "f")
        out = self._new(self.nstate) if out is None else out
        _check(lib().pb_scatter_rates(self._h, fp, _dev_vec(out, self.nstate, "out"), _stream_ptr(stream)))
        return out

    def rk4(self, f, dt: float, nsteps: int = 1, stream=None):
        """nsteps classic RK4 steps of df/dt = I[f], in place on the CUDA tensor f."""
        _check(lib().pb_rtbte_rk4_step(self._h, _dev_vec(f, self.nstate, "f"), float(dt), int(nsteps),
                                       _stream_ptr(stream)))
        return f

    def rk4_host(self, f_host, dt: float, nsteps: int = 1, out=None, stream=None):
        """RK4 through host buffers: H2D copy, nsteps steps, D2H copy (synchronous).
        ``f_host`` and ``out`` may be numpy arrays or (pinned) CPU torch tensors."""
        def ptr(a):
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.data_ptr())
            return ctypes.c_void_p(a.ctypes.data)

        src = f_host if hasattr(f_host, "data_ptr") else _f64(f_host)
        if out is None:
            out = np.empty(self.nstate)
        _check(lib().pb_rtbte_rk4_host(self._h, ptr(src), ptr(out), float(dt), int(nsteps), _stream_ptr(stream)))
        return out

    def transport(self, f0, vel3, tol: float = 1e-10, maxit: int = 1000, out=None, stream=None):
        """Iterative transport for x, y, z at once.  Returns (F [nstate,3], iters, resid, converged)."""
        out = self._new(self.nstate, 3) if out is None else out
        it = ctypes.c_int32(0)
        res = ctypes.c_double(0.0)
        rc = lib().pb_iter_transport(self._h, _dev_vec(f0, self.nstate, "f0"), _dev_vec(vel3, self.nstate, "vel3", 3),
                                     float(tol), int(maxit), _dev_vec(out, self.nstate, "out", 3),
                                     ctypes.byref(it), ctypes.byref(res), _stream_ptr(stream))
        if rc not in (PB_OK, PB_ENOCONV):
            _check(rc)
        return out, int(it.value), float(res.value), rc == PB_OK

    def transport_iterate_host(self, vel3, F_in, out=None, resid=None, stream=None):
        """pb_transport_iterate_host: one pass with the iterates in host memory (numpy arrays
        or pinned CPU torch tensors of shape [nstate, 3]); synchronous.  ``resid`` (3 doubles in
        host memory) receives the residual numbers if given."""
        def ptr(a):
            return ctypes.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else ctypes.c_void_p(a.ctypes.data)

        src = F_in if hasattr(F_in, "data_ptr") else np.ascontiguousarray(F_in, dtype=np.float64)
        if out is None:
            out = np.empty((self.nstate, 3))
        _check(lib().pb_transport_iterate_host(self._h, _dev_vec(vel3, self.nstate, "vel3", 3), ptr(src), ptr(out),
                                               None if resid is None else ptr(resid), _stream_ptr(stream)))
        return out

    def transport_map(self, f0, vel3, F_in, out=None, stream=None):
        out = self._new(self.nstate, 3) if out is None else out
        _check(lib().pb_transport_map(self._h, _dev_vec(f0, self.nstate, "f0"), _dev_vec(vel3, self.nstate, "vel3", 3),
                                      _dev_vec(F_in, self.nstate, "F_in", 3), _dev_vec(out, self.nstate, "out", 3),
                                      _stream_ptr(stream)))
        return out

    def transport_setup(self, f0, stream=None):
        """Weights W_c and tau_s at f0, kept on the device for transport_iterate."""
        _check(lib().pb_transport_setup(self._h, _dev_vec(f0, self.nstate, "f0"), _stream_ptr(stream)))

    def transport_iterate(self, vel3, F_in, out=None, resid=None, stream=None):
        """One device-only pass F_out = tau (v + W F_in); resid (CUDA double[3]) optional."""
        out = self._new(self.nstate, 3) if out is None else out
        rp = None if resid is None else _dev_vec(resid, 3, "resid")
        _check(lib().pb_transport_iterate(self._h, _dev_vec(vel3, self.nstate, "vel3", 3),
                                          _dev_vec(F_in, self.nstate, "F_in", 3), _dev_vec(out, self.nstate, "out", 3),
                                          rp, _stream_ptr(stream)))
        return out

    # ------------------------------------------------------------ adjoint

    def collision_vjp(self, f, lam, out=None, grad_g2=None, stream=None):
        """grad_f = J(f)^T lam; grad_g2 (CUDA double[nchannels], CSR order) accumulates dL/dg2."""
        out = self._new(self.nstate) if out is None else out
        gp = None if grad_g2 is None else _dev_vec(grad_g2, self.nchannels, "grad_g2")
        _check(lib().pb_collision_vjp(self._h, _dev_vec(f, self.nstate, "f"), _dev_vec(lam, self.nstate, "lam"),
                                      _dev_vec(out, self.nstate, "out"), gp, _stream_ptr(stream)))
        return out

    def rk4_vjp(self, f, lam, dt, grad_g2=None, stream=None):
        """In place: lam = dL/df_n from dL/df_{n+1} for the RK4 step from f."""
        gp = None if grad_g2 is None else _dev_vec(grad_g2, self.nchannels, "grad_g2")
        _check(lib().pb_rtbte_rk4_vjp(self._h, _dev_vec(f, self.nstate, "f"), _dev_vec(lam, self.nstate, "lam"),
                                      float(dt), gp, _stream_ptr(stream)))
        return lam

    def rk4_vjp_defer(self, f, lam, dt, stream=None):
        """rk4_vjp whose |g|^2 gradient goes to the device's per-pair accumulators (a device
        made with adjoint=True); g2grad_flush adds it to a gradient vector."""
        _check(lib().pb_rtbte_rk4_vjp_defer(self._h, _dev_vec(f, self.nstate, "f"),
                                            _dev_vec(lam, self.nstate, "lam"), float(dt), _stream_ptr(stream)))
        return lam

    def g2grad_flush(self, grad_g2, stream=None):
        """grad_g2 (CUDA double[nchannels], CSR order) += the deferred |g|^2 gradient; clears it."""
        _check(lib().pb_dev_g2grad_flush(self._h, _dev_vec(grad_g2, self.nchannels, "grad_g2"),
                                         _stream_ptr(stream)))
        return grad_g2

    def set_g2(self, g2, stream=None):
        """Replace |g|^2 (CUDA double[nchannels], CSR order) and recompute the coefficients."""
        _check(lib().pb_dev_set_g2(self._h, _dev_vec(g2, self.nchannels, "g2"), _stream_ptr(stream)))
        self._g2 = g2.detach().clone()

    def g2_values(self):
        """The |g|^2 the device computes with (CUDA double[nchannels], CSR order): the channel
        list's couplings, or the last values given to set_g2."""
        import torch

        if self._g2 is None:
            self._g2 = torch.tensor(self.channels.export()["g2"], dtype=torch.float64, device="cuda")
        return self._g2

    def observables(self, f, out=None, stream=None):
        """(sum f, sum eps f, sum I[f]) as a CUDA tensor of 3 doubles."""
        out = self._new(3) if out is None else out
        _check(lib().pb_observables(self._h, _dev_vec(f, self.nstate, "f"), _dev_vec(out, 3, "out"),
                                    _stream_ptr(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().pb_dev_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class _BatchOpts(ctypes.Structure):
    _fields_ = [("item_channels", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("layout", ctypes.c_int32)]


class Batch:
    """Many channel lists advanced together (pb_batch_*), one sweep launch per stage:
    precision "fp32" (|g|^2 in FP32, literal per-channel form), "ff" (FP64-accurate
    branch-merged coefficients) or "c32" (those coefficients as FP32 pairs with the net-term
    arithmetic of the c32 device variant)."""

    PRECISIONS = {"fp32": 0, "ff": 1, "c32": 2}

    def __init__(self, channels, item_channels: int = 0, ctas_per_sm: int = 0, precision: str = "fp32", layout: int = 0,
                 stream=None):
        import torch

        self.channels = list(channels)
        arr = (ctypes.c_void_p * len(self.channels))(*[c._h.value for c in self.channels])
        self._arr = arr
        self.precision = precision
        o = _BatchOpts(int(item_channels), int(ctas_per_sm), Batch.PRECISIONS[precision], int(layout))
        nbytes = ctypes.c_size_t(0)
        _check(lib().pb_batch_arena_bytes(arr, len(self.channels), ctypes.byref(o), ctypes.byref(nbytes)))
        self.arena = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        _check(lib().pb_batch_create(arr, len(self.channels), ctypes.byref(o), ctypes.c_void_p(self.arena.data_ptr()),
                                     ctypes.c_size_t(int(nbytes.value)), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.refresh_info()

    def refresh_info(self):
        ns, nc = ctypes.c_int64(0), ctypes.c_int64(0)
        ic, ct = ctypes.c_int32(0), ctypes.c_int32(0)
        offs = np.empty(len(self.channels) + 1, np.int64)
        _check(lib().pb_batch_get_info(self._h, ctypes.byref(ns), ctypes.byref(nc), offs.ctypes.data, ctypes.byref(ic),
                                       ctypes.byref(ct)))
        self.nstate, self.nchannels = int(ns.value), int(nc.value)
        self.offsets = offs
        self.item_channels, self.ctas_per_sm = int(ic.value), int(ct.value)
        self.tiled = self.item_channels == 0  # symmetric tiles (precision ff / c32)

    def check(self, stream=None):
        """Raise if a bounded device-side wait of the tile sweep gave up since the last check."""
        _check(lib().pb_batch_check(self._h, _stream_ptr(stream)))

    def collision(self, f, out=None, stream=None):
        out = torch_empty(self.nstate) if out is None else out
        _check(lib().pb_batch_collision(self._h, _dev_vec(f, self.nstate, "f"), _dev_vec(out, self.nstate, "out"),
                                        _stream_ptr(stream)))
        return out

    def rk4(self, f, dt: float, nsteps: int = 1, stream=None):
        _check(lib().pb_batch_rk4_step(self._h, _dev_vec(f, self.nstate, "f"), float(dt), int(nsteps),
                                       _stream_ptr(stream)))
        return f

    def autotune(self, f, stream=None):
        bi, bc, bm = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
        _check(lib().pb_batch_autotune(self._h, _dev_vec(f, self.nstate, "f"), _stream_ptr(stream), ctypes.byref(bi),
                                       ctypes.byref(bc), ctypes.byref(bm)))
        self.refresh_info()
        return int(bi.value), int(bc.value), float(bm.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().pb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def torch_empty(n):
    import torch

    return torch.empty(n, dtype=torch.float64, device="cuda")


# fail loudly at import time when the native library is missing
lib()
