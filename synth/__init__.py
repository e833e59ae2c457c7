"""Seeded synthetic e-ph model inputs (test and benchmark input generation only).

The paper's inputs are first-principles band energies eps_nk, phonon energies
hbar*omega_nuq and couplings |g_mnnu(k,q)|^2 on commensurate k/q grids (Eq. 2,
Sec. "Collision integral, e-ph coupling matrix, and scattering channels").  Its
DFT data (Table 1) is not available, so this module builds stand-ins with the
same structure:

* tight-binding bands  eps_n(k) = E_n + 2t sum_i (1 - cos k_i),  k_i = 2 pi j_i / N_i;
* band velocities      v_n(k) = (2t/hbar) sin k  (lattice constant 1);
* phonons with an acoustic branch shape s(q) = sqrt(sum_i sin^2(q_i/2) / 3);
* |g|^2 log-normal, drawn from a hash of a canonical channel key (synth.c);
* a hot Gaussian initial population and a Fermi-Dirac equilibrium.

All arrays are over the FULL grid: choosing the states inside the energy window
is part of the method and is done separately by each consumer.  The module holds
none of the collision-integral arithmetic (no Gaussian delta, no Bose factor, no
occupation factors).  Every value is bitwise invariant under the cubic group
acting on k (sums are taken over sorted per-axis terms, odd functions are built
from folded indices), so the synthetic problem has exact inversion and cubic
symmetry.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

HBAR_EVFS = 0.6582119569  # eV fs
KB_EVK = 8.617333262e-5  # eV / K

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")


class G2Params(ctypes.Structure):
    _fields_ = [
        ("nk", ctypes.c_int32 * 3),
        ("nbands", ctypes.c_int32),
        ("nmodes", ctypes.c_int32),
        ("cubic", ctypes.c_int32),
        ("mu", ctypes.c_double),
        ("sigma_ln", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (plain C, -O2, portable flags)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.synth_g2.restype = ctypes.c_double
        _lib.synth_g2.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        _lib.synth_g2_dense.restype = None
        _lib.synth_g2_dense.argtypes = [
            ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
            ctypes.c_void_p, ctypes.c_void_p]
    return _lib


@dataclass
class Model:
    """One synthetic e-ph system on an N1 x N2 x N3 grid (q grid = k grid)."""

    name: str
    nk: tuple
    nbands: int
    nmodes: int
    eps: np.ndarray  # [Nk, nb] eV
    vel: np.ndarray  # [Nk, nb, 3] lattice units / fs
    omega: np.ndarray  # [Nq, nmodes] hbar*omega in eV (Nq = Nk)
    win: np.ndarray | None  # [nb, 2] per-band energy window (eV) or None
    T: float  # K
    sigma: float  # eV, Gaussian smearing of the delta function
    g2_mu: float = -7.0
    g2_sigma_ln: float = 1.0
    seed: int = 20251103
    cubic: bool = True
    _params: G2Params | None = field(default=None, repr=False)

    @property
    def nkt(self) -> int:
        return int(np.prod(self.nk))

    def g2_params(self) -> G2Params:
        if self._params is None:
            p = G2Params()
            for i in range(3):
                p.nk[i] = int(self.nk[i])
            p.nbands = self.nbands
            p.nmodes = self.nmodes
            p.cubic = 1 if (self.cubic and len(set(self.nk)) == 1) else 0
            p.mu = self.g2_mu
            p.sigma_ln = self.g2_sigma_ln
            p.seed = self.seed
            self._params = p
        return self._params

    def g2_fn_ptr(self) -> int:
        """Address of the C function double synth_g2(int s, int p, int nu, const void*)."""
        return ctypes.cast(lib().synth_g2, ctypes.c_void_p).value

    def g2_batch_ptr(self) -> int:
        """Address of int synth_g2_batch(int64 n, const int32*, const int32*, const int32*, double*, void*)."""
        return ctypes.cast(lib().synth_g2_batch, ctypes.c_void_p).value

    def g2_user_ptr(self) -> int:
        return ctypes.addressof(self.g2_params())

    def g2(self, s: int, p: int, nu: int) -> float:
        return lib().synth_g2(s, p, nu, ctypes.byref(self.g2_params()))

    def g2_dense(self, s_ids: np.ndarray, p_ids: np.ndarray) -> np.ndarray:
        """|g|^2 for every (s, p, nu) of two id lists, shape [len(s), len(p), nmodes]."""
        s_ids = np.ascontiguousarray(s_ids, dtype=np.int32)
        p_ids = np.ascontiguousarray(p_ids, dtype=np.int32)
        out = np.empty((len(s_ids), len(p_ids), self.nmodes), dtype=np.float64)
        lib().synth_g2_dense(len(s_ids), s_ids.ctypes.data, len(p_ids), p_ids.ctypes.data, self.nmodes,
                             out.ctypes.data, ctypes.byref(self.g2_params()))
        return out

    def kcoords(self) -> np.ndarray:
        """Integer grid coordinates j[ik] = (j1, j2, j3), ik = (j1*N2 + j2)*N3 + j3."""
        return grid_coords(self.nk)

    def f_hot(self, e_exc: float = 0.3, amp: float = 0.1, width: float = 0.05) -> np.ndarray:
        """Hot Gaussian population centred e_exc above the lowest window energy, [Nk, nb]."""
        emin = self.emin()
        return amp * np.exp(-((self.eps - emin - e_exc) ** 2) / (2.0 * width * width))

    def f_fermi(self, mu: float) -> np.ndarray:
        """Fermi-Dirac occupations at the model temperature, [Nk, nb]."""
        return 1.0 / (np.exp((self.eps - mu) / (KB_EVK * self.T)) + 1.0)

    def emin(self) -> float:
        """Lowest band energy inside the window (used only to place input populations)."""
        if self.win is None:
            return float(self.eps.min())
        inwin = (self.eps >= self.win[None, :, 0]) & (self.eps <= self.win[None, :, 1])
        return float(self.eps[inwin].min())

    def with_(self, **kw) -> "Model":
        kw.setdefault("_params", None)
        return replace(self, **kw)


def grid_coords(nk) -> np.ndarray:
    """Integer grid coordinates j[ik] = (j1, j2, j3), ik = (j1*N2 + j2)*N3 + j3."""
    n1, n2, n3 = nk
    j1, j2, j3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    return np.stack([j1.ravel(), j2.ravel(), j3.ravel()], axis=1).astype(np.int64)


def _folded(j: np.ndarray, n: int) -> np.ndarray:
    return np.minimum(j, (n - j) % n)


def _sorted_axis_sum(terms: np.ndarray) -> np.ndarray:
    """Sum three per-axis terms in ascending order (bitwise permutation invariant)."""
    t = np.sort(terms, axis=1)
    return (t[:, 0] + t[:, 1]) + t[:, 2]


def tight_binding(nk, offsets, t=0.3):
    """eps[ik, n] = E_n + 2t sum_i (1 - cos k_i) and v = (2t/hbar) sin k."""
    j = grid_coords(nk)
    nkt = j.shape[0]
    cosine = np.empty((nkt, 3))
    sine = np.empty((nkt, 3))
    for i in range(3):
        n = nk[i]
        jj = _folded(j[:, i], n)
        cosine[:, i] = 1.0 - np.cos(2.0 * np.pi * jj / n)
        s = np.sin(2.0 * np.pi * jj / n)
        s[(jj == 0) | (2 * jj == n)] = 0.0
        sign = np.where(j[:, i] > n // 2, -1.0, 1.0)
        sine[:, i] = sign * s
    disp = 2.0 * t * _sorted_axis_sum(cosine)
    eps = np.asarray(offsets, dtype=np.float64)[None, :] + disp[:, None]
    vel = np.repeat(((2.0 * t / HBAR_EVFS) * sine)[:, None, :], len(offsets), axis=1)
    return eps, vel


def acoustic_shape(nk) -> np.ndarray:
    """s(q) = sqrt(sum_i sin^2(q_i / 2) / 3) in [0, 1], per q on the grid."""
    j = grid_coords(nk)
    terms = np.empty((j.shape[0], 3))
    for i in range(3):
        n = nk[i]
        jj = _folded(j[:, i], n)
        terms[:, i] = np.sin(np.pi * jj / n) ** 2
    return np.sqrt(_sorted_axis_sum(terms) / 3.0)


def make_tiny(n: int = 8, seed: int = 20251103, **kw) -> Model:
    """8^3 full-BZ grid, 2 bands (E_n = 0.5 n eV, t = 0.3 eV), 3 modes
    hbar*omega_nu(q) = 10 + 5 nu + 5 s(q) meV, sigma = 5 meV, T = 300 K, no window."""
    nk = (n, n, n)
    eps, vel = tight_binding(nk, [0.0, 0.5])
    s = acoustic_shape(nk)
    omega = np.stack([(10.0 + 5.0 * nu + 5.0 * s) * 1e-3 for nu in range(3)], axis=1)
    m = Model(f"tiny{n}", nk, 2, 3, eps, vel, omega, None, 300.0, 0.005, seed=seed)
    return m.with_(**kw) if kw else m


def make_window4(n: int = 40, seed: int = 20251104, **kw) -> Model:
    """n^3 grids, 4 bands (offsets 0/0.2/1.1/1.3 eV, t = 0.3 eV), 6 modes (3 acoustic
    15/20/25 meV * s(q), 3 optical flat 35/47.5/60 meV), per-band window 0.3 eV above
    each band minimum, sigma = 8 meV, T = 300 K."""
    nk = (n, n, n)
    offsets = [0.0, 0.2, 1.1, 1.3]
    eps, vel = tight_binding(nk, offsets)
    s = acoustic_shape(nk)
    ac = [15e-3 * s, 20e-3 * s, 25e-3 * s]
    op = [np.full_like(s, 35e-3), np.full_like(s, 47.5e-3), np.full_like(s, 60e-3)]
    omega = np.stack(ac + op, axis=1)
    win = np.array([[e - 1.0, e + 0.3] for e in offsets])
    m = Model(f"win4_{n}", nk, 4, 6, eps, vel, omega, win, 300.0, 0.008, seed=seed)
    return m.with_(**kw) if kw else m


def make_flat_einstein(n: int = 4, w0: float = 0.04, e0: float = 0.1, g2: float = 1e-3,
                       sigma: float = 0.01, T: float = 300.0, seed: int = 7) -> Model:
    """One flat band eps = e0, one Einstein mode hbar*omega = w0, constant |g|^2 = g2."""
    nk = (n, n, n)
    nkt = n ** 3
    eps = np.full((nkt, 1), e0)
    vel = np.zeros((nkt, 1, 3))
    omega = np.full((nkt, 1), w0)
    return Model(f"flat{n}", nk, 1, 1, eps, vel, omega, None, T, sigma, g2_mu=float(np.log(g2)),
                 g2_sigma_ln=0.0, seed=seed)


def make_two_level(n: int = 3, e0: float = 0.0, w0: float = 0.05, g2: float = 2e-3,
                   sigma: float = 0.004, T: float = 300.0, seed: int = 11) -> Model:
    """Two flat bands e0 and e0 + w0 joined by one Einstein mode of energy w0 (constant |g|^2)."""
    nk = (n, n, n)
    nkt = n ** 3
    eps = np.stack([np.full(nkt, e0), np.full(nkt, e0 + w0)], axis=1)
    vel = np.zeros((nkt, 2, 3))
    omega = np.full((nkt, 1), w0)
    return Model(f"twolevel{n}", nk, 2, 1, eps, vel, omega, None, T, sigma, g2_mu=float(np.log(g2)),
                 g2_sigma_ln=0.0, seed=seed)


_BAND_OFFSETS = [0.0, 0.2, 1.1, 1.3]


def make_batch_instance(i: int, seed: int = 20251107) -> tuple:
    """Instance i of the batched workload: grid N^3 with N uniform in 16..36, 2-4 bands
    (offsets from 0/0.2/1.1/1.3 eV), 3-6 modes (acoustic 15/20/25 meV x s(q), then optical
    flat 35/47.5/60 meV), T uniform in 100..500 K, per-band 0.3 eV window, sigma 8 meV.
    Returns (model, excitation energy in eV, uniform in 0.1..0.5)."""
    rng = np.random.default_rng([seed, i])
    n = int(rng.integers(16, 37))
    nb = int(rng.integers(2, 5))
    nm = int(rng.integers(3, 7))
    T = float(rng.uniform(100.0, 500.0))
    e_exc = float(rng.uniform(0.1, 0.5))
    nk = (n, n, n)
    offsets = _BAND_OFFSETS[:nb]
    eps, vel = tight_binding(nk, offsets)
    s = acoustic_shape(nk)
    branches = [15e-3 * s, 20e-3 * s, 25e-3 * s, np.full_like(s, 35e-3), np.full_like(s, 47.5e-3),
                np.full_like(s, 60e-3)]
    omega = np.stack(branches[:nm], axis=1)
    win = np.array([[e - 1.0, e + 0.3] for e in offsets])
    m = Model(f"batch{i}_{n}", nk, nb, nm, eps, vel, omega, win, T, 0.008, seed=seed * 1000 + i)
    return m, e_exc


def make_config(name: str) -> Model:
    """Named workloads: 'tiny' (8^3, ~3.1M channels), 'window40' (40^3, ~1.36e8 channels),
    'window24' (24^3, ~6.3e6 channels), and 'window<N>' for the same rule on an N^3 grid."""
    if name == "tiny":
        return make_tiny(8, seed=20251103)
    if name == "window40":
        return make_window4(40, seed=20251104)
    if name == "window24":
        return make_window4(24, seed=20251106)
    if name.startswith("window") and name[6:].isdigit():
        return make_window4(int(name[6:]), seed=20251100 + int(name[6:]))
    raise KeyError(name)
