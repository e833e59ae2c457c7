"""Dense numpy brute force of Eq. 2 for tiny grids (TEST INFRASTRUCTURE ONLY).

Builds full [s, p, nu] arrays over every pair of window states: the momentum
transfer q = k_p - k_s is taken per pair (modulo the grid), not looped over as in
``oracle.c``, so the two oracle forms enumerate the channel set differently.
Follows Eq. 2 of arXiv:2511.03683 with the F_abs / F_em readings stated in
``oracle.c``.  Memory grows as nstate^2 * nmodes: keep nstate below ~1000.
"""
from __future__ import annotations

import numpy as np

HBAR_EVFS = 0.6582119569
KB_EVK = 8.617333262e-5


class Dense:
    def __init__(self, model, g2_min: float = 0.0, delta_nsigma: float = 0.0):
        self.model = model
        nb, nm = model.nbands, model.nmodes
        N1, N2, N3 = model.nk
        eps = np.asarray(model.eps, dtype=np.float64).reshape(-1)
        band = np.arange(eps.size) % nb
        if model.win is None:
            mask = np.ones(eps.size, dtype=bool)
        else:
            mask = (eps >= model.win[band, 0]) & (eps <= model.win[band, 1])
        self.ids = np.nonzero(mask)[0].astype(np.int32)
        ik = self.ids // nb
        j = np.stack([ik // (N2 * N3), (ik // N3) % N2, ik % N3], axis=1)
        dq = (j[None, :, :] - j[:, None, :]) % np.array([N1, N2, N3])
        iq = (dq[..., 0] * N2 + dq[..., 1]) * N3 + dq[..., 2]  # [s, p]
        self.w = np.asarray(model.omega, dtype=np.float64)[iq]  # [s, p, nu]
        self.valid = self.w > 0.0
        wv = np.where(self.valid, self.w, 1.0)
        self.N = np.where(self.valid, 1.0 / (np.exp(wv / (KB_EVK * model.T)) - 1.0), 0.0)
        self.g2 = np.where(self.valid, model.g2_dense(self.ids, self.ids), 0.0)
        self.eps_w = eps[self.ids]
        x = self.eps_w[:, None] - self.eps_w[None, :]
        sig = model.sigma
        norm = 1.0 / (np.sqrt(2.0 * np.pi) * sig)
        self.Ga = norm * np.exp(-((x[..., None] + self.w) ** 2) / (2 * sig * sig))
        self.Ge = norm * np.exp(-((x[..., None] - self.w) ** 2) / (2 * sig * sig))
        self.c = 2.0 * np.pi / (HBAR_EVFS * N1 * N2 * N3)
        keep = self.valid.copy()
        if g2_min > 0.0:
            keep &= self.g2 >= g2_min
        if delta_nsigma > 0.0:
            lim = delta_nsigma * sig
            keep &= ~((np.abs(x[..., None] + self.w) > lim) & (np.abs(x[..., None] - self.w) > lim))
        self.g2 = np.where(keep, self.g2, 0.0)
        self.valid = keep
        self.nchannels = int(keep.sum())

    @property
    def nstate(self) -> int:
        return len(self.ids)

    def terms(self, f):
        """Per-channel summand of Eq. 2 times (2 pi / hbar)(1/Nq): [s, p, nu] (sign: I = -sum)."""
        fs = f[:, None, None]
        fp = f[None, :, None]
        N = self.N
        Fabs = fs * (1 - fp) * N - (1 - fs) * fp * (N + 1)
        Fem = fs * (1 - fp) * (N + 1) - (1 - fs) * fp * N
        return self.c * self.g2 * (self.Ga * Fabs + self.Ge * Fem)

    def collision(self, f):
        return -self.terms(np.asarray(f, dtype=np.float64)).sum(axis=(1, 2))

    def W(self, f0):
        """Dense transport kernel W[s, p] = sum_nu (2pi/hbar)(1/Nq) g2 [Ga (N + f0_p) + Ge (N + 1 - f0_p)]."""
        fp = np.asarray(f0, dtype=np.float64)[None, :, None]
        N = self.N
        return (self.c * self.g2 * (self.Ga * (N + fp) + self.Ge * (N + 1 - fp))).sum(axis=2)

    def rates(self, f):
        return self.W(f).sum(axis=1)
