"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

The paper (arXiv:2511.03683) prints no collision-integral values, so each pin
is a closed form, an invariant, a library solver or a brute force that a
plausible slip in the oracle (dropped term, wrong sign, N <-> N+1, wrong k+q
fold, transposed W) would break.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.dense import Dense

HBAR = 0.6582119569
KB = 8.617333262e-5


def gauss(x, s):
    return np.exp(-x * x / (2 * s * s)) / (np.sqrt(2 * np.pi) * s)


def nrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("model", [synth.make_tiny(4), synth.make_window4(12), synth.make_tiny(5)],
                         ids=["tiny4", "win12", "tiny5"])
def test_loop_matches_dense_bruteforce(model):
    """oracle.c (loop over q and m) == numpy brute force over all state pairs (Eq. 2)."""
    o, d = oracle.Oracle(model), Dense(model)
    assert np.array_equal(o.ids, d.ids)
    assert o.count_channels() == d.nchannels
    f = np.random.default_rng(1).uniform(0, 1, o.nstate)
    assert nrel(o.collision(f), d.collision(f)) < 1e-13
    assert nrel(o.rates(f), d.rates(f)) < 1e-13


def test_channel_count_tiny_closed_form():
    """8^3 grid, 2 bands, 3 modes with w > 0 everywhere, no window: (8^3*2)^2*3 channels."""
    o = oracle.Oracle(synth.make_config("tiny"))
    assert o.nstate == 1024
    assert o.count_channels() == 1024 * 1024 * 3 == 3145728


def test_pair_antisymmetry_and_conservation():
    """A channel adds equal and opposite amounts to I(nk) and I(mk+q) (Sec. 'Optimized GPU
    algorithm', step 1), so sum_s I_s = 0 for any f."""
    d = Dense(synth.make_tiny(4))
    f = np.random.default_rng(2).uniform(0, 1, d.nstate)
    t = d.terms(f)
    assert np.abs(t + np.transpose(t, (1, 0, 2))).max() <= 1e-15 * np.abs(t).max()
    o = oracle.Oracle(synth.make_config("tiny"))
    f = o.window_values(synth.make_config("tiny").f_hot())
    I, ab = o.collision(f, with_abs=True)
    assert abs(I.sum()) <= 1e-13 * ab.sum()


def test_two_level_detailed_balance():
    """Two flat bands split by exactly hbar*w0 with one Einstein mode w0: for Fermi-Dirac f at
    the phonon temperature every channel obeys detailed balance, so I = 0 up to rounding.
    Swapping N and N+1 in either occupation factor breaks it at O(1)."""
    m = synth.make_two_level(3, w0=0.05, sigma=0.004)
    o = oracle.Oracle(m)
    for mu in (-0.1, 0.02, 0.2):
        f = o.window_values(m.f_fermi(mu))
        I = o.collision(f)
        N = 1.0 / np.expm1(0.05 / (KB * m.T))
        c = 2 * np.pi / (HBAR * 27)
        scale = c * 27 * np.exp(m.g2_mu) * gauss(0.0, m.sigma) * max(f.max() * (1 - f.min()) * (N + 1), 1e-300)
        assert np.abs(I).max() <= 1e-13 * scale
    # a non-equilibrium f gives O(scale) values, so the pin has teeth
    f = o.window_values(m.f_fermi(0.02)) * 0.5
    assert np.abs(o.collision(f)).max() > 1e-3 * scale


@pytest.mark.parametrize("w0,T", [(0.04, 300.0), (0.02, 77.0)])
def test_flat_band_closed_forms(w0, T):
    """One flat band, Einstein mode w0, constant |g|^2 = g0: x = 0 for every channel, so
    1/tau = (2pi/hbar) g0 G_sigma(w0) (2N+1) for any f, and I_s = -(f_s - <f>)/tau."""
    m = synth.make_flat_einstein(4, w0=w0, T=T)
    o = oracle.Oracle(m)
    f = np.random.default_rng(3).uniform(0, 1, o.nstate)
    g0 = np.exp(m.g2_mu)
    N = 1.0 / np.expm1(w0 / (KB * T))
    inv_tau = 2 * np.pi / HBAR * g0 * gauss(w0, m.sigma) * (2 * N + 1)
    assert nrel(o.rates(f), np.full(o.nstate, inv_tau)) < 1e-13
    assert nrel(o.collision(f), -(f - f.mean()) * inv_tau) < 1e-12


def test_dispersive_band_rates_dos():
    """One tight-binding band, Einstein mode w0, constant |g|^2, uniform f:
    1/tau_s = (2pi/hbar) g0 [(N+1-f) D(eps_s - w0) + (N+f) D(eps_s + w0)],
    D(E) = (1/Nk) sum_k G_sigma(E - eps_k), the smeared density of states."""
    n, w0, fu = 6, 0.03, 0.3
    eps, vel = synth.tight_binding((n, n, n), [0.0])
    m = synth.Model("disp", (n, n, n), 1, 1, eps, vel, np.full((n ** 3, 1), w0), None, 300.0, 0.02,
                    g2_mu=np.log(2e-3), g2_sigma_ln=0.0, seed=5)
    o = oracle.Oracle(m)
    e = eps[:, 0]
    D = lambda E: gauss(E[:, None] - e[None, :], m.sigma).mean(axis=1)
    N = 1.0 / np.expm1(w0 / (KB * m.T))
    ref = 2 * np.pi / HBAR * 2e-3 * ((N + 1 - fu) * D(e - w0) + (N + fu) * D(e + w0))
    assert nrel(o.rates(np.full(o.nstate, fu)), ref) < 1e-13


def test_rates_are_minus_dI_dfs():
    """1/tau_s = -dI_s/df_s (central differences) on a model with no q = 0 channel (every
    mode acoustic, so hbar*w(Gamma) = 0 removes the self channel)."""
    n = 4
    eps, vel = synth.tight_binding((n, n, n), [0.0, 0.15])
    s = synth.acoustic_shape((n, n, n))
    omega = np.stack([0.02 * s, 0.035 * s], axis=1)
    m = synth.Model("acoustic", (n, n, n), 2, 2, eps, vel, omega, None, 300.0, 0.01, seed=9)
    o = oracle.Oracle(m)
    f = np.random.default_rng(4).uniform(0.1, 0.9, o.nstate)
    rows = np.array([0, 5, 17, 63, 100, o.nstate - 1])
    h = 1e-5
    num = []
    for r in rows:
        fp, fm = f.copy(), f.copy()
        fp[r] += h
        fm[r] -= h
        num.append(-(o.collision(fp, rows=[r])[0] - o.collision(fm, rows=[r])[0]) / (2 * h))
    # I_s is quadratic in f_s, so the central difference is exact up to rounding
    assert nrel(np.array(num), o.rates(f, rows=rows)) < 1e-8


def _narrow_model(n=3):
    """Narrow bands (t = 10 meV) so that phonon energies resonate on a 3^3 grid."""
    eps, vel = synth.tight_binding((n, n, n), [0.0, 0.03], t=0.01)
    s = synth.acoustic_shape((n, n, n))
    omega = np.stack([(10 + 5 * nu + 5 * s) * 1e-3 for nu in range(3)], axis=1)
    return synth.Model("narrow", (n, n, n), 2, 3, eps, vel, omega, None, 300.0, 0.005, seed=21)


def test_rk4_fourth_order_and_scipy():
    """Classic RK4: global error falls 16x per halving of dt, and the trajectory matches
    scipy's DOP853 at rtol 1e-13 (rt-BTE, Eq. 1 with no field)."""
    scipy_integrate = pytest.importorskip("scipy.integrate")
    m = _narrow_model()
    o = oracle.Oracle(m)
    f0 = o.window_values(m.f_hot(e_exc=0.02, width=0.02))
    T = 40.0
    ref = scipy_integrate.solve_ivp(lambda t, y: o.collision(y), (0, T), f0, method="DOP853", rtol=1e-13,
                                    atol=1e-16).y[:, -1]
    assert np.abs(ref - f0).max() > 0.1 * f0.max()  # the populations really move
    errs = [np.abs(o.rk4(f0, T / n, n) - ref).max() for n in (40, 80, 160)]
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20
    assert np.abs(o.rk4(f0, T / 400, 400) - ref).max() < 1e-10 * np.abs(f0).max()


def _transport_model(n=4):
    return synth.make_tiny(n).with_(sigma=0.01)


def test_transport_first_iterate_is_rta():
    """F^0 = tau v: the transport map applied to F = 0 gives the relaxation-time limit, and
    its tau is 1/rates(f0)."""
    m = _transport_model()
    o = oracle.Oracle(m)
    f0 = o.window_values(m.f_fermi(0.0))
    v = o.window_values(m.vel)
    F1, tau = o.transport_map(f0, v, np.zeros_like(v))
    inv_tau = o.rates(f0)
    assert nrel(tau, 1.0 / inv_tau) < 1e-14
    assert nrel(F1, v / inv_tau[:, None]) < 1e-14


def test_transport_fixed_point_matches_lstsq():
    """The converged iterate solves (1 - tau W) F = tau v: compare the shift-invariant
    conductivity-like observable with numpy.linalg.lstsq on the dense system."""
    m = _transport_model()
    o, d = oracle.Oracle(m), Dense(m)
    f0 = o.window_values(m.f_fermi(0.0))
    v = o.window_values(m.vel)
    F, iters, res, ok = o.transport(f0, v, tol=1e-12, maxit=3000)
    assert ok and res <= 1e-12
    W = d.W(f0)
    tau = 1.0 / W.sum(axis=1)
    A = np.eye(d.nstate) - tau[:, None] * W
    Fl = np.linalg.lstsq(A, tau[:, None] * v, rcond=None)[0]
    wgt = (f0 * (1 - f0))[:, None]
    s_it = (wgt * v * F).sum(axis=0)
    s_ls = (wgt * v * Fl).sum(axis=0)
    assert np.abs(s_it - s_ls).max() <= 1e-8 * np.abs(s_ls).max()
    # the residual of the linear system itself
    r = A @ F - tau[:, None] * v
    assert np.abs(r).max() <= 1e-9 * np.abs(F).max()


def test_transport_cubic_symmetry():
    """With cubic-invariant bands, phonons and |g|^2 the tensor sum_s f0(1-f0) v_a F_b is
    isotropic: equal diagonal, vanishing off-diagonal."""
    m = _transport_model(4)
    o = oracle.Oracle(m)
    f0 = o.window_values(m.f_fermi(0.0))
    v = o.window_values(m.vel)
    F, iters, res, ok = o.transport(f0, v, tol=1e-12, maxit=3000)
    assert ok
    S = ((f0 * (1 - f0))[:, None, None] * v[:, :, None] * F[:, None, :]).sum(axis=0)
    diag = np.diag(S)
    assert np.abs(diag - diag.mean()).max() <= 1e-10 * abs(diag.mean())
    assert np.abs(S - np.diag(diag)).max() <= 1e-10 * abs(diag.mean())


@pytest.mark.parametrize("g2_min,nsig", [(1e-3, 0.0), (0.0, 3.0), (5e-4, 4.0)])
def test_cutoffs_loop_matches_dense(g2_min, nsig):
    """The paper's optional |g| and delta cutoffs: C loop == brute force with the same mask,
    and the pruned sum stays antisymmetric (conservation)."""
    m = synth.make_window4(12)
    o, d = oracle.Oracle(m, g2_min=g2_min, delta_nsigma=nsig), Dense(m, g2_min=g2_min, delta_nsigma=nsig)
    assert o.count_channels() == d.nchannels < Dense(m).nchannels
    f = np.random.default_rng(2).uniform(0, 1, o.nstate)
    assert nrel(o.collision(f), d.collision(f)) < 1e-13
    assert nrel(o.rates(f), d.rates(f)) < 1e-13
    I, ab = o.collision(f, with_abs=True)
    assert abs(I.sum()) <= 1e-13 * ab.sum()
