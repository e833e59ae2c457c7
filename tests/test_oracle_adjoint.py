"""Pins of the oracle's reverse-mode pieces against central finite differences of the
oracle's own forward map (the definition of a derivative, not a retyped formula).

I[f] is quadratic in f and linear in each |g|^2, so central differences of L = sum lam I
are exact up to rounding for those two; the RK4 adjoint is checked along random
directions with an O(h^2) difference."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
import test_oracle_pins as pins


def test_collision_vjp_matches_central_differences():
    m = synth.make_tiny(4)
    o = oracle.Oracle(m)
    rng = np.random.default_rng(5)
    f = rng.uniform(0, 1, o.nstate)
    lam = rng.normal(size=o.nstate)
    g = o.collision_vjp(f, lam)
    for _ in range(5):
        d = rng.normal(size=o.nstate)
        h = 1e-3
        fd = (lam @ o.collision(f + h * d) - lam @ o.collision(f - h * d)) / (2 * h)
        assert abs(g @ d - fd) <= 1e-10 * (np.abs(g).sum() * np.abs(d).max())


def test_g2_gradient_matches_perturbed_callback():
    m = synth.make_tiny(3)
    o = oracle.Oracle(m)
    rng = np.random.default_rng(6)
    f = rng.uniform(0, 1, o.nstate)
    lam = rng.normal(size=o.nstate)
    base = synth.lib().synth_g2
    user = m.g2_user_ptr()
    CB = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p)
    for s, p, nu in [(0, 5, 1), (7, 7, 0), (12, 40, 2), (40, 12, 2)]:
        target = (int(o.ids[s]), int(o.ids[p]), nu)
        vals = []
        for scale in (1.0 + 1e-4, 1.0 - 1e-4):
            def g2(a, b, v, _u, scale=scale):
                x = base(a, b, v, user)
                return x * scale if (a, b, v) == target else x

            cb = CB(g2)
            o._m.g2 = ctypes.cast(cb, ctypes.c_void_p).value
            vals.append(lam @ o.collision(f))
            o._m.g2 = m.g2_fn_ptr()
        g2c = base(target[0], target[1], nu, user)
        fd = (vals[0] - vals[1]) / (2e-4 * g2c)
        an = o.g2_grad(f, lam, [s], [p], [nu])[0]
        assert abs(an - fd) <= 1e-7 * abs(an) + 1e-18


def test_rk4_adjoint_matches_central_differences():
    m = pins._narrow_model()
    o = oracle.Oracle(m)
    f0 = o.window_values(m.f_hot(e_exc=0.02, width=0.02))
    eps = o.window_values(m.eps)
    dt, n = 1.0, 8
    grad = o.rk4_vjp(f0, dt, n, eps)  # L = sum eps f(T)
    rng = np.random.default_rng(8)
    for _ in range(5):
        d = rng.normal(size=o.nstate) * f0.max()
        h = 1e-6
        fd = (eps @ o.rk4(f0 + h * d, dt, n) - eps @ o.rk4(f0 - h * d, dt, n)) / (2 * h)
        assert abs(grad @ d - fd) <= 1e-7 * abs(fd) + 1e-12
