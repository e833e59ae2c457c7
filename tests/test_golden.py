"""Regression pin of the oracle against fixtures written by tests/golden/make_golden.py
(which calls only the oracle).  Tolerance allows for libm differences between hosts."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name,model", [("tiny4", synth.make_tiny(4)), ("window12", synth.make_window4(12))])
def test_oracle_matches_fixture(name, model):
    data = np.loadtxt(os.path.join(GOLDEN, f"oracle_{name}.txt"))
    f, I_ref, r_ref = data[:, 0], data[:, 1], data[:, 2]
    o = oracle.Oracle(model)
    assert np.array_equal(f, np.random.default_rng(20251103).uniform(0.0, 1.0, o.nstate))
    assert np.abs(o.collision(f) - I_ref).max() <= 1e-12 * np.abs(I_ref).max()
    assert np.abs(o.rates(f) - r_ref).max() <= 1e-12 * np.abs(r_ref).max()


@pytest.mark.parametrize("name", ["window24", "window40"])
def test_trajectory_fixture_conserves_carriers_and_cools(name):
    """The stored oracle trajectories (tests/golden/make_trajectory.py) keep the physics the
    rt-BTE fixes: the carrier number sum_s f_s is conserved (sum_s I_s = 0 on the closed channel
    list, so every RK4 step conserves it up to rounding), occupations stay in [0, 1], and the hot
    carriers lose energy to the phonon bath (carrier energy decreases from checkpoint to checkpoint)."""
    m = synth.make_config(name)
    o = oracle.Oracle(m)
    f0 = o.window_values(m.f_hot())
    eps = o.window_values(m.eps)
    data = np.loadtxt(os.path.join(GOLDEN, f"trajectory_{name}.txt"), ndmin=2)
    assert data.shape[0] == o.nstate
    energies = [(eps * f0).sum()]
    for k in range(data.shape[1]):
        f = data[:, k]
        assert abs(f.sum() - f0.sum()) <= 1e-12 * f0.sum()
        assert f.min() >= -1e-12 and f.max() <= 1.0
        energies.append((eps * f).sum())
    assert all(b < a for a, b in zip(energies, energies[1:]))
