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
