"""The oracle pins have teeth: each plausible slip, planted in a separate build of
oracle.c (ORACLE_PLANT=k), makes at least one pin of test_oracle_pins.py fail."""
import numpy as np
import pytest

import oracle
import synth
import test_oracle_pins as pins

PLANTS = {
    1: "F_abs with N and N+1 swapped",
    2: "emission term dropped",
    3: "absorption and emission deltas swapped",
    4: "phonon energy taken at k+q instead of q",
    5: "rate occupation factors swapped",
    6: "rate factor uses f_s instead of f_p",
    7: "RK4 weights 1/4 each",
    8: "RK4 last stage at dt/2",
}


def _pin_calls():
    return [
        ("loop_vs_dense_tiny4", lambda: pins.test_loop_matches_dense_bruteforce(synth.make_tiny(4))),
        ("loop_vs_dense_win12", lambda: pins.test_loop_matches_dense_bruteforce(synth.make_window4(12))),
        ("conservation", pins.test_pair_antisymmetry_and_conservation),
        ("two_level", pins.test_two_level_detailed_balance),
        ("flat_300", lambda: pins.test_flat_band_closed_forms(0.04, 300.0)),
        ("dispersive_dos", pins.test_dispersive_band_rates_dos),
        ("rates_dIdf", pins.test_rates_are_minus_dI_dfs),
        ("rk4", pins.test_rk4_fourth_order_and_scipy),
        ("transport_rta", pins.test_transport_first_iterate_is_rta),
        ("transport_lstsq", pins.test_transport_fixed_point_matches_lstsq),
    ]


@pytest.mark.parametrize("plant", sorted(PLANTS), ids=[PLANTS[k] for k in sorted(PLANTS)])
def test_planted_mistake_is_caught(plant, monkeypatch):
    class Planted(oracle.Oracle):
        def __init__(self, model, nthreads=0):
            super().__init__(model, nthreads=nthreads, plant=plant)

    monkeypatch.setattr(pins.oracle, "Oracle", Planted)
    caught = []
    for name, call in _pin_calls():
        try:
            with np.errstate(all="ignore"):
                call()
        except (AssertionError, FloatingPointError, ValueError, np.linalg.LinAlgError):
            caught.append(name)
    assert caught, f"no pin catches: {PLANTS[plant]}"


def test_unplanted_build_passes_every_pin():
    for name, call in _pin_calls():
        call()
