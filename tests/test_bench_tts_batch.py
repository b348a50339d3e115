"""Host logic of the batched time-to-stationary summary in bench.py: which
forms get a wall-time ratio against the plain FP64 batch, which only a lower
bound, and how the ensemble window means are compared."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _form(cells, stationary, wall, p=None, x=None):
    done = stationary == cells
    return {"cells": cells, "stationary_cells": stationary, "wall_s": wall,
            "ensemble_window_means": {"p": p, "x_abs": x} if done else None}


def test_ratio_and_accuracy_when_every_cell_is_stationary():
    p64, x64 = [60.0, 12.0, 1.5, 48.0], [2.0, 1.0, 1e-6, 4.0]
    out = {"fp64": _form(4, 4, 124.2, p64, x64),
           "fused_ml": _form(4, 4, 18.1, [60.06, 11.97, 1.5, 48.0], [2.001, 1.0, 5e-6, 4.0])}
    ratio, lower, acc = bench.tts_batch_ratios(out)
    assert lower == {}
    assert np.isclose(ratio["fused_ml"], 124.2 / 18.1)
    # largest relative difference: P_port 1e-3 against P_ind 2.5e-3
    assert np.isclose(acc["fused_ml"]["ensemble_power_rel_diff"], 0.03 / 12.0)
    # the state entry below 1e-3 of the largest is left out of the comparison
    assert np.isclose(acc["fused_ml"]["ensemble_state_rel_diff"], 0.001 / 2.0)


def test_a_form_short_of_the_criterion_gets_no_ratio():
    out = {"fp64": _form(4, 4, 124.2, [1.0] * 4, [1.0]),
           "fused": _form(4, 2, 56.6),
           "fused_ml": _form(4, 4, 18.1, [1.0] * 4, [1.0])}
    ratio, lower, acc = bench.tts_batch_ratios(out)
    assert set(ratio) == {"fused_ml"} and set(acc) == {"fused_ml"} and lower == {}


def test_fp64_short_of_the_criterion_gives_a_lower_bound():
    out = {"fp64": _form(4, 3, 400.0), "fused": _form(4, 4, 50.0, [1.0] * 4, [1.0])}
    ratio, lower, acc = bench.tts_batch_ratios(out)
    assert ratio == {} and acc == {}
    assert np.isclose(lower["fused"], 8.0)


def test_without_an_fp64_run_there_is_nothing_to_compare():
    out = {"fused": _form(2, 2, 10.0, [1.0] * 4, [1.0])}
    assert bench.tts_batch_ratios(out) == ({}, {}, {})
