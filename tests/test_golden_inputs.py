"""The stored oracle values still describe the inputs the generators make."""

import importlib.util
import os

import numpy as np

from rqc import make_workload


def _mg():
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(__file__), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


def test_grid5x6_golden_matches_generated_inputs():
    mg = _mg()
    digest, amps = mg.read("grid5x6_m14")
    w = make_workload("grid5x6_m14")
    assert digest == mg.input_digest(w.circuit, w.bits)
    assert amps.shape == (4096,)
    # Porter-Thomas scale: 2^30 <|amp|^2> = 1 + F with F ~ 0 for uniform bitstrings
    f = (2.0 ** 30) * np.mean(np.abs(amps) ** 2) - 1.0
    assert abs(f) < 4 * np.sqrt(1.0 / 4096)
