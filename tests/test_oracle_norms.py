"""Pins of the oracle's norm reductions against numpy library routines."""
import math

import numpy as np

import oracle
from paper_2406_08923_gb300 import synth


def test_norms_match_numpy():
    f = synth.uniform(1, 1, 10007, -3, 2)
    s, s2, m = oracle.norms(f)
    assert math.isclose(s, math.fsum(f), rel_tol=1e-15, abs_tol=1e-12)
    assert math.isclose(s2, math.fsum(f * f), rel_tol=1e-15)
    assert m == np.abs(f).max()


def test_mass_matches_numpy():
    l = synth.uniform(2, 1, 999, -1e-3, 1e-3)
    assert math.isclose(oracle.mass(l), math.fsum(np.exp(l)), rel_tol=1e-14)
