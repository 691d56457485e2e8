"""The oracle reproduces its stored golden outputs (tests/golden/, see make_golden.py)."""
import json
import os

import numpy as np

import oracle

G = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_xcorr_int32_golden_bit_exact():
    rec = json.load(open(os.path.join(G, "xcorr_int32_n16.json")))
    out = oracle.xcorr1d(np.array(rec["data"], np.int32), np.array(rec["weights"], np.int32),
                         rec["sweeps"])
    assert out.tolist() == rec["expected"]


def test_xcorr_f64_golden():
    rec = json.load(open(os.path.join(G, "xcorr_f64_n32.json")))
    x = np.array([float.fromhex(v) for v in rec["data"]])
    g = np.array([float.fromhex(v) for v in rec["weights"]])
    exp = np.array([float.fromhex(v) for v in rec["expected"]])
    np.testing.assert_allclose(oracle.xcorr1d(x, g, rec["sweeps"]), exp, rtol=1e-12,
                               atol=1e-12 * np.abs(exp).max())
