"""Writes the stored expected values under tests/golden/ by calling only the oracle.

The paper prints no worked numerical example, so the fixtures here are oracle outputs on
tiny seeded inputs, kept as regression anchors: they must reproduce bit for bit on every
machine (the integer case) or to rounding (the FP64 case).  Run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2406_08923_gb300 import synth  # noqa: E402


def main():
    data, g = synth.xcorr_int32(16, seed=synth.SEED_XCORR)
    out = oracle.xcorr1d(data, g, 10)
    rec = {
        "what": "Eq. 3, 1D periodic cross-correlation, radius 3, 10 sweeps, int32 modulo 2^32",
        "cite": "Sec. 3.1 Eq. 3; padding Eq. 2 (periodic beta)",
        "seed": synth.SEED_XCORR, "n": 16, "sweeps": 10,
        "data": data.tolist(), "weights": g.tolist(), "expected": out.tolist(),
    }
    with open(os.path.join(HERE, "xcorr_int32_n16.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
    x = synth.xcorr_f64(32, seed=synth.SEED_XCORR)
    d2 = [1 / 90, -3 / 20, 3 / 2, -49 / 18, 3 / 2, -3 / 20, 1 / 90]
    y = oracle.xcorr1d(x, np.array(d2), 10)
    rec = {
        "what": "Eq. 3 with the 6th-order 2nd-derivative weights (dx = 1), 10 sweeps, FP64",
        "cite": "Sec. 3.1 Eq. 3; Sec. 3.3 (6th-order central differences)",
        "seed": synth.SEED_XCORR, "n": 32, "sweeps": 10,
        "data": [float.hex(float(v)) for v in x], "weights": [float.hex(v) for v in d2],
        "expected": [float.hex(float(v)) for v in y],
    }
    with open(os.path.join(HERE, "xcorr_f64_n32.json"), "w") as fh:
        json.dump(rec, fh, indent=1)


if __name__ == "__main__":
    main()
