"""Host-side checks of the seeded serving request mix (no GPU)."""
import math

import numpy as np

from paper_2406_08923_gb300 import _lib as L
from paper_2406_08923_gb300 import serving


def test_request_mix_distribution_and_determinism():
    a = serving.make_requests(1024)
    b = serving.make_requests(1024)
    assert [(r.kind, r.n, r.nsteps) for r in a] == [(r.kind, r.n, r.nsteps) for r in b]
    n = np.array([r.n for r in a])
    assert n.min() >= 32 and n.max() <= 192 and np.all(n % 8 == 0)
    # log-uniform: the median of log n sits near the middle of [log 32, log 192]
    assert abs(np.median(np.log(n)) - 0.5 * (math.log(32) + math.log(192))) < 0.1
    steps = np.array([r.nsteps for r in a])
    assert steps.min() >= 10 and steps.max() <= 50
    kinds = np.bincount([serving.KINDS.index(r.kind) for r in a], minlength=3)
    assert np.all(np.abs(kinds - 1024 / 3) < 80)


def test_poisson_arrivals_rate():
    reqs = serving.poisson_arrivals(serving.make_requests(2000), rate_per_s=500.0)
    t = np.array([r.arrival for r in reqs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert abs((len(t) - 1) / t[-1] - 500.0) < 40.0


def test_serving_xcorr_weights_are_a_stable_smoother():
    w = np.array(serving.XC_WEIGHTS)
    assert math.isclose(w.sum(), 1.0, rel_tol=1e-12)
    k = np.linspace(0, math.pi, 257)
    sym = w[3] + 2 * sum(w[3 + j] * np.cos(j * k) for j in range(1, 4))
    assert np.all(np.abs(sym) <= 1.0 + 1e-12)


def test_request_params_fill_the_struct():
    q = serving.request_params(L.STENCIL_XCORR, 16)
    assert q.kind == L.STENCIL_XCORR and q.dims[0] == 16 ** 3 and q.dims[1] == 1
    q = serving.request_params(L.STENCIL_MHD8, 32)
    assert q.dims[2] == 32 and q.params.gamma > 1.0 and q.params.dt > 0
