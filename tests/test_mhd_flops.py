"""The algorithmic work count of one MHD cell-substep (the numerator of the MHD roofline).

The counted evaluation in mhd_flops.py must compute what the oracle computes (Eqs. A1-A4
with the Sec. 3.3 differences, then the 2N-storage RK3 update), so that its operation count
is the count of a correct evaluation of the method; the count itself is pinned, and the
benchmark uses exactly this value.
"""
import os
import re

import numpy as np
import pytest

import mhd_flops as MF
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAR = dict(cs0=1.1, gamma=5.0 / 3.0, cp=1.3, lnrho0=0.2, nu=7e-3, eta=4e-3, zeta=3e-3, mu0=1.2, dt=0.02)
H = (0.31, 0.27, 0.36)


def _oracle_par():
    return oracle.MhdParams(dx=H[0], dy=H[1], dz=H[2], cs0=PAR["cs0"], gamma=PAR["gamma"], cp=PAR["cp"],
                            lnrho0=PAR["lnrho0"], nu=PAR["nu"], eta=PAR["eta"], zeta=PAR["zeta"],
                            mu0=PAR["mu0"], K=0.0)


def _box(m, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.2, 0.2, size=(8, m, m, m))


def test_counted_rhs_equals_the_oracle():
    box = _box(7, 1)
    ref = oracle.mhd_rhs_box(box, _oracle_par())[:, 0, 0, 0]
    rhs, _, _, _ = MF.cell_substep(box, (0, 0, 0), H, PAR, [0.0] * 8, 0)
    np.testing.assert_allclose(rhs, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_counted_rk_substeps_equal_the_oracle():
    # substep 0 at the centre of a 7^3 box, then substep 1 at the centre of a 13^3 box after
    # substep 0 over the 7^3 neighbourhood it needs
    box = _box(13, 2)
    ref1 = oracle.mhd_rk3_box(box[:, 3:10, 3:10, 3:10], _oracle_par(), PAR["dt"], 1)[:, 3, 3, 3]
    _, f0, w0, _ = MF.cell_substep(box, (3, 3, 3), H, PAR, [0.0] * 8, 0)
    np.testing.assert_allclose(f0, ref1, rtol=1e-13)
    mid = box.copy()
    wmid = np.zeros((8, 7, 7, 7))
    for k in range(7):
        for j in range(7):
            for i in range(7):
                _, f, w, _ = MF.cell_substep(box, (k, j, i), H, PAR, [0.0] * 8, 0)
                mid[:, k + 3, j + 3, i + 3] = f
                wmid[:, k, j, i] = w
    ref2 = oracle.mhd_rk3_box(box, _oracle_par(), PAR["dt"], 2)[:, 6, 6, 6]
    _, f1, _, _ = MF.cell_substep(mid[:, 3:10, 3:10, 3:10], (0, 0, 0), H, PAR, wmid[:, 3, 3, 3], 1)
    np.testing.assert_allclose(f1, ref2, rtol=1e-12)


def test_count_per_substep():
    avg, nexp, per = MF.flops_per_cell_substep()
    # derivatives: 21 first (8 flop), 18 second (10), 18 mixed (14) = 600; then the RHS
    # (187 flop) and the RK update (24 on the first substep, 40 on the others)
    assert [p[0] for p in per] == [811, 827, 827]
    assert nexp == 2
    assert avg == pytest.approx(2465 / 3)


def test_bench_uses_this_count():
    src = open(os.path.join(ROOT, "bench.py")).read()
    m = re.search(r"^MHD_FLOPS_PER_CELL_SUBSTEP\s*=\s*([0-9.]+)\s*/\s*3", src, re.M)
    assert m, "bench.py must define MHD_FLOPS_PER_CELL_SUBSTEP = <flops per RK step> / 3"
    assert float(m.group(1)) == sum(p[0] for p in MF.flops_per_cell_substep()[2])
