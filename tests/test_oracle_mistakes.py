"""Planted mistakes in the oracle: each one must fail at least one of the oracle's pins.

Every case is a plausible slip in the oracle: in its C arithmetic (oracle/oracle.c: a dropped
term, a wrong sign, a transposed operand or index, a wrong constant, an off-by-one window) or
in its Python wrapper (oracle/__init__.py: axis order, array shapes, parameter order, integer
masking).  The test copies the package into a temporary directory with the one mistake in
it, compiles the copy's library there, and runs the oracle's pin tests
(tests/test_oracle_*.py, this file excluded) in a subprocess with STENCIL_ORACLE_MUTANT_PKG
naming the copy (conftest.py loads it in place of the package).  A mistake that passes every
pin would be one the pins cannot tell from the paper's arithmetic.  The committed oracle is
only read.  Everything runs on the host.
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PY = os.path.join(ROOT, "oracle", "__init__.py")
PIN_FILES = sorted(f for f in glob.glob(os.path.join(HERE, "test_oracle_*.py"))
                   if os.path.basename(f) != os.path.basename(__file__))

# (name, exact text in oracle.c, replacement).  Each text occurs exactly once.
MUTANTS = [
    # Eq. 2: periodic image
    ("pad_x_shift", "int64_t si = wrap(i - hx, nx)", "int64_t si = wrap(i + hx, nx)"),
    ("pad_y_off_by_one", "sj = wrap(j - hy, ny)", "sj = wrap(j - hy + 1, ny)"),
    ("pad_z_shift", "sk = wrap(k - hz, nz)", "sk = wrap(k + hz, nz)"),
    # Eq. 3: cross-correlation
    ("xcorr_f64_convolution", "acc += g[j + r] * fhat[i + r + j];", "acc += g[j + r] * fhat[i + r - j];"),
    ("xcorr_u32_dropped_term", "for (int j = -r; j <= r; ++j) acc += (uint32_t)g[j + r]",
     "for (int j = -r; j < r; ++j) acc += (uint32_t)g[j + r]"),
    ("xcorr_sweeps_one_short", "for (int s = 0; s < sweeps; ++s) {\n        pad_periodic(cur, n, 1, 1, r, sizeof(double), hat);\n        oracle_xcorr1d_box_f64",
     "for (int s = 1; s < sweeps; ++s) {\n        pad_periodic(cur, n, 1, 1, r, sizeof(double), hat);\n        oracle_xcorr1d_box_f64"),
    # Sec. 2.1: max filter
    ("maxfilter_window_short", "double m = fhat[i];\n        for (int j = 1; j <= 2 * r; ++j)",
     "double m = fhat[i];\n        for (int j = 1; j < 2 * r; ++j)"),
    ("maxfilter_i32_min", "int32_t m = fhat[i];\n        for (int j = 1; j <= 2 * r; ++j)\n            if (fhat[i + j] > m)",
     "int32_t m = fhat[i];\n        for (int j = 1; j <= 2 * r; ++j)\n            if (fhat[i + j] < m)"),
    # Sec. 3.3: 6th-order central differences
    ("d1_sign", "static const double C1[7] = {-1.0 / 60.0", "static const double C1[7] = {1.0 / 60.0"),
    ("d1_constant", "3.0 / 4.0,   -3.0 / 20.0, 1.0 / 60.0}", "3.0 / 4.0,   -3.0 / 20.0, 1.0 / 61.0}"),
    ("d1_spacing_squared", "acc += C1[j + R] * f[p + j * s];\n    return acc / h;",
     "acc += C1[j + R] * f[p + j * s];\n    return acc / (h * h);"),
    ("d2_centre", "-49.0 / 18.0", "-49.0 / 17.0"),
    ("d2_spacing_linear", "return acc / (h * h);\n}\n\nstatic double dermix", "return acc / h;\n}\n\nstatic double dermix"),
    ("mixed_constant", "{270.0, -27.0, 2.0}", "{270.0, -27.0, 3.0}"),
    ("mixed_sign", "double d = f[p + a * s1 + a * s2] - f[p + a * s1 - a * s2]",
     "double d = f[p + a * s1 + a * s2] + f[p + a * s1 - a * s2]"),
    ("mixed_spacing_transposed", "acc / (720.0 * h1 * h2)", "acc / (720.0 * h1 * h1)"),
    ("derivs_dz_uses_y_stride", "out[2 * ncell + o] = der1(fhat, p, sz, h[2]);", "out[2 * ncell + o] = der1(fhat, p, sy, h[2]);"),
    ("derivs_dyz_uses_dxz", "out[8 * ncell + o] = dermix(fhat, p, sy, sz, h[1], h[2]);",
     "out[8 * ncell + o] = dermix(fhat, p, sx, sz, h[1], h[2]);"),
    # Eq. 4: diffusion
    ("diffusion_dropped_z_axis", "for (int a = 0; a < 3; ++a)\n                    if (n[a] > 1) lap += der2(fhat",
     "for (int a = 0; a < 2; ++a)\n                    if (n[a] > 1) lap += der2(fhat"),
    ("diffusion_sign", "lap += der2(fhat, p, s[a], h[a]);\n                out[(k * ny + j) * nx + i] = fhat[p] + dt * alpha * lap;",
     "lap += der2(fhat, p, s[a], h[a]);\n                out[(k * ny + j) * nx + i] = fhat[p] - dt * alpha * lap;"),
    ("diffusion_alpha_dropped", "lap += der2(fhat, p, s[a], h[a]);\n                out[(k * ny + j) * nx + i] = fhat[p] + dt * alpha * lap;",
     "lap += der2(fhat, p, s[a], h[a]);\n                out[(k * ny + j) * nx + i] = fhat[p] + dt * lap;"),
    ("diffusion_spacing_axis", "if (n[a] > 1) lap += der2(fhat, p, s[a], h[a]);", "if (n[a] > 1) lap += der2(fhat, p, s[a], h[0]);"),
    # radius-r second derivative (Sec. 5.3 radius sweep)
    ("d2r_weight_k_not_k_squared", "((double)k * (double)k * factorial(r - k)", "((double)k * factorial(r - k)"),
    ("d2r_sign_alternation", "double sign = (k % 2 == 1) ? 1.0 : -1.0;", "double sign = (k % 2 == 0) ? 1.0 : -1.0;"),
    ("d2r_centre", "c[0] = -2.0 * centre;", "c[0] = -centre;"),
    ("d2r_stride_dropped", "(f[p + k * s] + f[p - k * s])", "(f[p + k * s] + f[p - k])"),
    # Eqs. A1-A4: MHD right-hand side
    ("A1_divu_sign", "rhs[LNRHO][o] = -ugradlnrho - divu;", "rhs[LNRHO][o] = -ugradlnrho + divu;"),
    ("A1_advection_dropped", "rhs[LNRHO][o] = -ugradlnrho - divu;", "rhs[LNRHO][o] = -divu;"),
    ("A2_advection_transposed", "double adv = u[0] * du[c][0] + u[1] * du[c][1] + u[2] * du[c][2];",
     "double adv = u[0] * du[0][c] + u[1] * du[1][c] + u[2] * du[2][c];"),
    ("A2_pressure_cp", "- cs2 * (gss[c] / cp + glnrho[c])", "- cs2 * (gss[c] * cp + glnrho[c])"),
    ("A2_pressure_sign", "- cs2 * (gss[c] / cp + glnrho[c])", "- cs2 * (gss[c] / cp - glnrho[c])"),
    ("A2_lorentz_density", "+ jxB[c] / rho +", "+ jxB[c] * rho +"),
    ("A2_lorentz_sign", "+ jxB[c] / rho +", "- jxB[c] / rho +"),
    ("A2_viscous_third", "graddivu[c] / 3.0 + 2.0 * Sg", "graddivu[c] / 2.0 + 2.0 * Sg"),
    ("A2_viscous_2S", "graddivu[c] / 3.0 + 2.0 * Sg", "graddivu[c] / 3.0 + Sg"),
    ("A2_bulk_viscosity_lap", "zeta * graddivu[c];", "zeta * lapu[c];"),
    ("A2_nu_on_S_only", "nu * (lapu[c] + graddivu[c] / 3.0 + 2.0 * Sg)", "nu * (lapu[c] + graddivu[c] / 3.0) + 2.0 * Sg"),
    ("graddiv_is_laplacian", "graddivu[c] = Hu[0][c][0] + Hu[1][c][1] + Hu[2][c][2];",
     "graddivu[c] = Hu[c][0][0] + Hu[c][1][1] + Hu[c][2][2];"),
    ("shear_trace_half", "- (a == b ? divu / 3.0 : 0.0)", "- (a == b ? divu / 2.0 : 0.0)"),
    ("shear_not_symmetrised", "S[a][b] = 0.5 * (du[a][b] + du[b][a])", "S[a][b] = (du[a][b])"),
    ("curl_sign", "double B[3] = {dA[2][1] - dA[1][2]", "double B[3] = {dA[1][2] - dA[2][1]"),
    ("current_graddiv_dropped", "jj[c] = (graddivA[c] - lapA[c]) / mu0;", "jj[c] = (-lapA[c]) / mu0;"),
    ("current_mu0_dropped", "jj[c] = (graddivA[c] - lapA[c]) / mu0;", "jj[c] = (graddivA[c] - lapA[c]);"),
    ("jxB_component", "double jxB[3] = {jj[1] * B[2] - jj[2] * B[1]", "double jxB[3] = {jj[2] * B[1] - jj[1] * B[2]"),
    ("cs2_gamma_minus_one", "exp(gam * ss / cp + (gam - 1.0) * (lnrho - lnrho0))", "exp(gam * ss / cp + gam * (lnrho - lnrho0))"),
    ("cs2_lnrho0_sign", "(gam - 1.0) * (lnrho - lnrho0))", "(gam - 1.0) * (lnrho + lnrho0))"),
    ("temperature_cp", "double TT = cs2 / (cp * (gam - 1.0));", "double TT = cs2 / (gam - 1.0);"),
    ("A3_advection_sign", "rhs[SS][o] = -ugrads +", "rhs[SS][o] = ugrads +"),
    ("A3_ohmic_mu0", "(eta * mu0 * j2 +", "(eta * j2 +"),
    ("A3_viscous_factor", "2.0 * rho * nu * SS2 +", "rho * nu * SS2 +"),
    ("A3_bulk_square", "zeta * rho * divu * divu) / (rho * TT)", "zeta * rho * divu) / (rho * TT)"),
    ("A3_over_T_only", "/ (rho * TT);", "/ TT;"),
    ("A3_conduction_grad_dropped", "rhs[SS][o] += K / rho * (lapphi + gphi2);", "rhs[SS][o] += K / rho * lapphi;"),
    ("A3_conduction_density", "rhs[SS][o] += K / rho * (lapphi + gphi2);", "rhs[SS][o] += K * rho * (lapphi + gphi2);"),
    ("A3_conduction_phi_gamma", "double gphi = gam / cp * gss[a] + (gam - 1.0) * glnrho[a];",
     "double gphi = gam / cp * gss[a] + gam * glnrho[a];"),
    ("A3_conduction_lap_lnrho", "(gam - 1.0) * der2(fhat[LNRHO], p, st[a], h[a]);", "(gam - 1.0) * der2(fhat[SS], p, st[a], h[a]);"),
    ("A4_induction_sign", "rhs[AX + c][o] = uxB[c] + eta * lapA[c];", "rhs[AX + c][o] = -uxB[c] + eta * lapA[c];"),
    ("A4_resistivity_dropped", "rhs[AX + c][o] = uxB[c] + eta * lapA[c];", "rhs[AX + c][o] = uxB[c];"),
    ("uxB_component", "double uxB[3] = {u[1] * B[2] - u[2] * B[1]", "double uxB[3] = {u[2] * B[1] - u[1] * B[2]"),
    # Sec. 3.3: RK3 (Williamson 2N-storage reading)
    ("rk_alpha2", "-5.0 / 9.0", "-5.0 / 8.0"),
    ("rk_alpha3", "-153.0 / 128.0", "-153.0 / 127.0"),
    ("rk_beta1", "{1.0 / 3.0, 15.0 / 16.0", "{1.0 / 2.0, 15.0 / 16.0"),
    ("rk_beta2", "15.0 / 16.0", "15.0 / 17.0"),
    ("rk_beta3", "8.0 / 15.0}", "8.0 / 16.0}"),
    ("rk_dt_dropped", "w[c] = RK_ALPHA[s] * w[c] + dt * rhs[c];", "w[c] = RK_ALPHA[s] * w[c] + rhs[c];"),
    ("rk_box_memory_dropped", "w[c] = RK_ALPHA[s] * w[c] + dt * r;", "w[c] = dt * r;"),
    ("rk_box_halo_offset", "(i + lo + R);\n", "(i + lo + R - 1);\n"),
    ("d1_dropped_outer_point", "for (int j = -R; j <= R; ++j) acc += C1[j + R]", "for (int j = -R; j < R; ++j) acc += C1[j + R]"),
    ("mixed_dropped_outer_ring", "for (int a = 1; a <= R; ++a) {", "for (int a = 1; a < R; ++a) {"),
    ("d2r_dropped_axis", "if (n[a] > 1) lap += der2_r(fhat, p, s[a], h[a], r, c);",
     "if (n[a] > 1 && a < 2) lap += der2_r(fhat, p, s[a], h[a], r, c);"),
    ("density_uses_lnrho0", "double rho = exp(lnrho);", "double rho = exp(lnrho - lnrho0);"),
    ("cs2_linear_in_cs0", "double cs2 = cs0 * cs0 * exp(", "double cs2 = cs0 * exp("),
    ("A3_conduction_cp_dropped", "lapphi += gam / cp * der2(fhat[SS]", "lapphi += gam * der2(fhat[SS]"),
    ("rk_one_register", "w[c] = RK_ALPHA[s] * w[c] + dt * rhs[c];\n                f[c] = f[c] + RK_BETA[s] * w[c];",
     "w[c] = RK_ALPHA[s] * w[c] + dt * rhs[c];\n                f[c] = f[c] + RK_BETA[s] * dt * rhs[c];"),
    ("rk_two_substeps", "for (int s = 0; s < 3; ++s) {\n            for (int q = 0; q < NF; ++q)",
     "for (int s = 0; s < 2; ++s) {\n            for (int q = 0; q < NF; ++q)"),
    ("norms_sum_is_sumsq", "out[0] = (double)s;", "out[0] = (double)s2;"),
    # field norms
    ("norms_sumsq", "s2 += (long double)f[i] * f[i];", "s2 += (long double)f[i];"),
    ("norms_maxabs_signed", "double a = fabs(f[i]);", "double a = f[i];"),
    ("mass_log", "s += exp(lnrho[i]);", "s += lnrho[i];"),
]


# The same for the Python wrapper.  None of these makes the C code read or write outside the
# arrays the wrapper allocates: a changed shape keeps the element count, or enlarges the array.
PY_MUTANTS = [
    ("py_dims_reversed", "return s[2], s[1], s[0]", "return s[0], s[1], s[2]"),
    ("py_pad_halo_on_unit_axes", "h = lambda n: n + 2 * r if n > 1 else 1", "h = lambda n: n + 2 * r"),
    ("py_xcorr_box_mask_31_bits", "fh = _c(np.asarray(fhat).astype(np.int64) & 0xFFFFFFFF, np.uint32)",
     "fh = _c(np.asarray(fhat).astype(np.int64) & 0x7FFFFFFF, np.uint32)"),
    ("py_xcorr_mask_31_bits", "d = _c(np.asarray(data).astype(np.int64) & 0xFFFFFFFF, np.uint32)",
     "d = _c(np.asarray(data).astype(np.int64) & 0x7FFFFFFF, np.uint32)"),
    ("py_xcorr_box_radius", "r = (len(g) - 1) // 2\n    n = len(fhat) - 2 * r", "r = (len(g) - 1) // 2 - 1\n    n = len(fhat) - 2 * r"),
    ("py_params_nu_eta_swapped", "self.nu, self.eta, self.zeta", "self.eta, self.nu, self.zeta"),
    ("py_for_grid_axis_order", "nz, ny, nx = (n, n, n) if np.isscalar(n) else tuple(n)",
     "nx, ny, nz = (n, n, n) if np.isscalar(n) else tuple(n)"),
    ("py_mhd_rhs_shape_transposed", "out = np.empty((8, nz, ny, nx), dtype=np.float64)",
     "out = np.empty((8, nx, ny, nz), dtype=np.float64)"),
    ("py_derivs_shape_transposed", "out = np.empty((9, nz, ny, nx), dtype=np.float64)",
     "out = np.empty((9, nx, ny, nz), dtype=np.float64)"),
    ("py_rk3_in_place", "f = _c(f8, np.float64).copy()\n    nz, ny, nx = f.shape[1:]",
     "f = _c(f8, np.float64)\n    nz, ny, nx = f.shape[1:]"),
    ("py_diffusion_spacing_reversed", "rc = _load().oracle_diffusion(_p(f), nx, ny, nz, dt, alpha, _p(_c(h, np.float64)), steps,",
     "rc = _load().oracle_diffusion(_p(f), nx, ny, nz, dt, alpha, _p(_c(h[::-1], np.float64)), steps,"),
]

CASES = [("c",) + m for m in MUTANTS] + [("py",) + m for m in PY_MUTANTS]


def test_every_mutant_applies_exactly_once():
    text = {"c": open(SRC).read(), "py": open(PY).read()}
    names = [m[1] for m in CASES]
    assert len(names) == len(set(names))
    for where, name, old, new in CASES:
        assert text[where].count(old) == 1, f"{name}: text occurs {text[where].count(old)} times"
        assert old != new, name


def _run_mutant(tmp, where, name, old, new):
    """Copy the package with one mistake into tmp/name/oracle, compile it, run the pins."""
    d = os.path.join(tmp, name, "oracle")
    os.makedirs(d)
    for path, kind in ((SRC, "c"), (PY, "py")):
        text = open(path).read()
        if kind == where:
            text = text.replace(old, new, 1)
        with open(os.path.join(d, os.path.basename(path)), "w") as fh:
            fh.write(text)
    oracle.build(force=True, src=os.path.join(d, "oracle.c"), lib=os.path.join(d, "liboracle.so"))  # must compile
    env = dict(os.environ, STENCIL_ORACLE_MUTANT_PKG=d, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *PIN_FILES], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-1500:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda m: _run_mutant(str(tmp_path), *m), CASES))
    survivors = [n for n, rc, _ in results if rc == 0]
    broken = [(n, rc, out) for n, rc, out in results if rc not in (0, 1)]
    assert not broken, broken
    assert not survivors, f"planted mistakes that pass every pin: {survivors}"


def test_unmutated_copy_passes_every_pin(tmp_path):
    """The harness itself: the same run on an unmodified copy passes, so a failing mutant
    fails because of its mistake."""
    name, rc, out = _run_mutant(str(tmp_path), "c", "unmodified", "", "")
    assert rc == 0, out
    assert "passed" in out
