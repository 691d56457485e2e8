"""Seeded synthetic inputs for the stencil workloads.

This module holds no stencil arithmetic: it only draws numbers and evaluates the smooth
initial fields the workloads start from.  Both the CUDA path (through the tests and the
benchmark) and the FP64 oracle take their inputs from here, so the two sides see the same
bits.

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea & Flood 2014,
finaliser constants as published by Vigna): value i of stream s for seed k is
mix(mix(k) ^ (s * C) + (i + 1) * golden_gamma).  It is written out here in numpy uint64
arithmetic, so its output does not depend on numpy's own generators or version.

Workload shapes follow the paper's benchmark protocol (randomised inputs, Sec. 5.1) and the
initial-value ranges of its Table B2; the exact recipes are:

* 1D cross-correlation (Eq. 3): int32 data uniform in [-1000, 1000], 7 int32 weights uniform
  in [-8, 8]; FP64 variant: data uniform in [-1, 1).
* 3D heat equation (Eqs. 4-7): the sum of 4 sine modes of amplitude 1, integer wave vector
  components in [1, 8], random phase, plus Gaussian noise of standard deviation 1e-3.
* 8-field MHD-shaped system (Appendix A): each field is the sum of 4 sine modes with amplitude
  uniform in [-1e-3, 1e-3), integer wave vector components in [1, 4] and random phase.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = np.uint64(0xD1B54A32D192ED03)

SEED_XCORR = 2406089231
SEED_HEAT = 2406089232
SEED_MHD = 2406089233
SEED_MHD_LOWP = 2406089234


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def bits(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n 64-bit words of stream ``stream`` for ``seed``, counters start..start+n-1."""
    key = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        base = key ^ (np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _STREAM)
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = base + ctr * _GAMMA
    return _mix(z)


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Doubles in [lo, hi): the top 53 bits scaled by 2**-53."""
    u = (bits(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def integers(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers in [lo, hi] (inclusive) by the multiply-shift map of the top 32 bits."""
    span = np.uint64(hi - lo + 1)
    top = bits(seed, stream, n) >> np.uint64(32)
    return (lo + ((top * span) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normal doubles by the Box-Muller transform of two uniform streams."""
    u1 = uniform(seed, 2 * stream + 1, n)
    u2 = uniform(seed, 2 * stream + 2, n)
    u1 = np.where(u1 <= 0.0, 2.0 ** -53, u1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------- workloads


def xcorr_int32(n: int, seed: int = SEED_XCORR):
    """(data[n] int32 in [-1000, 1000], weights[7] int32 in [-8, 8])."""
    data = integers(seed, 1, n, -1000, 1000).astype(np.int32)
    w = integers(seed, 2, 7, -8, 8).astype(np.int32)
    return data, w


def xcorr_f64(n: int, seed: int = SEED_XCORR) -> np.ndarray:
    """data[n] float64 uniform in [-1, 1)."""
    return uniform(seed, 3, n, -1.0, 1.0)


def _mode_sum(shape, amps, kvecs, phases, out=None):
    """sum_m amps[m] * sin(k_m . x + phase_m) on the periodic grid x_i = 2*pi*i/n_i.

    Evaluated as the imaginary part of a product of 1D complex exponentials, one z-plane at a
    time, so a 384^3 field needs no full-size complex temporaries.
    """
    nz, ny, nx = shape
    if out is None:
        out = np.zeros(shape, dtype=np.float64)
    xs = [2.0 * math.pi * np.arange(n) / n for n in (nx, ny, nz)]
    for a, k, ph in zip(amps, kvecs, phases):
        ex = np.exp(1j * k[0] * xs[0])
        ey = np.exp(1j * k[1] * xs[1])
        ez = np.exp(1j * (k[2] * xs[2] + ph))
        plane = np.outer(ey, ex)
        for z in range(nz):
            out[z] += a * (ez[z] * plane).imag
    return out


def heat_field(n, seed: int = SEED_HEAT, nmodes: int = 4, kmax: int = 8, noise: float = 1e-3):
    """3D heat-equation initial field of shape (nz, ny, nx), float64."""
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    k = integers(seed, 10, 3 * nmodes, 1, kmax).reshape(nmodes, 3)
    ph = uniform(seed, 11, nmodes, 0.0, 2.0 * math.pi)
    f = _mode_sum(shape, np.ones(nmodes), k, ph)
    if noise:
        f += noise * normal(seed, 12, int(np.prod(shape))).reshape(shape)
    return f


MHD_FIELDS = ("lnrho", "ux", "uy", "uz", "ax", "ay", "az", "ss")


def mhd_fields(n, seed: int = SEED_MHD, nmodes: int = 4, kmax: int = 4, amp: float = 1e-3):
    """8 MHD-shaped fields, shape (8, nz, ny, nx), float64, order ``MHD_FIELDS``."""
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    out = np.zeros((8,) + shape, dtype=np.float64)
    for f in range(8):
        s = 100 + 10 * f
        a = uniform(seed, s, nmodes, -amp, amp)
        k = integers(seed, s + 1, 3 * nmodes, 1, kmax).reshape(nmodes, 3)
        ph = uniform(seed, s + 2, nmodes, 0.0, 2.0 * math.pi)
        _mode_sum(shape, a, k, ph, out=out[f])
    return out
