"""Error budget of the tensor-core far-wing evaluation, emulated on the CPU.

Where a Voigt w4 line is in region I and u = delta^2 >= C / 0.012 (grid units,
C = b + g^2, b = a^2 / (2 ln 2)), the far-wing kernel replaces the rational
(u + C) / (u^2 + E u + F) by the four-term series r (1 + c1 r + c2 r^2 + c3 r^3),
r = 1/u, and sums the terms as TF32 matrix products: for j = 0 both factors split
hi + lo (hi = the 13 low mantissa bits cleared) in three products; for j = 1 both
factors rounded to the nearest TF32 value in one product; the j = 2, 3 terms as the
tensor core reads them (truncated to TF32).  The products of two TF32 values are
exact in FP32.  This test emulates that operand handling in numpy and checks it
against the rational in FP64 over the widths of the workloads: the relative error
stays below 5e-5 (the j = 1 rounding, at most 2 x 2^-11 x 0.036), and its mean over
many (line, point) pairs is far smaller (the rounding is unbiased), which a
truncation of the j = 1 operands would not be.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _trunc(x):
    """TF32 as the tensor core reads an FP32 operand: the 13 low mantissa bits dropped."""
    return (np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def _round(x):
    """The nearest TF32 value (ties away from zero): half a TF32 unit added to the bits."""
    u = np.asarray(x, np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def _series_coefficients(a, g):
    b = a * a / (2.0 * np.log(2.0))
    g2 = g * g
    C = b + g2
    E = 2.0 * (g2 - b)
    F = C * C
    c1 = 3.0 * b - g2
    c2 = (g2 - 5.0 * b) ** 2 - 20.0 * b * b
    c3 = -E * c2 - F * c1
    return C, E, F, c1, c2, c3


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    a = np.exp(rng.uniform(np.log(0.05), np.log(20.0), n))     # Doppler HWHM in grid steps
    g = np.exp(rng.uniform(np.log(1e-3), np.log(300.0), n))    # Lorentz HWHM in grid steps
    C = a * a / (2.0 * np.log(2.0)) + g * g
    u_lo = C / 0.012                                           # the kernel's far radius
    u = u_lo * np.exp(rng.uniform(0.0, np.log(50.0), n))       # from the radius outwards
    return a, g, u


def _emulated(a, g, u, round_j1=True):
    C, E, F, c1, c2, c3 = _series_coefficients(a, g)
    P = np.ones_like(a)
    p = [(P * c).astype(np.float32) for c in (np.ones_like(a), c1, c2, c3)]
    r = (np.float32(1.0) / u.astype(np.float32)).astype(np.float32)
    r2 = (r * r).astype(np.float32)
    r3 = (r2 * r).astype(np.float32)
    r4 = (r2 * r2).astype(np.float32)
    rh = _trunc(r)
    rl = (r - rh).astype(np.float32)
    p0h = _trunc(p[0])
    p0l = (p[0] - p0h).astype(np.float32)
    if round_j1:
        t1 = _round(r2).astype(np.float64) * _round(p[1])
    else:
        t1 = _trunc(r2).astype(np.float64) * _trunc(p[1])
    terms = [rh.astype(np.float64) * p0h, rh.astype(np.float64) * _trunc(p0l), _trunc(rl).astype(np.float64) * p0h,
             t1, _trunc(r3).astype(np.float64) * _trunc(p[2]), _trunc(r4).astype(np.float64) * _trunc(p[3])]
    return np.sum(terms, axis=0)


def _exact(a, g, u):
    C, E, F, *_ = _series_coefficients(a, g)
    return (u + C) / (u * (u + E) + F)


def test_far_wing_operands_stay_within_the_budget():
    a, g, u = _samples(200_000, 11)
    ref = _exact(a, g, u)
    rel = (_emulated(a, g, u) - ref) / ref
    assert np.all(np.isfinite(rel))
    assert np.max(np.abs(rel)) < 5e-5
    # the rounding of the j = 1 operands is unbiased: its mean error is small against its
    # largest (near the far radius, where the j = 1 term weighs most)
    near = u < 2.0 * (a * a / (2.0 * np.log(2.0)) + g * g) / 0.012
    assert abs(np.mean(rel[near])) < 2e-6


def test_truncated_j1_operands_would_bias_the_sum():
    """The same emulation with the j = 1 operands truncated instead of rounded: the error
    is then one-signed near the far radius, the bias the rounding avoids."""
    a, g, u = _samples(200_000, 12)
    C = a * a / (2.0 * np.log(2.0)) + g * g
    near = u < 2.0 * C / 0.012
    ref = _exact(a, g, u)
    rel_t = (_emulated(a, g, u, round_j1=False) - ref) / ref
    rel_r = (_emulated(a, g, u) - ref) / ref
    assert abs(np.mean(rel_t[near])) > 5.0 * abs(np.mean(rel_r[near]))


def test_series_matches_the_rational_beyond_the_far_radius():
    """The four-term series itself (FP64, no TF32) within 2e-7 of the rational for
    u >= C / 0.012, and the coefficients satisfy the recurrence of the expansion
    (1 + E r + F r^2) sum_n c_n r^n = 1 + C r."""
    a, g, u = _samples(50_000, 13)
    C, E, F, c1, c2, c3 = _series_coefficients(a, g)
    r = 1.0 / u
    s = r * (1.0 + r * (c1 + r * (c2 + r * c3)))
    ref = _exact(a, g, u)
    assert np.max(np.abs(s / ref - 1.0)) < 2e-7
    assert np.allclose(c1, C - E, rtol=1e-12, atol=0)
    assert np.allclose(c2, -E * c1 - F, rtol=1e-9, atol=1e-9 * np.abs(F))
