"""The FP32 kernels' arctangent of the binned Lorentzian and binned Gauss-Hermite Voigt.

`atan2_ypos` in the CUDA source replaces the library atan2f for y >= 0: a reciprocal, a
degree-8 polynomial in s = t^2 and two reflections.  Its coefficients are read from the
source here and the function is replayed in numpy float32 (the reciprocal exact instead of
the hardware's approximate one, which adds at most an ulp), then compared with numpy's
float64 arctan2 over the ranges the profiles produce: y = gamma in grid steps (zero
included), x = delta^2 +- ... of either sign, and the reflections' boundaries (y = |x|).
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1801_09803_gb300", "csrc", "xc_batched.cuh")


def _coefficients():
    s = open(SRC).read()
    body = s[s.index("__device__ __forceinline__ float atan2_ypos("):]
    body = body[:body.index("\n}\n")]
    lead = re.search(r"float q = ([-+0-9.eE]+)f;", body).group(1)
    rest = re.findall(r"q = fmaf\(q, s, ([-+0-9.eE]+)f\);", body)
    return [np.float32(float(lead))] + [np.float32(float(c)) for c in rest]   # highest degree first


def atan2_ypos(y, x, coef):
    y = np.asarray(y, np.float32)
    x = np.asarray(x, np.float32)
    ax = np.abs(x)
    mx = np.maximum(ax, y)
    mn = np.minimum(ax, y)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(mx > 0, mn * (np.float32(1) / mx), np.float32(0)).astype(np.float32)
    s = (t * t).astype(np.float32)
    q = np.full_like(s, coef[0])
    for c in coef[1:]:
        q = (q * s + c).astype(np.float32)
    p = (q * t).astype(np.float32)
    p = np.where(y > ax, np.float32(np.pi / 2) - p, p).astype(np.float32)
    p = np.where(x < 0, np.float32(np.pi) - p, p).astype(np.float32)
    return p


def test_polynomial_is_the_source_one():
    c = _coefficients()
    assert len(c) == 9
    assert abs(float(c[-1]) - 1.0) < 1e-7          # atan(t) / t -> 1 as t -> 0
    assert abs(float(c[-2]) + 1.0 / 3.0) < 1e-5    # the t^3 / 3 term of atan


def test_arctangent_against_float64():
    coef = _coefficients()
    rng = np.random.default_rng(180109803)
    n = 1_000_000
    y = np.exp(rng.uniform(np.log(1e-6), np.log(1e3), n)).astype(np.float32)
    x = (np.exp(rng.uniform(np.log(1e-6), np.log(1e7), n)) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    got = atan2_ypos(y, x, coef).astype(np.float64)
    assert np.max(np.abs(got - ref) / ref) < 4e-7
    # near the reflections (y = |x|) and at small t
    t = np.linspace(0.0, 2.0, 200001).astype(np.float32)
    for sgn in (1.0, -1.0):
        xx = (sgn * np.ones_like(t)).astype(np.float32)
        ref = np.arctan2(t.astype(np.float64), xx.astype(np.float64))
        got = atan2_ypos(t, xx, coef).astype(np.float64)
        nz = ref > 0
        assert np.max(np.abs(got[nz] - ref[nz]) / ref[nz]) < 4e-7
        assert np.all(got[~nz] == 0.0)


def test_arctangent_special_cases():
    coef = _coefficients()
    # gamma = 0: the bin average of a delta function -- pi inside the bin (x < 0), 0 outside
    assert atan2_ypos(0.0, -0.25, coef) == np.float32(np.pi)
    assert atan2_ypos(0.0, 3.0, coef) == 0.0
    assert atan2_ypos(0.0, 0.0, coef) == 0.0
    assert abs(float(atan2_ypos(1.0, 0.0, coef)) - np.pi / 2) < 2e-7
    # far wing: atan2(y, x) -> y / x
    assert abs(float(atan2_ypos(1e-3, 1e6, coef)) / 1e-9 - 1.0) < 3e-7
