"""Provenance and error bound of the FP32 atan2 used by the guarded FP32 wedge
projection of the self-energy kernels (atan2_poly in csrc/sigma.cu).

* The coefficients in csrc/atan_poly.h are the output of the committed Remez
  fit csrc/atan_fit.py (regenerated here and compared byte for byte).
* The FP32 evaluation -- Horner with fused multiply-adds, an approximate
  quotient t = min/max (2 ulp), the octant reflections pi/2 - a and pi - a --
  stays within 2.3e-6 rad of the FP64 atan2 on a dense set of directions, the
  figure the projection's guard band (8e-6 rad) is built on.
"""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIT = os.path.join(ROOT, "paper_2005_00827_gb300", "csrc", "atan_fit.py")


def _fit_module():
    spec = importlib.util.spec_from_file_location("atan_fit", FIT)
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_header_is_the_fit_output():
    """Coefficients in the header equal the fit's to one FP32 unit (a platform's
    FP64 linear algebra may move a coefficient across an FP32 rounding tie)."""
    import re
    m = _fit_module()
    c32, lev, bound = m.fit()
    text = open(m.HEADER).read()
    got = [float(re.search(rf"kAtanC{k} = ([-0-9.e+]+)f;", text).group(1)) for k in range(6)]
    for g, c in zip(got, c32):
        assert abs(g - c) <= 1.2e-7 * abs(c)
    # the minimax level of a degree-11 odd fit of atan on [0, 1]
    assert 1e-6 < lev < 2e-6 and bound < 1.8e-6


def _atan2_poly_f32(y, x, c32, tscale=1.0):
    f32 = np.float32
    ax, ay = np.abs(x).astype(f32), np.abs(y).astype(f32)
    t = (np.minimum(ax, ay) / np.maximum(ax, ay)).astype(f32)
    t = (t * f32(tscale)).astype(f32)           # the approximate quotient's error
    s = (t * t).astype(f32)
    p = np.full_like(s, f32(c32[5]))
    for ck in (c32[4], c32[3], c32[2], c32[1], c32[0]):
        p = (s.astype(np.float64) * p + np.float64(ck)).astype(f32)
    a = (t * p).astype(f32)
    a = np.where(ay > ax, (f32(1.57079633) - a).astype(f32), a)
    a = np.where(x < 0, (f32(3.14159265) - a).astype(f32), a)
    return np.copysign(a, y).astype(np.float64)


def test_fp32_atan2_within_guard_bound():
    m = _fit_module()
    c32, _, bound = m.fit()
    th = np.linspace(-np.pi, np.pi, 400001)
    worst = 0.0
    for rad in (1e-3, 0.7, 3.0, 4.4):
        x = (rad * np.cos(th)).astype(np.float32)
        y = (rad * np.sin(th)).astype(np.float32)
        ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
        for ts in (1.0 - 2.0 ** -22, 1.0, 1.0 + 2.0 ** -22):
            got = _atan2_poly_f32(y, x, c32, ts)
            d = np.abs(np.angle(np.exp(1j * (got - ref))))
            worst = max(worst, float(d.max()))
    assert worst < 2.3e-6
