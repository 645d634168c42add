#!/usr/bin/env python3
"""Minimax fit of the odd polynomial behind atan2_poly (csrc/sigma.cu).

atan(t) on t in [0, 1] is approximated by t * P(t^2), P of degree 5 (an odd
polynomial of degree 11), minimising the largest absolute error with the Remez
exchange algorithm (E. Remez, 1934): solve for the coefficients and the level
E on 7 reference points where the error alternates in sign, move the
references to the extrema of the new error curve, repeat until the levels
agree.  The coefficients are rounded to FP32 and written to atan_poly.h.

Run from anywhere: ``python atan_fit.py`` rewrites atan_poly.h next to this
file; ``python atan_fit.py --check`` exits non-zero when the header differs.
"""
from __future__ import annotations

import os
import sys

import numpy as np

DEGREE = 5                 # P(s), s = t^2
HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "atan_poly.h")


def basis(t):
    return np.stack([t ** (2 * k + 1) for k in range(DEGREE + 1)], axis=-1)


def remez(iters=60, grid=200001):
    n = DEGREE + 1                      # unknown coefficients; n + 1 references
    tt = np.linspace(0.0, 1.0, grid)[1:]
    # initial references: Chebyshev extrema mapped into (0, 1]
    k = np.arange(n + 1)
    ref = 0.5 * (1.0 - np.cos(np.pi * (k + 1) / (n + 1)))
    for _ in range(iters):
        Amat = np.hstack([basis(ref), ((-1.0) ** np.arange(n + 1))[:, None]])
        sol = np.linalg.solve(Amat, np.arctan(ref))
        c, lev = sol[:n], sol[n]
        err = basis(tt) @ c - np.arctan(tt)
        # local extrema of the error (and the end point t = 1)
        idx = [i for i in range(1, len(tt) - 1) if (err[i] - err[i - 1]) * (err[i + 1] - err[i]) <= 0]
        idx.append(len(tt) - 1)
        # keep the largest of each run of equal sign, then n + 1 of them
        pts = []
        for i in idx:
            if pts and np.sign(err[i]) == np.sign(err[pts[-1]]):
                if abs(err[i]) > abs(err[pts[-1]]):
                    pts[-1] = i
            else:
                pts.append(i)
        while len(pts) > n + 1:         # drop the smaller end
            pts = pts[1:] if abs(err[pts[0]]) < abs(err[pts[-1]]) else pts[:-1]
        new = tt[pts]
        if len(new) == n + 1 and np.allclose(new, ref, atol=1e-12):
            break
        if len(new) == n + 1:
            ref = new
    return c, abs(lev)


def f32_coeffs(c):
    return [float(np.float32(x)) for x in c]


def eval_f32(t, c32):
    """Horner evaluation in FP32 with fused multiply-adds emulated in FP64
    then rounded (one rounding per FMA, as the device's fmaf)."""
    t = np.asarray(t, dtype=np.float32)
    s = (t * t).astype(np.float32)
    p = np.float32(c32[-1])
    for ck in reversed(c32[:-1]):
        p = (s.astype(np.float64) * p + np.float64(ck)).astype(np.float32)
    return (t * p).astype(np.float32)


def header_text(c32, bound):
    lines = [
        "// Generated by atan_fit.py (Remez minimax fit, do not edit): atan(t) ~ t P(t^2)",
        "// on t in [0, 1], P of degree 5, coefficients of s^0 .. s^5 rounded to FP32.",
        f"// Maximum absolute error of the FP32 evaluation over [0, 1]: {bound:.3e} rad.",
        "#pragma once",
        "namespace qpfrg {",
        *[f"constexpr float kAtanC{k} = {x:.9e}f;" for k, x in enumerate(c32)],
        f"constexpr float kAtanErr = {bound:.3e}f;",
        "}  // namespace qpfrg",
        "",
    ]
    return "\n".join(lines)


def fit():
    c, lev = remez()
    c32 = f32_coeffs(c)
    t = np.linspace(0.0, 1.0, 2000001, dtype=np.float64).astype(np.float32)
    err = np.abs(eval_f32(t, c32).astype(np.float64) - np.arctan(t.astype(np.float64)))
    # bound: the measured FP32 error, rounded up to 2 significant digits
    bound = float(np.ceil(err.max() * 1e8) / 1e8)
    return c32, lev, bound


def main():
    c32, lev, bound = fit()
    text = header_text(c32, bound)
    if "--check" in sys.argv:
        ok = os.path.exists(HEADER) and open(HEADER).read() == text
        print("atan_poly.h up to date" if ok else "atan_poly.h differs from the fit")
        sys.exit(0 if ok else 1)
    with open(HEADER, "w") as f:
        f.write(text)
    print(f"minimax level {lev:.3e}, FP32 bound {bound:.3e}; wrote {HEADER}")


if __name__ == "__main__":
    main()
