"""The fixed-point wedge decision of the FP32 kernels against the oracle.

The self-energy kernels and the wedge-mode partner maps decide the patch of a
folded momentum r without FP64: components as 32-bit fixed-point turns (the
fold is the wrap of integer arithmetic), a 256 x 256 cell table over the zone
(each cell: the lower of the at most two wedges it touches, widened by 2e-5;
255 where three or more wedges meet), and one FP32 cross product with the ray
between the two wedges.  Within 4e-6 rad of that ray or of the zone edge the
kernels fall back to the exact FP64 projection.  This test restates that
scheme in numpy and checks that, outside the guard bands, it returns exactly
the oracle's FP64 projection (fold to [-pi, pi], atan2, nearest wedge centre),
on random pairs of which a third lie within 1e-4 rad of a wedge ray.
"""
import numpy as np
import pytest

W = 256
GUARD = np.float32(4e-6 * 2.0**32 / (2 * np.pi))
EDGE = np.float32((np.pi - 4e-6) * 2.0**32 / (2 * np.pi))


def cell_table(N):
    h, m, dth = 2 * np.pi / W, 2e-5, 2 * np.pi / N
    k = np.arange(W)
    x0 = (-np.pi + k * h - m)[None, :]
    x1 = (-np.pi + (k + 1) * h + m)[None, :]
    y0 = (-np.pi + k * h - m)[:, None]
    y1 = (-np.pi + (k + 1) * h + m)[:, None]
    cx = [x0 + 0 * y0, x1 + 0 * y0, x0 + 0 * y0, x1 + 0 * y0]
    cy = [y0 + 0 * x0, y0 + 0 * x0, y1 + 0 * x0, y1 + 0 * x0]
    a0 = np.arctan2(cy[0], cx[0])
    lo = np.zeros_like(a0)
    hi = np.zeros_like(a0)
    for c in range(1, 4):
        d = np.remainder(np.arctan2(cy[c], cx[c]) - a0 + np.pi, 2 * np.pi) - np.pi
        lo, hi = np.minimum(lo, d), np.maximum(hi, d)
    jl = np.floor((a0 + lo) / dth + 0.5).astype(np.int64)
    jh = np.floor((a0 + hi) / dth + 0.5).astype(np.int64)
    tab = np.where(jh - jl <= 1, jl % N, 255)
    origin = (x0 <= 0) & (x1 >= 0) & (y0 <= 0) & (y1 >= 0)
    return np.where(origin, 255, tab)


def fixed(v):
    t = v / (2 * np.pi)
    return (np.rint((t - np.rint(t)) * 2.0**32).astype(np.int64) & 0xFFFFFFFF).astype(np.uint32)


def decide(X, Y, tab, N):
    """(patch, slow) from wrapped fixed-point components, as in the kernels."""
    ang = (np.arange(N + 1) - 0.5) * 2 * np.pi / N
    ray = np.zeros((257, 2), np.float32)
    ray[:N + 1, 0] = np.cos(ang)
    ray[:N + 1, 1] = np.sin(ang)
    ray[N] = ray[0]
    x, y = X.astype(np.float32), Y.astype(np.float32)
    e = tab[(Y >> 24) + 128, (X >> 24) + 128]
    rr = ray[e + 1]
    cr = (rr[:, 0] * y).astype(np.float32) - (rr[:, 1] * x).astype(np.float32)
    slow = (np.maximum(np.abs(x), np.abs(y)) > EDGE) | (np.abs(cr) < GUARD)
    return (e + (cr >= 0)) % N, slow


@pytest.mark.parametrize("N", [16, 48, 96])
def test_fixed_point_decision_equals_fp64_projection(oracle_mod, N):
    o = oracle_mod.Oracle(N, 2, 2)
    tab = cell_table(N)
    rng = np.random.default_rng(N)
    n = 40000
    a = rng.uniform(-np.pi, np.pi, (n, 2))       # k + p, or Q
    b = rng.uniform(-np.pi, np.pi, (n, 2))       # q, or p
    near = rng.random(n) < 0.33                   # r within 1e-4 rad of a wedge ray
    r = rng.uniform(0.01, np.pi, n)
    th = (rng.integers(0, N, n) - 0.5) * 2 * np.pi / N + rng.uniform(-1e-4, 1e-4, n)
    a[near] = b[near] + np.stack([r * np.cos(th), r * np.sin(th)], 1)[near]
    fa, fb = fixed(a), fixed(b)
    checked = 0
    for sign in (-1, 1):                          # a - b (self-energy, pp maps), a + b (ph maps)
        # uint32 arithmetic wraps: the fold
        X = ((fa[:, 0] + fb[:, 0]) if sign > 0 else (fa[:, 0] - fb[:, 0])).astype(np.int32)
        Y = ((fa[:, 1] + fb[:, 1]) if sign > 0 else (fa[:, 1] - fb[:, 1])).astype(np.int32)
        c, slow = decide(X, Y, tab, N)
        rx, ry = a[:, 0] + sign * b[:, 0], a[:, 1] + sign * b[:, 1]
        for i in np.flatnonzero(~slow)[:6000]:
            assert c[i] == o.proj(rx[i], ry[i]), (N, sign, rx[i], ry[i])
            checked += 1
        assert slow.mean() < 0.1                  # the guarded paths stay rare
    assert checked == 12000
