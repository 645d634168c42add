"""Pins of the oracle's Fermi functions and closed-form bubbles.

The closed forms (Matsubara sums done through Fermi functions, the loop
kernels of the one-loop flow, App. A.1 Eq. (vertex_flow_general) with
G0 = 1/(i w - xi), Eq. (both_propagators_Z) at Z = 1) are checked against
term-by-term Matsubara sums and finite differences -- not against themselves.
"""
import numpy as np
import pytest

from tests import brute

PAIRS = [(0.3, -0.7), (1.2, 1.5), (-2.0, 0.4), (0.05, 0.06), (-3.9, 3.9), (0.0, 0.8)]
TEMPS = [0.05, 0.3, 1.0]


@pytest.mark.parametrize("T", TEMPS)
def test_fermi_closed_forms(oracle_mod, T):
    o = oracle_mod
    assert o.fermi(0.0, T) == 0.5
    for x in [-3.0, -0.4, 0.01, 0.7, 2.5]:
        assert o.fermi(x, T) + o.fermi(-x, T) == pytest.approx(1.0, abs=1e-15)
        assert o.fermi(x, T) == pytest.approx(1.0 / (np.exp(x / T) + 1.0), rel=1e-13)
        d = brute.ddT(lambda TT: 1.0 / (np.exp(x / TT) + 1.0), T)
        assert o.dfermi_dT(x, T) == pytest.approx(d, rel=1e-7, abs=1e-12)


@pytest.mark.parametrize("T", TEMPS)
@pytest.mark.parametrize("a,b", PAIRS)
def test_ph_bubble_equals_matsubara_sum(oracle_mod, a, b, T):
    ref = brute.matsubara_ph(a, b, T)
    assert oracle_mod.Lph(a, b, T) == pytest.approx(ref, rel=1e-11, abs=1e-14)


@pytest.mark.parametrize("T", TEMPS)
@pytest.mark.parametrize("a,b", PAIRS)
def test_pp_bubble_equals_matsubara_sum(oracle_mod, a, b, T):
    ref = brute.matsubara_pp(a, b, T)
    assert oracle_mod.Lpp(a, b, T) == pytest.approx(ref, rel=1e-11, abs=1e-14)


@pytest.mark.parametrize("T", [0.1, 0.5])
@pytest.mark.parametrize("a,b", [(0.3, -0.7), (0.2, 0.2 + 3e-7), (-1.1, 1.1), (0.6, -0.6 + 1e-7)])
def test_scale_derivatives_equal_matsubara_differences(oracle_mod, a, b, T):
    o = oracle_mod
    dph = brute.ddT(lambda TT: brute.matsubara_ph(a, b, TT, nmax=40000), T)
    dpp = brute.ddT(lambda TT: brute.matsubara_pp(a, b, TT, nmax=40000), T)
    assert o.dLph_dT(a, b, T) == pytest.approx(dph, rel=2e-6, abs=1e-10)
    assert o.dLpp_dT(a, b, T) == pytest.approx(dpp, rel=2e-6, abs=1e-10)


@pytest.mark.parametrize("T", [0.02, 0.2, 1.0])
def test_degenerate_limit_is_fermi_derivative(oracle_mod, T):
    """x -> y limit of (f(x) - f(y))/(x - y) is f'(x); continuous across the
    switch to the analytic derivative."""
    o = oracle_mod
    for x in [-0.3 * T, 0.0, 0.7 * T, 2.0 * T]:
        fprime = -np.exp(x / T) / (T * (np.exp(x / T) + 1.0) ** 2)
        assert o.D(x, x, T) == pytest.approx(fprime, rel=1e-12)
        for eps in [3e-6 * T, 9.9e-6 * T, 1.01e-5 * T, 1e-4 * T]:
            m = x + 0.5 * eps   # D(x, x+eps) = f'(midpoint) + O(eps^2)
            fm = -np.exp(m / T) / (T * (np.exp(m / T) + 1.0) ** 2)
            assert o.D(x, x + eps, T) == pytest.approx(fm, rel=(eps / T) ** 2 + 1e-10)
        # analytic T-derivative of f' against differences of f'
        d = brute.ddT(lambda TT: -np.exp(x / TT) / (TT * (np.exp(x / TT) + 1.0) ** 2), T)
        assert o.dD_dT(x, x, T) == pytest.approx(d, rel=1e-7, abs=1e-12)
        below, above = o.dD_dT(x, x + 0.99e-5 * T, T), o.dD_dT(x, x + 1.01e-5 * T, T)
        assert below == pytest.approx(above, rel=1e-6, abs=1e-9 / T ** 2)


def test_pp_is_reflected_ph(oracle_mod):
    o = oracle_mod
    for a, b in PAIRS:
        assert o.Lpp(a, b, 0.2) == -o.D(a, -b, 0.2)
        assert o.Lph(a, b, 0.2) < 0.0
        assert o.Lpp(a, b, 0.2) > 0.0


@pytest.mark.parametrize("T", TEMPS)
def test_loop_kernel_magnitude_bounds(oracle_mod, T):
    """|D| <= 1/(4T) and |dD/dT| <= 1/(4T^2) for every pair of line energies
    (mean value theorem: D is f' and dD/dT is d^2f/dxdT somewhere between the
    energies, both largest at x = 0).  The FP32 loop-kernel rows accumulate as
    fixed point with a scale taken from exactly these bounds, so they must hold
    for the pp and ph kernels alike, including near-degenerate pairs."""
    o = oracle_mod
    xs = np.concatenate([np.linspace(-6.0, 6.0, 121), np.linspace(-4.0, 4.0, 17) * T])
    pairs = [(a, b) for a in xs for b in xs] + [(a, a + e * T) for a in xs for e in (1e-7, 9.9e-6, 1e-3)]
    bD, bT = 0.25 / T, 0.25 / T ** 2
    worst_D = max(max(abs(o.Lph(a, b, T)), abs(o.Lpp(a, b, T))) for a, b in pairs)
    worst_T = max(max(abs(o.dLph_dT(a, b, T)), abs(o.dLpp_dT(a, b, T))) for a, b in pairs)
    assert worst_D <= bD * (1.0 + 1e-12)
    assert worst_T <= bT * (1.0 + 1e-12)
    # the bounds are attained at the Fermi level (degenerate pair at x = 0)
    assert abs(o.Lph(0.0, 0.0, T)) == pytest.approx(bD, rel=1e-12)
    assert abs(o.dLph_dT(0.0, 0.0, T)) == pytest.approx(bT, rel=1e-12)
