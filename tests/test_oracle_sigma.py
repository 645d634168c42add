"""Pins of the oracle's real-frequency two-loop self-energy and Z.

* V = U, Z = 1 is second-order perturbation theory (SOPT, Sec. 3.1): the pole
  sum continued to z = i w_n must equal an imaginary-time quadrature of
  -U^2 G G G, and Im Sigma(i w_n > 0) < 0 (causality).
* Sum rule: Sigma(w) -> U^2 n(1-n) / w for large w (exact in lattice mode).
* The SU(2) weight W = 2V(k,p,q)^2 - V(k,p,q)V(k,p,r) must equal the spin
  sum (1/2) sum G(k,p;q,r) G(q,r;k,p) of the antisymmetrised vertex.
* Half filling / perfect nesting: Im Sigma(k_F, w) even, Re Sigma odd
  (no Fermi-surface shift, Sec. A.2 Comment 2).
* Sigma = 0 gives Z = 1 (start of the flow, App. B).
"""
import numpy as np
import pytest

from oracle.oracle import MODE_LATTICE, PROP_QP, Oracle
from paper_2005_00827_gb300 import inputs
from tests import brute
from tests.brute import Lattice, gamma_su2


@pytest.mark.parametrize("n_mats", [0, 1, 3])
@pytest.mark.parametrize("kidx", [0, 5, 6])
def test_sopt_matches_imaginary_time_quadrature(n_mats, kidx):
    L, U, T = 4, 1.3, 0.5
    lat = Lattice(L)
    wn = (2 * n_mats + 1) * np.pi * T
    o = Oracle(lat.K, mode=MODE_LATTICE, eta=wn)          # w + i eta = i w_n
    V = np.full((lat.K,) * 3, U)
    got = o.sigma(T, V, np.ones(lat.K), kidx, [0.0])[0]
    ref = brute.sigma_tau_quadrature(lat, kidx, U, T, n_mats)
    assert ref.imag < 0
    assert abs(got - ref) < 1e-11 * abs(ref)


def test_sum_rule_lattice():
    """-(1/pi) int Im Sigma = sum W F = U^2 n (1 - n) = U^2/4 at half filling."""
    L, U, T = 6, 1.7, 0.2
    o = Oracle(L * L, mode=MODE_LATTICE, eta=0.05)
    V = np.full((L * L,) * 3, U)
    for k in (0, 4, 9):
        w = 1e7
        s = o.sigma(T, V, np.ones(L * L), k, [w])[0]
        assert (w * s).real == pytest.approx(U * U / 4, rel=1e-5)


@pytest.mark.parametrize("qp", [False, True])
def test_su2_weight_equals_spin_sum(qp):
    L, T, eta = 4, 0.3, 0.07
    lat = Lattice(L)
    K = lat.K
    V = inputs.random_vertex(K, 2.0, seed=9, c4v=False)
    for _ in range(4):
        V = lat.exchange_symmetrise(lat.tr_symmetrise(V))
    rng = np.random.default_rng(1)
    Z = rng.uniform(0.8, 1.0, K)
    o = Oracle(K, mode=MODE_LATTICE, eta=eta, prop_mode=PROP_QP if qp else 0)
    omega = np.array([-1.3, -0.2, 0.0, 0.45, 2.2])
    fer = lambda e: 0.5 * (1.0 - np.tanh(0.5 * e / T))
    ar = np.arange(K)
    p, q = np.meshgrid(ar, ar, indexing="ij")
    for k in (1, 6, 11):
        r = lat.sub(lat.add(np.full_like(p, k), p), q)
        xp, xq, xr = lat.xi[p], lat.xi[q], lat.xi[r]
        if qp:
            xp, xq, xr = Z[p] * xp, Z[q] * xq, Z[r] * xr
        F = fer(xp) * (1 - fer(xq)) * (1 - fer(xr)) + (1 - fer(xp)) * fer(xq) * fer(xr)
        E = xq + xr - xp
        W = np.zeros_like(F)
        kk = np.full_like(p, k)
        for s2 in (0, 1):
            for s3 in (0, 1):
                for s4 in (0, 1):
                    W += gamma_su2(V, kk, 0, p, s2, q, s3, s4) * gamma_su2(V, q, s3, r, s4, kk, 0, s2)
        W *= 0.5 * Z[p] * Z[q] * Z[r]
        ref = np.array([(W * F / (w + 1j * eta - E)).sum() / K ** 2 for w in omega])
        got = o.sigma(T, V, Z, k, omega)
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_particle_hole_symmetry_at_fermi_surface():
    L, U, T = 4, 2.0, 0.25
    lat = Lattice(L)
    o = Oracle(lat.K, mode=MODE_LATTICE, eta=0.03)
    kF = 1 * L + 1                                   # (pi/2, pi/2), xi = 0
    assert abs(lat.xi[kF]) < 1e-15
    V = np.full((lat.K,) * 3, U)
    w = np.linspace(-3, 3, 13)
    s = o.sigma(T, V, np.ones(lat.K), kF, w)
    assert np.allclose(s.imag, s.imag[::-1], rtol=1e-12, atol=1e-15)
    assert np.allclose(s.real, -s.real[::-1], rtol=1e-12, atol=1e-15)
    assert np.all(s.imag < 0)


def test_zero_vertex_gives_unit_z():
    o = Oracle(16, 4, 4)
    Z = o.zfactor(0.3, np.zeros((16, 16, 16)), np.ones(16))
    assert np.array_equal(Z, np.ones(16))


def test_sopt_z_below_one_at_weak_coupling_wedge():
    """SOPT at weak coupling: the chord slope from outside is negative, so
    0 < Z < 1 along the Fermi surface (Sec. 3.1.1)."""
    N, n = 8 * 2, 4
    o = Oracle(N, n, n, eta=0.02)
    Z = o.zfactor(0.3, np.full((N, N, N), 1.0), np.ones(N))
    assert np.all(Z > 0.9) and np.all(Z < 1.0)
    # C4v: Z is constant on symmetry-related patches
    for g in inputs.c4v_patch_maps(N):
        assert np.allclose(Z[g], Z, rtol=1e-12)


def _single_pole_chord(A, E, eta, centre, margin, denom):
    """Chord of Re[A/(w + i eta - E)] = A (w - E)/((w - E)^2 + eta^2) between
    centre - margin and centre + margin, divided by denom (closed form)."""
    re = lambda w: A * (w - E) / ((w - E) ** 2 + eta ** 2)
    return (re(centre + margin) - re(centre - margin)) / denom


@pytest.mark.parametrize("case", [
    dict(t=0.25, U=2.0, T=0.5, eta=0.05, z=1.0, qp=False),
    dict(t=0.25, U=1.5, T=0.2, eta=0.02, z=0.8, qp=False),
    dict(t=0.3, U=2.5, T=0.35, eta=0.1, z=0.7, qp=True),
    dict(t=1.0, U=3.0, T=1.5, eta=0.02, z=1.0, qp=False),
], ids=["z1", "zlines", "qp", "wide"])
def test_z_chord_single_pole_closed_form(case):
    """Pin of the Z chord (Eq. (definition_Z), slope "from outside" with a
    margin of 2T, Sec. 3.1.1): on the one-point lattice (L = 1: p = q = r = 0)
    the self-energy is a single pole, Sigma(w) = A / (w + i eta - E) with
    E = x_0 (x_0 = Z xi_0 for quasi-particle lines, else xi_0 = -4t),
    A = Z^3 V^2 f(x_0)(1 - f(x_0)) (W = Z^3 (2V^2 - V^2), F = f(1-f)).  Its
    chord over xi_0 +- 2T is A (E-terms in closed form) / 4T, so Z is fixed
    without the oracle's pole sum.  The alternative readings -- margin T,
    denominator 2T, centre w = 0 instead of xi_0 -- give Z values far from it."""
    t, U, T, eta, z, qp = (case[k] for k in ("t", "U", "T", "eta", "z", "qp"))
    o = Oracle(1, mode=MODE_LATTICE, t=t, eta=eta, prop_mode=PROP_QP if qp else 0)
    xi0 = -4.0 * t
    x0 = z * xi0 if qp else xi0
    f = 1.0 / (1.0 + np.exp(x0 / T))
    A = z ** 3 * U * U * f * (1.0 - f)
    slope = _single_pole_chord(A, x0, eta, xi0, 2 * T, 4 * T)
    ref = 1.0 / (1.0 - slope)
    got = o.zfactor(T, np.full((1, 1, 1), U), np.full(1, z))[0]
    assert got == pytest.approx(ref, rel=1e-12)
    # discriminating power of the pin: each misreading moves Z by > 1 %
    for alt in (_single_pole_chord(A, x0, eta, xi0, T, 2 * T),        # margin T
                _single_pole_chord(A, x0, eta, xi0, 2 * T, 2 * T),    # denominator 2T
                _single_pole_chord(A, x0, eta, 0.0, 2 * T, 4 * T)):   # centred on w = 0
        assert abs(1.0 / (1.0 - alt) - ref) > 1e-2 * abs(ref)
