"""Pins of the oracle's spectral function and its Fermi-liquid (Gaussian)
approximation (Sec. 3.1.1, Figs. 2-3; the SOPT spectral workload).

* Sum rule: A(k, w) = -(1/pi) Im G of a causal self-energy integrates to 1
  (G ~ 1/w at large w); checked on a wide, fine grid for SOPT (V = U) on the
  4 x 4 lattice and for a random SU(2) vertex in wedge mode.
* A >= 0 (causality: Im Sigma <= 0) and, at half filling on the Fermi
  surface, A(w) = A(-w) (Re Sigma odd, Im Sigma even).
* The Gaussian of Fig. 3 has weight Z (closed form) and equals A at xi_k.
"""
import numpy as np

from oracle.oracle import MODE_LATTICE, Oracle
from paper_2005_00827_gb300 import inputs


def _spectral(o, T, V, Z, j, w):
    s = o.sigma(T, V, Z, j, w)
    z = o.zfactor_targets(T, V, Z, [j])[0]
    A, Afl = o.spectral(j, w, s, z)
    return A, Afl, z


def test_sum_rule_and_symmetry_sopt_lattice():
    L, U, T = 4, 2.0, 0.3
    o = Oracle(L * L, mode=MODE_LATTICE, eta=0.05)
    w = np.linspace(-40.0, 40.0, 80001)
    kF = 1 * L + 1                                     # (pi/2, pi/2), xi = 0
    A, Afl, z = _spectral(o, T, np.full((L * L,) * 3, U), np.ones(L * L), kF, w)
    dw = w[1] - w[0]
    assert abs(A.sum() * dw - 1.0) < 1e-6
    assert np.all(A >= 0.0)
    assert np.abs(A - A[::-1]).max() < 1e-10 * A.max()
    assert abs(Afl.sum() * dw - z) < 1e-9 * z
    assert Afl[len(w) // 2] == A[len(w) // 2]


def test_sum_rule_random_vertex_wedge():
    N, n, T = 8, 4, 0.25
    o = Oracle(N, n, n, eta=0.05)
    V = inputs.random_vertex(N, 2.0, seed=3, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    w = np.linspace(-60.0, 60.0, 120001)
    for j in (0, 1):
        A, Afl, z = _spectral(o, T, V, Z, j, w)
        dw = w[1] - w[0]
        assert abs(A.sum() * dw - 1.0) < 1e-5
        assert np.all(A >= 0.0)
        assert abs(Afl.sum() * dw - z) < 1e-9 * z


def test_gaussian_constrained_at_xi_off_grid_point():
    """A_FL at xi_j equals the linear interpolation of A there, on a grid
    that does not contain xi_j = 0."""
    L, U, T = 4, 1.5, 0.2
    o = Oracle(L * L, mode=MODE_LATTICE, eta=0.05)
    w = np.linspace(-3.0, 3.0, 64)                     # 0 lies between two points
    kF = 1 * L + 1
    A, Afl, z = _spectral(o, T, np.full((L * L,) * 3, U), np.ones(L * L), kF, w)
    m = np.searchsorted(w, 0.0) - 1
    u = (0.0 - w[m]) / (w[m + 1] - w[m])
    A0 = (1 - u) * A[m] + u * A[m + 1]
    ref = A0 * np.exp(-np.pi * A0 ** 2 * w ** 2 / z ** 2)
    assert np.abs(Afl - ref).max() < 1e-14 * A0
