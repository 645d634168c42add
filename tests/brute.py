"""Brute-force references used to pin the oracle (numpy only, no oracle code).

* Matsubara sums T sum_n G G evaluated term by term with an analytic
  1/w^2 + 1/w^4 tail (trigamma / tetragamma), not through Fermi functions.
* Scale derivatives d/dT by Richardson-extrapolated central differences.
* Finite-lattice momenta 2 pi m / L, for lattice-mode comparisons.
* Imaginary-time quadrature of the second-order self-energy.
"""
from __future__ import annotations

import numpy as np
from scipy.special import polygamma, roots_legendre


def matsubara_ph(a, b, T, nmax=20000):
    """T sum_n 1/((i w_n - a)(i w_n - b)) for arrays a, b (same shape)."""
    a = np.asarray(a, dtype=float)[..., None]
    b = np.asarray(b, dtype=float)[..., None]
    n = np.arange(-nmax, nmax)
    w = (2 * n + 1) * np.pi * T
    z = 1j * w
    s = (T / ((z - a) * (z - b))).sum(axis=-1).real
    # tail |n| >= nmax: -1/w^2 + (a^2+ab+b^2)/w^4, both signs of n
    t2 = polygamma(1, nmax + 0.5) / (4 * np.pi ** 2 * T ** 2)
    t4 = polygamma(3, nmax + 0.5) / 6.0 / (16 * np.pi ** 4 * T ** 4)
    a = a[..., 0]; b = b[..., 0]
    return s + 2 * T * (-t2 + (a * a + a * b + b * b) * t4)


def matsubara_pp(a, b, T, nmax=20000):
    """T sum_n 1/((i w_n - a)(-i w_n - b))."""
    a = np.asarray(a, dtype=float)[..., None]
    b = np.asarray(b, dtype=float)[..., None]
    n = np.arange(-nmax, nmax)
    z = 1j * (2 * n + 1) * np.pi * T
    s = (T / ((z - a) * (-z - b))).sum(axis=-1).real
    # large w: 1/((iw-a)(-iw-b)) = 1/w^2 - (a^2 - ab + b^2)/w^4 + ...
    t2 = polygamma(1, nmax + 0.5) / (4 * np.pi ** 2 * T ** 2)
    t4 = polygamma(3, nmax + 0.5) / 6.0 / (16 * np.pi ** 4 * T ** 4)
    a = a[..., 0]; b = b[..., 0]
    return s + 2 * T * (t2 - (a * a - a * b + b * b) * t4)


def ddT(fun, T, rel=1e-3):
    """Richardson-extrapolated central difference of fun(T) (O(h^4))."""
    h = rel * T
    d1 = (fun(T + h) - fun(T - h)) / (2 * h)
    d2 = (fun(T + h / 2) - fun(T - h / 2)) / h
    return (4 * d2 - d1) / 3


class Lattice:
    """L x L square lattice, momenta k_m = 2 pi (m1, m2)/L, index m1*L + m2."""

    def __init__(self, L, t=1.0, tp=0.0, mu=0.0):
        self.L = L
        self.K = L * L
        m = np.arange(self.K)
        self.m1, self.m2 = m // L, m % L
        kx, ky = 2 * np.pi * self.m1 / L, 2 * np.pi * self.m2 / L
        self.xi = -2 * t * (np.cos(kx) + np.cos(ky)) - 4 * tp * np.cos(kx) * np.cos(ky) - mu

    def add(self, a, b):
        L = self.L
        return ((self.m1[a] + self.m1[b]) % L) * L + (self.m2[a] + self.m2[b]) % L

    def sub(self, a, b):
        L = self.L
        return ((self.m1[a] - self.m1[b]) % L) * L + (self.m2[a] - self.m2[b]) % L

    def k4(self, k1, k2, k3):
        return self.sub(self.add(k1, k2), k3)

    def exchange_symmetrise(self, V):
        """V(k1,k2,k3) -> [V(k1,k2,k3) + V(k2,k1,k4)]/2 (exchange symmetry)."""
        K = self.K
        k1, k2, k3 = np.meshgrid(np.arange(K), np.arange(K), np.arange(K), indexing="ij")
        k4 = self.k4(k1, k2, k3)
        return 0.5 * (V + V[k2, k1, k4])

    def tr_symmetrise(self, V):
        """V(k1,k2,k3) -> [V(k1,k2,k3) + V(k3,k4,k1)]/2 (real static vertex)."""
        K = self.K
        k1, k2, k3 = np.meshgrid(np.arange(K), np.arange(K), np.arange(K), indexing="ij")
        k4 = self.k4(k1, k2, k3)
        return 0.5 * (V + V[k3, k4, k1])


def gamma_su2(V, k1, s1, k2, s2, k3, s3, s4):
    """Antisymmetrised spin-resolved vertex of an SU(2) coupling function:
    G(1,2;3,4) = V(k1,k2,k3) d(s1,s3) d(s2,s4) - V(k2,k1,k3) d(s1,s4) d(s2,s3)."""
    return (V[k1, k2, k3] * float(s1 == s3) * float(s2 == s4)
            - V[k2, k1, k3] * float(s1 == s4) * float(s2 == s3))


def sigma_tau_quadrature(lat: Lattice, k, U, T, n_mats, nodes=400):
    """Second-order self-energy at i w_n from the imaginary-time product
    Sigma(k, tau) = -U^2 (1/K^2) sum_{p,q} G(q,tau) G(k+p-q,tau) G(p,-tau),
    Fourier transformed by Gauss-Legendre quadrature over [0, beta]."""
    K = lat.K
    beta = 1.0 / T
    x, wq = roots_legendre(nodes)
    tau = 0.5 * beta * (x + 1.0)
    wq = 0.5 * beta * wq
    p, q = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
    r = lat.sub(lat.add(np.full_like(p, k), p), q)
    xp, xq, xr = lat.xi[p][..., None], lat.xi[q][..., None], lat.xi[r][..., None]
    fer = lambda e: 0.5 * (1.0 - np.tanh(0.5 * e / T))
    # G(e, tau>0) = -exp(-e tau)(1 - f(e));  G(e, -tau) = exp(e tau) f(e)
    prod = (-np.exp(-xq * tau) * (1 - fer(xq))) * (-np.exp(-xr * tau) * (1 - fer(xr))) \
        * (np.exp(xp * tau) * fer(xp))
    s_tau = -U * U * prod.sum(axis=(0, 1)) / K ** 2
    w = (2 * n_mats + 1) * np.pi * T
    return (wq * np.exp(1j * w * tau) * s_tau).sum()
