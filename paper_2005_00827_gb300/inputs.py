"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the method's arithmetic: it draws random numbers,
permutes patch indices by the C4v symmetry of the angular patching, and
names the workloads.  The paper (arXiv:2005.00827) uses no dataset: its runs
are parameter scans of the half-filled square-lattice Hubbard model (t = 1,
t' = 0, mu = 0; Sec. 3) on patch discretisations of 16-728 patches (Sec. 3.2).
The workloads below reproduce those shapes with seeded draws.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed: int):
    """Counter-based generator (Steele, Lea, Flood 2014): yields uniform
    floats in [0, 1) with 53 random bits."""
    state = seed & MASK64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        z ^= z >> 31
        yield (z >> 11) * (1.0 / (1 << 53))


def splitmix64_array(seed: int, count: int) -> np.ndarray:
    """The first `count` values of splitmix64(seed) at once (numpy uint64
    arithmetic wraps modulo 2^64 as the generator's masks do)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def c4v_patch_maps(N: int, n_shell: int = 1):
    """The 8 index permutations of the angular patches under C4v (wedge
    centres at 2 pi w / N_a, N_a = N / n_shell a multiple of 4; patch
    j = w n_shell + s): w -> +-w + m N_a/4 (mod N_a), the shell s kept."""
    Na = N // n_shell
    if N % n_shell or Na % 4:
        raise ValueError("C4v needs N / n_shell % 4 == 0")
    w, sh = np.divmod(np.arange(N), n_shell)
    maps = []
    for m in range(4):
        maps.append(((w + m * Na // 4) % Na) * n_shell + sh)
        maps.append(((-w + m * Na // 4) % Na) * n_shell + sh)
    return maps


def c4v_symmetrise(V: np.ndarray, n_shell: int = 1) -> np.ndarray:
    """Average a coupling array V[k1,k2,k3] over the C4v patch permutations."""
    N = V.shape[0]
    out = np.zeros_like(V)
    for g in c4v_patch_maps(N, n_shell):
        out += V[np.ix_(g, g, g)]
    return out / 8.0


def random_vertex(N: int, U: float, seed: int = 1, amp: float = 0.5, c4v: bool = True,
                  n_shell: int = 1) -> np.ndarray:
    """V = U + amp U s with s uniform in [-1, 1] (splitmix64), FP64, [k1][k2][k3]."""
    s = 2.0 * splitmix64_array(seed, N ** 3) - 1.0
    V = (U + amp * U * s).reshape(N, N, N)
    return c4v_symmetrise(V, n_shell) if c4v else V


def z_profile(N: int, kind: str = "one", n_shell: int = 1) -> np.ndarray:
    """Quasi-particle weights per patch: 'one' (Z = 1) or 'aniso'
    (Z_j = 0.9 + 0.05 cos(4 theta_j) - 0.02 s', theta_j = 2 pi w / N_a the
    angle of patch j = w n_shell + s and s' = |s - n_shell // 2| its distance
    from the Fermi shell; C4v symmetric)."""
    if kind == "one":
        return np.ones(N)
    w, sh = np.divmod(np.arange(N), n_shell)
    th = 2 * np.pi * w / (N // n_shell)
    return 0.9 + 0.05 * np.cos(4 * th) - 0.02 * np.abs(sh - n_shell // 2)


def batch_specs(count: int = 128, seed: int = 20050082):
    """Phase-boundary sweep: for i = 0..count-1 in order, U = 1 + 3u,
    T_end = exp(ln 0.01 + u ln 20), N_p = {24,48,72,96}[floor(4u)] (one u each)."""
    gen = splitmix64(seed)
    specs = []
    for _ in range(count):
        U = 1.0 + 3.0 * next(gen)
        T_end = math.exp(math.log(0.01) + next(gen) * math.log(20.0))
        Np = (24, 48, 72, 96)[min(3, int(4 * next(gen)))]
        specs.append(dict(U=U, T_end=T_end, N=Np))
    return specs


# Workloads shaped like the paper's runs (t = 1, t' = 0, mu = 0; T-flow from
# T = 1 with d ln T = ln 0.98, stop at max|V| > 20).
WORKLOADS = {
    "np16_n8": dict(N=16, n=8, U=2.0, T_end=0.05, z_feedback=False, n_omega=0),
    "np48_n16": dict(N=48, n=16, U=3.0, T_end=0.05, z_feedback=True, n_omega=512),
    "np48_n32": dict(N=48, n=32, U=3.0, T_end=0.05, z_feedback=True, n_omega=512),
    "np96_n32": dict(N=96, n=32, U=2.5, T_end=0.02, z_feedback=True, n_omega=1024),
    "np192_n32": dict(N=192, n=32, U=2.0, T_end=0.01, z_feedback=True, n_omega=2048),
    # energy-shell patching (Sec. 3.2): 32 angular sections x 7 shells = 224 patches,
    # per patch 8 angular x 8 radial fine points
    "np224_s7": dict(N=224, n=8, U=2.0, T_end=0.05, z_feedback=True, n_omega=0, n_shell=7),
}
