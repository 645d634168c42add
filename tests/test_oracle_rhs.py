"""Pins of the oracle's one-loop right-hand side (App. A.1,
Eq. (vertex_flow_general); Z weights of Eq. (vertex_flow_feedback_Z)).

* Lattice mode makes the patch scheme the exact finite-lattice one-loop flow,
  so the SU(2) channel formulas of the oracle must equal the generic one-loop
  equation for the antisymmetrised spin-resolved vertex, evaluated by brute
  force with explicit spin sums and term-by-term Matsubara bubbles.
* For V = U the flow reduces to RPA ladders with closed-form solutions:
  V = U / (1 + U dchi(Q)); the crossed channel diverges (Stoner), the pp
  channel screens (Sec. 3.2: ph-only flows reach strong coupling first).
* Symmetries: C4v in wedge mode, exchange in lattice mode.
"""
import numpy as np
import pytest

from oracle.oracle import (CH_ALL, CH_CR, CH_D, CH_PP, MODE_LATTICE, PROP_QP, REG_INTERACTION,
                           Oracle)
from paper_2005_00827_gb300 import inputs
from tests import brute
from tests.brute import Lattice, gamma_su2


def bubbles(lat, T, Z, regulator="T", g=1.0, qp=False):
    """Z-weighted loop kernels for every ordered pair (p5, p6) of momenta."""
    K = lat.K
    p5, p6 = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
    x5, x6 = lat.xi[p5], lat.xi[p6]
    if qp:
        x5, x6 = Z[p5] * x5, Z[p6] * x6
    if regulator == "T":
        lpp = brute.ddT(lambda TT: brute.matsubara_pp(x5, x6, TT), T)
        lph = brute.ddT(lambda TT: brute.matsubara_ph(x5, x6, TT), T)
        w = Z[p5] * Z[p6]
    else:
        lpp = brute.matsubara_pp(x5, x6, T)
        lph = brute.matsubara_ph(x5, x6, T)
        w = g * Z[p5] * Z[p6] * (Z[p5] + Z[p6])
    return w * lpp, w * lph


def generic_one_loop(lat, V, Lpp, Lph):
    """d Gamma(1 up, 2 dn; 3 up, 4 dn) from the generic one-loop equation
      -1/2 sum G(1,2;5,6) Lpp(5,6) G(5,6;3,4)
      +    sum G(1,6;3,5) Lph(5,6) G(5,2;6,4)      (direct particle-hole)
      -    sum G(1,6;4,5) Lph(5,6) G(5,2;6,3)      (crossed particle-hole)
    with explicit spin sums; returns the three channel arrays (pp, cr, d)."""
    K = lat.K
    ar = np.arange(K)
    k1, k2, k3 = np.meshgrid(ar, ar, ar, indexing="ij")
    k4 = lat.k4(k1, k2, k3)
    up, dn = 0, 1
    pp = np.zeros((K, K, K)); cr = np.zeros((K, K, K)); d = np.zeros((K, K, K))
    for p in range(K):
        pv = np.full_like(k1, p)
        a5, a6 = pv, lat.sub(lat.add(k1, k2), pv)
        for s5 in (up, dn):
            for s6 in (up, dn):
                g1 = gamma_su2(V, k1, up, k2, dn, a5, s5, s6)
                g2 = gamma_su2(V, a5, s5, a6, s6, k3, up, dn)
                pp += -0.5 * g1 * Lpp[a5, a6] * g2 / K
        b6 = pv
        b5 = lat.sub(lat.add(k1, pv), k3)
        c5 = lat.sub(lat.add(k1, pv), k4)
        for s5 in (up, dn):
            for s6 in (up, dn):
                g1 = gamma_su2(V, k1, up, b6, s6, k3, up, s5)
                g2 = gamma_su2(V, b5, s5, k2, dn, b6, s6, dn)
                d += g1 * Lph[b5, b6] * g2 / K
                h1 = gamma_su2(V, k1, up, b6, s6, k4, dn, s5)
                h2 = gamma_su2(V, c5, s5, k2, dn, b6, s6, up)
                cr += -h1 * Lph[c5, b6] * h2 / K
    return pp, cr, d


def oracle_channels(o, lam, V, Z):
    N = o.N
    out = np.zeros((3, N, N, N))
    for i in range(N):
        for j in range(N):
            for l in range(N):
                out[:, i, j, l] = o.rhs_triple(lam, V, Z, i, j, l)
    return out


def normwise(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def exchange_symmetric_vertex(lat, U, seed, tr=False):
    V = inputs.random_vertex(lat.K, U, seed=seed, c4v=False)
    V = lat.exchange_symmetrise(V)
    if tr:
        for _ in range(3):
            V = lat.exchange_symmetrise(lat.tr_symmetrise(V))
    return V


@pytest.mark.parametrize("case", ["T-paper", "T-qp", "g-paper"])
def test_su2_channels_equal_spin_resolved_one_loop(case):
    L = 4
    lat = Lattice(L)
    rng = np.random.default_rng(7)
    Z = rng.uniform(0.75, 1.0, lat.K)
    V = exchange_symmetric_vertex(lat, 2.0, seed=11)
    if case == "T-paper":
        o = Oracle(lat.K, mode=MODE_LATTICE)
        lam, T = 0.4, 0.4
        Lpp, Lph = bubbles(lat, T, Z)
    elif case == "T-qp":
        o = Oracle(lat.K, mode=MODE_LATTICE, prop_mode=PROP_QP)
        lam, T = 0.3, 0.3
        Lpp, Lph = bubbles(lat, T, Z, qp=True)
    else:
        T = 0.25
        o = Oracle(lat.K, mode=MODE_LATTICE, regulator=REG_INTERACTION, T_fixed=T)
        lam = 0.7
        Lpp, Lph = bubbles(lat, T, Z, regulator="g", g=lam)
    ref = generic_one_loop(lat, V, Lpp, Lph)
    got = oracle_channels(o, lam, V, Z)
    for ch in range(3):
        assert normwise(got[ch], ref[ch]) < 1e-7, ("pp", "cr", "d")[ch]
    # the full RHS is the sum of the channels
    assert normwise(o.rhs(lam, V, Z), got.sum(axis=0)) < 1e-14


def test_constant_vertex_is_second_order_pt():
    """V = U: dV = -U^2 d/dT[chi_pp(k1+k2) + chi_ph(k3-k2)], direct channel 0."""
    L, U, T = 4, 2.0, 0.35
    lat = Lattice(L)
    o = Oracle(lat.K, mode=MODE_LATTICE)
    Z = np.ones(lat.K)
    V = np.full((lat.K,) * 3, U)
    Lpp, Lph = bubbles(lat, T, Z)
    ar = np.arange(lat.K)
    chi_pp = np.array([Lpp[ar, lat.sub(Q, ar)].mean() for Q in ar])
    chi_ph = np.array([Lph[ar, lat.add(ar, Q)].mean() for Q in ar])
    got = oracle_channels(o, T, V, Z)
    k1, k2, k3 = np.meshgrid(ar, ar, ar, indexing="ij")
    assert normwise(got[0], -U * U * chi_pp[lat.add(k1, k2)]) < 1e-7
    assert normwise(got[1], -U * U * chi_ph[lat.sub(k3, k2)]) < 1e-7
    assert np.abs(got[2]).max() < 1e-14 * np.abs(got[1]).max()
    # pp screens a repulsive U (dchi_pp/dT < 0 -> dV/dT > 0, V falls as T falls)
    assert np.all(got[0] > 0)


def chi_lattice(lat, T, Q, kind):
    ar = np.arange(lat.K)
    if kind == "pp":
        return brute.matsubara_pp(lat.xi[ar], lat.xi[lat.sub(np.full_like(ar, Q), ar)], T).mean()
    return brute.matsubara_ph(lat.xi[ar], lat.xi[lat.add(ar, np.full_like(ar, Q))], T).mean()


@pytest.mark.parametrize("kind", ["pp", "cr"])
def test_ladder_flow_matches_rpa_closed_form(kind):
    """Single-channel T-flow from V(T0) = U: V(Q, T) = U/(1 + U[chi(Q,T) - chi(Q,T0)])."""
    L, U, T0, T1 = 4, 1.5, 1.0, 0.3
    lat = Lattice(L)
    o = Oracle(lat.K, mode=MODE_LATTICE, channels=CH_PP if kind == "pp" else CH_CR)
    V0 = np.full((lat.K,) * 3, U)
    r = o.flow(V0, np.ones(lat.K), T0, T1, np.log(0.98), stop_abs_v=1e9)
    assert r["status"] == "REACHED_END"
    assert r["lam"] == pytest.approx(T1, rel=1e-14)
    ar = np.arange(lat.K)
    k1, k2, k3 = np.meshgrid(ar, ar, ar, indexing="ij")
    Qidx = lat.add(k1, k2) if kind == "pp" else lat.sub(k3, k2)
    chname = "pp" if kind == "pp" else "ph"
    Vq = np.array([U / (1 + U * (chi_lattice(lat, T1, Q, chname) - chi_lattice(lat, T0, Q, chname)))
                   for Q in ar])
    assert normwise(r["V"], Vq[Qidx]) < 1e-8
    if kind == "pp":
        assert r["V"].max() <= U + 1e-12          # repulsion screened
    else:
        assert r["V"].max() > U                    # antiferromagnetic enhancement


def test_crossed_ladder_divergence_scale():
    """Flow to strong coupling (Sec. 3.2): the crossed ladder at Q = (pi, pi)
    crosses |V| = 20 where 1 + U dchi_ph = U/20; Lambda_c within 0.5%."""
    L, U, T0 = 4, 2.0, 1.0
    lat = Lattice(L)
    o = Oracle(lat.K, mode=MODE_LATTICE, channels=CH_CR)
    r = o.flow(np.full((lat.K,) * 3, U), np.ones(lat.K), T0, 0.01, np.log(0.98), stop_abs_v=20.0)
    assert r["status"] == "DIVERGED"
    Qpi = (L // 2) * L + L // 2
    c0 = chi_lattice(lat, T0, Qpi, "ph")

    def past_crossing(T):   # V(T) above the bound, or past the pole of the ladder
        den = 1 + U * (chi_lattice(lat, T, Qpi, "ph") - c0)
        return den <= 0 or U / den > 20.0

    hi, lo = T0, 0.05       # V(T0) = U < 20; find a temperature past the crossing
    while not past_crossing(lo):
        lo *= 0.9
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if past_crossing(mid):
            lo = mid
        else:
            hi = mid
    Tc = 0.5 * (lo + hi)
    assert r["lambda_c"] == pytest.approx(Tc, rel=5e-3)


def test_exchange_symmetry_preserved_lattice():
    lat = Lattice(4)
    o = Oracle(lat.K, mode=MODE_LATTICE)
    V = exchange_symmetric_vertex(lat, 2.0, seed=5)
    dV = o.rhs(0.3, V, np.ones(lat.K))
    ar = np.arange(lat.K)
    k1, k2, k3 = np.meshgrid(ar, ar, ar, indexing="ij")
    assert normwise(dV[k2, k1, lat.k4(k1, k2, k3)], dV) < 1e-13


def test_nesting_identity_lattice():
    """Half filling, t' = 0: xi(k + (pi,pi)) = -xi(k) gives
    chi_pp(Q) = -chi_ph((pi,pi) - Q), seen through single-channel RHS at V = U."""
    L, U, T = 4, 1.0, 0.3
    lat = Lattice(L)
    Z = np.ones(lat.K)
    V = np.full((lat.K,) * 3, U)
    opp = Oracle(lat.K, mode=MODE_LATTICE, channels=CH_PP)
    ocr = Oracle(lat.K, mode=MODE_LATTICE, channels=CH_CR)
    Qpi = (L // 2) * L + L // 2
    for Q in range(lat.K):
        # pp at k1 + k2 = Q (k1 = Q, k2 = 0); cr at k3 - k2 = Pi - Q (k2 = 0, k3 = Pi - Q)
        a = opp.rhs_triple(T, V, Z, Q, 0, 0)[0]
        b = ocr.rhs_triple(T, V, Z, 0, 0, lat.sub(Qpi, Q))[1]
        assert a == pytest.approx(-b, rel=1e-12, abs=1e-15)


def test_c4v_covariance_wedge():
    N, n = 16, 4
    o = Oracle(N, n, n)
    V = inputs.random_vertex(N, 2.0, seed=3, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    dV = o.rhs(0.2, V, Z)
    for g in inputs.c4v_patch_maps(N):
        assert normwise(dV[np.ix_(g, g, g)], dV) < 1e-12


def test_interaction_flow_scales_with_g():
    lat = Lattice(4)
    o = Oracle(lat.K, mode=MODE_LATTICE, regulator=REG_INTERACTION, T_fixed=0.2)
    V = exchange_symmetric_vertex(lat, 1.0, seed=2)
    Z = np.ones(lat.K)
    r1, r2 = o.rhs(1.0, V, Z), o.rhs(0.37, V, Z)
    assert normwise(r2, 0.37 * r1) < 1e-14


@pytest.mark.parametrize("ch", [1, 2, 4], ids=["pp", "cr", "d"])
def test_each_channel_is_c4v_invariant(ch):
    """The premise of the contraction's row orbits: for a C4v-symmetric V and
    Z every channel's contribution is invariant by itself."""
    N, n = 16, 4
    V = inputs.random_vertex(N, 2.0, seed=5, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    dV = Oracle(N, n, n, channels=ch).rhs(0.2, V, Z)
    assert np.abs(dV).max() > 0
    for g in inputs.c4v_patch_maps(N):
        assert normwise(dV[np.ix_(g, g, g)], dV) < 1e-12


def test_row_orbit_expansion_rebuilds_every_channel():
    """The row-orbit expansion restated on the oracle's channels: a channel
    GEMM row is a transfer pair Q = (x, y), its column n (pp: row (k1, k2),
    column k3; cr: row (k3, k2), column k1; d: row (k1, k3), column k2); keeping
    only the representative rows (the image of Q with the smallest index) and
    reading row Q = g rep at column g^-1 n reproduces the whole channel."""
    N, n = 16, 4
    V = inputs.random_vertex(N, 2.0, seed=6, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    maps = inputs.c4v_patch_maps(N)
    # representative of every pair and the element g with Q = g(rep)
    rep, gof = {}, {}
    for x in range(N):
        for y in range(N):
            imgs = [(int(g[x]) * N + int(g[y]), k) for k, g in enumerate(maps)]
            best, k = min(imgs)
            rep[(x, y)] = divmod(best, N)
            gof[(x, y)] = k          # maps[k] sends (x, y) to its representative
    reps = sorted(set(rep.values()))
    assert len(reps) == (N * N + 16) // 8          # Burnside: 256 pairs, 16 fixed by the mirrors
    for ch, row_col in ((1, lambda k1, k2, k3: ((k1, k2), k3)), (2, lambda k1, k2, k3: ((k3, k2), k1)),
                        (4, lambda k1, k2, k3: ((k1, k3), k2))):
        full = Oracle(N, n, n, channels=ch).rhs(0.2, V, Z)
        # the channel's GEMM output rows out[(x, y)][col] = full at the triple they fill
        out = {}
        for k1 in range(N):
            for k2 in range(N):
                for k3 in range(N):
                    q, col = row_col(k1, k2, k3)
                    out.setdefault(q, np.zeros(N))[col] = full[k1, k2, k3]
        rebuilt = np.empty_like(full)
        for k1 in range(N):
            for k2 in range(N):
                for k3 in range(N):
                    q, col = row_col(k1, k2, k3)
                    g = maps[gof[q]]                  # rep = g(q), so q = g^-1(rep), col -> g(col)
                    rebuilt[k1, k2, k3] = out[rep[q]][int(g[col])]
        assert normwise(rebuilt, full) < 1e-12
