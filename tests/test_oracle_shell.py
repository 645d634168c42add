"""Pins of the oracle's energy-shell patching (Sec. 3.2: "7 shells in total in
the energy direction and 32 angular sections"; shell mode of the oracle's
geometry).  Each test checks the geometry against something other than the
geometry code itself: wedge mode (one shell), a Cartesian count of the zone,
the lattice's C4v symmetry and the energies the construction promises."""
import math

import numpy as np
import pytest

from oracle.oracle import MODE_SHELL, MODE_WEDGE, Oracle


def shells(Na, ns, nt=4, nr=4, **kw):
    return Oracle(Na * ns, nt, nr, mode=MODE_SHELL, n_shell=ns, **kw)


def test_one_shell_is_wedge_mode():
    """n_s = 1: the same representatives, fine points, weights and patches as
    the angular wedges, and the same projection of arbitrary momenta."""
    a, b = Oracle(16, 4, 6), shells(16, 1, 4, 6)
    for x, y in zip(a.geometry(), b.geometry()):
        assert np.array_equal(x, y)
    rng = np.random.default_rng(3)
    for kx, ky in rng.uniform(-7, 7, (500, 2)):
        assert a.proj(kx, ky) == b.proj(kx, ky)


@pytest.mark.parametrize("ns,tp", [(3, 0.0), (7, 0.0), (5, -0.1)])
def test_shell_areas_match_a_cartesian_count(ns, tp):
    """The weight of each shell (summed over its wedges) is the fraction of
    the zone whose energy lies in the shell, counted on a 2000 x 2000
    Cartesian midpoint grid; the total weight is the wedge mode's."""
    Na, nt = 8, 24
    o = shells(Na, ns, nt, 4, tp=tp)
    kf, fk, fw, fp = o.geometry()
    wedge_total = Oracle(Na, nt, 4, tp=tp).geometry()[2].sum()
    assert fw.sum() == pytest.approx(wedge_total, rel=1e-12)
    D = o.shell_width()
    n = 2000
    k = -math.pi + (np.arange(n) + 0.5) * (2 * math.pi / n)
    cx, cy = np.meshgrid(np.cos(k), np.cos(k), indexing="ij")
    xi = -2.0 * (cx + cy) - 4.0 * tp * cx * cy
    edges = (np.arange(1, ns) - ns / 2) * D
    s_cart = np.searchsorted(edges, xi, side="right")
    frac = np.bincount(s_cart.ravel(), minlength=ns) / n ** 2
    got = np.bincount(fp % ns, weights=fw, minlength=ns) / fw.sum()
    assert np.abs(got - frac).max() < 4e-3


def test_fine_points_project_to_their_patch():
    o = shells(8, 7, 3, 4)
    kf, fk, fw, fp = o.geometry()
    for p in np.flatnonzero(fw > 0):
        assert o.proj(*fk[p]) == fp[p]


def test_representatives():
    """Fermi-shell representatives are the wedge mode's k_F; the others lie on
    the wedge's centre ray at the shell's middle energy, or at the zone edge
    of the ray when the band ends below that energy along it."""
    Na, ns = 8, 5
    o = shells(Na, ns)
    kf = o.geometry()[0]
    kw = Oracle(Na, 4, 4).geometry()[0]
    D = o.shell_width()
    for w in range(Na):
        th = 2 * math.pi * w / Na
        for s in range(ns):
            k = kf[w * ns + s]
            if s == ns // 2:
                assert np.array_equal(k, kw[w])
                continue
            r = math.hypot(*k)
            assert abs(math.atan2(k[1], k[0]) - math.remainder(th, 2 * math.pi)) < 1e-12 or r == 0.0
            want = (s - ns // 2) * D
            rbz = math.pi / max(abs(math.cos(th)), abs(math.sin(th)))
            if abs(o.xi(*k) - want) > 1e-9:
                # clamped: the ray's range of energies ends short of the shell's middle
                assert (r == pytest.approx(rbz, abs=1e-12) and o.xi(*k) < want) or (r == 0.0 and o.xi(0, 0) > want)


def test_projection_is_c4v_covariant():
    """Rotating a momentum by pi/2 moves its wedge by N_a/4 and keeps its
    shell; the mirror k_y -> -k_y sends wedge w to -w.  Momenta within 1e-9
    of a wedge ray or a shell edge are skipped (the tie rules are not
    covariant there)."""
    Na, ns = 16, 3
    o = shells(Na, ns)
    D = o.shell_width()
    rng = np.random.default_rng(11)
    n_checked = 0
    for kx, ky in rng.uniform(-math.pi, math.pi, (4000, 2)):
        u = math.atan2(ky, kx) / (2 * math.pi / Na) + 0.5
        e = o.xi(kx, ky) / D + ns / 2
        if abs(u - round(u)) < 1e-9 or abs(e - round(e)) < 1e-9:
            continue
        j = o.proj(kx, ky)
        w, s = divmod(j, ns)
        assert o.proj(-ky, kx) == ((w + Na // 4) % Na) * ns + s
        assert o.proj(kx, -ky) == ((-w) % Na) * ns + s
        n_checked += 1
    assert n_checked > 3900


def test_shell_follows_the_energy():
    """Along a ray the shell index never decreases, and a momentum just below
    or above a shell edge falls in the shell below or above it."""
    Na, ns = 8, 7
    o = shells(Na, ns)
    D = o.shell_width()
    th = 2 * math.pi * 1 / Na + 0.05
    rb = math.pi / max(abs(math.cos(th)), abs(math.sin(th)))
    last = -1
    for r in np.linspace(0.0, rb * (1 - 1e-9), 400):
        s = o.proj(r * math.cos(th), r * math.sin(th)) % ns
        assert s >= last
        last = s
    assert last == ns - 1
    for b in range(1, ns):
        edge = (b - ns / 2) * D
        lo, hi = 0.0, rb
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if o.xi(mid * math.cos(th), mid * math.sin(th)) < edge:
                lo = mid
            else:
                hi = mid
        if hi >= rb * (1 - 1e-12):
            continue          # the ray ends below this edge
        below = o.proj(lo * (1 - 1e-6) * math.cos(th), lo * (1 - 1e-6) * math.sin(th)) % ns
        above = o.proj(hi * (1 + 1e-6) * math.cos(th), hi * (1 + 1e-6) * math.sin(th)) % ns
        assert (below, above) == (b - 1, b)


def test_rejected_shell_parameters():
    with pytest.raises(ValueError):
        shells(8, 2)                               # even shell count: no Fermi shell
    with pytest.raises(ValueError):
        Oracle(30, 4, 4, mode=MODE_SHELL, n_shell=3)   # 10 wedges: not C4v
    with pytest.raises(ValueError):
        shells(8, 3, tp=0.6)                       # xi not monotone along the rays
    assert MODE_WEDGE == 0
