"""Pins of the oracle's patch geometry (Sec. 3.2 gives only patch counts; the
wedge reading: N angular wedges about the origin, fine polar grid per wedge).
Checked against closed forms: the Fermi surface at half filling, the area of
the Brillouin zone, the C4v group of the square lattice."""
import numpy as np
import pytest

from oracle.oracle import MODE_LATTICE, Oracle


@pytest.mark.parametrize("N,n", [(16, 8), (24, 4), (48, 6)])
def test_patch_reps_on_fermi_surface(N, n):
    o = Oracle(N, n, n)
    kf, fk, fw, fp = o.geometry()
    # half filling, t' = 0: FS is the diamond |kx| + |ky| = pi
    assert np.allclose(np.abs(kf).sum(axis=1), np.pi, atol=1e-14)
    th = np.arctan2(kf[:, 1], kf[:, 0]) % (2 * np.pi)
    assert np.allclose(th, 2 * np.pi * np.arange(N) / N, atol=1e-13)
    for j in range(N):
        assert abs(o.xi(*kf[j])) < 1e-14
        assert o.proj(*kf[j]) == j


@pytest.mark.parametrize("N,n", [(16, 8), (24, 4)])
def test_every_fine_point_projects_to_its_wedge(N, n):
    o = Oracle(N, n, n)
    kf, fk, fw, fp = o.geometry()
    assert np.all(fp == np.repeat(np.arange(N), n * n))
    for p in range(o.M):
        assert o.proj(*fk[p]) == fp[p]
        # periodicity of the projection
        assert o.proj(fk[p, 0] + 2 * np.pi, fk[p, 1] - 4 * np.pi) == fp[p]
    # fine points inside the Brillouin zone
    assert np.all(np.abs(fk) < np.pi)


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_weights_integrate_brillouin_zone(n):
    """sum w -> area / (2 pi)^2 = 1; the midpoint rule in angle converges as 1/n^2."""
    N = 16
    o = Oracle(N, n, n)
    kf, fk, fw, fp = o.geometry()
    err = abs(fw.sum() - 1.0)
    assert err < 0.03 / n ** 2
    # exact area of one wedge: int 1/2 r_BZ(theta)^2 dtheta, r_BZ = pi / max(|c|,|s|)
    th = np.linspace(-np.pi / N, np.pi / N, 200001)
    rbz = np.pi / np.maximum(np.abs(np.cos(th)), np.abs(np.sin(th)))
    area0 = np.trapezoid(0.5 * rbz ** 2, th) / (2 * np.pi) ** 2
    assert fw[: n * n].sum() == pytest.approx(area0, rel=0.05 / n ** 2)


def test_projection_c4v_covariant():
    N = 48
    o = Oracle(N, 4, 4)
    rng = np.random.default_rng(3)
    dth = 2 * np.pi / N
    done = 0
    for _ in range(400):
        k = rng.uniform(-np.pi, np.pi, 2)
        th = np.arctan2(k[1], k[0])
        frac = (th / dth + 0.5) % 1.0
        if min(frac, 1 - frac) < 1e-6:
            continue
        j = o.proj(*k)
        assert o.proj(-k[1], k[0]) == (j + N // 4) % N        # rotation by pi/2
        assert o.proj(k[1], k[0]) == (N // 4 - j) % N         # reflection x <-> y
        assert o.proj(k[0], -k[1]) == (-j) % N                # reflection y -> -y
        done += 1
    assert done > 350


def test_lattice_mode_geometry():
    L = 4
    o = Oracle(L * L, mode=MODE_LATTICE)
    kf, fk, fw, fp = o.geometry()
    assert o.M == L * L
    assert np.allclose(fw, 1.0 / (L * L))
    assert np.array_equal(fp, np.arange(L * L))
    for j in range(L * L):
        m1, m2 = divmod(j, L)
        assert np.allclose(kf[j], [2 * np.pi * m1 / L, 2 * np.pi * m2 / L])
        assert o.proj(*kf[j]) == j
        assert o.proj(kf[j, 0] - 2 * np.pi, kf[j, 1] + 2 * np.pi) == j


def test_rejects_bad_parameters():
    with pytest.raises(ValueError):
        Oracle(18, 4, 4)        # N not a multiple of 4
    with pytest.raises(ValueError):
        Oracle(16, 4, 3)        # odd radial count
    with pytest.raises(ValueError):
        Oracle(15, mode=MODE_LATTICE)
