"""Seeded synthetic inputs: reproducible, with the ranges the workloads state."""
import math

import numpy as np

from paper_2005_00827_gb300 import inputs


def test_splitmix64_reference_values():
    # first outputs of splitmix64 from seed 0 (Steele, Lea, Flood 2014): 0xe220a8397b1dcdaf, ...
    g = inputs.splitmix64(0)
    first = next(g)
    assert first == (0xE220A8397B1DCDAF >> 11) * (1.0 / (1 << 53))
    assert 0.0 <= next(g) < 1.0


def test_batch_specs_ranges_and_determinism():
    a, b = inputs.batch_specs(), inputs.batch_specs()
    assert a == b and len(a) == 128
    for s in a:
        assert 1.0 <= s["U"] <= 4.0
        assert 0.01 <= s["T_end"] <= 0.2 + 1e-12
        assert s["N"] in (24, 48, 72, 96)
    # all four patch counts occur
    assert {s["N"] for s in a} == {24, 48, 72, 96}
    lt = [math.log(s["T_end"]) for s in a]
    assert min(lt) < math.log(0.02) and max(lt) > math.log(0.1)


def test_random_vertex_is_c4v_symmetric_and_seeded():
    V = inputs.random_vertex(16, 2.0, seed=3)
    assert np.array_equal(V, inputs.random_vertex(16, 2.0, seed=3))
    for g in inputs.c4v_patch_maps(16):
        assert np.allclose(V[np.ix_(g, g, g)], V, rtol=0, atol=1e-15)
    assert np.all(V > 2.0 * 0.5 - 1e-12) and np.all(V < 2.0 * 1.5 + 1e-12)


def test_splitmix64_array_equals_the_generator():
    for seed in (0, 1, 20050082, (1 << 64) - 5):
        g = inputs.splitmix64(seed)
        ref = np.array([next(g) for _ in range(2000)])
        assert np.array_equal(inputs.splitmix64_array(seed, 2000), ref)


def test_shell_patch_maps_keep_the_shell():
    N, ns = 24, 3
    for g in inputs.c4v_patch_maps(N, ns):
        assert sorted(g) == list(range(N))
        assert np.array_equal(g % ns, np.arange(N) % ns)
    V = inputs.random_vertex(N, 2.0, seed=5, n_shell=ns)
    for g in inputs.c4v_patch_maps(N, ns):
        assert np.allclose(V[np.ix_(g, g, g)], V, rtol=0, atol=1e-15)
