"""GPU parity at the sizes of the paper-shaped workloads, through the C ABI.

* The divergence scale of the Z-feedback temperature flow (Sec. 3.2 flow to
  strong coupling, Z from Eq. (definition_Z) once per step) against the
  oracle: FP64 to 1e-9, mixed and tensor-core forms to 0.5 %.
* np96_n32 (N = 96 wedges, 32 x 32 fine points each, the bench workload):
  - the one-loop RHS (App. A.1, Eq. (vertex_flow_general)) on sampled output
    triples against the oracle, degenerate transfers included (ph at Q = 0,
    pp on the nesting vector (pi, pi)), normalised by the oracle's largest
    sampled value: FP64 1e-10, mixed and tensor-core 1e-4;
  - the whole RHS of the mixed and tensor-core forms against the FP64 GPU form
    (normwise 1e-4: the accuracy behind their speed-up over FP64);
  - Z of the flow step (C4v-irreducible targets, mirror-line targets over half
    of the loop points) against the oracle on a mirror-line and a generic
    patch, 1e-4;
  - the tensor-core flow against the FP64 flow up to the step half-way (in
    ln T) to the divergence scale, vertex normwise 1e-4.
* np48_n16 and np16_n8 complete flows; np192_n32 sampled RHS.
"""
import concurrent.futures as cf
import math
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2005_00827_gb300 import api, inputs

pytestmark = pytest.mark.gpu

STEP = math.log(0.98)


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()


def zeros(n):
    import torch
    return torch.zeros(n, dtype=torch.float64, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_triples(o, lam, V, Z, triples):
    """Oracle RHS of each (i, j, l) on all host cores (the C call releases the
    interpreter lock)."""
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return np.array(list(ex.map(lambda t: o.rhs_triple(lam, V, Z, *t).sum(), triples)))


def sample_triples(N, count, seed, extra=()):
    rng = np.random.default_rng(seed)
    t = [tuple(int(x) for x in rng.integers(0, N, 3)) for _ in range(count)]
    return list(extra) + t


def degenerate_triples(N):
    """ph transfers at Q = 0 (cr: k3 = k2, d: k1 = k3), pp on the nesting
    vector (k_F(N/8) + k_F(N/8) = (pi, pi) and k_F(3N/8) + k_F(3N/8) =
    (-pi, pi), the same lattice momentum) and pp at Q = (0, pi)."""
    a, b = N // 8, 3 * N // 8
    return [(5, 7, 7), (9, 3, 9), (a, a, 0), (a, a, a), (b, b, 2), (a, b, 1), (0, 0, 0), (N // 4, 0, N // 4)]


# --------------------------------------------------------------------------- #
# divergence scale with Z feedback
# --------------------------------------------------------------------------- #
@pytest.fixture(scope="module")
def zflow_ref():
    N, n, U = 16, 4, 3.0
    o = Oracle(N, n, n, eta=0.02)
    r = o.flow(np.full((N, N, N), U), np.ones(N), 1.0, 0.01, STEP, z_feedback=True)
    assert r["status"] == "DIVERGED"
    return dict(N=N, n=n, U=U, ref=r)


@pytest.mark.parametrize("prec,rel", [(api.QPFRG_FP64, 1e-9), (api.QPFRG_MIXED, 5e-3), (api.QPFRG_MIXED_TC, 5e-3)],
                         ids=["fp64", "mixed", "tc"])
def test_z_feedback_flow_divergence_matches_oracle(zflow_ref, prec, rel):
    N, n, U, ref = zflow_ref["N"], zflow_ref["n"], zflow_ref["U"], zflow_ref["ref"]
    with api.Context(N, n, n, U=U, lambda0=1.0, precision=prec, lambda_end=0.01, z_feedback=1, eta=0.02) as c:
        r = api.qpfrg_flow(c.h).as_dict()
        Zg = zeros(N)
        api.qpfrg_read_state(c.h, None, Zg)
        Zg = host(Zg)
    assert r["status"] == "DIVERGED"
    assert r["lambda_c"] == pytest.approx(ref["lambda_c"], rel=rel)
    if prec == api.QPFRG_FP64:
        assert r["steps"] == ref["steps"]
        assert np.abs(Zg - ref["Z"]).max() < 1e-9
    else:
        assert abs(r["steps"] - ref["steps"]) <= 1


# --------------------------------------------------------------------------- #
# np96_n32: the bench workload
# --------------------------------------------------------------------------- #
@pytest.fixture(scope="module")
def np96():
    N, n, U = 96, 32, 2.5
    o = Oracle(N, n, n, eta=0.02)
    V = inputs.random_vertex(N, U, seed=1)
    Z = inputs.z_profile(N, "aniso")
    return dict(N=N, n=n, U=U, o=o, V=V, Z=Z)


@pytest.mark.parametrize("prec,tol", [(api.QPFRG_FP64, 1e-10), (api.QPFRG_MIXED, 1e-4), (api.QPFRG_MIXED_TC, 1e-4)],
                         ids=["fp64", "mixed", "tc"])
def test_rhs_np96_sampled_triples_against_oracle(np96, prec, tol):
    N, n, U, o, V, Z = (np96[k] for k in ("N", "n", "U", "o", "V", "Z"))
    T = 0.1
    triples = sample_triples(N, 200, seed=7, extra=degenerate_triples(N))
    ref = oracle_triples(o, T, V, Z, triples)
    with api.Context(N, n, n, U=U, precision=prec) as c:
        if prec == api.QPFRG_MIXED_TC:
            api.qpfrg_autotune(c.h, T)           # the bench's launch configuration
        out = zeros(N ** 3)
        api.qpfrg_rhs(c.h, T, dev(V), dev(Z), out)
        got = host(out).reshape(N, N, N)
    g = np.array([got[t] for t in triples])
    assert np.abs(g - ref).max() < tol * np.abs(ref).max()


def test_rhs_np96_mixed_forms_against_fp64_gpu(np96):
    """Equal accuracy behind the speed-up: every one of the N^3 outputs of the
    mixed and tensor-core RHS against the FP64 GPU RHS (itself pinned to the
    oracle at 1e-10 above), at T = 1, 0.1 and 0.02."""
    N, n, U, V, Z = (np96[k] for k in ("N", "n", "U", "V", "Z"))
    for T in (1.0, 0.1, 0.02):
        outs = {}
        for prec in (api.QPFRG_FP64, api.QPFRG_MIXED, api.QPFRG_MIXED_TC):
            with api.Context(N, n, n, U=U, precision=prec) as c:
                out = zeros(N ** 3)
                api.qpfrg_rhs(c.h, T, dev(V), dev(Z), out)
                outs[prec] = host(out)
        ref = outs[api.QPFRG_FP64]
        for prec in (api.QPFRG_MIXED, api.QPFRG_MIXED_TC):
            assert np.abs(outs[prec] - ref).max() < 1e-4 * np.abs(ref).max(), (T, prec)


def sparse_c4v_vertex(N, U, targets, a_set, b_set, seed):
    """A C4v-symmetric vertex whose Sigma weight V(k_j, a, b) is nonzero for
    the targets j only on a_set x b_set (16 patch pairs of the 96^2): the
    oracle then sums those pairs alone, every GPU pair is still evaluated."""
    rng = np.random.default_rng(seed)
    V = np.zeros((N, N, N))
    for j in targets:
        for a in a_set:
            for b in b_set:
                V[j, a, b] = U * (1.0 + 0.5 * rng.uniform(-1, 1))
    V = inputs.c4v_symmetrise(V)
    # any (j, a, b) that C4v maps onto a target's support carries a value too;
    # the vertex stays sparse (zero elsewhere) and symmetric
    return V


def test_z_np96_flow_step_against_oracle(np96):
    """Z of one tensor-core flow step at np96_n32 (the bench's self-energy
    launch: 13 irreducible targets, mirror-line targets over half of the loop
    points, autotuned shapes) against the oracle on patch N/8 (a mirror line)
    and patch 5 (generic), for a C4v-symmetric vertex supported on 16 patch
    pairs per target (all M^2 pairs still run on the GPU; the oracle skips
    the pairs of zero weight, which add exactly nothing)."""
    N, n, U, o, Z0 = (np96[k] for k in ("N", "n", "U", "o", "Z"))
    T0 = 0.4
    targets = [N // 8, 5]
    # 60 U on the support: slopes 1 - 1/Z of a few per cent, as for a dense vertex
    V = sparse_c4v_vertex(N, 60.0 * U, targets, (3, 5, 20, 47), (0, 7, 12, 60), seed=5)
    ref = o.zfactor_targets(T0, V, Z0, targets)
    assert np.all(np.abs(1.0 - ref) > 1e-2)          # a slope well above the tolerance
    with api.Context(N, n, n, U=U, lambda0=T0, z_feedback=1, lambda_end=0.02, precision=api.QPFRG_MIXED_TC) as c:
        api.qpfrg_autotune(c.h, T0)
        img = bytearray(api.qpfrg_get_state(c.h))
        img[64:] = np.concatenate([V.ravel(), Z0]).tobytes()
        api.qpfrg_set_state(c.h, bytes(img))
        api.qpfrg_step(c.h, 1)
        Zg = zeros(N)
        api.qpfrg_read_state(c.h, None, Zg)
        Zg = host(Zg)
    assert np.abs(Zg[targets] - ref).max() < 1e-4
    # the C4v images carry the representative's Z
    for g in inputs.c4v_patch_maps(N):
        assert np.abs(Zg[g[targets]] - Zg[targets]).max() < 1e-12


def test_flow_np96_tc_against_fp64_to_half_scale():
    """np96_n32 flow with fixed anisotropic Z: the tensor-core flow and the FP64
    flow agree to 1e-4 (normwise) at the step half-way in ln T between T = 1
    and the divergence scale (the comparison point of the mixed tolerance)."""
    N, n, U = 96, 32, 2.5
    Z0 = inputs.z_profile(N, "aniso")

    def start(c):
        img = bytearray(api.qpfrg_get_state(c.h))
        img[64:] = np.concatenate([np.full(N ** 3, U), Z0]).tobytes()
        api.qpfrg_set_state(c.h, bytes(img))

    with api.Context(N, n, n, U=U, lambda0=1.0, lambda_end=0.02, precision=api.QPFRG_MIXED_TC) as c:
        start(c)
        r = api.qpfrg_flow(c.h).as_dict()
    assert r["status"] == "DIVERGED"
    k = int(round(0.5 * math.log(r["lambda_c"]) / STEP))
    states = {}
    for prec in (api.QPFRG_FP64, api.QPFRG_MIXED_TC):
        with api.Context(N, n, n, U=U, lambda0=1.0, lambda_end=0.02, precision=prec) as c:
            start(c)
            rr = api.qpfrg_step(c.h, k).as_dict()
            assert rr["steps"] == k and rr["status"] == "RUNNING"
            Vg = zeros(N ** 3)
            api.qpfrg_read_state(c.h, Vg, None)
            states[prec] = host(Vg)
    ref = states[api.QPFRG_FP64]
    assert np.abs(states[api.QPFRG_MIXED_TC] - ref).max() < 1e-4 * np.abs(ref).max()
    assert np.abs(ref).max() > 1.5 * U        # the comparison point lies inside the growth


# --------------------------------------------------------------------------- #
# np48_n16, np16_n8, np192_n32
# --------------------------------------------------------------------------- #
def test_flow_np48_n16_divergence_mixed_forms_against_fp64():
    """np48_n16 (U = 3): the divergence scale of the mixed and tensor-core
    flows within 0.5 % of the FP64 flow (Z = 1), and with Z feedback the mixed
    and tensor-core flows within 0.5 % of each other."""
    N, n, U = 48, 16, 3.0
    lc = {}
    for prec in (api.QPFRG_FP64, api.QPFRG_MIXED, api.QPFRG_MIXED_TC):
        with api.Context(N, n, n, U=U, lambda0=1.0, lambda_end=0.02, precision=prec) as c:
            r = api.qpfrg_flow(c.h).as_dict()
        assert r["status"] == "DIVERGED"
        lc[prec] = r["lambda_c"]
    for prec in (api.QPFRG_MIXED, api.QPFRG_MIXED_TC):
        assert lc[prec] == pytest.approx(lc[api.QPFRG_FP64], rel=5e-3)
    lz = {}
    for prec in (api.QPFRG_MIXED, api.QPFRG_MIXED_TC):
        with api.Context(N, n, n, U=U, lambda0=1.0, lambda_end=0.02, precision=prec, z_feedback=1) as c:
            r = api.qpfrg_flow(c.h).as_dict()
        assert r["status"] == "DIVERGED"
        lz[prec] = r["lambda_c"]
    assert lz[api.QPFRG_MIXED_TC] == pytest.approx(lz[api.QPFRG_MIXED], rel=5e-3)


def test_flow_np16_n8_fp64_complete_against_oracle():
    """np16_n8 at its own fine grid: the complete FP64 flow (U = 2, T = 1 to
    0.05, Z = 1) against the oracle's, vertex normwise 1e-10 at the end."""
    import torch
    N, n, U = 16, 8, 2.0
    o = Oracle(N, n, n)
    ref = o.flow(np.full((N, N, N), U), np.ones(N), 1.0, 0.05, STEP)
    with api.Context(N, n, n, U=U, lambda0=1.0, lambda_end=0.05, precision=api.QPFRG_FP64) as c:
        r = api.qpfrg_flow(c.h).as_dict()
        Vg = zeros(N ** 3)
        api.qpfrg_read_state(c.h, Vg, None)
        Vg = host(Vg).reshape(N, N, N)
    assert r["status"] == "REACHED_END" and ref["status"] == "REACHED_END"
    assert r["steps"] == ref["steps"] == 149
    assert np.abs(Vg - ref["V"]).max() < 1e-10 * np.abs(ref["V"]).max()


@pytest.mark.parametrize("prec,tol", [(api.QPFRG_FP64, 1e-10), (api.QPFRG_MIXED_TC, 1e-4)], ids=["fp64", "tc"])
def test_rhs_np192_sampled_triples_against_oracle(prec, tol):
    N, n, U, T = 192, 32, 2.0, 0.05
    o = Oracle(N, n, n)
    V = inputs.random_vertex(N, U, seed=3)
    Z = inputs.z_profile(N, "aniso")
    triples = sample_triples(N, 40, seed=11, extra=degenerate_triples(N))
    ref = oracle_triples(o, T, V, Z, triples)
    with api.Context(N, n, n, U=U, precision=prec) as c:
        out = zeros(N ** 3)
        api.qpfrg_rhs(c.h, T, dev(V), dev(Z), out)
        got = host(out).reshape(N, N, N)
    g = np.array([got[t] for t in triples])
    assert np.abs(g - ref).max() < tol * np.abs(ref).max()
