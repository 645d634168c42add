"""Tensor-core contraction (QPFRG_MIXED_TC: tcgen05 MMA on BF16 hi/lo split
operands, FP32 accumulation) against the FP64 oracle through the C ABI.
Tolerance: 1e-4 normwise, as for the other mixed-precision forms."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2005_00827_gb300 import api, inputs

pytestmark = pytest.mark.gpu
TC = api.QPFRG_MIXED_TC


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()


def gpu_rhs(ctx, lam, V, Z):
    import torch
    N = V.shape[0]
    dV = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    api.qpfrg_rhs(ctx.h, lam, dev(V), dev(Z), dV)
    torch.cuda.synchronize()
    return dV.cpu().numpy().reshape(N, N, N)


def normwise(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("case", [(16, 4, 4, 0, 7, 1), (24, 4, 6, 0, 7, 1), (16, 1, 1, 1, 7, 0), (16, 4, 4, 0, 1, 1),
                                  (16, 4, 4, 0, 2, 1), (16, 4, 4, 0, 4, 1), (36, 1, 1, 1, 7, 0), (20, 2, 4, 0, 7, 1),
                                  (16, 4, 4, 0, 7, 0), (24, 4, 6, 0, 7, 0), (20, 2, 4, 0, 2, 0)],
                         ids=["w16", "w24_ragged", "lat4", "pp_only", "cr_only", "d_only", "lat6", "w20_ragged_k",
                              "w16_asym", "w24_asym", "w20_cr_asym"])
def test_tc_rhs_matches_oracle(case):
    """Symmetric (V, Z) in wedge mode take the row orbits of the contraction
    (representative rows, expanded); the asymmetric vertices and the lattice
    take every row."""
    N, nt, nr, mode, ch, sym = case
    T = 0.25
    V = inputs.random_vertex(N, 2.0, seed=N + 3, c4v=bool(sym))
    Z = inputs.z_profile(N, "aniso") if mode == 0 else np.random.default_rng(1).uniform(0.8, 1.0, N)
    ref = Oracle(N, nt, nr, mode=mode, channels=ch).rhs(T, V, Z)
    with api.Context(N, nt, nr, U=2.0, mode=mode, precision=TC, channel_mask=ch) as ctx:
        got = gpu_rhs(ctx, T, V, Z)
        work = api.qpfrg_rhs_work(ctx.h)
    assert normwise(got, ref) < 1e-4
    if mode == 0:
        maps = inputs.c4v_patch_maps(N)
        reps = {min(g[x] * N + g[y] for g in maps) for x in range(N) for y in range(N)}
        assert (work["loop_evals"] == 2 * len(reps) * N * nt * nr) == bool(sym)
        assert work["contraction_rows"] == (len(reps) if sym else N * N)


def test_tc_rhs_full_size_sampled():
    N, n, T = 96, 32, 0.1
    V = inputs.random_vertex(N, 2.5, seed=1)
    Z = inputs.z_profile(N, "aniso")
    with api.Context(N, n, n, U=2.5, precision=TC) as ctx:
        got = gpu_rhs(ctx, T, V, Z)
    o = Oracle(N, n, n)
    rng = np.random.default_rng(6)
    trip = [tuple(rng.integers(0, N, 3)) for _ in range(10)] + [(0, 0, 0), (N - 1, 7, 48)]
    ref = np.array([o.rhs_triple(T, V, Z, *t).sum() for t in trip])
    g = np.array([got[t] for t in trip])
    assert np.abs(g - ref).max() / np.abs(got).max() < 1e-4


def test_tc_flow_divergence_scale():
    import math
    N, n, U = 16, 4, 3.0
    ref = Oracle(N, n, n).flow(np.full((N, N, N), U), np.ones(N), 1.0, 0.01, math.log(0.98))
    with api.Context(N, n, n, U=U, precision=TC, lambda_end=0.01) as ctx:
        r = api.qpfrg_flow(ctx.h).as_dict()
    assert r["status"] == "DIVERGED" and abs(r["steps"] - ref["steps"]) <= 1
    assert r["lambda_c"] == pytest.approx(ref["lambda_c"], rel=5e-3)
