"""GPU parity of the one-loop right-hand side against the FP64 oracle, through
the C ABI (qpfrg_rhs).  Tolerances (normwise, max|diff| / max|ref|): FP64
path 1e-10; mixed path (FP32 loop kernels and contraction) 1e-4."""
import numpy as np
import pytest

from oracle.oracle import MODE_LATTICE, Oracle
from paper_2005_00827_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL = {api.QPFRG_FP64: 1e-10, api.QPFRG_MIXED: 1e-4}


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


CASES = [
    # (N, n_theta, n_r, mode, regulator, propagator, channels, lam, Zkind)
    (16, 8, 8, 0, 0, 0, 7, 0.3, "aniso"),         # np16_n8 workload shape
    (24, 4, 6, 0, 0, 0, 7, 0.05, "aniso"),        # ragged contraction tiles, low T
    (16, 4, 4, 0, 0, 1, 7, 0.2, "aniso"),         # Z in the pole
    (16, 4, 4, 0, 1, 0, 7, 0.8, "aniso"),         # interaction flow
    (16, 4, 4, 0, 0, 0, 3, 0.4, "one"),           # no direct channel
    (16, 4, 4, 0, 0, 0, 4, 0.4, "one"),           # direct only
    (16, 1, 1, 1, 0, 0, 7, 0.25, "aniso"),        # lattice L = 4
    (36, 1, 1, 1, 0, 0, 7, 0.3, "aniso"),         # lattice L = 6, ragged tiles
    (12, 3, 2, 0, 0, 0, 7, 0.5, "one"),           # odd angular count, tiny grid
]


@pytest.mark.parametrize("prec", [api.QPFRG_FP64, api.QPFRG_MIXED])
@pytest.mark.parametrize("case", CASES, ids=[f"N{c[0]}_n{c[1]}x{c[2]}_m{c[3]}_r{c[4]}_p{c[5]}_c{c[6]}" for c in CASES])
def test_rhs_matches_oracle(case, prec):
    N, nt, nr, mode, reg, prop, ch, lam, zk = case
    Tfix = 0.15
    o = Oracle(N, nt, nr, mode=mode, regulator=reg, prop_mode=prop, channels=ch, T_fixed=Tfix)
    V = inputs.random_vertex(N, 2.0, seed=N + nt, c4v=(mode == 0))
    Z = inputs.z_profile(N, zk) if mode == 0 else np.random.default_rng(3).uniform(0.8, 1.0, N)
    ref = o.rhs(lam, V, Z)
    opts = dict(precision=prec, propagator=prop, channel_mask=ch, T_fixed=Tfix)
    if reg == 1:
        opts.update(step=0.01, lambda_end=1.0)
    with api.Context(N, nt, nr, U=2.0, lambda0=0.0 if reg == 1 else 1.0, mode=mode, regulator=reg,
                     **opts) as ctx:
        got = gpu_rhs(ctx, lam, V, Z)
    assert normwise(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [api.QPFRG_FP64, api.QPFRG_MIXED, api.QPFRG_MIXED_TC])
def test_rhs_matches_oracle_next_nearest_hopping(prec):
    """t' = -0.2, mu = -0.3 (no nesting): the general line energy of the loop
    kernels (the t' = 0 lattice takes a compile-time specialisation)."""
    N, nt, nr, lam = 16, 4, 4, 0.3
    o = Oracle(N, nt, nr, tp=-0.2, mu=-0.3)
    V = inputs.random_vertex(N, 2.0, seed=21, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    ref = o.rhs(lam, V, Z)
    with api.Context(N, nt, nr, U=2.0, tp=-0.2, mu=-0.3, precision=prec) as ctx:
        got = gpu_rhs(ctx, lam, V, Z)
    assert normwise(got, ref) < (1e-10 if prec == api.QPFRG_FP64 else 1e-4)


def test_geometry_matches_oracle():
    o = Oracle(48, 16, 16)
    kf, fk, fw, fp = o.geometry()
    with api.Context(48, 16, 16) as ctx:
        gkf, fine = api.qpfrg_geometry(ctx.h)
    # same formulas on both sides; compilers may round a few ulp differently
    assert np.abs(gkf - kf).max() < 4e-15
    assert np.abs(fine[:, :2] - fk).max() < 4e-15
    assert np.abs(fine[:, 2] - fw).max() / fw.max() < 1e-14
    assert np.array_equal(fine[:, 3].astype(int), fp)


@pytest.mark.parametrize("prec", [api.QPFRG_FP64, api.QPFRG_MIXED])
def test_rhs_full_size_sampled(prec):
    """N = 96, 32 x 32 fine grid per patch (the np96_n32 workload), Z anisotropic:
    the whole RHS on the GPU, sampled output triples from the oracle."""
    N, n, T = 96, 32, 0.1
    V = inputs.random_vertex(N, 2.5, seed=1)
    Z = inputs.z_profile(N, "aniso")
    with api.Context(N, n, n, U=2.5, precision=prec) as ctx:
        got = gpu_rhs(ctx, T, V, Z)
    o = Oracle(N, n, n)
    rng = np.random.default_rng(5)
    trip = [tuple(rng.integers(0, N, 3)) for _ in range(12)] + [(0, 0, 0), (0, N // 2, N // 2), (N - 1, 5, 48)]
    ref = np.array([o.rhs_triple(T, V, Z, *t).sum() for t in trip])
    g = np.array([got[t] for t in trip])
    scale = np.abs(got).max()
    assert np.abs(g - ref).max() / scale < TOL[prec]
    # C4v covariance of the whole GPU output (V and Z are C4v symmetric)
    for gmap in inputs.c4v_patch_maps(N)[1:3]:
        assert np.abs(got[np.ix_(gmap, gmap, gmap)] - got).max() / scale < 10 * TOL[prec]


SYM_CASES = [
    # (N, n_theta, n_r, regulator, propagator, lam)
    (16, 4, 4, 0, 0, 0.3),
    (24, 4, 6, 0, 1, 0.05),      # quasi-particle lines with a C4v-symmetric Z
    (12, 3, 2, 0, 0, 0.5),       # odd angular count: points on the wedge centre lines
    (16, 4, 4, 1, 0, 0.8),       # interaction flow
    (48, 8, 8, 0, 0, 0.1),
]


@pytest.mark.parametrize("prec", [api.QPFRG_FP64, api.QPFRG_MIXED, api.QPFRG_MIXED_TC])
@pytest.mark.parametrize("case", SYM_CASES, ids=[f"N{c[0]}_n{c[1]}x{c[2]}_r{c[3]}_p{c[4]}" for c in SYM_CASES])
def test_loop_symmetry_matches_unreduced(case, prec):
    """The C4v-reduced loop kernels (one row per orbit of (transfer, patch),
    written to its images) give the results of the unreduced launch: to
    rounding in FP64, to FP32 rounding of the image points' coordinates
    otherwise.  Checked on qpfrg_rhs and on one flow step from a symmetric
    (V, Z) state (the path that reduces with quasi-particle lines, whose loop
    kernels depend on Z); the work report says how many evaluations the
    reduced RHS does.  With tensor cores the symmetric state also takes the
    row orbits of the contraction (one output row per orbit of transfer pairs,
    expanded); no_loop_symmetry = 2 keeps the loop-kernel orbits only."""
    import torch
    N, nt, nr, reg, prop, lam = case
    tc = prec == api.QPFRG_MIXED_TC
    if tc and (N * N) % 8:
        pytest.skip("tensor-core path needs N^2 % 8 == 0")
    V = inputs.random_vertex(N, 2.0, seed=N + 1, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    out, step, work = {}, {}, {}
    for nosym in ((0, 1, 2) if tc else (0, 1)):
        opts = dict(precision=prec, propagator=prop, T_fixed=0.15, no_loop_symmetry=nosym)
        lam0 = 0.0 if reg == 1 else 1.0
        if reg == 1:
            opts.update(step=0.01, lambda_end=1.0)
        with api.Context(N, nt, nr, U=2.0, lambda0=lam0, regulator=reg, **opts) as ctx:
            out[nosym] = gpu_rhs(ctx, lam, V, Z)
            img = bytearray(api.qpfrg_get_state(ctx.h))
            img[64:] = np.concatenate([V.ravel(), Z]).tobytes()
            api.qpfrg_set_state(ctx.h, bytes(img))
            api.qpfrg_step(ctx.h, 1)
            Vs = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
            api.qpfrg_read_state(ctx.h, Vs, None)
            torch.cuda.synchronize()
            step[nosym] = Vs.cpu().numpy() - V.ravel()
            work[nosym] = api.qpfrg_rhs_work(ctx.h)
    tol = 1e-12 if prec == api.QPFRG_FP64 else 1e-5
    for k in out:
        assert normwise(out[k], out[1]) < tol
        assert normwise(step[k], step[1]) < tol
    full = 2 * N * N * N * nt * nr
    assert work[1]["loop_evals"] == full and work[0]["loop_evals_full"] == full
    if nt % 2 == 0:
        assert work[0]["rows_unreduced"] == 0
        assert work[0]["loop_evals"] < full / 6
        if tc:
            # row orbits: every patch of each representative transfer pair
            maps = inputs.c4v_patch_maps(N)
            reps = {min(g[x] * N + g[y] for g in maps) for x in range(N) for y in range(N)}
            assert work[0]["loop_evals"] == 2 * len(reps) * N * nt * nr
            assert work[2]["loop_evals"] < full / 6 and work[2]["loop_evals"] != work[0]["loop_evals"]
