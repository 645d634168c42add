"""GPU parity of the self-energy / Z and of the RK4 flow against the FP64
oracle, plus checkpoint/resume and host-side failure detection, through the
C ABI.  Tolerances: Z absolute 1e-10 (FP64) / 1e-4 (mixed); vertex normwise
1e-10 / 1e-4; divergence scale relative 1e-9 / 5e-3."""
import math

import numpy as np
import pytest

from oracle.oracle import MODE_LATTICE, Oracle
from paper_2005_00827_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()


def zeros(n):
    import torch
    return torch.zeros(n, dtype=torch.float64, device="cuda")


def gpu_z(ctx, T, V, Z):
    import torch
    out = zeros(len(Z))
    api.qpfrg_selfenergy(ctx.h, T, dev(V), dev(Z), None, None, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [(api.QPFRG_FP64, 1e-10), (api.QPFRG_MIXED, 1e-4)])
@pytest.mark.parametrize("geo", [(16, 4, 4, 0, 0), (16, 1, 1, 1, 0), (16, 4, 6, 0, 1)],
                         ids=["wedge", "lattice", "wedge_qp"])
def test_z_matches_oracle(geo, prec, tol):
    N, nt, nr, mode, prop = geo
    T = 0.2
    o = Oracle(N, nt, nr, mode=mode, eta=0.02, prop_mode=prop)
    V = inputs.random_vertex(N, 2.0, seed=4, c4v=(mode == 0))
    Z = inputs.z_profile(N, "aniso") if mode == 0 else np.random.default_rng(2).uniform(0.85, 1.0, N)
    ref = o.zfactor(T, V, Z)
    with api.Context(N, nt, nr, U=2.0, mode=mode, precision=prec, propagator=prop) as ctx:
        got = gpu_z(ctx, T, V, Z)
    assert np.abs(got - ref).max() < tol


@pytest.mark.parametrize("case", [
    dict(N=16, nt=4, nr=4, tp=-0.2, mu=-0.3, prop=1),   # t' != 0 line energies, QP lines
    dict(N=8, nt=34, nr=32, tp=0.0, mu=0.0, prop=0),    # P = 1088 loop points: two record passes
    dict(N=48, nt=4, nr=4, tp=0.0, mu=0.0, prop=1),     # 48 wedges, ragged last block of q
    dict(N=8, nt=32, nr=32, tp=-0.2, mu=-0.3, prop=1),  # 1024 points per patch: per-patch weight table
], ids=["tp_mu_qp", "two_passes", "np48", "p1024_tp"])
def test_z_mixed_wedge_cases(case):
    """Mixed-precision Z (table-driven wedge projection) against the oracle."""
    N, nt, nr = case["N"], case["nt"], case["nr"]
    T = 0.2
    o = Oracle(N, nt, nr, tp=case["tp"], mu=case["mu"], eta=0.02, prop_mode=case["prop"])
    V = inputs.random_vertex(N, 2.0, seed=5, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    ref = o.zfactor(T, V, Z)
    with api.Context(N, nt, nr, U=2.0, tp=case["tp"], mu=case["mu"], precision=api.QPFRG_MIXED,
                     propagator=case["prop"]) as ctx:
        got = gpu_z(ctx, T, V, Z)
    assert np.abs(got - ref).max() < 1e-4


@pytest.mark.parametrize("prec,sym", [(api.QPFRG_FP64, True), (api.QPFRG_MIXED, True), (api.QPFRG_MIXED, False)],
                         ids=["fp64", "mixed-c4v", "mixed-asym"])
def test_sigma_grid_matches_exact_pole_sum(prec, sym):
    """Sigma on the frequency grid against the exact pole sum.  In mixed
    precision a C4v-symmetric (V, Z) is evaluated on the irreducible patches
    (the mirror-line ones over half of the loop points) and copied to the
    others; an asymmetric vertex takes every patch."""
    import torch
    N, n, T, nw = 16, 4, 0.15, 64
    o = Oracle(N, n, n, eta=0.05)
    V = inputs.random_vertex(N, 2.0, seed=8, c4v=sym)
    Z = inputs.z_profile(N, "aniso")
    w = np.linspace(-4.0, 4.0, nw)
    with api.Context(N, n, n, U=2.0, precision=prec, eta=0.05, n_omega=nw, omega_min=-4.0,
                     omega_max=4.0) as ctx:
        re, im = zeros(N * nw), zeros(N * nw)
        api.qpfrg_selfenergy(ctx.h, T, dev(V), dev(Z), re, im, None)
        torch.cuda.synchronize()
        got = (re.cpu().numpy() + 1j * im.cpu().numpy()).reshape(N, nw)
    for j in (0, 3, 5, 8, 13):
        ref = o.sigma(T, V, Z, j, w)
        assert np.abs(got[j] - ref).max() / np.abs(ref).max() < 1e-4
        assert np.all(got[j].imag <= 1e-12)


def test_sigma_grid_qp_p512_matches_exact_pole_sum():
    """Frequency grid in mixed precision with quasi-particle lines, t' and mu
    nonzero and 512 points per patch (the per-patch weight table of the
    shared-memory histogram kernel)."""
    import torch
    N, nt, nr, T, nw = 8, 32, 16, 0.2, 48
    o = Oracle(N, nt, nr, tp=-0.2, mu=-0.3, prop_mode=1, eta=0.05)
    V = inputs.random_vertex(N, 2.0, seed=13, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    w = np.linspace(-3.0, 3.0, nw)
    with api.Context(N, nt, nr, U=2.0, tp=-0.2, mu=-0.3, precision=api.QPFRG_MIXED, propagator=1, eta=0.05,
                     n_omega=nw, omega_min=-3.0, omega_max=3.0) as ctx:
        re, im = zeros(N * nw), zeros(N * nw)
        api.qpfrg_selfenergy(ctx.h, T, dev(V), dev(Z), re, im, None)
        torch.cuda.synchronize()
        got = (re.cpu().numpy() + 1j * im.cpu().numpy()).reshape(N, nw)
    for j in (0, 3):
        ref = o.sigma(T, V, Z, j, w)
        assert np.abs(got[j] - ref).max() / np.abs(ref).max() < 1e-4


def run_oracle_flow(o, U, T0, T_end, z_feedback, steps=None):
    N = o.N
    return o.flow(np.full((N, N, N), U), np.ones(N), T0, T_end, math.log(0.98), stop_abs_v=20.0,
                  z_feedback=z_feedback, max_steps=steps or 100000)


@pytest.mark.parametrize("prec", [api.QPFRG_FP64, api.QPFRG_MIXED])
def test_flow_to_divergence_matches_oracle(prec):
    """np16-shaped T-flow (N=16, coarse 4x4 fine grid for oracle speed), U=3."""
    N, n, U = 16, 4, 3.0
    o = Oracle(N, n, n)
    ref = run_oracle_flow(o, U, 1.0, 0.01, False)
    assert ref["status"] == "DIVERGED"
    with api.Context(N, n, n, U=U, lambda0=1.0, precision=prec, lambda_end=0.01) as ctx:
        r = api.qpfrg_flow(ctx.h).as_dict()
    assert r["status"] == "DIVERGED" and r["steps"] == ref["steps"]
    rel = 1e-9 if prec == api.QPFRG_FP64 else 5e-3
    assert r["lambda_c"] == pytest.approx(ref["lambda_c"], rel=rel)


@pytest.mark.parametrize("prec,tol", [(api.QPFRG_FP64, 1e-10), (api.QPFRG_MIXED, 1e-4)])
def test_flow_with_z_feedback_trajectory(prec, tol):
    """Z feedback on: vertex and Z after a fixed number of steps."""
    import torch
    N, n, U, steps = 16, 4, 2.0, 12
    o = Oracle(N, n, n, eta=0.02)
    ref = run_oracle_flow(o, U, 1.0, 0.02, True, steps=steps)
    with api.Context(N, n, n, U=U, lambda0=1.0, precision=prec, lambda_end=0.02, z_feedback=1) as ctx:
        r = api.qpfrg_step(ctx.h, steps).as_dict()
        V, Z = zeros(N ** 3), zeros(N)
        api.qpfrg_read_state(ctx.h, V, Z)
        torch.cuda.synchronize()
    assert r["steps"] == steps and r["lam"] == pytest.approx(ref["lam"], rel=1e-13)
    Vg = V.cpu().numpy().reshape(N, N, N)
    assert np.abs(Vg - ref["V"]).max() / np.abs(ref["V"]).max() < tol
    assert np.abs(Z.cpu().numpy() - ref["Z"]).max() < tol
    assert np.all(ref["Z"] > 0.0)


def test_flow_z_full_size_matches_all_targets():
    """np96_n32, the bench workload, in its launch configuration (MIXED_TC,
    autotuned shapes): Z from the flow's self-energy (the 13 C4v-irreducible
    targets, mirror-line targets over half of the loop points) equals Z from
    all 96 targets evaluated independently (qpfrg_selfenergy).  The chord
    slope 1 - 1/Z is quadratic in the vertex, and doubling V is exact in
    floating point, so slope(2V) = 4 slope(V) to the reduction order."""
    import torch
    N, n, T0 = 96, 32, 0.7
    V = inputs.random_vertex(N, 2.5, seed=21, c4v=True)
    Z0 = inputs.z_profile(N, "aniso")
    with api.Context(N, n, n, U=2.5, lambda0=T0, z_feedback=1, lambda_end=0.05,
                     precision=api.QPFRG_MIXED_TC) as c:
        api.qpfrg_autotune(c.h, T0)
        img = bytearray(api.qpfrg_get_state(c.h))
        img[64:] = np.concatenate([V.ravel(), Z0]).tobytes()
        api.qpfrg_set_state(c.h, bytes(img))
        api.qpfrg_step(c.h, 1)
        Zflow = zeros(N)
        api.qpfrg_read_state(c.h, None, Zflow)
        torch.cuda.synchronize()
        Zall = gpu_z(c, T0, V, Z0)
        Z2 = gpu_z(c, T0, 2.0 * V, Z0)
    Zflow = Zflow.cpu().numpy()
    assert np.all(np.isfinite(Zall)) and np.all(np.isfinite(Zflow))
    assert np.abs(Zflow - Zall).max() < 1e-4
    s1, s2 = 1.0 - 1.0 / Zall, 1.0 - 1.0 / Z2
    assert np.abs(s2 - 4.0 * s1).max() < 1e-9 * np.abs(4.0 * s1).max()


@pytest.mark.parametrize("symmetric,prec,N,n", [
    (True, api.QPFRG_FP64, 16, 4), (False, api.QPFRG_FP64, 16, 4),
    (True, api.QPFRG_MIXED, 16, 4),     # irreducible targets, mirror halving of targets 0 and N/8
    (True, api.QPFRG_MIXED, 8, 32),     # the same with 1024 points per patch (per-patch weight table)
    (False, api.QPFRG_MIXED, 8, 32),    # all targets, per-patch weight table
], ids=["sym-fp64", "asym-fp64", "sym-mixed", "sym-mixed-p1024", "asym-mixed-p1024"])
def test_z_feedback_after_set_state(symmetric, prec, N, n):
    """The flow evaluates Sigma only on the C4v-irreducible patches while the
    state is symmetric (mixed precision; the two targets on mirror lines sum
    over half of the loop points); a state image without the symmetry
    switches back to all patches.  Either way Z must equal the oracle's on
    every patch."""
    import torch
    U, T0 = 2.0, 0.7
    V = inputs.random_vertex(N, U, seed=12, c4v=symmetric)
    Z0 = inputs.z_profile(N, "aniso") if symmetric else np.random.default_rng(4).uniform(0.9, 1.0, N)
    ref = Oracle(N, n, n, eta=0.02).zfactor(T0, V, Z0)
    with api.Context(N, n, n, U=U, lambda0=T0, z_feedback=1, lambda_end=0.05, precision=prec) as c:
        img = bytearray(api.qpfrg_get_state(c.h))
        img[64:] = np.concatenate([V.ravel(), Z0]).tobytes()
        api.qpfrg_set_state(c.h, bytes(img))
        api.qpfrg_step(c.h, 1)
        Zt = zeros(N)
        api.qpfrg_read_state(c.h, None, Zt)
        torch.cuda.synchronize()
    tol = 1e-10 if prec == api.QPFRG_FP64 else 1e-4
    assert np.abs(Zt.cpu().numpy() - ref).max() < tol


def test_checkpoint_resume():
    N, n, U = 16, 4, 2.5
    with api.Context(N, n, n, U=U, lambda_end=0.05) as a:
        api.qpfrg_step(a.h, 6)
        img = api.qpfrg_get_state(a.h)
        ra = api.qpfrg_step(a.h, 5).as_dict()
        full = api.qpfrg_get_state(a.h)
    with api.Context(N, n, n, U=U, lambda_end=0.05) as b:
        api.qpfrg_set_state(b.h, img)
        rb = api.qpfrg_step(b.h, 5).as_dict()
        resumed = api.qpfrg_get_state(b.h)
    assert ra["steps"] == rb["steps"] == 11 and ra["lam"] == rb["lam"]
    va = np.frombuffer(full[64:], dtype=np.float64)
    vb = np.frombuffer(resumed[64:], dtype=np.float64)
    assert np.abs(va - vb).max() / np.abs(va).max() < 1e-13


def test_state_round_trip_through_pinned_buffer():
    """qpfrg_get_state_into / qpfrg_set_state_from with a page-locked buffer
    write and read the same image as the bytes interface."""
    import torch
    N, n = 16, 4
    with api.Context(N, n, n, U=2.5, lambda_end=0.05) as c:
        api.qpfrg_step(c.h, 3)
        ref = api.qpfrg_get_state(c.h)
        buf = torch.empty(api.qpfrg_state_size(c.h), dtype=torch.uint8, pin_memory=True)
        api.qpfrg_get_state_into(c.h, buf)
        assert bytes(buf.numpy()) == ref
        api.qpfrg_step(c.h, 2)
        api.qpfrg_set_state_from(c.h, buf)
        assert api.qpfrg_get_state(c.h) == ref
        assert api.qpfrg_step(c.h, 1).as_dict()["steps"] == 4


def test_failure_detection_host_side(monkeypatch):
    N, n = 16, 4
    with api.Context(N, n, n, U=2.0) as c:
        img = bytearray(api.qpfrg_get_state(c.h))
        bad = np.frombuffer(img, dtype=np.float64, offset=64).copy()
        bad[17] = np.nan
        img[64:] = bad.tobytes()
        with pytest.raises(api.QpfrgError) as ei:
            api.qpfrg_set_state(c.h, bytes(img))
        assert ei.value.status == api.QPFRG_ERR_NONFINITE
        with pytest.raises(api.QpfrgError) as ei:
            api.qpfrg_set_state(c.h, bytes(img[:-8]))
        assert ei.value.status == api.QPFRG_ERR_INVALID
        # state untouched by the rejected images
        r = api.qpfrg_step(c.h, 1).as_dict()
        assert r["status"] == "RUNNING" and np.isfinite(r["max_abs_v"])
    # wall-clock budget
    with api.Context(N, n, n, U=2.0, timeout_s=1e-9) as c:
        api.qpfrg_step(c.h, 1)
        r = api.qpfrg_flow(c.h).as_dict()
        assert r["status"] == "TIMEOUT"
    # Z leaves (0, z_max]
    with api.Context(N, n, n, U=2.0, z_feedback=1, z_max=0.5) as c:
        r = api.qpfrg_flow(c.h).as_dict()
        assert r["status"] == "Z_OUT_OF_RANGE" and r["steps"] == 0
    # injected allocation failure
    monkeypatch.setenv("QPFRG_TEST_FAIL_ALLOC", "1")
    with pytest.raises(api.QpfrgError) as ei:
        api.Context(N, n, n, U=2.0)
    assert ei.value.status == api.QPFRG_ERR_OOM


def test_invalid_arguments_rejected():
    with pytest.raises(api.QpfrgError) as ei:
        api.Context(18, 4, 4)
    assert ei.value.status == api.QPFRG_ERR_INVALID
    with pytest.raises(api.QpfrgError) as ei:
        api.Context(16, 4, 3)
    assert ei.value.status == api.QPFRG_ERR_INVALID
    with pytest.raises(api.QpfrgError) as ei:
        api.Context(16, 64, 64)
    assert ei.value.status == api.QPFRG_ERR_UNSUPPORTED
    with api.Context(16, 4, 4) as c:
        with pytest.raises(api.QpfrgError):
            api.qpfrg_rhs(c.h, -1.0, 1, None, 2)


def test_profiler_counts_launches():
    with api.Context(16, 4, 4, U=2.0) as c:
        api.qpfrg_set_profiling(c.h, True)
        api.qpfrg_step(c.h, 2)
        prof = api.qpfrg_profile(c.h)
    assert prof["bubble"][1] == 8 and prof["contract_pp"][1] == 8 and prof["rk_final"][1] == 2
    assert prof["bubble"][0] > 0


def test_sigma_table_holds_the_fp64_projection():
    """The self-energy's patch-of-r table (built by the first Z of a
    C4v-symmetric state): 40 000 sampled entries against the oracle's FP64
    projection of r = (k_j + p) - q (a byte N stands for patch 0), with the context's own exported
    geometry; and Z with the table against Z decided per pair (1e-6: the
    FP64 atomics of the CTA sums add in a run-dependent order)."""
    import torch
    N, n = 48, 16
    o = Oracle(N, n, n)
    res = []
    for table in (0, -1):
        with api.Context(N, n, n, U=3.0, lambda0=1.0, precision=api.QPFRG_MIXED, lambda_end=0.05, z_feedback=1,
                         sigma_table=table) as c:
            api.qpfrg_step(c.h, 2)
            Z = zeros(N)
            api.qpfrg_read_state(c.h, None, Z)
            torch.cuda.synchronize()
            size, _ = api.qpfrg_sigma_table(c.h)
            if table == 0:
                kf, fine = api.qpfrg_geometry(c.h)
                M, P, nirr = len(fine), n * n, N // 8 + 1
                assert size == nirr * N * M * P
                rng = np.random.default_rng(17)
                idx = np.sort(rng.integers(0, size, 40000))
                got = np.array([api.qpfrg_sigma_table(c.h, int(x), 1)[1][0] for x in idx])
            else:
                assert size == 0
        res.append(Z.cpu().numpy())
    assert np.abs(res[0] - res[1]).max() < 1e-6
    bad = 0
    for x, g in zip(idx, got):
        # byte (((j N + a) P/8 + i/8) M + iq) 8 + i % 8
        word, i8 = divmod(int(x), 8)
        grp, iq = divmod(word, M)
        i = (grp % (P // 8)) * 8 + i8
        a = (grp // (P // 8)) % N
        j = grp // ((P // 8) * N)
        b, t = divmod(iq, P)
        q = b * P + (t % n) * n + t // n
        p = a * P + i
        rx = (kf[j, 0] + fine[p, 0]) - fine[q, 0]
        ry = (kf[j, 1] + fine[p, 1]) - fine[q, 1]
        # a byte N is the kernel's second slot of patch 0 (past the last ray)
        bad += int(o.proj(rx, ry) != int(g) % N)
    assert bad == 0
