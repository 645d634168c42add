"""Energy-shell patching (QPFRG_GRID_SHELL; Sec. 3.2: 32 angular sections x 7
energy shells = 224 patches) on the GPU against the FP64 oracle, through the
C ABI: the exported geometry, the right-hand side in every precision, Z of
every patch (chord about its own xi_j), a Z-feedback temperature flow and an
interaction flow with the self-energy ODE and the Katanin factor.
Tolerances as for the angular patching: FP64 1e-10 (vertex normwise, Z
absolute), mixed and tensor-core 1e-4."""
import numpy as np
import pytest

from oracle.oracle import A_AVG, MODE_SHELL, REG_INTERACTION, Oracle
from paper_2005_00827_gb300 import api, inputs

pytestmark = pytest.mark.gpu
SHELL = api.QPFRG_GRID_SHELL


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()


def zeros(n):
    import torch
    return torch.zeros(n, dtype=torch.float64, device="cuda")


def ctx(Na, ns, nt, nr, **kw):
    return api.Context(Na * ns, nt, nr, mode=SHELL, n_shell=ns, **kw)


def orc(Na, ns, nt, nr, **kw):
    return Oracle(Na * ns, nt, nr, mode=MODE_SHELL, n_shell=ns, **kw)


def test_geometry_matches_oracle():
    Na, ns, nt, nr = 8, 5, 3, 4
    kf_o, fk_o, fw_o, fp_o = orc(Na, ns, nt, nr).geometry()
    with ctx(Na, ns, nt, nr) as c:
        kf, fine = api.qpfrg_geometry(c.h)
    assert np.abs(kf - kf_o).max() < 1e-13
    assert np.abs(fine[:, :2] - fk_o).max() < 1e-13
    assert np.abs(fine[:, 2] - fw_o).max() < 1e-16
    assert np.array_equal(fine[:, 3].astype(int), fp_o)


@pytest.mark.parametrize("prec,tol", [(api.QPFRG_FP64, 1e-10), (api.QPFRG_MIXED, 1e-4),
                                      (api.QPFRG_MIXED_TC, 1e-4)], ids=["fp64", "mixed", "tc"])
@pytest.mark.parametrize("shape", [(8, 3, 2, 4), (4, 5, 3, 4)], ids=["8x3", "4x5_ragged"])
def test_rhs_matches_oracle(shape, prec, tol):
    import torch
    Na, ns, nt, nr = shape
    N, T = Na * ns, 0.2
    V = inputs.random_vertex(N, 2.0, seed=N + 1, n_shell=ns)
    Z = inputs.z_profile(N, "aniso", n_shell=ns)
    ref = orc(Na, ns, nt, nr).rhs(T, V, Z)
    out = zeros(N ** 3)
    with ctx(Na, ns, nt, nr, U=2.0, precision=prec) as c:
        api.qpfrg_rhs(c.h, T, dev(V), dev(Z), out)
        torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(N, N, N)
    assert np.abs(got - ref).max() / np.abs(ref).max() < tol


def test_one_shell_equals_wedge_mode():
    """n_shell = 1 takes the FP64 partner maps and the generic self-energy
    kernel, wedge mode the fixed-point maps and the wedge kernels: the same
    right-hand side and Z."""
    import torch
    N, n, T = 16, 4, 0.2
    V = inputs.random_vertex(N, 2.0, seed=9)
    Z = inputs.z_profile(N, "aniso")
    res = []
    for mode in (api.QPFRG_GRID_WEDGE, SHELL):
        out, zo = zeros(N ** 3), zeros(N)
        with api.Context(N, n, n, U=2.0, mode=mode, n_shell=1, precision=api.QPFRG_FP64) as c:
            api.qpfrg_rhs(c.h, T, dev(V), dev(Z), out)
            api.qpfrg_selfenergy(c.h, T, dev(V), dev(Z), None, None, zo)
            torch.cuda.synchronize()
        res.append((out.cpu().numpy(), zo.cpu().numpy()))
    assert np.abs(res[0][0] - res[1][0]).max() <= 1e-13 * np.abs(res[0][0]).max()
    assert np.abs(res[0][1] - res[1][1]).max() < 1e-13


@pytest.mark.parametrize("prec,tol", [(api.QPFRG_FP64, 1e-10), (api.QPFRG_MIXED, 1e-4)], ids=["fp64", "mixed"])
def test_z_every_patch_matches_oracle(prec, tol):
    import torch
    Na, ns, nt, nr = 8, 3, 2, 4
    N, T = Na * ns, 0.2
    V = inputs.random_vertex(N, 2.0, seed=5, n_shell=ns)
    Z = inputs.z_profile(N, "aniso", n_shell=ns)
    ref = orc(Na, ns, nt, nr, eta=0.02).zfactor(T, V, Z)
    out = zeros(N)
    with ctx(Na, ns, nt, nr, U=2.0, precision=prec, eta=0.02) as c:
        api.qpfrg_selfenergy(c.h, T, dev(V), dev(Z), None, None, out)
        torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() < tol


@pytest.mark.parametrize("prec,tol", [(api.QPFRG_FP64, 1e-10), (api.QPFRG_MIXED, 1e-4),
                                      (api.QPFRG_MIXED_TC, 1e-4)], ids=["fp64", "mixed", "tc"])
def test_z_feedback_flow_matches_oracle(prec, tol):
    import math

    import torch
    Na, ns, nt, nr = 8, 3, 2, 4
    N, U, steps = Na * ns, 2.0, 8
    o = orc(Na, ns, nt, nr, eta=0.02)
    ref = o.flow(np.full((N, N, N), U), np.ones(N), 1.0, 0.05, math.log(0.98), z_feedback=True,
                 max_steps=steps)
    with ctx(Na, ns, nt, nr, U=U, lambda0=1.0, precision=prec, lambda_end=0.05, z_feedback=1, eta=0.02) as c:
        r = api.qpfrg_step(c.h, steps).as_dict()
        V, Z = zeros(N ** 3), zeros(N)
        api.qpfrg_read_state(c.h, V, Z)
        torch.cuda.synchronize()
    assert r["steps"] == steps
    Vg = V.cpu().numpy().reshape(N, N, N)
    assert np.abs(Vg - ref["V"]).max() / np.abs(ref["V"]).max() < tol
    assert np.abs(Z.cpu().numpy() - ref["Z"]).max() < tol


def test_gflow_katanin_matches_oracle():
    """Interaction flow with the self-energy ODE, Z feedback and the Katanin
    factor; A-bar averages over the Fermi shell."""
    import torch
    Na, ns, nt, nr = 4, 3, 2, 4
    N, U, dg, steps, T = Na * ns, 2.5, 0.1, 5, 0.3
    o = orc(Na, ns, nt, nr, regulator=REG_INTERACTION, T_fixed=T, eta=0.05)
    var = dict(z_feedback=1, katanin=1, a_mode=A_AVG)
    ref = o.gflow(U, g_end=dg * steps, dg=dg, **var)
    with ctx(Na, ns, nt, nr, U=U, lambda0=0.0, regulator=api.QPFRG_REG_INTERACTION, T_fixed=T, eta=0.05,
             step=dg, lambda_end=1.0, sigma_ode=1, precision=api.QPFRG_FP64, **var) as c:
        r = api.qpfrg_step(c.h, steps).as_dict()
        V = zeros(N ** 3)
        api.qpfrg_read_state(c.h, V, None)
        torch.cuda.synchronize()
    assert r["steps"] == steps
    assert np.abs(V.cpu().numpy().reshape(N, N, N) - ref["V"]).max() < 1e-10 * np.abs(ref["V"]).max()


def test_shell_parameters_rejected():
    with pytest.raises(api.QpfrgError):
        ctx(8, 2, 2, 4)                 # even shell count
    with pytest.raises(api.QpfrgError):
        api.Context(30, 2, 4, mode=SHELL, n_shell=3)   # 10 wedges
    with pytest.raises(api.QpfrgError):
        ctx(8, 3, 2, 4, tp=0.6)         # xi not monotone along the rays
