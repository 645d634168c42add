"""GPU parity of the interaction flow with the self-energy ODE (App.
A.2-A.5, Eq. (nutshell_2); options.sigma_ode) against the oracle, through
the C ABI: the vertex, the chord slopes of Sigma and Sigma', Z, K, A and
Sigma on the frequency grid after a few steps, for the feedback variants
(none, patch average with the Katanin factor, minimum of A, one-loop term
dropped); and the divergence scale with feedback and the Katanin factor.
Tolerances: FP64 1e-10 (vertex normwise, slopes and Z/K/A absolute), mixed
and tensor-core 1e-4; the binned frequency grid 1e-4 of max|Sigma|;
divergence scale relative 1e-9 (FP64) and 0.5 %."""
import numpy as np
import pytest

from oracle.oracle import A_AVG, A_DROP, A_MIN, REG_INTERACTION, Oracle
from paper_2005_00827_gb300 import api

pytestmark = pytest.mark.gpu

T, ETA = 0.3, 0.05


def zeros(n):
    import torch
    return torch.zeros(n, dtype=torch.float64, device="cuda")


VARIANTS = [
    dict(z_feedback=0, katanin=0, a_mode=A_AVG),
    dict(z_feedback=1, katanin=1, a_mode=A_AVG),
    dict(z_feedback=1, katanin=0, a_mode=A_MIN),
    dict(z_feedback=1, katanin=1, a_mode=A_DROP),
]


@pytest.mark.parametrize("prec", [api.QPFRG_FP64, api.QPFRG_MIXED, api.QPFRG_MIXED_TC], ids=["fp64", "mixed", "tc"])
@pytest.mark.parametrize("var", VARIANTS, ids=["nofeedback", "avg-katanin", "min", "drop-katanin"])
def test_sigma_ode_flow_matches_oracle(var, prec):
    import torch
    N, n, U, dg, steps, nw = 8, 4, 2.5, 0.1, 6, 9
    w = np.linspace(-2.0, 2.0, nw)
    o = Oracle(N, n, n, regulator=REG_INTERACTION, T_fixed=T, eta=ETA)
    ref = o.gflow(U, g_end=dg * steps, dg=dg, omega=w, **var)
    Zr, Kr, Ar, Abr = o.gflow_zka(dg * steps, ref["S"], ref["D"], omega=w, **var)
    with api.Context(N, n, n, U=U, lambda0=0.0, regulator=api.QPFRG_REG_INTERACTION, T_fixed=T, eta=ETA,
                     step=dg, lambda_end=1.0, sigma_ode=1, precision=prec, n_omega=nw, omega_min=-2.0,
                     omega_max=2.0, **var) as c:
        r = api.qpfrg_step(c.h, steps).as_dict()
        V, sl, sg, zka = zeros(N ** 3), zeros(2 * N), zeros(4 * N * nw), zeros(3 * N + 1)
        api.qpfrg_read_state(c.h, V, None)
        api.qpfrg_read_sigma_flow(c.h, sl, sg, zka)
        torch.cuda.synchronize()
        V, sl, sg, zka = (x.cpu().numpy() for x in (V, sl, sg, zka))
    assert r["steps"] == steps and r["lam"] == pytest.approx(dg * steps, rel=1e-13)
    tol = 1e-10 if prec == api.QPFRG_FP64 else 1e-4
    assert np.abs(V.reshape(N, N, N) - ref["V"]).max() < tol * np.abs(ref["V"]).max()
    s1 = (ref["S"][:, 0].real - ref["S"][:, 1].real) / (4 * T)
    s2 = (ref["D"][:, 0].real - ref["D"][:, 1].real) / (4 * T)
    scale = max(np.abs(s1).max(), np.abs(s2).max())
    assert np.abs(sl[:N] - s1).max() < tol * scale and np.abs(sl[N:] - s2).max() < tol * scale
    for got, want in ((zka[:N], Zr), (zka[N:2 * N], Kr), (zka[2 * N:3 * N], Ar)):
        assert np.abs(got - want).max() < tol
    assert zka[3 * N] == pytest.approx(Abr, abs=tol)
    sg = sg.reshape(4, N, nw)
    Sg, Dg = sg[0] + 1j * sg[1], sg[2] + 1j * sg[3]
    for got, want in ((Sg, ref["S"][:, 2:]), (Dg, ref["D"][:, 2:])):
        assert np.abs(got - want).max() < 1e-4 * np.abs(want).max()


@pytest.mark.parametrize("prec,rel", [(api.QPFRG_FP64, 1e-9), (api.QPFRG_MIXED, 5e-3), (api.QPFRG_MIXED_TC, 5e-3)],
                         ids=["fp64", "mixed", "tc"])
def test_sigma_ode_divergence_with_katanin(prec, rel):
    """Flow to strong coupling (max|V| > 20) with Z feedback and the Katanin
    factor, N = 16, T = 0.1: the divergence scale g_c (U* = g_c^2 U, Sec.
    3.2) against the oracle, and above the one of the flow without feedback.
    In tensor-core precision the symmetric state takes the contraction's row
    orbits, with the Katanin factors in the loop-kernel weights."""
    N, n, U, dg = 16, 4, 2.0, 0.1
    o = Oracle(N, n, n, regulator=REG_INTERACTION, T_fixed=0.1, eta=ETA)
    ref = o.gflow(U, g_end=3.0, dg=dg, z_feedback=True, katanin=True)
    ref0 = o.gflow(U, g_end=3.0, dg=dg, z_feedback=False)
    assert ref["status"] == "DIVERGED" and ref["g_c"] > ref0["g_c"]
    with api.Context(N, n, n, U=U, lambda0=0.0, regulator=api.QPFRG_REG_INTERACTION, T_fixed=0.1, eta=ETA,
                     step=dg, lambda_end=3.0, sigma_ode=1, z_feedback=1, katanin=1, precision=prec) as c:
        r = api.qpfrg_flow(c.h).as_dict()
    assert r["status"] == "DIVERGED"
    assert r["lambda_c"] == pytest.approx(ref["g_c"], rel=rel)


def test_sigma_ode_checkpoint_resume():
    """The state image carries (V, Z, s1, s2, Sigma, Sigma'): a flow resumed
    from it continues as the uninterrupted one."""
    N, n = 8, 4
    kw = dict(U=2.5, lambda0=0.0, regulator=api.QPFRG_REG_INTERACTION, T_fixed=T, eta=ETA, step=0.1,
              lambda_end=2.0, sigma_ode=1, z_feedback=1, katanin=1, n_omega=5, omega_min=-1.0, omega_max=1.0)
    with api.Context(N, n, n, **kw) as a:
        api.qpfrg_step(a.h, 3)
        img = api.qpfrg_get_state(a.h)
        api.qpfrg_step(a.h, 2)
        full = api.qpfrg_get_state(a.h)
    with api.Context(N, n, n, **kw) as b:
        api.qpfrg_set_state(b.h, img)
        api.qpfrg_step(b.h, 2)
        resumed = api.qpfrg_get_state(b.h)
    va = np.frombuffer(full[64:], dtype=np.float64)
    vb = np.frombuffer(resumed[64:], dtype=np.float64)
    assert va.shape == vb.shape == (N ** 3 + N + 2 * N + 4 * N * 5,)
    assert np.abs(va - vb).max() < 1e-13 * np.abs(va).max()
