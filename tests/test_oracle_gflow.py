"""Pins of the oracle's interaction flow with the self-energy ODE (App.
A.2-A.5, Eq. (nutshell_2)): state (V, Sigma, Sigma') in g at fixed T.

* Frozen vertex, no feedback (Z = K = 1, A = 0): d^2 Sigma/dg^2 = 6 g T2 is
  exactly integrated by RK4 (Sigma_g = g^3 T2), so g Sigma_g at g = 1 equals
  the second-order self-energy of U (App. A.3: g Sigma_g is the self-energy
  of the bare coupling g^2 U), which orc_sigma computes and the SOPT pins of
  test_oracle_sigma fix.  A wrong prefactor or power of g fails it.
* With feedback: A_g = 2 (dZ/dg)/Z along the trajectory (Eq.
  (single_scale_derivative_Z)), dZ/dg from a Richardson-extrapolated central
  difference of Z between flows; A_g = -(2/g)(1 - Z K) (Eq. (A_g_simple)).
* g = 0: Sigma = Sigma' = 0, Z = K = 1, A = 0 (App. B).
* Without feedback the vertex part is the plain interaction flow.
* Weak coupling (App. A.4, App. B): the flows with A_min and A_max bracket the
  averaged flow's Sigma, and dropping the one-loop term changes Sigma by
  less than 1 %.
"""
import numpy as np
import pytest

from oracle.oracle import A_AVG, A_DROP, A_MAX, A_MIN, MODE_LATTICE, REG_INTERACTION, Oracle

N, n, T = 8, 4, 0.3


@pytest.fixture(scope="module")
def o():
    return Oracle(N, n, n, regulator=REG_INTERACTION, T_fixed=T, eta=0.05)


@pytest.mark.parametrize("dg", [0.25, 0.3])
def test_frozen_vertex_sigma_is_second_order(o, dg):
    U = 2.0
    w = np.linspace(-2.0, 2.0, 9)
    r = o.gflow(U, g_end=1.0, dg=dg, omega=w, z_feedback=False, freeze_vertex=True)
    assert r["status"] == "REACHED_END" and r["g"] == pytest.approx(1.0)
    V = np.full((N, N, N), U)
    sopt = np.array([o.sigma(T, V, np.ones(N), j, w) for j in range(N)])
    assert np.abs(r["S"][:, 2:] - sopt).max() < 1e-12 * np.abs(sopt).max()
    # the chord points xi_j +- 2T as well
    xij = np.array([o.xi(*o.geometry()[0][j]) for j in range(N)])
    for j in (0, 3):
        s2 = o.sigma(T, V, np.ones(N), j, [xij[j] + 2 * T, xij[j] - 2 * T])
        assert np.abs(r["S"][j, :2] - s2).max() < 1e-12 * np.abs(s2).max()


def test_z_k_a_identities_along_the_flow(o):
    U, g, d = 3.0, 0.6, 0.04
    kw = dict(z_feedback=True, katanin=True, freeze_vertex=True, dg=0.01)
    Zs = {}
    for ge in (g - d, g - d / 2, g, g + d / 2, g + d):
        r = o.gflow(U, g_end=ge, **kw)
        Zs[ge] = o.gflow_zka(ge, r["S"], r["D"], **kw)
    Z, K, A, _ = Zs[g]
    D1 = (Zs[g + d][0] - Zs[g - d][0]) / (2 * d)
    D2 = (Zs[g + d / 2][0] - Zs[g - d / 2][0]) / d
    dZ = (4 * D2 - D1) / 3
    assert np.abs(2 * dZ / Z - A).max() < 2e-5 * np.abs(A).max()
    assert np.abs(-(2.0 / g) * (1.0 - Z * K) - A).max() < 1e-12 * np.abs(A).max()
    assert np.all(Z < 1.0) and np.all(A < 0.0)      # Fermi-liquid-like weak coupling


def test_initial_state(o):
    S = np.zeros((N, 2), dtype=complex)
    Z, K, A, Ab = o.gflow_zka(0.0, S, S, z_feedback=True, katanin=True)
    assert np.all(Z == 1.0) and np.all(K == 1.0) and np.all(A == 0.0) and Ab == 0.0


def test_vertex_without_feedback_is_the_interaction_flow():
    L = 4
    o = Oracle(L * L, mode=MODE_LATTICE, regulator=REG_INTERACTION, T_fixed=0.2, eta=0.05)
    U = 2.0
    r = o.gflow(U, g_end=0.9, dg=0.1, z_feedback=False)
    ref = o.flow(np.full((L * L,) * 3, U), np.ones(L * L), 0.0, 0.9, 0.1)
    assert r["steps"] == ref["steps"] == 9
    assert np.abs(r["V"] - ref["V"]).max() < 1e-13 * np.abs(ref["V"]).max()


def test_bracket_and_dropped_term_at_weak_coupling(o):
    kw = dict(g_end=0.8, dg=0.05, z_feedback=True, katanin=True)
    S = {m: o.gflow(1.5, a_mode=m, **kw)["S"] for m in (A_AVG, A_MIN, A_MAX, A_DROP)}
    lo = np.minimum(S[A_MIN].imag, S[A_MAX].imag)
    hi = np.maximum(S[A_MIN].imag, S[A_MAX].imag)
    assert np.all(lo <= S[A_AVG].imag + 1e-15) and np.all(S[A_AVG].imag <= hi + 1e-15)
    assert np.abs(S[A_DROP] - S[A_AVG]).max() < 1e-2 * np.abs(S[A_AVG]).max()
