"""GPU parity of the SOPT spectral workload (Sec. 3.1.1, Figs. 1-3): the
spectral function and its Fermi-liquid (Gaussian) approximation from the
real-frequency self-energy, and Z along the Fermi surface against U.

* qpfrg_spectral on the oracle's own Sigma: A and A_FL to 1e-12 (the kernel
  alone), wedge and lattice mode.
* End to end (qpfrg_selfenergy at V = U, Z = 1, then qpfrg_spectral) against
  the oracle's exact pole sum: A normwise 1e-3 (the frequency grid is
  binned, Sigma to 1e-4 of its maximum).
* SOPT scaling: the chord slope 1 - 1/Z is exactly quadratic in U.
"""
import numpy as np
import pytest

from oracle.oracle import MODE_LATTICE, Oracle
from paper_2005_00827_gb300 import api

pytestmark = pytest.mark.gpu


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()


def zeros(n):
    import torch
    return torch.zeros(n, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("mode", [0, 1], ids=["wedge", "lattice"])
def test_spectral_kernel_on_oracle_sigma(mode):
    import torch
    N, n, U, T, nw = 16, 4, 2.0, 0.3, 129
    o = Oracle(N, n, n, mode=mode, eta=0.05) if mode == 0 else Oracle(N, mode=MODE_LATTICE, eta=0.05)
    V = np.full((N, N, N), U)
    w = np.linspace(-4.0, 4.0, nw)
    sig = np.array([o.sigma(T, V, np.ones(N), j, w) for j in range(N)])
    Z = o.zfactor(T, V, np.ones(N))
    ref = [o.spectral(j, w, sig[j], Z[j]) for j in range(N)]
    nt, nr = (n, n) if mode == 0 else (1, 1)
    with api.Context(N, nt, nr, U=U, mode=mode, eta=0.05, n_omega=nw, omega_min=-4.0, omega_max=4.0) as c:
        A, Afl = zeros(N * nw), zeros(N * nw)
        api.qpfrg_spectral(c.h, dev(sig.real), dev(sig.imag), dev(Z), A, Afl)
        torch.cuda.synchronize()
        A, Afl = A.cpu().numpy().reshape(N, nw), Afl.cpu().numpy().reshape(N, nw)
    for j in range(N):
        assert np.abs(A[j] - ref[j][0]).max() < 1e-12 * max(1.0, ref[j][0].max())
        assert np.abs(Afl[j] - ref[j][1]).max() < 1e-12 * max(1.0, ref[j][1].max())


@pytest.mark.parametrize("prec", [api.QPFRG_FP64, api.QPFRG_MIXED])
def test_sopt_spectral_end_to_end(prec):
    import torch
    N, n, U, T, nw = 16, 4, 2.0, 0.3, 256
    o = Oracle(N, n, n, eta=0.05)
    V = np.full((N, N, N), U)
    w = np.linspace(-4.0, 4.0, nw)
    with api.Context(N, n, n, U=U, precision=prec, eta=0.05, n_omega=nw, omega_min=-4.0, omega_max=4.0) as c:
        re, im, Zg = zeros(N * nw), zeros(N * nw), zeros(N)
        api.qpfrg_selfenergy(c.h, T, dev(V), None, re, im, Zg)
        A, Afl = zeros(N * nw), zeros(N * nw)
        api.qpfrg_spectral(c.h, re, im, Zg, A, Afl)
        torch.cuda.synchronize()
        A = A.cpu().numpy().reshape(N, nw)
        Zg = Zg.cpu().numpy()
    for j in (0, 1, 2):
        sig = o.sigma(T, V, np.ones(N), j, w)
        z = o.zfactor_targets(T, V, np.ones(N), [j])[0]
        ref, _ = o.spectral(j, w, sig, z)
        assert np.abs(A[j] - ref).max() < 1e-3 * ref.max()
        assert abs(Zg[j] - z) < (1e-10 if prec == api.QPFRG_FP64 else 1e-4)


def test_sopt_z_scales_with_u_squared():
    """Z along the Fermi surface for U = 1, 2, 4 at T = 0.3: in SOPT the
    self-energy is U^2 times that of U = 1, so 1 - 1/Z scales as U^2."""
    import torch
    N, n, T = 16, 4, 0.3
    s = {}
    with api.Context(N, n, n, U=1.0, precision=api.QPFRG_FP64, eta=0.05) as c:
        for U in (1.0, 2.0, 4.0):
            Zg = zeros(N)
            api.qpfrg_selfenergy(c.h, T, dev(np.full((N, N, N), U)), None, None, None, Zg)
            torch.cuda.synchronize()
            s[U] = 1.0 - 1.0 / Zg.cpu().numpy()
    assert np.abs(s[2.0] - 4.0 * s[1.0]).max() < 1e-9 * np.abs(s[1.0]).max()
    assert np.abs(s[4.0] - 16.0 * s[1.0]).max() < 1e-9 * np.abs(s[1.0]).max()
