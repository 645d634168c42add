"""The allocation-free Z entry point (qpfrg_zfactor_static) against the
context-based qpfrg_selfenergy, through the C ABI, on two calls in a row.

It serves callers that cannot allocate device memory while they run; its
scratch is a static device array shared by all calls.  The test's own
buffers come from torch (the test is not such a caller); the entry point
under test allocates nothing.  Both sides compute in FP64: tolerance 1e-10.
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2005_00827_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()


@pytest.mark.parametrize("geo", [(16, 4, 4, api.QPFRG_GRID_WEDGE, api.QPFRG_PROP_PAPER),
                                 (16, 4, 6, api.QPFRG_GRID_WEDGE, api.QPFRG_PROP_QP),
                                 (16, 1, 1, api.QPFRG_GRID_LATTICE, api.QPFRG_PROP_PAPER)],
                         ids=["wedge", "wedge_qp", "lattice"])
def test_static_z_matches_selfenergy_twice(geo):
    import torch
    N, nt, nr, mode, prop = geo
    T, eta = 0.2, 0.02
    stream = torch.cuda.current_stream().cuda_stream
    V = inputs.random_vertex(N, 2.0, seed=21, c4v=(mode == api.QPFRG_GRID_WEDGE))
    Z = inputs.z_profile(N, "aniso") if mode == api.QPFRG_GRID_WEDGE else \
        np.random.default_rng(5).uniform(0.85, 1.0, N)
    Vd, Zd = dev(V), dev(Z)
    with api.Context(N, nt, nr, U=2.0, mode=mode, propagator=prop, eta=eta, stream=stream) as ctx:
        ref = torch.zeros(N, dtype=torch.float64, device="cuda")
        api.qpfrg_selfenergy(ctx.h, T, Vd, Zd, None, None, ref)
        kf, fine = api.qpfrg_geometry(ctx.h)
    torch.cuda.synchronize()
    lat = api.qpfrg_lattice(1.0, 0.0, 0.0)
    fine_d, kf_d = dev(fine), dev(kf)
    for call in range(2):
        out = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        api.qpfrg_zfactor_static(lat, N, fine.shape[0], mode, prop, fine_d, kf_d, Vd, Zd, T, eta, stream, out)
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref.cpu().numpy()).max() < 1e-10, f"call {call}"


def test_static_z_rejects_too_many_patches():
    import torch
    lat = api.qpfrg_lattice(1.0, 0.0, 0.0)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(api.QpfrgError) as ei:
        api.qpfrg_zfactor_static(lat, 260, 260, api.QPFRG_GRID_WEDGE, 0, buf, buf, buf, buf, 0.2, 0.02, 0, buf)
    assert ei.value.status == api.QPFRG_ERR_INVALID
