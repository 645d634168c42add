"""Launch-shape autotuner: shapes change only the order of floating-point
sums, so every shape must give the same right-hand side, Z and flows up to
FP32 reassociation; the tuner must return shapes from its candidate sets.
Split-K regroups FP32 partial sums of up to K = 2 N^2 terms before they
reach the FP64 output, so the RHS is compared normwise at 1e-5 (K eps32 with
K = 512 is 3e-5 in the worst case; the mixed parity bar is 1e-4)."""
import numpy as np
import pytest

from paper_2005_00827_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).ravel()).cuda()


def rhs(ctx, lam, V, Z):
    import torch
    out = torch.zeros(V.size, dtype=torch.float64, device="cuda")
    api.qpfrg_rhs(ctx.h, lam, dev(V), dev(Z), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def zfac(ctx, T, V, Z):
    import torch
    out = torch.zeros(len(Z), dtype=torch.float64, device="cuda")
    api.qpfrg_selfenergy(ctx.h, T, dev(V), dev(Z), None, None, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_autotune_returns_candidate_shapes_and_keeps_results():
    N, n = 16, 8
    V = inputs.random_vertex(N, 2.0, seed=3, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    with api.Context(N, n, n, U=2.0, precision=api.QPFRG_MIXED_TC, z_feedback=1) as c:
        before = rhs(c, 0.3, V, Z)
        t = api.qpfrg_autotune(c.h, 0.3)
        after = rhs(c, 0.3, V, Z)
    assert t["bubble_qchunk"] in (8, 16, 32, 64, 128, 256)
    assert t["bubble_transfers"] in (2, 4)
    assert t["sigma_qblocks"] in (1, 2, 4, 8)
    assert all(s in (0, 1, 2, 3, 4, 6, 8, 12, 16) for s in t["tc_splits"])
    assert t["ms_bubble"] > 0 and t["ms_sigma"] > 0 and t["ms_contract"] > 0
    assert np.abs(after - before).max() <= 1e-5 * np.abs(before).max()


@pytest.mark.parametrize("prec", [api.QPFRG_MIXED, api.QPFRG_MIXED_TC])
def test_extreme_shapes_agree(prec):
    """Smallest and largest shapes of every knob give the same RHS and Z
    (8 patches x 1024 points: 16 q blocks, several CTAs of the self-energy)."""
    N, n = 8, 32
    V = inputs.random_vertex(N, 2.0, seed=9, c4v=True)
    Z = inputs.z_profile(N, "aniso")
    res = []
    with api.Context(N, n, n, U=2.0, precision=prec) as c:
        for shape in (dict(bubble_qchunk=8, sigma_qblocks=1, tc_splits=(1, 1, 1)),
                      dict(bubble_qchunk=256, sigma_qblocks=8, tc_splits=(16, 16, 16), bubble_transfers=4),
                      dict(bubble_qchunk=32, sigma_qblocks=3, tc_splits=(3, 2, 5), bubble_transfers=4),
                      dict(bubble_qchunk=8, bubble_transfers=4)):
            api.qpfrg_set_tuning(c.h, **shape)
            res.append((rhs(c, 0.2, V, Z), zfac(c, 0.2, V, Z)))
    for r, z in res[1:]:
        assert np.abs(r - res[0][0]).max() <= 1e-5 * np.abs(res[0][0]).max()
        assert np.abs(z - res[0][1]).max() <= 1e-6


def test_set_tuning_rejects_negative_shapes():
    with api.Context(8, 4, 4, U=2.0, precision=api.QPFRG_MIXED) as c:
        with pytest.raises(api.QpfrgError):
            api.qpfrg_set_tuning(c.h, bubble_qchunk=-1)
        with pytest.raises(api.QpfrgError):
            api.qpfrg_set_tuning(c.h, sigma_qblocks=65)
        with pytest.raises(api.QpfrgError):
            api.qpfrg_set_tuning(c.h, bubble_transfers=3)


def test_batch_with_autotune_matches_batch_without():
    import torch
    n = 8
    specs = [(16, 3.0, 1.0, 0.02), (24, 2.0, 1.0, 0.05), (16, 1.5, 1.0, 0.2)]
    stream = torch.cuda.current_stream().cuda_stream
    out = []
    for tune in (0, 1):
        o = api.qpfrg_default_options()
        o.precision = api.QPFRG_MIXED_TC
        o.autotune = tune
        out.append(api.qpfrg_flow_batch(api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(n, n, 0),
                                        api.QPFRG_REG_TEMPERATURE, o, specs, stream))
    for a, b in zip(*out):
        assert a["status"] == b["status"] and a["steps"] == b["steps"]
        assert b["max_abs_v"] == pytest.approx(a["max_abs_v"], rel=1e-5)
        if a["status"] == "DIVERGED":
            assert b["lambda_c"] == pytest.approx(a["lambda_c"], rel=1e-5)
