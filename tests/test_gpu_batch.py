"""Batched flows (qpfrg_flow_batch): each flow of a sweep over (N_p, U, T_end)
must end exactly as the same flow run alone through qpfrg_flow, and one flow
as the FP64 oracle's; flows stop independently."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2005_00827_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def specs_small():
    gen = inputs.splitmix64(7)
    out = []
    for i in range(7):
        N = (16, 24)[i % 2]
        U = 2.0 + 2.0 * next(gen)
        T_end = math.exp(math.log(0.02) + next(gen) * math.log(10.0))
        out.append((N, U, 1.0, T_end))
    return out


@pytest.mark.parametrize("prec", [api.QPFRG_FP64, api.QPFRG_MIXED])
def test_batch_matches_single_flows(prec):
    import torch
    n = 4
    specs = specs_small()
    stream = torch.cuda.current_stream().cuda_stream
    o = api.qpfrg_default_options()
    o.precision = prec
    res = api.qpfrg_flow_batch(api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(n, n, 0),
                               api.QPFRG_REG_TEMPERATURE, o, specs, stream)
    statuses = set()
    for (N, U, T0, Tend), r in zip(specs, res):
        with api.Context(N, n, n, U=U, lambda0=T0, precision=prec, lambda_end=Tend, stream=stream) as c:
            single = api.qpfrg_flow(c.h).as_dict()
        assert r["status"] == single["status"] and r["steps"] == single["steps"]
        assert r["lam"] == pytest.approx(single["lam"], rel=1e-12)
        if r["status"] == "DIVERGED":
            assert r["lambda_c"] == pytest.approx(single["lambda_c"], rel=1e-9)
        assert r["max_abs_v"] == pytest.approx(single["max_abs_v"], rel=1e-9 if prec == api.QPFRG_FP64 else 1e-6)
        statuses.add(r["status"])
    assert statuses == {"DIVERGED", "REACHED_END"}   # the sweep straddles the boundary


def test_batch_flow_matches_oracle():
    import torch
    n = 4
    specs = [(16, 3.2, 1.0, 0.01), (16, 1.5, 1.0, 0.3)]
    o = api.qpfrg_default_options()
    res = api.qpfrg_flow_batch(api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(n, n, 0),
                               api.QPFRG_REG_TEMPERATURE, o, specs, torch.cuda.current_stream().cuda_stream)
    for (N, U, T0, Tend), r in zip(specs, res):
        ref = Oracle(N, n, n).flow(np.full((N, N, N), U), np.ones(N), T0, Tend, math.log(0.98))
        assert r["status"] == ref["status"] and r["steps"] == ref["steps"]
        if r["status"] == "DIVERGED":
            assert r["lambda_c"] == pytest.approx(ref["lambda_c"], rel=1e-9)


def test_batch_rejects_bad_specs():
    o = api.qpfrg_default_options()
    with pytest.raises(api.QpfrgError):
        api.qpfrg_flow_batch(api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(4, 4, 0),
                             api.QPFRG_REG_TEMPERATURE, o, [(16, 2.0, -1.0, 0.1)], 0)


def test_batch_device_path_config4_shapes_match_single_flows():
    """The batched device path (tensor-core precision, Z = 1, one graph per
    chunk of steps and group): 16 draws of the phase-boundary sweep (N_p in
    {24, 48, 72, 96}, 16 x 16 fine grid) end as the same flows run alone.
    The batched launch splits the contraction's reduction differently, so its
    FP32 partial sums add in another order: step counts and statuses agree
    exactly, Lambda_c to 1e-5 and max|V| at the last step (past |V| = 20,
    where the flow amplifies rounding) to the tensor-core tolerance 1e-4.
    Both sides take the row orbits of the contraction (every flow's state
    stays C4v symmetric)."""
    import torch
    n = 16
    specs = [(d["N"], d["U"], 1.0, d["T_end"]) for d in inputs.batch_specs(16)]
    assert len({s[0] for s in specs}) >= 3
    stream = torch.cuda.current_stream().cuda_stream
    o = api.qpfrg_default_options()
    o.precision = api.QPFRG_MIXED_TC
    res = api.qpfrg_flow_batch(api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(n, n, 0),
                               api.QPFRG_REG_TEMPERATURE, o, specs, stream)
    statuses = set()
    for (N, U, T0, Tend), r in zip(specs, res):
        with api.Context(N, n, n, U=U, lambda0=T0, precision=api.QPFRG_MIXED_TC, lambda_end=Tend,
                         stream=stream) as c:
            single = api.qpfrg_flow(c.h).as_dict()
        assert r["status"] == single["status"] and r["steps"] == single["steps"]
        assert r["lam"] == pytest.approx(single["lam"], rel=1e-12)
        if r["status"] == "DIVERGED":
            assert r["lambda_c"] == pytest.approx(single["lambda_c"], rel=1e-5)
        assert r["max_abs_v"] == pytest.approx(single["max_abs_v"], rel=1e-4)
        statuses.add(r["status"])
    assert statuses == {"DIVERGED", "REACHED_END"}


def test_batch_device_path_matches_oracle():
    import torch
    n = 4
    specs = [(16, 3.2, 1.0, 0.01), (16, 1.5, 1.0, 0.3), (24, 2.4, 1.0, 0.05)]
    o = api.qpfrg_default_options()
    o.precision = api.QPFRG_MIXED_TC
    res = api.qpfrg_flow_batch(api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(n, n, 0),
                               api.QPFRG_REG_TEMPERATURE, o, specs, torch.cuda.current_stream().cuda_stream)
    for (N, U, T0, Tend), r in zip(specs, res):
        ref = Oracle(N, n, n).flow(np.full((N, N, N), U), np.ones(N), T0, Tend, math.log(0.98))
        assert r["status"] == ref["status"] and abs(r["steps"] - ref["steps"]) <= 1
        if r["status"] == "DIVERGED":
            assert r["lambda_c"] == pytest.approx(ref["lambda_c"], rel=5e-3)


def test_tensor_core_wait_expiry_is_reported(monkeypatch):
    """A bounded wait of the tensor-core contraction that runs out (a barrier
    nothing arrives on) aborts its CTA and surfaces as QPFRG_ERR_TIMEOUT, for a
    single flow and for the batched path; the device stays usable."""
    import torch
    n = 4
    monkeypatch.setenv("QPFRG_TEST_TC_WAIT", "1")
    with api.Context(16, n, n, U=2.0, precision=api.QPFRG_MIXED_TC) as c:
        with pytest.raises(api.QpfrgError) as ei:
            api.qpfrg_step(c.h, 1)
        assert ei.value.status == api.QPFRG_ERR_TIMEOUT
    o = api.qpfrg_default_options()
    o.precision = api.QPFRG_MIXED_TC
    with pytest.raises(api.QpfrgError) as ei:
        api.qpfrg_flow_batch(api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(n, n, 0),
                             api.QPFRG_REG_TEMPERATURE, o, [(16, 2.0, 1.0, 0.9)],
                             torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == api.QPFRG_ERR_TIMEOUT
    monkeypatch.delenv("QPFRG_TEST_TC_WAIT")
    with api.Context(16, n, n, U=2.0, precision=api.QPFRG_MIXED_TC) as c:
        r = api.qpfrg_step(c.h, 2).as_dict()
    assert r["steps"] == 2 and np.isfinite(r["max_abs_v"])
