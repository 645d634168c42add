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
