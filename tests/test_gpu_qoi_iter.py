"""GPU parity of the iterated QoI retrieval (Algorithm 3) for the total
velocity V = vx^2 + vy^2 + vz^2: for every next-bound estimator the GPU must
take the oracle's decisions exactly (same iterations, same groups, same FP64
bound), so components and V_hat match bit for bit."""
import math

import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2505_00227_gb300 import binding
    binding.lib()
    return binding


def _triplet(shape, seed):
    from paper_2505_00227_gb300 import synthetic as S
    return [S.spectral(shape, seed=seed + c).numpy() for c in range(3)]


CASES = {"small": ((12, 13, 14), 70), "cells": ((20, 24, 64), 71), "general": ((40, 45, 50), 72)}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("est", ["EST_CP", "EST_MA", "EST_MAPE"])
@pytest.mark.parametrize("tau", [1e-1, 1e-3, 1e-5])
def test_iterated_qoi_matches_oracle(B, case, est, tau):
    shape, seed = CASES[case]
    v = _triplet(shape, seed)
    ctx = B.Context()
    dev = [torch.from_numpy(x).cuda() for x in v]
    hs = [ctx.refactor(d) for d in dev]
    ctx.prepare_vtotal(hs, *dev)
    outs = [torch.empty(shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    q, rep, st = ctx.retrieve_qoi_vtotal(hs, tau, getattr(B, est), outs=outs)
    lo, hi = O.vtotal_range(*v)
    Fs = [O.Field(x) for x in v]
    ost, oouts, oq, orep = O.qoi_vtotal(Fs, lo, hi, tau, getattr(O, est))
    assert st == ost and rep.status == orep.status
    assert rep.iterations == orep.iterations
    assert rep.tau_abs == orep.tau_abs and rep.est == orep.est
    assert list(rep.prefix) == list(orep.prefix) and list(rep.eps) == list(orep.eps)
    for o, r in zip(outs, oouts):
        assert np.array_equal(o.cpu().numpy().view(np.uint32), r.view(np.uint32))
    assert np.array_equal(q.cpu().numpy().view(np.uint32), oq.view(np.uint32))
    if st == 0:
        Vt = sum(x.astype(np.float64) ** 2 for x in v)
        assert np.abs(q.cpu().numpy().astype(np.float64) - Vt).max() <= rep.est * (1 + 1e-12)
        assert rep.est <= rep.tau_abs


def test_mape_without_threshold_is_ma(B):
    v = _triplet((12, 13, 14), 75)
    ctx = B.Context()
    dev = [torch.from_numpy(x).cuda() for x in v]
    hs = [ctx.refactor(d) for d in dev]
    ctx.prepare_vtotal(hs, *dev)
    _, ma, _ = ctx.retrieve_qoi_vtotal(hs, 1e-4, B.EST_MA)
    for h in hs:
        h.reset()
    _, mape, _ = ctx.retrieve_qoi_vtotal(hs, 1e-4, B.EST_MAPE, c=math.inf)
    assert ma.iterations == mape.iterations and list(ma.prefix) == list(mape.prefix)


@pytest.mark.parametrize("est", ["EST_MA", "EST_CP"])
def test_repeated_handle_matches_oracle(B, est):
    """The same handle for two components (vx = vy): its one selection record
    serves both retrievals of an iteration, which take the per-retrieval path.
    A reconstruction depends only on the bound, so the decisions, components and
    V_hat equal the oracle's on three separate fields."""
    shape = (20, 24, 64)
    a, _, c = _triplet(shape, 76)
    v = [a, a, c]
    ctx = B.Context()
    da, dc = torch.from_numpy(a).cuda(), torch.from_numpy(c).cuda()
    ha, hc = ctx.refactor(da), ctx.refactor(dc)
    hs = [ha, ha, hc]
    ctx.prepare_vtotal(hs, da, da, dc)
    outs = [torch.empty(shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    q, rep, st = ctx.retrieve_qoi_vtotal(hs, 1e-4, getattr(B, est), outs=outs)
    lo, hi = O.vtotal_range(*v)
    ost, oouts, oq, orep = O.qoi_vtotal([O.Field(x) for x in v], lo, hi, 1e-4, getattr(O, est))
    assert st == ost and rep.iterations == orep.iterations and rep.est == orep.est
    assert list(rep.prefix) == list(orep.prefix) and list(rep.eps) == list(orep.eps)
    for o, r in zip(outs, oouts):
        assert np.array_equal(o.cpu().numpy().view(np.uint32), r.view(np.uint32))
    assert np.array_equal(q.cpu().numpy().view(np.uint32), oq.view(np.uint32))
