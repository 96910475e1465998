"""Asynchronous retrieval (hpmdr_retrieve_async + hpmdr_ctx_wait): retrievals
enqueued back to back without host round trips give, bit for bit, the oracle's
reconstructions and the synchronous path's infos, across handles, past the
64-slot ring, and with an unattainable bound in the middle."""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu

TAUS = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6]


@pytest.fixture(scope="module")
def B():
    from paper_2505_00227_gb300 import binding
    binding.lib()
    return binding


def _field(shape, seed):
    from paper_2505_00227_gb300 import synthetic as S
    return S.spectral(shape, seed=seed).numpy()


def _same_info(a, b):
    return (a.status == b.status and a.est_linf == b.est_linf and
            a.bytes_fetched_total == b.bytes_fetched_total and
            a.bytes_fetched_new == b.bytes_fetched_new and
            list(a.groups_per_level[:a.nlevels]) == list(b.groups_per_level[:b.nlevels]))


@pytest.mark.parametrize("shape", [(33, 20, 70), (64, 64, 128)])
def test_async_matches_oracle_and_sync(B, shape):
    f = _field(shape, 3)
    F = O.Field(f)
    ctx = B.Context()
    d = torch.from_numpy(f).cuda()
    h = ctx.refactor(d)
    outs = [torch.empty(shape, dtype=torch.float32, device="cuda") for _ in TAUS]
    infos = [h.retrieve_async(t, o) for t, o in zip(TAUS, outs)]
    assert ctx.wait() == 0
    h2 = ctx.refactor(d)
    for t, o, info in zip(TAUS, outs, infos):
        rc, ref, g, E = F.retrieve(t * F.range)
        assert info.status == rc and info.est_linf == E
        assert list(info.groups_per_level[:info.nlevels]) == list(g)
        assert np.array_equal(o.cpu().numpy().view(np.uint32), ref.view(np.uint32)), t
        so, sinfo, _ = h2.retrieve(t)
        assert torch.equal(so.view(torch.int32), o.view(torch.int32)) and _same_info(info, sinfo)


def test_async_two_handles_and_ring_drain(B):
    fa, fb = _field((40, 36, 64), 5), _field((17, 50, 33), 6)
    ctx = B.Context()
    ha, hb = ctx.refactor(torch.from_numpy(fa).cuda()), ctx.refactor(torch.from_numpy(fb).cuda())
    rng = np.random.default_rng(1)
    taus = [float(10.0 ** rng.uniform(-6, -1)) for _ in range(75)]  # more than the 64 slots
    work = []
    for i, t in enumerate(taus):
        h, f = (ha, fa) if i % 2 == 0 else (hb, fb)
        o = torch.empty(f.shape, dtype=torch.float32, device="cuda")
        work.append((f, t, o, h.retrieve_async(t, o)))
    assert ctx.wait() == 0
    Fa, Fb = O.Field(fa), O.Field(fb)
    for f, t, o, info in work:
        F = Fa if f is fa else Fb
        rc, ref, g, E = F.retrieve(t * F.range)
        assert info.status == rc and list(info.groups_per_level[:info.nlevels]) == list(g)
        assert np.array_equal(o.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_async_unattainable_and_bad_arguments(B):
    f = _field((20, 20, 20), 8)
    f[3, 4, 5] = np.float32(1e-20)  # below the fixed-point unit: no retrieval is exact
    ctx = B.Context()
    h = ctx.refactor(torch.from_numpy(f).cuda())
    o1, o2, o3 = (torch.empty(f.shape, dtype=torch.float32, device="cuda") for _ in range(3))
    i1 = h.retrieve_async(1e-2, o1)
    i2 = h.retrieve_async(0.0, o2)  # no prefix meets a zero bound
    i3 = h.retrieve_async(1e-3, o3)
    assert ctx.wait() == B.ERR_UNATTAINABLE
    assert i1.status == 0 and i2.status == B.ERR_UNATTAINABLE and i3.status == 0
    F = O.Field(f)
    rc, ref, g, E = F.retrieve(1e-3 * F.range)
    assert np.array_equal(o3.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    with pytest.raises(B.HpmdrError):
        h.retrieve_async(-1.0, o1)
    assert ctx.wait() == 0  # nothing pending


def test_profile_selected_stages_only(B):
    f = _field((64, 64, 128), 9)
    ctx = B.Context()
    h = ctx.refactor(torch.from_numpy(f).cuda())
    out = torch.empty(f.shape, dtype=torch.float32, device="cuda")
    ctx.profile(True, stages=["cells_recompose_out", "select"])
    infos = [h.retrieve_async(t, out) for t in TAUS]
    ctx.wait()
    prof = {p[0]: p for p in ctx.profile_entries()}
    ctx.profile(False)
    assert prof["cells_recompose_out"][2] == len(TAUS) and prof["select"][2] == len(TAUS)
    assert prof["cells_recompose_out"][1] > 0 and prof["cells_recompose_out"][3] > 0
    assert all(p[2] == 0 for k, p in prof.items() if k not in ("cells_recompose_out", "select"))
    assert all(i.status == 0 for i in infos)


def test_async_into_host_memory(B):
    f = _field((40, 64, 128), 12)
    F = O.Field(f)
    ctx = B.Context()
    h = ctx.refactor(torch.from_numpy(f).cuda())
    outs = [torch.empty(f.shape, dtype=torch.float32).pin_memory() for _ in TAUS]
    infos = [h.retrieve_async(t, o) for t, o in zip(TAUS, outs)]
    shared = torch.empty(f.shape, dtype=torch.float32).pin_memory()
    last = [h.retrieve_async(t, shared) for t in reversed(TAUS)]  # one buffer: the last wins
    assert ctx.wait() == 0
    for t, o, info in zip(TAUS, outs, infos):
        rc, ref, g, E = F.retrieve(t * F.range)
        assert info.status == rc and info.est_linf == E
        assert np.array_equal(o.numpy().view(np.uint32), ref.view(np.uint32)), t
    rc, ref, g, E = F.retrieve(TAUS[0] * F.range)
    assert np.array_equal(shared.numpy().view(np.uint32), ref.view(np.uint32))
    assert all(i.status == 0 for i in last)
    # a larger handle afterwards grows the context's output buffers
    f2 = _field((64, 64, 128), 13)
    h2 = ctx.refactor(torch.from_numpy(f2).cuda())
    o2 = torch.empty(f2.shape, dtype=torch.float32).pin_memory()
    i2 = h2.retrieve_async(1e-4, o2)
    assert ctx.wait() == 0
    F2 = O.Field(f2)
    rc, ref, g, E = F2.retrieve(1e-4 * F2.range)
    assert i2.status == rc and np.array_equal(o2.numpy().view(np.uint32), ref.view(np.uint32))
