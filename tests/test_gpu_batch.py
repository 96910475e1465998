"""GPU parity of the batched persistent path (one graph launch per pass).

Fields of uneven shapes (ragged, cell-eligible, tiny, single value) are
refactored together; every field's stored groups and greedy sequence must
equal the oracle's, every batched retrieval must equal the oracle's
reconstruction bit for bit, and the results must equal the one-field-per-
launch path, before and after autotuning.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu

SHAPES = [(33, 20, 64), (17, 23, 30), (9, 40, 128), (32, 32, 32), (5, 7, 200), (1, 64, 128),
          (12, 100, 9), (40, 37, 192), (3, 3, 3), (1, 1, 1), (2, 64, 64), (20, 24, 40),
          (45, 47, 49), (30, 50, 70), (3, 9, 512), (2, 5, 1024)]


@pytest.fixture(scope="module")
def B():
    from paper_2505_00227_gb300 import binding
    binding.lib()
    return binding


def _fields(dtype=torch.float32, shapes=SHAPES):
    from paper_2505_00227_gb300 import synthetic as S
    out = []
    for i, sh in enumerate(shapes):
        if i % 2 == 0 or np.prod(sh) < 8:  # a one-value spectral field is 0/0 after rescaling
            f = S.blobs(sh, seed=100 + i, dtype=dtype)
        else:
            f = S.spectral(sh, seed=100 + i, dtype=dtype)
        out.append(f.numpy())
    return out


def _taus(n, seed):
    rng = np.random.default_rng(seed)
    return [float(10.0 ** rng.uniform(-6, -1)) for _ in range(n)]


def _run(B, dtype, shapes):
    ctx = B.Context()
    fs = _fields(dtype, shapes)
    dev = [torch.from_numpy(f).cuda() for f in fs]
    batch = B.Batch(ctx, shapes, dtype)
    batch.refactor(dev)
    return ctx, fs, dev, batch


def _check_refactor(batch, fs):
    for h, f in zip(batch.handles, fs):
        F = O.Field(f)
        info = h.field_info()
        assert info["E_f"] == F.E_f and info["range"] == F.range
        for l in range(F.nlev):
            assert h.level_info(l)[:2] == F.levels[l][:2]
            for g in range(F.ngroups):
                gb, m, est = h.group(l, g)
                ob, om, oH, oR = F.group(l, g)
                assert m == om and est == (oH, oR) and np.array_equal(gb, ob), (f.shape, l, g)
        assert h.sequence() == F.sequence()


def _check_retrieve(batch, fs, taus, outs, infos, st):
    worst = 0
    for f, tau, o, info in zip(fs, taus, outs, infos):
        F = O.Field(f)
        rc, ref, g, E = F.retrieve(tau * F.range)
        assert info.status == rc and info.groups == list(g) and info.est_linf == E, f.shape
        got = o.cpu().numpy()
        assert np.array_equal(got.view(np.uint8), ref.view(np.uint8)), f.shape
        err = np.abs(got.astype(np.float64) - f.astype(np.float64)).max()
        assert err <= info.est_linf
        worst = rc if rc != 0 else worst
    assert st == worst


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_matches_oracle_and_plain_path(B, dtype):
    shapes = SHAPES if dtype == torch.float32 else SHAPES[:6] + SHAPES[-4:]
    ctx, fs, dev, batch = _run(B, dtype, shapes)
    _check_refactor(batch, fs)
    prev = [0] * len(fs)
    for rnd, seed in enumerate([1, 2, 3]):
        taus = _taus(len(fs), seed)
        if rnd == 2:
            taus = [t * 1e-2 for t in taus]  # tighter: decodes only new groups
        outs = [torch.empty(f.shape, dtype=dtype, device="cuda") for f in fs]
        infos, st = batch.retrieve(taus, outs)
        _check_retrieve(batch, fs, taus, outs, infos, st)
        # the plain one-field-per-launch path gives the same bytes
        for f, d, tau, o in zip(fs, dev, taus, outs):
            h = ctx.refactor(d)
            po, pinfo, pst = h.retrieve(tau)
            assert torch.equal(po.view(torch.uint8), o.view(torch.uint8)), f.shape
        if rnd == 2:
            for i, info in enumerate(infos):
                assert info.bytes_fetched_total >= prev[i]
        prev = [i.bytes_fetched_total for i in infos]
    batch.close()


def test_batch_autotune_keeps_results(B):
    ctx, fs, dev, batch = _run(B, torch.float32, SHAPES)
    taus = _taus(len(fs), 5)
    outs = [torch.empty(f.shape, dtype=torch.float32, device="cuda") for f in fs]
    best = batch.autotune(dev, taus, outs)
    assert best == batch.tuning()
    assert best[0] in (2, 4, 8) and best[1] in (16384, 65536) and best[2] in (4, 8)
    _check_refactor(batch, fs)
    outs = [torch.empty(f.shape, dtype=torch.float32, device="cuda") for f in fs]
    infos, st = batch.retrieve(taus, outs)
    _check_retrieve(batch, fs, taus, outs, infos, st)
    for sm, seg, dm in [(1, 1024, 1), (3, 4096, 2)]:  # odd tunings: same bytes
        batch.set_tuning(sm, seg, dm)
        batch.refactor(dev)
        _check_refactor(batch, fs[:3])
        o2 = [torch.empty_like(o) for o in outs]
        infos, st = batch.retrieve(taus, o2)
        for a, b in zip(outs, o2):
            assert torch.equal(a.view(torch.uint8), b.view(torch.uint8))
    ms = batch.last_ms()
    assert ms[0] > 0 and ms[1] > 0
    batch.close()


def test_batch_rejects_bad_arguments(B):
    ctx = B.Context()
    batch = B.Batch(ctx, [(8, 8, 8)], torch.float32)
    outs = [torch.empty((8, 8, 8), dtype=torch.float32, device="cuda")]
    with pytest.raises(B.HpmdrError):
        batch.retrieve([1e-3], outs)  # not refactored yet
    f = torch.zeros(8 * 8 * 8 + 1, dtype=torch.float32, device="cuda")[1:].view(8, 8, 8)
    with pytest.raises(B.HpmdrError):
        batch.refactor([f])  # not 16-byte aligned
    with pytest.raises(B.HpmdrError):
        batch.set_tuning(0, 65536, 4)
    batch.close()
