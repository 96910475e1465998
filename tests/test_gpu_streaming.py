"""GPU parity of the chunk-streamed path and of compacted handles.

Chunk streaming (Sec. 5.3 pipeline): a field is cut into independent
sub-blocks, each refactored as a field of its own on one of several CUDA
streams, and retrieved against the whole field's value range.  The oracle
refactors each sub-block on its own and retrieves it with the same absolute
bound; the assembled reconstruction must match bit for bit.

Compaction: a handle whose stored groups were packed and whose plane buffer
became a cache must give exactly the reconstructions of the plain handle, and
dropping the cache must only cost re-decoding.
"""
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


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context()


def _boxes(shape, chunk):
    cnt = [(s + c - 1) // c for s, c in zip(shape, chunk)]
    for iz in range(cnt[0]):
        for iy in range(cnt[1]):
            for ix in range(cnt[2]):
                org = (iz * chunk[0], iy * chunk[1], ix * chunk[2])
                yield tuple(slice(o, min(o + c, s)) for o, c, s in zip(org, chunk, shape))


def _cases():
    from paper_2505_00227_gb300 import synthetic as S
    return {
        # FP64 spectral + trend, ragged chunk grid on two axes
        "f64_trend_ragged": (S.spectral_trend((20, 24, 40), seed=3, dtype=torch.float64).numpy(),
                             (8, 16, 40)),
        # FP32, chunks whose large levels take the cell kernels
        "f32_cells": (S.spectral((16, 16, 128), seed=21).numpy(), (8, 16, 128)),
        # FP32 chunks with a 512-wide finest level (the widest cell tile), ragged along y
        "f32_cells_512": (S.spectral((6, 13, 512), seed=30).numpy(), (3, 7, 512)),
        # FP64 chunks whose large levels take the 64-plane cell kernels
        "f64_cells": (S.spectral_trend((8, 16, 256), seed=35, dtype=torch.float64).numpy(),
                      (4, 8, 256)),
        # one chunk covering everything (equals a plain refactor)
        "f32_single_chunk": (S.blobs((9, 10, 11), seed=22).numpy(), (64, 64, 64)),
        # chunks of one x-row
        "f64_rows": (S.spectral((3, 4, 50), seed=23, dtype=torch.float64).numpy(), (1, 1, 50)),
    }


CASES = list(_cases())


def _oracle_chunks(f, chunk):
    return [(sl, O.Field(np.ascontiguousarray(f[sl]))) for sl in _boxes(f.shape, chunk)]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("where", ["host", "device"])
def test_chunked_matches_oracle(ctx, name, where):
    f, chunk = _cases()[name]
    src = torch.from_numpy(f)
    src = src.pin_memory() if where == "host" else src.cuda()
    hs = ctx.refactor_chunked(src, chunk, nstreams=3)
    OF = _oracle_chunks(f, chunk)
    assert len(hs) == len(OF)
    for h, (sl, F) in zip(hs, OF):
        assert tuple(h.shape) == f[sl].shape
        for l in range(F.nlev):
            assert h.level_info(l)[:2] == F.levels[l][:2]
            for g in range(F.ngroups):
                gb, m, _ = h.group(l, g)
                ob, om, _, _ = F.group(l, g)
                assert m == om and np.array_equal(gb, ob), (sl, l, g)
        assert h.sequence() == F.sequence()
    lo = min(F.vmin for _, F in OF)
    hi = max(F.vmax for _, F in OF)
    tol = 1e-6 if f.dtype == np.float32 else 1e-12
    for tau in TAUS:
        tau_abs = tau * (hi - lo)
        out = torch.empty(f.shape, dtype=src.dtype)
        out = out.pin_memory() if where == "host" else out.cuda()
        infos, st = ctx.retrieve_chunked(hs, f.shape, chunk, tau, out, nstreams=3)
        got = out.cpu().numpy()
        ref = np.empty_like(f)
        worst = 0
        for info, (sl, F) in zip(infos, OF):
            rc, r, g, E = F.retrieve(tau_abs)
            ref[sl] = r
            assert info.groups == list(g) and info.est_linf == E
            worst = rc if rc != 0 else worst
        assert st == worst
        assert np.array_equal(got.view(np.uint8), ref.view(np.uint8)), tau
        err = np.abs(got.astype(np.float64) - f.astype(np.float64)).max()
        assert err <= max(i.est_linf for i in infos)
        assert np.abs(got.astype(np.float64) - ref).max() <= tol * max(hi - lo, 1.0)
        if st == 0:
            assert err <= tau_abs


def test_chunked_rejects_mismatched_handles(ctx, B):
    f, chunk = _cases()["f32_cells"]
    hs = ctx.refactor_chunked(torch.from_numpy(f).cuda(), chunk)
    out = torch.empty(f.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(B.HpmdrError):
        ctx.retrieve_chunked(hs[:1], f.shape, chunk, 1e-3, out)
    with pytest.raises(B.HpmdrError):
        ctx.retrieve_chunked(hs, f.shape, (4, 16, 128), 1e-3, out)


@pytest.mark.parametrize("shape,dtype", [((32, 40, 128), torch.float32),
                                         ((17, 23, 30), torch.float32),
                                         ((12, 10, 9), torch.float64)])
def test_compact_and_drop_cache(ctx, shape, dtype):
    from paper_2505_00227_gb300 import synthetic as S
    f = S.spectral(shape, seed=31, dtype=dtype).numpy()
    F = O.Field(f)
    h = ctx.refactor(torch.from_numpy(f).cuda())
    blob = h.export()
    res0, _, _ = h.memory()
    h.compact()
    res1, cache, cache_max = h.memory()
    # all-DC fields (groups at most T_s bytes) keep every byte: no saving there
    assert cache == 0 and res1 <= res0 and cache_max > 0
    assert h.export() == blob  # packing moves bytes, it changes none
    for rnd in range(2):
        prev = 0
        for tau in TAUS:
            out, info, st = h.retrieve(tau)
            rc, ref, g, E = F.retrieve(tau * F.range)
            assert st == rc and info.groups == list(g) and info.est_linf == E
            assert np.array_equal(out.cpu().numpy().view(np.uint8), ref.view(np.uint8))
            assert info.bytes_fetched_total >= prev
            prev = info.bytes_fetched_total
        assert 0 < h.memory()[1] <= cache_max  # the transient staging is not held
        # tightening decoded only new groups; after dropping the cache the next
        # retrieval fetches everything it uses again
        h.drop_cache()
        assert h.memory()[1] == 0
        out, info, st = h.retrieve(1e-3)
        assert info.bytes_fetched_new == info.bytes_fetched_total > 0
        h.drop_cache()
