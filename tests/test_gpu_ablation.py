"""GPU tests of the lossless-strategy comparison (Sec. 7.2.2): every group
stored with one forced method.  The stored bytes must equal the oracle's coder
applied to the oracle's planes, and the reconstructions must still meet their
bounds; retrieving everything must give the same field as Algorithm 2."""
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


def _group_bytes(F, l, g):
    planes = F.planes(l)  # (B+1, W) uint32
    off, size = O.group_slice(planes.shape[1], g)  # bytes within the level's planes
    return np.ascontiguousarray(planes).view(np.uint8).reshape(-1)[off:off + size]


@pytest.mark.parametrize("shape,dtype", [((33, 20, 64), torch.float32),
                                         ((17, 23, 30), torch.float64)])
@pytest.mark.parametrize("method", ["DC", "HUFFMAN", "RLE"])
def test_forced_method(B, shape, dtype, method):
    from paper_2505_00227_gb300 import synthetic as S
    f = S.spectral(shape, seed=61, dtype=dtype).numpy()
    F = O.Field(f)
    m = getattr(B, method)
    ctx = B.Context(method=m)
    h = ctx.refactor(torch.from_numpy(f).cuda())
    for l in range(F.nlev):
        for g in range(F.ngroups):
            gb, gm, _ = h.group(l, g)
            assert gm == m
            G = _group_bytes(F, l, g)
            ref = {B.DC: G, B.HUFFMAN: O.huffman_encode(G), B.RLE: O.rle_encode(G)}[m]
            assert np.array_equal(gb, ref), (l, g)
    for tau in [1e-1, 1e-3, 1e-6]:
        out, info, st = h.retrieve(tau)
        err = np.abs(out.cpu().numpy().astype(np.float64) - f.astype(np.float64)).max()
        assert err <= info.est_linf
        if st == 0:
            assert info.est_linf <= tau * F.range
    # everything fetched: the same field as the hybrid coder gives
    out, info, st = h.retrieve(0.0)
    _, ref, _, _ = F.retrieve(0.0)
    assert np.array_equal(out.cpu().numpy().view(np.uint8), ref.view(np.uint8))


def test_bad_method_rejected(B):
    with pytest.raises(B.HpmdrError):
        B.Context(method=7)
