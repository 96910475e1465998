"""The bitplane encoder designs of Sec. 4 (locality block, register shuffling
with ballot / shift / match-any / reduce, register block) on the GPU: every
design writes the oracle's Algorithm 1 planes byte for byte and decodes them as
the oracle does, for ragged sizes (1, one partial word, one full word, partial
128-element groups, several tiles) and every number of kept planes tested."""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu

DESIGNS = ["register_block", "locality_block", "shuffle_ballot", "shuffle_shift",
           "shuffle_match_any", "shuffle_reduce"]


@pytest.fixture(scope="module")
def B():
    from paper_2505_00227_gb300 import binding
    binding.lib()
    return binding


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    q = rng.integers(0, 1 << 32, size=n, dtype=np.uint64)
    q[::5] >>= np.uint64(20)  # leading zero planes
    q[3::11] = 0
    q[7::13] = 0xffffffff
    sign = (rng.random(n) < 0.4).astype(np.uint8)
    sign[::9] = 3  # any nonzero byte is a negative sign
    return q, sign


@pytest.mark.parametrize("n", [1, 31, 32, 33, 127, 1000, 1025, 4097, 70001, 1 << 20])
@pytest.mark.parametrize("design", DESIGNS)
def test_design_matches_algorithm1(B, design, n):
    q, sign = _inputs(n, n)
    ref = O.bitplane_encode(q, (sign != 0).astype(np.uint8), 32).reshape(-1)
    qt = torch.from_numpy(q.astype(np.uint32).view(np.int32)).cuda()
    st = torch.from_numpy(sign).cuda()
    d = B.BP_DESIGNS[design]
    planes = B.bitplane_encode_design(qt, st, d)
    assert np.array_equal(planes.cpu().numpy().view(np.uint32), ref)
    for k in (0, 1, 4, 13, 31, 32):
        qh, sh = B.bitplane_decode_design(planes, n, d, k)
        rq, rs = O.bitplane_decode(ref, n, 32, k)
        assert np.array_equal(qh.cpu().numpy().view(np.uint32).astype(np.uint64), rq), k
        assert np.array_equal(sh.cpu().numpy(), rs), k


def test_design_padding_is_zero_over_garbage(B):
    n = 1000  # W = 32 words per plane, 31.25 of them in use
    q, sign = _inputs(n, 3)
    qt = torch.from_numpy(q.astype(np.uint32).view(np.int32)).cuda()
    st = torch.from_numpy(sign).cuda()
    W = 4 * ((n + 127) // 128)
    for d in range(6):
        planes = torch.full((33 * W,), -1, dtype=torch.int32, device="cuda")
        B.bitplane_encode_design(qt, st, d, planes=planes)
        p = planes.cpu().numpy().view(np.uint32).reshape(33, W)
        assert not p[:, n // 32 + 1:].any() and not (p[:, n // 32] >> (n % 32)).any(), d


def test_design_rejects_bad_arguments(B):
    q = torch.zeros(65, dtype=torch.int32, device="cuda")
    s = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.HpmdrError):
        B.bitplane_encode_design(q, s, 6)
    with pytest.raises(B.HpmdrError):
        B.bitplane_encode_design(q[1:], s, 1)  # q not 16-byte aligned
    planes = B.bitplane_encode_design(q[:64], s, 2)
    with pytest.raises(B.HpmdrError):
        B.bitplane_decode_design(planes, 64, 2, 33)
