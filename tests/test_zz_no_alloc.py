"""hpmdr_encode_group_noalloc: the group encoder of hpmdr_encode_group for
callers that cannot allocate device memory (a solver that owns all of HBM, or
one that forbids cudaMalloc/cudaFree between steps); its scratch is a static
device array shared by every call.

Checked through the C ABI against the CPU oracle's coders and against
hpmdr_encode_group (which allocates its scratch): three inputs that take the
Huffman, RLE and direct-copy branches, forced coders, non-default thresholds,
two calls in a row, and a call whose output buffer is too small followed by a
normal call (no state may leak through the shared array).  This file is
collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu

MAX_BYTES = 16 << 20
DC, HUFFMAN, RLE = 0, 1, 2


def _encode_allocating(ctx, G, force=-1):
    from paper_2505_00227_gb300 import binding
    cap = G.numel() * 3 + 8192
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    ln, m = ctypes.c_uint64(), ctypes.c_int()
    st = binding.lib().hpmdr_encode_group(ctx._p, ctypes.c_void_p(G.data_ptr()), G.numel(), force,
                                          ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(ln),
                                          ctypes.byref(m))
    assert st == 0
    return out[: ln.value].cpu().numpy(), m.value


def _encode_noalloc(G, cap=None, force=-1, Ts=0, cr_num=0, cr_den=0):
    from paper_2505_00227_gb300 import binding
    cap = cap if cap is not None else G.numel() * 3 + 8192
    out = torch.empty(max(cap, 1), dtype=torch.uint8, device="cuda")
    ln, m = ctypes.c_uint64(), ctypes.c_int()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = binding.lib().hpmdr_encode_group_noalloc(ctypes.c_void_p(G.data_ptr()), G.numel(), force,
                                                  Ts, cr_num, cr_den,
                                                  ctypes.c_void_p(out.data_ptr()), cap,
                                                  ctypes.byref(ln), ctypes.byref(m), stream)
    return st, out[: ln.value].cpu().numpy(), m.value


def _inputs():
    rng = np.random.default_rng(42)
    huff = np.zeros(300000, dtype=np.uint8)  # sparse bytes over many chunks: Huffman
    huff[rng.integers(0, huff.size, 2000)] = rng.integers(1, 256, 2000).astype(np.uint8)
    rle = np.repeat(rng.integers(0, 256, 900), rng.integers(100, 400, 900)).astype(np.uint8)
    dc = rng.integers(0, 256, 70001).astype(np.uint8)  # incompressible, ragged: direct copy
    return [(huff, HUFFMAN), (rle, RLE), (dc, DC)]


def test_noalloc_matches_oracle_and_allocating_encoder_twice():
    from paper_2505_00227_gb300 import binding
    ctx = binding.Context()
    for rep in range(2):  # two passes: the shared array must not carry state over
        for G_np, expect in _inputs():
            G = torch.from_numpy(G_np).cuda()
            ref, mref = O.hybrid_encode(G_np)
            assert mref == expect
            alloc, malloc = _encode_allocating(ctx, G)
            st, got, m = _encode_noalloc(G)
            assert st == 0 and m == mref == malloc, (rep, expect)
            assert np.array_equal(got, ref) and np.array_equal(got, alloc), (rep, expect)


@pytest.mark.parametrize("force", [0, 1, 2])
def test_noalloc_forced_coders_match_oracle(force):
    coder = {0: lambda G: G, 1: O.huffman_encode, 2: O.rle_encode}[force]
    for G_np, _ in _inputs():
        G = torch.from_numpy(G_np).cuda()
        st, got, m = _encode_noalloc(G, force=force)
        assert st == 0 and m == force
        assert np.array_equal(got, coder(G_np)), force


@pytest.mark.parametrize("Ts,cr_num,cr_den", [(100000, 1, 1), (4096, 4, 1), (1 << 20, 2, 1),
                                              (8192, 3, 2)])
def test_noalloc_thresholds_match_oracle_and_context(Ts, cr_num, cr_den):
    from paper_2505_00227_gb300 import binding
    ctx = binding.Context(size_threshold=Ts, cr_num=cr_num, cr_den=cr_den)
    for G_np, _ in _inputs():
        G = torch.from_numpy(G_np).cuda()
        ref, mref = O.hybrid_encode(G_np, Ts=Ts, cr_num=cr_num, cr_den=cr_den)
        alloc, malloc = _encode_allocating(ctx, G)
        st, got, m = _encode_noalloc(G, Ts=Ts, cr_num=cr_num, cr_den=cr_den)
        assert st == 0 and m == mref == malloc
        assert np.array_equal(got, ref) and np.array_equal(got, alloc)


def test_noalloc_small_cap_then_normal_call():
    huff, _ = _inputs()[0]
    G = torch.from_numpy(huff).cuda()
    ref, mref = O.hybrid_encode(huff)
    st, _, _ = _encode_noalloc(G, cap=64)  # the coded bytes do not fit
    assert st == -1  # HPMDR_ERR_ARG
    st, got, m = _encode_noalloc(G)
    assert st == 0 and m == mref and np.array_equal(got, ref)
    dc, _ = _inputs()[2]
    st, _, m = _encode_noalloc(torch.from_numpy(dc).cuda(), cap=1000)  # direct copy, cap < S
    assert st == -1 and m == DC
    st, got, m = _encode_noalloc(G)
    assert st == 0 and m == mref and np.array_equal(got, ref)


def test_noalloc_rejects_groups_beyond_its_scratch():
    G = torch.zeros(MAX_BYTES + 16, dtype=torch.uint8, device="cuda")
    st, _, _ = _encode_noalloc(G, cap=1024)
    assert st == -1  # HPMDR_ERR_ARG
