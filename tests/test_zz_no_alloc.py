"""hpmdr_encode_group_noalloc: the Algorithm 2 group encoder for callers that
cannot allocate device memory (its scratch is a static device array).  Checked
through the C ABI against hpmdr_encode_group, which allocates its scratch, on
two calls in a row (the shared array must not leak state between calls).
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MAX_BYTES = 16 << 20


def _encode_allocating(ctx, G):
    from paper_2505_00227_gb300 import binding
    cap = G.numel() * 3 + 8192
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    ln, m = ctypes.c_uint64(), ctypes.c_int()
    st = binding.lib().hpmdr_encode_group(ctx._p, ctypes.c_void_p(G.data_ptr()), G.numel(), -1,
                                          ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(ln),
                                          ctypes.byref(m))
    assert st == 0
    return out[: ln.value].cpu().numpy(), m.value


def _encode_noalloc(G, cap=None):
    from paper_2505_00227_gb300 import binding
    cap = cap if cap is not None else G.numel() * 3 + 8192
    out = torch.empty(max(cap, 1), dtype=torch.uint8, device="cuda")
    ln, m = ctypes.c_uint64(), ctypes.c_int()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = binding.lib().hpmdr_encode_group_noalloc(ctypes.c_void_p(G.data_ptr()), G.numel(), -1, 0, 0,
                                                  0, ctypes.c_void_p(out.data_ptr()), cap,
                                                  ctypes.byref(ln), ctypes.byref(m), stream)
    return st, out[: ln.value].cpu().numpy(), m.value


def test_noalloc_matches_allocating_encoder_twice():
    from paper_2505_00227_gb300 import binding
    ctx = binding.Context()
    rng = np.random.default_rng(42)
    first = np.zeros(300000, dtype=np.uint8)                      # Huffman, many chunks
    first[rng.integers(0, first.size, 2000)] = rng.integers(1, 256, 2000).astype(np.uint8)
    second = np.repeat(rng.integers(0, 256, 900), rng.integers(100, 400, 900)).astype(np.uint8)  # RLE
    third = rng.integers(0, 256, 70001).astype(np.uint8)          # direct copy, ragged
    for G_np in (first, second, third):
        G = torch.from_numpy(G_np).cuda()
        ref, mref = _encode_allocating(ctx, G)
        st, got, m = _encode_noalloc(G)
        assert st == 0 and m == mref
        assert np.array_equal(got, ref)


def test_noalloc_rejects_groups_beyond_its_scratch():
    G = torch.zeros(MAX_BYTES + 16, dtype=torch.uint8, device="cuda")
    st, _, _ = _encode_noalloc(G, cap=1024)
    assert st == -1  # HPMDR_ERR_ARG
