"""GPU parity on the full 512^3 FP32 field that the benchmark times.

The benchmark's field (Gaussian random field with P(k) ~ k^-11/3, rescaled to
[-1, 1], seed 2, made by the same generator call) is refactored by the CUDA
path in its benchmark launch configuration and by the CPU oracle; then six
incremental retrievals at relative L-infinity bounds 1e-1 .. 1e-6 run on the
same handle.  Bit-exact: the level bit lengths, every bitplane of every level,
every stored group (bytes, method, size estimates), the greedy sequence, the
selections, the 128-bit error estimates and the six reconstructions.  The FP32
tolerance (1e-6 x range) and the requested bounds are asserted as well.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu

TAUS = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6]
N = 512


@pytest.fixture(scope="module")
def case():
    from paper_2505_00227_gb300 import binding, synthetic
    binding.lib()
    fd = synthetic.spectral((N, N, N), seed=2, dtype=torch.float32, device="cuda")
    f = fd.cpu().numpy()
    ctx = binding.Context()
    h = ctx.refactor(fd)
    F = O.Field(f)
    yield f, fd, F, h
    h.free()
    ctx.close()


def test_refactor_512_bit_exact(case):
    f, fd, F, h = case
    info = h.field_info()
    assert info["nlevels"] == F.nlev
    assert info["E_f"] == F.E_f and info["input_exact"] == F.input_exact
    assert info["range"] == F.range
    for l in range(F.nlev):
        n, bl, ng, ex = h.level_info(l)
        assert (n, bl, ex) == F.levels[l], l
        assert np.array_equal(h.planes(l), F.planes(l).reshape(-1)), f"planes of level {l}"
        for g in range(F.ngroups):
            gb, m, est = h.group(l, g)
            ob, om, oH, oR = F.group(l, g)
            assert (m, est) == (om, (oH, oR)), (l, g)
            assert np.array_equal(gb, ob), f"stored bytes of level {l} group {g}"
    assert h.sequence() == F.sequence()


def test_incremental_retrievals_512_bit_exact(case):
    f, fd, F, h = case
    out = torch.empty_like(fd)
    prev = 0
    for tau in TAUS:
        tau_abs = tau * F.range
        out, info, st = h.retrieve(tau, out=out)
        rc, ref, g, E = F.retrieve(tau_abs)
        assert st == rc == 0
        assert info.groups == list(g) and info.est_linf == E
        got = out.cpu().numpy()
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), tau
        assert np.abs(got.astype(np.float64) - ref.astype(np.float64)).max() <= 1e-6 * F.range
        err = float(np.abs(got.astype(np.float64) - f.astype(np.float64)).max())
        assert err <= info.est_linf <= tau_abs
        assert info.bytes_fetched_total >= prev
        prev = info.bytes_fetched_total
