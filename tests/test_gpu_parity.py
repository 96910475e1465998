"""GPU parity: the sm_103a path through the C ABI against the CPU oracle.

Bit-exact for every integer and byte product (aligned integers via the
bitplanes, bitplane streams, stored group bytes, methods, estimates, greedy
sequence, 128-bit error estimates) and for the reconstructions, which are
integers converted once with round-to-nearest on both sides.  The FP
tolerance of the reconstruction (1e-6 x range for FP32, 1e-12 x range for
FP64) is asserted as well, and every retrieval must meet its bound.
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


def _spike(shape, at, value, extra=None):
    f = np.zeros(shape, dtype=np.float32)
    f[at] = np.float32(value)
    if extra is not None:
        f[extra[0]] = np.float32(extra[1])
    return f


def _fields():
    from paper_2505_00227_gb300 import synthetic as S
    rng = np.random.default_rng(11)
    return {
        "blobs64": S.blobs((64, 64, 64), seed=0).numpy(),
        "spectral_ragged": S.spectral((17, 23, 30), seed=4).numpy(),
        "spectral_2d_f64": S.spectral((1, 40, 33), seed=5, dtype=torch.float64).numpy(),
        "blobs_1d": S.blobs((1, 1, 300), seed=6).numpy(),
        "tiny_odd": rng.standard_normal((3, 5, 7)).astype(np.float32),
        "single": np.array([[[0.7]]], dtype=np.float32),
        "constant": np.full((5, 6, 7), -0.375, dtype=np.float32),
        "zero": np.zeros((4, 4, 9), dtype=np.float64),
        "integers": rng.integers(-50, 50, size=(9, 10, 11)).astype(np.float32),
        "f64_blobs": S.blobs((33, 20, 18), seed=8, dtype=torch.float64).numpy(),
        "long_x": S.spectral((2, 3, 2500), seed=9).numpy(),
        "subnormal_f32": (rng.standard_normal((6, 7, 8)) * 1e-40).astype(np.float32),
        # shapes whose large levels take the cell kernels (x extent a multiple of 64)
        "cells_ragged_yz": S.spectral((7, 37, 128), seed=12).numpy(),
        "cells_2d": S.blobs((1, 64, 128), seed=13).numpy(),
        "cells_three_words": S.spectral((5, 9, 192), seed=14).numpy(),
        "cells_256": S.spectral((24, 40, 256), seed=15).numpy(),
        # level x-extent 512, 1024 and 1536: the finest level takes the widest cell
        # tile (8 plane words, 256 cells per row of a tile, 4 rows), the tile of the
        # 512^3 field's finest level; 37 and 9 rows leave a ragged last row of tiles,
        # 1024 and 1536 put two and three tiles along x
        "cells_512": S.spectral((4, 6, 512), seed=25).numpy(),
        "cells_512_ragged": S.spectral((6, 37, 512), seed=28).numpy(),
        "cells_512_blobs": S.blobs((2, 9, 512), seed=27).numpy(),
        "cells_1024": S.spectral((3, 5, 1024), seed=26).numpy(),
        "cells_1536": S.spectral((2, 7, 1536), seed=29).numpy(),
        # FP64 levels of x-extent 128 .. 1024 take the cell kernels with 64 planes
        "cells_f64_128": S.spectral((8, 12, 128), seed=31, dtype=torch.float64).numpy(),
        "cells_f64_256_ragged": S.blobs((7, 37, 256), seed=33, dtype=torch.float64).numpy(),
        "cells_f64_512": S.spectral((4, 6, 512), seed=32, dtype=torch.float64).numpy(),
        "cells_f64_1024": S.spectral((2, 5, 1024), seed=34, dtype=torch.float64).numpy(),
        # a level maximum exactly at a power of two (C8 = 2^50): the FP32 estimate of
        # the level maximum is ambiguous there and the exact pass must decide
        "cells_power_of_two": _spike((8, 8, 128), (3, 5, 77), 2.0 ** -10),
        # all-zero finest level apart from one value below the fixed-point unit
        "cells_floored": _spike((8, 8, 128), (2, 2, 6), 1.0, extra=((4, 4, 9), 1e-30)),
        # the statistics pass decides input exactness from the least set-bit
        # exponent: integers are exact; values spanning the FP32 subnormals (E_f far
        # below -78) lose bits; a single half-unit value among exact ones loses bits
        "cells_integers": rng.integers(-1000, 1000, size=(6, 8, 128)).astype(np.float32),
        "cells_subnormal": (S.spectral((4, 8, 128), seed=36).numpy() *
                            np.float32(1e-36)).astype(np.float32),
        "cells_one_inexact": _spike((4, 8, 128), (1, 2, 3), 2.0 ** 40, extra=((3, 7, 100), 2.0 ** -9)),
        # values far below max|f|: the estimate's bound scales with max|f|
        "cells_wide_range": (S.spectral((8, 16, 128), seed=24).numpy() *
                             np.float32(1e-6)).astype(np.float32) +
                            _spike((8, 16, 128), (0, 0, 0), 3.0),
        # large levels of any size take the general cell kernels (staged transposes)
        "gcells_odd": S.spectral((45, 47, 49), seed=16).numpy(),
        "gcells_f64": S.blobs((40, 36, 44), seed=17, dtype=torch.float64).numpy(),
        "gcells_2d": S.spectral((1, 300, 250), seed=18).numpy(),
        "gcells_1d": S.blobs((1, 1, 70001), seed=19).numpy(),
        "gcells_two_levels": S.spectral((90, 100, 110), seed=20).numpy(),
    }


FIELDS = list(_fields())


def _pair(ctx, name):
    f = _fields()[name]
    F = O.Field(f)
    h = ctx.refactor(torch.from_numpy(f).cuda())
    return f, F, h


@pytest.mark.parametrize("name", FIELDS)
def test_refactor_bit_exact(ctx, name):
    f, F, h = _pair(ctx, name)
    info = h.field_info()
    assert info["nlevels"] == F.nlev
    assert info["E_f"] == F.E_f
    assert info["input_exact"] == F.input_exact
    assert info["range"] == F.range and info["vmin"] == F.vmin and info["vmax"] == F.vmax
    for l in range(F.nlev):
        n, bl, ng, ex = h.level_info(l)
        assert (n, bl, ex) == F.levels[l], l
        assert np.array_equal(h.planes(l), F.planes(l).reshape(-1)), f"planes of level {l}"
        for g in range(F.ngroups):
            gb, m, est = h.group(l, g)
            ob, om, oH, oR = F.group(l, g)
            assert m == om, (l, g)
            assert est == (oH, oR), (l, g)
            assert np.array_equal(gb, ob), f"stored bytes of level {l} group {g}"
    assert h.sequence() == F.sequence()


def _check_retrieval(f, F, out, info, st, tau_abs):
    rc, ref, g, E = F.retrieve(tau_abs)
    assert st == rc
    assert info.groups == list(g)
    assert info.est_linf == E
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint8), ref.view(np.uint8)), "reconstruction differs"
    rng = F.range if F.range > 0 else 1.0
    tol = 1e-6 if f.dtype == np.float32 else 1e-12
    assert np.abs(got.astype(np.float64) - ref.astype(np.float64)).max() <= tol * rng
    err = float(np.abs(got.astype(np.float64) - f.astype(np.float64)).max())
    assert err <= info.est_linf
    if st == 0:
        assert info.est_linf <= tau_abs


@pytest.mark.parametrize("name", FIELDS)
def test_incremental_retrieval_matches_oracle(ctx, name):
    f, F, h = _pair(ctx, name)
    prev_total = 0
    for tau in TAUS:
        tau_abs = tau * F.range
        out, info, st = h.retrieve(tau)
        _check_retrieval(f, F, out, info, st, tau_abs)
        assert info.bytes_fetched_total >= prev_total
        prev_total = info.bytes_fetched_total
    # a looser bound after tighter ones reuses the cached planes, masked
    out, info, st = h.retrieve(1e-2)
    _check_retrieval(f, F, out, info, st, 1e-2 * F.range)
    assert info.bytes_fetched_new == 0


@pytest.mark.parametrize("name", ["blobs64", "spectral_2d_f64", "long_x", "f64_blobs"])
def test_export_import_and_poisoned_cache(ctx, name):
    f, F, h = _pair(ctx, name)
    blob = h.export()
    h2 = ctx.import_handle(blob)
    assert h2.export() == blob
    for tau in (1e-3, 1e-6):
        out, info, st = h2.retrieve(tau)
        _check_retrieval(f, F, out, info, st, tau * F.range)
    # poisoning the coded groups' planes forces a real decode next time
    h.reset(poison=True)
    out, info, st = h.retrieve(1e-6)
    _check_retrieval(f, F, out, info, st, 1e-6 * F.range)


@pytest.mark.parametrize("tau_abs", [0.0, 1e-30, 0.5, 1e9])
def test_absolute_bounds_and_unattainable(ctx, tau_abs):
    f, F, h = _pair(ctx, "spectral_ragged")
    out, info, st = h.retrieve(tau_abs, absolute=True)
    _check_retrieval(f, F, out, info, st, tau_abs)


@pytest.mark.parametrize("name", ["cells_f64_512", "cells_f64_256_ragged"])
def test_f64_cells_deep_bounds(ctx, name):
    """FP64 cell levels retrieved with more than 32 planes (the low-half planes
    33..64): tight relative bounds, then every plane (absolute bound 0)."""
    f, F, h = _pair(ctx, name)
    for tau in (1e-9, 1e-12, 1e-14):
        out, info, st = h.retrieve(tau)
        _check_retrieval(f, F, out, info, st, tau * F.range)
    out, info, st = h.retrieve(0.0, absolute=True)
    _check_retrieval(f, F, out, info, st, 0.0)
    # the sequence stops once every bit of a level is fetched (bl <= 53 < 64),
    # which on the finest levels takes more than 32 planes
    assert max(info.groups) > 8


@pytest.mark.parametrize("n", [1, 31, 32, 1000, 1025, 4097, 70001])
@pytest.mark.parametrize("Bits", [32, 64])
def test_bitplane_stage_bit_exact(B, n, Bits):
    rng = np.random.default_rng(n + Bits)
    hi = 1 << Bits
    q = rng.integers(0, hi, size=n, dtype=np.uint64) if Bits == 64 else rng.integers(
        0, hi, size=n, dtype=np.uint64)
    q[::7] >>= np.uint64(Bits // 2)
    sign = (rng.random(n) < 0.5).astype(np.uint8)
    ref = O.bitplane_encode(q, sign, Bits).reshape(-1)
    qt = torch.from_numpy(q.view(np.int64) if Bits == 64 else q.astype(np.uint32).view(np.int32)).cuda()
    st = torch.from_numpy(sign).cuda()
    planes = B.bitplane_encode(qt, st, Bits)
    assert np.array_equal(planes.cpu().numpy().view(np.uint32), ref)
    for k in (0, 1, 5, Bits // 2, Bits - 1, Bits):
        qh, sh = B.bitplane_decode(planes, n, Bits, k)
        rq, rs = O.bitplane_decode(ref, n, Bits, k)
        got = qh.cpu().numpy().view(np.uint64 if Bits == 64 else np.uint32).astype(np.uint64)
        assert np.array_equal(got, rq), k
        assert np.array_equal(sh.cpu().numpy(), rs), k


def _groups():
    rng = np.random.default_rng(5)
    return {
        "zeros": np.zeros(50000, dtype=np.uint8),
        "ff": np.full(20000, 0xFF, dtype=np.uint8),
        "single": np.array([7], dtype=np.uint8),
        "random": rng.integers(0, 256, 40000).astype(np.uint8),
        "sparse": ((rng.random(70000) < 0.03) * rng.integers(1, 256, 70000)).astype(np.uint8),
        "runs": np.repeat(rng.integers(0, 5, 400), rng.integers(1, 300, 400)).astype(np.uint8),
        "ragged": rng.integers(0, 3, 16384 * 2 + 13).astype(np.uint8),
        # Fibonacci counts: an uncapped code would be 25 bits deep, so the
        # lengths are capped (counts halved and the code rebuilt, twice or more)
        "fibonacci": _fibonacci_group(),
        # code lengths 6..10 and mostly 8 / 9 (gcd 1): speculative parses of a
        # chunk's segments often stay out of step past the next segment, so
        # joins land several segments ahead
        "skewed": _weighted_group(1.0 / (1 + np.arange(256) / 40.0), 3 * 16384 + 100, 3),
        "near_uniform": _weighted_group(np.where(np.arange(256) < 200, 1.0, 0.55), 2 * 16384 + 77, 3),
    }


def _weighted_group(w, n, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(256, size=n, p=w / w.sum()).astype(np.uint8)


def _fibonacci_group():
    counts, a, b = [], 1, 1
    for _ in range(26):
        counts.append(a)
        a, b = b, a + b
    G = np.repeat(np.arange(26, dtype=np.uint8) * 7 + 1, counts)
    return np.random.default_rng(9).permutation(G).astype(np.uint8)


@pytest.mark.parametrize("name", list(_groups()))
@pytest.mark.parametrize("force", [-1, 0, 1, 2])
def test_group_coders_bit_exact(ctx, name, force):
    G = _groups()[name]
    Gt = torch.from_numpy(G).cuda()
    data, m = ctx.encode_group(Gt, force=force, cap=G.size * 3 + 8192)
    if force == -1:
        ref, om = O.hybrid_encode(G)
        assert m == om
    elif force == 0:
        ref = G
    elif force == 1:
        ref = O.huffman_encode(G)
    else:
        ref = O.rle_encode(G)
    assert np.array_equal(data.cpu().numpy(), ref)
    st, back = ctx.decode_group(data, m, G.size)
    assert st == 0 and np.array_equal(back.cpu().numpy(), G)


@pytest.mark.parametrize("method", [1, 2])
def test_decoders_flag_corruption(ctx, method):
    G = _groups()["runs"]
    ref = O.huffman_encode(G) if method == 1 else O.rle_encode(G)
    bad = ref.copy()
    bad[12] ^= 0x40  # nchunks field
    st, _ = ctx.decode_group(torch.from_numpy(bad).cuda(), method, G.size)
    assert st == -4
    st, _ = ctx.decode_group(torch.from_numpy(ref[: ref.size // 2].copy()).cuda(), method, G.size)
    assert st == -4


def test_invalid_fields_rejected(ctx, B):
    bad = torch.tensor([1.0, float("nan"), 2.0], device="cuda")
    with pytest.raises(B.HpmdrError) as e:
        ctx.refactor(bad)
    assert e.value.status == B.ERR_ARG
    big = torch.tensor([2.0 ** 125], device="cuda")
    with pytest.raises(B.HpmdrError):
        ctx.refactor(big)


def test_host_buffers_round_trip(ctx):
    f = _fields()["spectral_ragged"]
    F = O.Field(f)
    h = ctx.refactor(torch.from_numpy(f))  # host input
    out = torch.empty(f.shape, dtype=torch.float32)  # host output
    out, info, st = h.retrieve(1e-4, out=out)
    _check_retrieval(f, F, out, info, st, 1e-4 * F.range)


def test_qoi_vmag(ctx):
    from paper_2505_00227_gb300 import synthetic as S
    vs = [S.spectral((20, 21, 22), seed=s).numpy() for s in (11, 12, 13)]
    Fs = [O.Field(v) for v in vs]
    hs = [ctx.refactor(torch.from_numpy(v).cuda()) for v in vs]
    ctx.prepare_vmag(hs, *[torch.from_numpy(v).cuda() for v in vs])
    q, qmin, qmax = O.vmag_field(*vs)
    for tau in (1e-1, 1e-3, 1e-5):
        outs = [torch.empty(v.shape, dtype=torch.float32, device="cuda") for v in vs]
        vm, infos, st = ctx.retrieve_qoi_vmag(hs, tau, outs=outs)
        tq = tau * (qmax - qmin)
        eps = O.qoi_component_bound(tq, qmax)
        refs = []
        for c in range(3):
            rc, ref, g, E = Fs[c].retrieve(eps)
            assert np.array_equal(outs[c].cpu().numpy().view(np.uint32), ref.view(np.uint32))
            assert infos[c].est_linf == E
            refs.append(ref)
        qref, _, _ = O.vmag_field(*refs)
        assert np.array_equal(vm.cpu().numpy().view(np.uint32), qref.view(np.uint32))
        est = O.qoi_estimate(*[infos[c].est_linf for c in range(3)], qmax)
        assert infos[3].est_linf == est
        actual = float(np.abs(qref.astype(np.float64) - q.astype(np.float64)).max())
        assert actual <= est <= tq and st == 0
