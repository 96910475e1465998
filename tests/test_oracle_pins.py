"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks one oracle step against a closed form, a hand-derived
example under tests/golden/, an invariant of the mathematics, an independent
library routine, or brute force over tiny inputs (the paper prints no worked
numeric example).  Runs on the CPU only.
"""
import heapq
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import pyoracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ geometry
def _brute_levels(shape):
    """Assign every node to a level straight from the definition."""
    nz, ny, nx = shape
    maxn = max(shape)
    hs = []
    h = 1
    while h < maxn:
        hs.append(h)
        h *= 2
    counts = {0: 0}
    for h in hs:
        counts[h] = 0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if (z, y, x) == (0, 0, 0):
                    counts[0] += 1
                    continue
                found = [h for h in hs
                         if z % h == 0 and y % h == 0 and x % h == 0
                         and not (z % (2 * h) == 0 and y % (2 * h) == 0 and x % (2 * h) == 0)]
                assert len(found) == 1
                counts[found[0]] += 1
    L = len(hs)
    return [counts[0]] + [counts[1 << (L - l)] for l in range(1, L + 1)]


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 2), (1, 1, 7), (1, 5, 3), (3, 4, 5),
                                   (2, 9, 6), (8, 8, 8), (5, 1, 17)])
def test_level_sizes_match_definition(shape):
    nlev = O.num_levels(shape)
    sizes = [O.level_size(shape, l) for l in range(nlev)]
    assert sizes == _brute_levels(shape)
    assert sum(sizes) == int(np.prod(shape))


def test_level_sizes_64cube_worked_count():
    # every node but the 32^3 even ones is in the finest level, and so on
    shape = (64, 64, 64)
    sizes = [O.level_size(shape, l) for l in range(O.num_levels(shape))]
    assert sizes == [1, 7, 56, 448, 3584, 28672, 229376]


def test_plane_words_padding():
    assert [O.plane_words(n) for n in (1, 127, 128, 129, 256)] == [4, 4, 4, 8, 8]


# ------------------------------------------------------------ fixed point
@pytest.mark.parametrize("maxabs", [1.0, 0.999, 3.0, 2.0 ** -130, 1e-30, 12345.678, 2.0 ** 100])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_exponent_bound_is_frexp(maxabs, dt):
    f = np.array([0.0, -dt(maxabs), dt(maxabs) / 3], dtype=dt)
    rc, st = O.field_stats(f)
    assert rc == O.OK
    m = float(dt(maxabs))
    assert st.E_f == math.frexp(m)[1]  # m < 2^e, m >= 2^(e-1)
    assert st.range == pytest.approx(float(f.max()) - float(f.min()), rel=0, abs=0)


def test_fixed_point_values():
    f = np.array([1.0, -0.75, 2.0 ** -60, 0.5 + 2.0 ** -24], dtype=np.float32)
    E = 1  # max|f| = 1 < 2^1
    assert O.fixed_point(f, 0, E) == (2 ** 47, False)
    assert O.fixed_point(f, 1, E) == (-3 * 2 ** 45, False)
    assert O.fixed_point(f, 2, E) == (0, True)          # below U = 2^-47: floored away
    assert O.fixed_point(f, 3, E) == (2 ** 46 + 2 ** 23, False)
    d = np.array([1.0 + 2.0 ** -52], dtype=np.float64)  # 53 bits do not fit in 48
    assert O.fixed_point(d, 0, 1) == (2 ** 47, True)


def test_stats_reject_nonfinite_and_huge():
    assert O.field_stats(np.array([1.0, np.nan], dtype=np.float32))[0] == O.ERR_ARG
    assert O.field_stats(np.array([1.0, np.inf], dtype=np.float64))[0] == O.ERR_ARG
    assert O.field_stats(np.array([2.0 ** 125], dtype=np.float32))[0] == O.ERR_ARG


def test_zero_field_is_exact():
    rc, st = O.field_stats(np.zeros(10, dtype=np.float32))
    assert rc == O.OK and st.E_f == 0 and st.input_exact == 1


# ------------------------------------------------------------ decomposition
def test_decompose_1d_golden():
    f = np.array([0, 1, 4, 9], dtype=np.float32).reshape(1, 1, 4)
    rc, st = O.field_stats(f)
    U = 2.0 ** (st.E_f - 48)
    assert st.E_f == 4
    for row in _golden_rows("decompose_1d.txt"):
        l, vals = int(row[0]), [int(v) for v in row[1:]]
        c8 = O.level_coeffs(f, st.E_f, l)
        expect = [int(8 * v / U) for v in vals] if l > 0 else [int(8 * 0 / U)]
        assert c8.tolist() == expect


def _grid(shape):
    z, y, x = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    return z, y, x


@pytest.mark.parametrize("shape", [(9, 9, 9), (5, 17, 9), (1, 1, 33), (1, 17, 5)])
def test_trilinear_field_closed_form(shape):
    # multilinear interpolation reproduces a trilinear function exactly, so a
    # detail coefficient is zero unless a right neighbour falls outside the
    # grid; on 2^k+1 grids that happens only at h = n_d - 1 on axis d, where the
    # axis collapses to its left neighbour and the coefficient becomes
    # f(i) - f(i with the clamped coordinates moved left by h).
    z, y, x = _grid(shape)
    f = (3 + 2 * x - 5 * y + 7 * z + x * y - 2 * x * z + 3 * y * z + x * y * z).astype(np.float32)
    rc, st = O.field_stats(f)
    assert st.input_exact
    U = Fraction(2) ** (st.E_f - 48)
    L = O.num_levels(shape) - 1
    for l in range(1, L + 1):
        h = 1 << (L - l)
        got = [Fraction(int(v)) * U / 8 for v in O.level_coeffs(f, st.E_f, l)]
        expect = []
        for t in range(1, 8):
            odd = ((t >> 2) & 1, (t >> 1) & 1, t & 1)
            rng = [range(h, n, 2 * h) if o else range(0, n, 2 * h) for n, o in zip(shape, odd)]
            for a in rng[0]:
                for b in rng[1]:
                    for c in rng[2]:
                        i = [a, b, c]
                        j = [v - h if (o and v + h >= n) else v for v, o, n in zip(i, odd, shape)]
                        expect.append(Fraction(float(f[tuple(i)])) - Fraction(float(f[tuple(j)])))
        assert got == expect, l
        if l > 1 and shape[0] == shape[1] == shape[2]:
            assert not any(got)


def test_quadratic_field_closed_form():
    # f = x^2 + y^2 + z^2: on a node with odd-axis set O at half-stride h the
    # multilinear interpolant is f + |O| h^2, so the coefficient is -|O| h^2
    # (below the top level, where no right neighbour is clamped on a 9^3 grid)
    shape = (9, 9, 9)
    z, y, x = _grid(shape)
    f = (x * x + y * y + z * z).astype(np.float32)
    rc, st = O.field_stats(f)
    U = Fraction(2) ** (st.E_f - 48)
    L = O.num_levels(shape) - 1
    for l in range(2, L + 1):
        h = 1 << (L - l)
        c8 = O.level_coeffs(f, st.E_f, l)
        g = [(s + h - 1) // h for s in shape]
        j = 0
        for t in range(1, 8):
            odd = ((t >> 2) & 1, (t >> 1) & 1, t & 1)
            cnt = [(g[d] // 2) if odd[d] else ((g[d] + 1) // 2) for d in range(3)]
            n = cnt[0] * cnt[1] * cnt[2]
            expect = -sum(odd) * h * h
            assert all(Fraction(int(v)) * U / 8 == expect for v in c8[j:j + n]), (l, t)
            j += n
        assert j == c8.size


def test_power_of_two_grid_only_boundary_nonzero():
    # on n = 2^k the rightmost odd node of each level clamps to its left
    # neighbour; for f = x the coefficient there is f(x) - f(x-h) = h, else 0
    f = np.arange(16, dtype=np.float32).reshape(1, 1, 16)
    rc, st = O.field_stats(f)
    U = Fraction(2) ** (st.E_f - 48)
    L = O.num_levels(f.shape) - 1
    for l in range(1, L + 1):
        h = 1 << (L - l)
        c8 = [Fraction(int(v)) * U / 8 for v in O.level_coeffs(f, st.E_f, l)]
        xs = list(range(h, 16, 2 * h))
        for xv, c in zip(xs, c8):
            assert c == (h if xv + h >= 16 else 0)


# ---------------------------------------------------- quantize + Algorithm 1
def test_quantize_alignment():
    C8 = np.array([0, 5, -12, 7, 1], dtype=np.int64)
    bl = O.bitlen_max(C8)
    assert bl == (12).bit_length()
    q, s = O.quantize(C8, 8, bl)
    assert q.tolist() == [0, 5 << 4, 12 << 4, 7 << 4, 1 << 4]
    assert s.tolist() == [0, 0, 1, 0, 0]
    q, s = O.quantize(C8, 2, bl)  # B < bl: floor of the magnitude
    assert q.tolist() == [0, 1, 3, 1, 0]
    assert O.level_exact(C8, 8, bl) and not O.level_exact(C8, 2, bl)
    big = np.array([(1 << 52) - 1, -(1 << 40)], dtype=np.int64)
    bl = O.bitlen_max(big)
    q, _ = O.quantize(big, 32, bl)
    assert bl == 52 and q[0] == (1 << 32) - 1 and q[0] < (1 << 32)


def test_dequantize_is_truncation():
    bl, B = 10, 4
    for mag in range(0, 1 << bl):
        q = mag >> (bl - B)
        for k in range(B + 1):
            qk = q & (((1 << B) - 1) ^ ((1 << (B - k)) - 1))
            c = O.dequantize(qk, 1, B, bl)
            assert c <= 0 and 0 <= mag - (-c) < (1 << (bl - k))


def test_bitplane_bruteforce_roundtrip_b6():
    # every q in [0, 2^6)^4 with every k: decode keeps exactly the top k bits
    B = 6
    vals = np.arange(64, dtype=np.uint64)
    grids = np.stack(np.meshgrid(vals, vals, vals, vals, indexing="ij"), -1).reshape(-1, 4)
    rng = np.random.default_rng(0)
    for q in grids[rng.permutation(len(grids))[:4096]].tolist() + [[63, 0, 1, 32], [0, 0, 0, 0]]:
        q = np.array(q, dtype=np.uint64)
        s = (q & 1).astype(np.uint8)
        planes = O.bitplane_encode(q, s, B)
        assert planes.shape == (B + 1, 4)
        for k in range(B + 1):
            qh, sh = O.bitplane_decode(planes, 4, B, k)
            mask = ((1 << B) - 1) ^ ((1 << (B - k)) - 1)
            assert qh.tolist() == [int(v) & mask for v in q]
            assert sh.tolist() == (s.tolist() if k > 0 else [0, 0, 0, 0])


def test_bitplane_layout_hand_example():
    # plane p = 0 holds the MSB; element j sits at word j>>5, bit j&31
    n, B = 40, 8
    q = np.zeros(n, dtype=np.uint64)
    s = np.zeros(n, dtype=np.uint8)
    q[0] = 0x80       # MSB of element 0 -> plane 1 (first magnitude plane), bit 0
    q[33] = 0x01      # LSB of element 33 -> last plane, word 1, bit 1
    s[35] = 1         # sign of element 35 -> plane 0, word 1, bit 3
    planes = O.bitplane_encode(q, s, B)
    expect = np.zeros((B + 1, 4), dtype=np.uint32)
    expect[1, 0] = 1
    expect[B, 1] = 1 << 1
    expect[0, 1] = 1 << 3
    assert (planes == expect).all()


def test_group_slices():
    W = 8
    assert O.group_slice(W, 0) == (0, 5 * W * 4)
    assert O.group_slice(W, 1) == (5 * W * 4, 4 * W * 4)
    assert O.group_slice(W, 7) == ((4 * 7 + 1) * W * 4, 4 * W * 4)


# ---------------------------------------------------------------- Huffman
def _optimal_cost(freqs):
    """Minimum total code length of any prefix code (textbook Huffman, heapq)."""
    h = [f for f in freqs if f > 0]
    if len(h) <= 1:
        return sum(h)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def test_huffman_golden_tie_break_and_codes():
    hist = np.zeros(256, dtype=np.uint64)
    rows = _golden_rows("huffman_small.txt")
    freq = {97: 5, 98: 2, 99: 1, 100: 1}
    for s, f in freq.items():
        hist[s] = f
    lens = O.huffman_lengths(hist)
    for sym, ln, code in rows:
        assert lens[int(sym)] == int(ln)
    # encode "abacabad a a" style input and check the canonical bits
    G = np.array([97] * 5 + [98] * 2 + [99, 100], dtype=np.uint8)
    enc = O.huffman_encode(G)
    codes = {int(s): c for s, _, c in rows}
    bits = "".join(codes[int(b)] for b in G)
    payload = enc[272 + 8:]
    word = int.from_bytes(payload[:4].tobytes(), "little")
    assert format(word, "032b")[:len(bits)] == bits
    assert int(format(word, "032b")[len(bits):] or "0", 2) == 0


@pytest.mark.parametrize("seed", range(6))
def test_huffman_optimal_and_kraft(seed):
    rng = np.random.default_rng(seed)
    nsym = int(rng.integers(2, 256))
    hist = np.zeros(256, dtype=np.uint64)
    syms = rng.choice(256, nsym, replace=False)
    hist[syms] = rng.integers(1, 10000, nsym)
    lens = O.huffman_lengths(hist).astype(np.int64)
    if lens.max() <= 16:
        assert sum(Fraction(1, 2 ** int(l)) for l in lens if l) == 1
        assert int((hist.astype(np.int64) * lens).sum()) == _optimal_cost(hist.tolist())


def test_huffman_dyadic_lengths():
    hist = np.zeros(256, dtype=np.uint64)
    for i, e in enumerate([1, 2, 3, 4, 5, 6, 7, 7]):
        hist[10 + i] = 2 ** (7 - e)
    lens = O.huffman_lengths(hist)
    assert [int(lens[10 + i]) for i in range(8)] == [1, 2, 3, 4, 5, 6, 7, 7]


def test_huffman_length_cap():
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    hist = np.zeros(256, dtype=np.uint64)
    hist[:30] = fib
    lens = O.huffman_lengths(hist)
    assert 12 <= lens.max() <= 16  # uncapped, Fibonacci counts would reach depth 29
    assert sum(Fraction(1, 2 ** int(l)) for l in lens if l) <= 1
    assert (lens[:30] > 0).all()


def _coder_inputs():
    rng = np.random.default_rng(7)
    yield np.zeros(5000, dtype=np.uint8)
    yield np.full(40000, 0xFF, dtype=np.uint8)
    yield np.full(1, 3, dtype=np.uint8)
    yield rng.integers(0, 256, 50000).astype(np.uint8)                 # 4 chunks, ragged
    yield (rng.random(70000) < 0.05).astype(np.uint8) * rng.integers(0, 256, 70000).astype(np.uint8)
    yield np.repeat(rng.integers(0, 4, 300), rng.integers(1, 400, 300)).astype(np.uint8)
    yield np.array([1, 2], dtype=np.uint8)


@pytest.mark.parametrize("case", range(7))
def test_huffman_roundtrip_and_estimate(case):
    G = list(_coder_inputs())[case]
    enc = O.huffman_encode(G)
    rc, dec = O.huffman_decode(enc, G.size)
    assert rc == O.OK and (dec == G).all()
    lens = O.huffman_lengths(O.histogram(G))
    est = O.huffman_estimate(O.histogram(G), lens, G.size)
    nchunks = -(-G.size // O.CHUNK)
    assert est >= enc.size and est - enc.size <= 4 * nchunks + 1


@pytest.mark.parametrize("case", range(7))
def test_rle_roundtrip_and_exact_estimate(case):
    G = list(_coder_inputs())[case]
    enc = O.rle_encode(G)
    rc, dec = O.rle_decode(enc, G.size)
    assert rc == O.OK and (dec == G).all()
    assert O.rle_estimate(G) == enc.size


def test_rle_golden():
    payload = bytes(int(b, 16) for b in _golden_rows("rle_small.txt")[0])
    G = np.array([5] * 3 + [7] + [0] * 200, dtype=np.uint8)
    enc = O.rle_encode(G)
    hdr = 8 + 4 + 4 + 4 * 2
    assert enc[:8].tobytes() == (204).to_bytes(8, "little")
    assert enc[16:24].tobytes() == (0).to_bytes(4, "little") + (7).to_bytes(4, "little")
    assert enc[hdr:].tobytes() == payload


def test_rle_runs_break_at_chunks():
    G = np.zeros(O.CHUNK + 10, dtype=np.uint8)
    enc = O.rle_encode(G)
    # two runs: 16384 (LEB 16383 = 2 bytes) and 10 (1 byte)
    assert enc.size == (8 + 4 + 4 + 4 * 3) + (1 + 2) + (1 + 1)


def test_decoders_reject_corruption():
    G = np.arange(3000, dtype=np.uint32).astype(np.uint8)
    for enc_fn, dec_fn in ((O.huffman_encode, O.huffman_decode), (O.rle_encode, O.rle_decode)):
        enc = enc_fn(G)
        rc, _ = dec_fn(enc[:-3], G.size)
        assert rc == O.ERR_CORRUPT
        bad = enc.copy()
        bad[8] ^= 1  # chunk_bytes field
        assert dec_fn(bad, G.size)[0] == O.ERR_CORRUPT


# ------------------------------------------------------------- Algorithm 2
def test_hybrid_truth_table():
    cfg = O.hybrid_cfg(Ts=4096, cr_num=2, cr_den=1)
    S = 10000
    # S <= T_s: direct copy whatever the estimates
    assert O.hybrid_choose(4096, 1, 1, cfg) == O.DC
    # Huffman first when its ratio passes, even if RLE is better
    assert O.hybrid_choose(S, 4999, 10, cfg) == O.HUFFMAN
    # ratio exactly T_cr is not "greater": falls through
    assert O.hybrid_choose(S, 5000, 4999, cfg) == O.RLE
    assert O.hybrid_choose(S, 5000, 5000, cfg) == O.DC
    assert O.hybrid_choose(S, 20000, 20000, cfg) == O.DC
    cfg4 = O.hybrid_cfg(Ts=4096, cr_num=4, cr_den=1)
    assert O.hybrid_choose(S, 2499, 9999, cfg4) == O.HUFFMAN
    assert O.hybrid_choose(S, 2500, 2499, cfg4) == O.RLE


# -------------------------------------------------- estimator and selection
def test_tau_units_floor_exact():
    for tau, E_f, B in [(0.3, 2, 32), (1e-6, 1, 32), (2.5e-12, 0, 64), (7.0, -3, 64)]:
        u = O.tau_units(tau, E_f, B)
        exact = Fraction(tau) / (Fraction(2) ** (E_f - 51 - B))
        assert u == math.floor(exact)
    assert O.tau_units(0.0, 0, 32) == 0
    assert O.tau_units(1e300, 0, 64) == 1 << 127


def _meta_from_field(F):
    sizes = F.group_sizes()
    return O.make_meta(F.nlev, F.B, F.dtype_code, F.E_f, F.input_exact,
                       [lv[1] for lv in F.levels], [lv[2] for lv in F.levels], sizes)


def _fields():
    from paper_2505_00227_gb300 import synthetic as S
    yield S.blobs((32, 32, 32), seed=0).numpy()
    yield S.spectral((17, 23, 30), seed=4).numpy()
    yield S.spectral((1, 40, 33), seed=5, dtype=__import__("torch").float64).numpy()
    yield S.blobs((1, 1, 300), seed=6).numpy()


@pytest.mark.parametrize("case", range(4))
def test_every_retrieval_meets_its_bound(case):
    f = list(_fields())[case]
    F = O.Field(f)
    seq = F.sequence()
    prev = None
    for tau_rel in [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6]:
        tau = tau_rel * F.range
        rc, out, g, E = F.retrieve(tau)
        assert rc == O.OK
        err = float(np.abs(out.astype(np.float64) - f.astype(np.float64)).max())
        assert err <= E <= tau
        # the selection is a prefix of the tau-independent greedy sequence
        counts = np.zeros(F.nlev, dtype=np.int64)
        for i in range(int(g.sum())):
            counts[seq[i]] += 1
        assert (counts == g).all()
        if prev is not None:
            assert (g >= prev).all()  # monotone in tau
        prev = g


@pytest.mark.parametrize("case", range(4))
def test_all_planes_lossless_up_to_quantization(case):
    f = list(_fields())[case]
    F = O.Field(f)
    B = F.B
    g = [F.ngroups] * F.nlev
    rc, out = F.reconstruct(g)
    U = 2.0 ** (F.E_f - 48)
    step = sum(2.0 ** (bl - B - 3) for (_, bl, ex) in F.levels if bl > B and not ex) * U
    half_ulp = 2.0 ** (F.E_f - 24) if F.B == 32 else 2.0 ** (F.E_f - 53)
    bound = step + (F.nlev + 1) * U + half_ulp
    err = float(np.abs(out.astype(np.float64) - f.astype(np.float64)).max())
    assert err <= bound
    if F.B == 64:
        # B = 64 >= bl on every level: the fixed-point field comes back exactly
        Ff = np.array([O.fixed_point(f.reshape(-1), i, F.E_f)[0] for i in range(0, f.size, 97)])
        back = np.array([O.fixed_point(out.reshape(-1), i, F.E_f)[0] for i in range(0, f.size, 97)])
        assert (Ff == back).all()


def test_integer_field_full_retrieval_is_exact():
    rng = np.random.default_rng(1)
    f = rng.integers(-50, 50, size=(9, 10, 11)).astype(np.float32)
    F = O.Field(f)
    assert F.input_exact
    rc, out, g, E = F.retrieve(0.0)
    assert rc == O.OK and E == 0.0 and (out == f).all()


def test_constant_field_root_only():
    f = np.full((5, 6, 7), 0.375, dtype=np.float32)
    F = O.Field(f)
    assert F.range == 0.0
    rc, out, g, E = F.retrieve(0.0)
    assert rc == O.OK and E == 0.0 and (out == f).all()
    assert g[0] == F.ngroups and not g[1:].any()


def test_unattainable_reports_best():
    f = np.linspace(-1, 1, 1000, dtype=np.float64).reshape(1, 1, 1000) + 1e-9
    F = O.Field(f)
    rc, out, g, E = F.retrieve(1e-20)
    assert rc == O.ERR_UNATTAINABLE and E > 1e-20
    assert float(np.abs(out - f).max()) <= E


def test_greedy_tie_goes_to_smaller_level():
    sizes = [np.full(8, 100, dtype=np.uint64)] * 3
    meta = O.make_meta(3, 32, O.OR_F32, 1, True, [40, 40, 40], [False] * 3, sizes)
    seq = O.greedy_sequence(meta)
    assert seq[:6] == [0, 1, 2, 0, 1, 2]
    # a level with twice the delta per byte is taken first
    meta = O.make_meta(2, 32, O.OR_F32, 1, True, [40, 41], [False] * 2, sizes[:2])
    assert O.greedy_sequence(meta)[:2] == [1, 0]
    # an all-zero level is never taken
    meta = O.make_meta(2, 32, O.OR_F32, 1, True, [0, 30], [True, False], sizes[:2])
    assert 0 not in O.greedy_sequence(meta)


def test_estimate_units_closed_form():
    # one level, bl = 40, k = 4 planes of B = 32: delta = 2^(40-4-3) U, plus one
    # floor per level (2 levels) plus the input floor, plus 2^24 U rounding
    sizes = [np.full(8, 64, dtype=np.uint64)] * 2
    meta = O.make_meta(2, 32, O.OR_F32, 5, False, [0, 40], [True, False], sizes)
    E = O.estimate(meta, [0, 1])
    U = Fraction(2) ** (5 - 48)
    unit = Fraction(2) ** (5 - 51 - 32)
    assert Fraction(E) * unit == Fraction(2) ** 33 * U + 3 * U + 2 ** 24 * U


# ---------------------------------------------------------------------- QoI
def test_vmag_matches_numpy_float32():
    rng = np.random.default_rng(3)
    v = rng.standard_normal((3, 1000)).astype(np.float32)
    out, lo, hi = O.vmag_field(v[0], v[1], v[2])
    ref = np.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])  # float32, one rounding per op
    assert (out == ref).all() and lo == ref.min() and hi == ref.max()


def test_qoi_bound_holds():
    from paper_2505_00227_gb300 import synthetic as S
    vx, vy, vz = (S.spectral((20, 21, 22), seed=s).numpy() for s in (11, 12, 13))
    q, qmin, qmax = O.vmag_field(vx, vy, vz)
    for tau_rel in [1e-1, 1e-3, 1e-5]:
        tq = tau_rel * (qmax - qmin)
        eps = O.qoi_component_bound(tq, qmax)
        outs, Es = [], []
        for v in (vx, vy, vz):
            F = O.Field(v)
            rc, out, g, E = F.retrieve(eps)
            assert rc == O.OK and E <= eps
            outs.append(out)
            Es.append(E)
        qh, _, _ = O.vmag_field(*outs)
        est = O.qoi_estimate(*Es, qmax)
        actual = float(np.abs(qh.astype(np.float64) - q.astype(np.float64)).max())
        assert actual <= est <= tq


# ------------------------------------------------------------ recomposition
def test_recompose_tent_closed_form():
    # one nonzero coefficient at a level-h node reconstructs as a tent of
    # half-width h (multilinear hat), zero elsewhere
    shape = (1, 1, 17)
    L = O.num_levels(shape) - 1
    E_f = 1
    U = 2.0 ** (E_f - 48)
    for l in range(1, L + 1):
        h = 1 << (L - l)
        n = O.level_size(shape, l)
        c8s = [None] * (L + 1)
        c = np.zeros(n, dtype=np.int64)
        c[0] = 8 * 64 * (2 ** 20)  # coefficient 64 * 2^20 U at node x = h
        c8s[l] = c
        out = O.recompose(shape, O.OR_F32, E_f, c8s).reshape(-1).astype(np.float64)
        xs = np.arange(17)
        tent = np.maximum(0.0, 1.0 - np.abs(xs - h) / h) * 64 * 2 ** 20 * U
        assert np.array_equal(out, tent)
