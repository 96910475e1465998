"""The output conversion of every retrieval, f = RN(X) * 2^(E_f - 48), against
its definition written with exact integer arithmetic: round-to-nearest-even of
the integer to 24 (FP32) or 53 (FP64) significant bits, then the power-of-two
scale (for FP32 below E_f = -78 and above 121 the value is rounded to FP64
first, scaled, then rounded to FP32).  Covers every exponent range, the 2^48
boundary of the fast FP32 construction, exact ties, and the extreme integers."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _rn_int(x, bits):
    """RN-even of the integer x to `bits` significant bits, as an exact integer"""
    if x == 0:
        return 0
    s, m = (-1 if x < 0 else 1), abs(x)
    sh = m.bit_length() - bits
    if sh <= 0:
        return x
    q, r = divmod(m, 1 << sh)
    half = 1 << (sh - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return s * (q << sh)


def _expect32(x, E_f):
    e = E_f - 48
    with np.errstate(over="ignore"):
        if -126 <= e and E_f <= 121:  # exact: 24 bits, normal (or past the FP32 range)
            return np.float32(math.ldexp(float(_rn_int(x, 24)), e))
        d = float(x)  # RN to FP64 (Python's int -> float is correctly rounded)
        return np.float32(np.ldexp(np.float64(d), e))


def _expect64(x, E_f):
    e = E_f - 48
    d = np.float64(float(x))
    with np.errstate(over="ignore", under="ignore"):
        if e >= -1022:
            return np.ldexp(d, e)
        return np.ldexp(np.ldexp(d, -500), e + 500)


def _values(seed=0):
    rng = np.random.default_rng(seed)
    v = [0, 1, -1, 2**24, -(2**24), 2**24 + 1, 2**48 - 1, -(2**48 - 1), 2**48, -(2**48),
         2**48 + 1, -(2**48) - 1, 2**53 - 1, 2**53 + 1, -(2**53) - 1, 2**62, 2**63 - 1, -(2**63)]
    for p in range(25, 63):  # exact ties and their neighbours at every bit length
        for q in (2**23, 2**23 + 1, 2**24 - 1, 0xABCDEF):
            base = q << (p - 24)
            for d in (-1, 0, 1):
                t = base + (1 << (p - 25)) + d
                v += [t, -t]
    for p in range(54, 63):  # FP64 ties
        t = ((2**52 + 5) << (p - 53)) + (1 << (p - 54))
        v += [t, -t, t + 1, -t - 1]
    bl = rng.integers(0, 63, 4000)
    mag = [int(rng.integers(0, 2**62)) >> (62 - int(b)) for b in bl]
    v += [m if rng.random() < 0.5 else -m for m in mag]
    v += [int(x) for x in rng.integers(-(2**48), 2**48, 4000)]
    return [int(x) for x in v]


@pytest.fixture(scope="module")
def ctx():
    from paper_2505_00227_gb300 import binding
    return binding.Context()


@pytest.mark.parametrize("E_f", [-148, -100, -79, -78, -77, 0, 1, 2, 48, 100, 121, 122, 128])
def test_fixed_to_f32(ctx, E_f):
    v = _values(E_f + 1000)
    X = torch.tensor(v, dtype=torch.int64, device="cuda")
    got = ctx.fixed_to_float(X, E_f, torch.float32).cpu().numpy()
    exp = np.array([_expect32(x, E_f) for x in v], dtype=np.float32)
    bad = np.nonzero(got.view(np.uint32) != exp.view(np.uint32))[0]
    assert bad.size == 0, [(v[i], got[i], exp[i]) for i in bad[:5]]


@pytest.mark.parametrize("E_f", [-1073, -1000, -975, -974, -973, 0, 1, 49, 500, 970, 1024])
def test_fixed_to_f64(ctx, E_f):
    v = _values(E_f + 5000)
    X = torch.tensor(v, dtype=torch.int64, device="cuda")
    got = ctx.fixed_to_float(X, E_f, torch.float64).cpu().numpy()
    exp = np.array([_expect64(x, E_f) for x in v], dtype=np.float64)
    bad = np.nonzero(got.view(np.uint64) != exp.view(np.uint64))[0]
    assert bad.size == 0, [(v[i], got[i], exp[i]) for i in bad[:5]]


def test_fixed_to_float_rejects_bad_arguments(ctx):
    from paper_2505_00227_gb300 import binding as B
    X = torch.zeros(4, dtype=torch.int64, device="cuda")
    for E_f, dt in [(-149, torch.float32), (129, torch.float32), (-1074, torch.float64),
                    (1025, torch.float64)]:
        with pytest.raises(B.HpmdrError):
            ctx.fixed_to_float(X, E_f, dt)
    assert ctx.fixed_to_float(X[:0], 0, torch.float32).numel() == 0
