"""GPU parity of one QoI bounding step for V = vx^2 + vy^2 + vz^2 (Sec. 6.2,
Algorithm 3's error estimate), through hpmdr_qoi_vtotal_bound.

V_hat is checked bit for bit against its definition (FP64 squares and sums,
one rounding each, then one rounding to FP32; numpy gives exactly that) and
against the oracle's evaluation on samples; the largest pointwise bound and its
first point against the oracle's scan.  The inputs include values whose V_hat
lies on or next to an FP32 rounding midpoint (where rounding twice differs from
rounding once), values outside the range of the FP32 evaluation, overflow to
+inf, zeros, subnormals, and ties of the largest bound.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import pyoracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2505_00227_gb300 import binding
    binding.lib()
    return binding.Context()


def _definition(x, y, z):
    X, Y, Z = (np.asarray(a, dtype=np.float32).astype(np.float64) for a in (x, y, z))
    with np.errstate(over="ignore"):
        return ((X * X + Y * Y) + Z * Z).astype(np.float32)


def _check(ctx, x, y, z, e, sample=2000, seed=0):
    x, y, z = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z))
    d = [torch.from_numpy(a).cuda() for a in (x, y, z)]
    out, b, pt = ctx.vtotal_bound(*d, e)
    got = out.cpu().numpy()
    ref = _definition(x, y, z)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    rng = np.random.default_rng(seed)
    idx = rng.choice(x.size, size=min(sample, x.size), replace=False)
    for i in idx:
        with np.errstate(over="ignore"):  # V past FLT_MAX rounds to +inf
            v = np.float32(O.vtotal(x.flat[i], y.flat[i], z.flat[i]))
        assert v.view(np.uint32) == got.flat[i].view(np.uint32), i
    ob, opt = O.vtotal_bound(x, y, z, e)
    assert pt == opt
    assert b * (1.0 + 2.0 ** -40) == ob
    assert b == O.vtotal_point_bound(x.flat[pt], y.flat[pt], z.flat[pt], e)
    return got, b, pt


def test_spectral_triplet(ctx):
    from paper_2505_00227_gb300 import synthetic as S
    v = [c.numpy() for c in S.velocity_triplet((24, 40, 64), seed=51)]
    for e in ([1e-3, 2e-3, 5e-4], [0.0, 0.0, 0.0], [1e-7, 0.3, 1e-12]):
        _check(ctx, *v, e)


def _midpoints(rng, n):
    """x^2 = 1 + 2^-11 + 2^-24 (an FP32 midpoint) with small y, z that either
    vanish in the FP64 sum or push it across, at many binades and signs."""
    base = np.float32(1.0 + 2.0 ** -12)
    scale = (2.0 ** rng.integers(-20, 21, n)).astype(np.float32)
    x = (base * scale) * rng.choice([-1, 1], n).astype(np.float32)
    kind = rng.integers(0, 4, n)
    tiny = scale * np.float32(2.0 ** -30)
    y = np.where(kind == 0, 0.0, np.where(kind == 1, tiny, np.where(kind == 2, -tiny, scale * 2.0 ** -12)))
    z = np.where(kind == 3, scale * 2.0 ** -13, np.where(kind == 1, tiny * 2.0 ** -4, 0.0))
    return x.astype(np.float32), y.astype(np.float32), z.astype(np.float32)


def _rn32(q):
    """FP32 round-to-nearest-even of an exact rational q >= 0 (a normal result)."""
    f = np.float32(float(q))
    best = None
    for c in (np.nextafter(f, np.float32(0)), f, np.nextafter(f, np.float32(np.inf))):
        d = abs(Fraction(float(c)) - q)
        if best is None or d < best[0] or (d == best[0] and not (c.view(np.uint32) & 1)):
            best = (d, c)
    return best[1]


def test_rounding_midpoints(ctx):
    rng = np.random.default_rng(52)
    x, y, z = _midpoints(rng, 20000)
    ref = _definition(x, y, z)
    # the set holds exact FP32 ties and values where rounding the FP64 sum
    # differs from rounding the exact sum once
    ties = twice = 0
    for i in range(3000):
        q = sum(Fraction(float(a[i])) ** 2 for a in (x, y, z))
        v64 = Fraction(float((np.float64(x[i]) ** 2 + np.float64(y[i]) ** 2) + np.float64(z[i]) ** 2))
        lo = Fraction(float(np.float32(float(v64))))
        ties += v64 != lo and 2 * abs(v64 - lo) == Fraction(float(np.spacing(np.float32(float(v64)))))
        twice += _rn32(q) != ref[i]
    assert ties > 0 and twice > 0
    _check(ctx, x, y, z, [1e-6, 1e-6, 1e-6], sample=500)


def test_ranges_overflow_and_zeros(ctx):
    vals = np.array([0.0, -0.0, 1e-45, 1e-40, 2.0 ** -33, 2.0 ** -32, 2.0 ** -31, 1.0,
                     2.0 ** 59, 2.0 ** 60, 2.0 ** 61, 2.0 ** 64, 1.8e19, 3e38, -3e38],
                    dtype=np.float32)
    g = np.array(np.meshgrid(vals, vals, vals, indexing="ij")).reshape(3, -1)
    for e in ([0.0, 0.0, 0.0], [1e-3, 1e-3, 1e-3], [1e30, 1.0, 1e-300]):
        got, b, pt = _check(ctx, g[0], g[1], g[2], e, sample=g.shape[1])
    assert np.isinf(got).any() and b == float("inf")


def test_ties_and_first_point(ctx):
    rng = np.random.default_rng(53)
    n = 5_000_003  # several points per thread, a ragged last block
    x = rng.uniform(-1, 1, n).astype(np.float32)
    y = rng.uniform(-1, 1, n).astype(np.float32)
    z = rng.uniform(-1, 1, n).astype(np.float32)
    for at in (4_000_000, n - 1, 0):
        xx, yy, zz = x.copy(), y.copy(), z.copy()
        for j in sorted({at, min(at + 777, n - 1), n - 1}):  # equal maxima: the first wins
            xx[j], yy[j], zz[j] = 1.5, -1.5, 1.5
        _, b, pt = _check(ctx, xx, yy, zz, [1e-4, 2e-4, 3e-4], sample=300)
        assert pt == at
    c = np.full(1000, 0.25, dtype=np.float32)  # all equal: point 0
    _, b, pt = _check(ctx, c, c, c, [1e-3, 1e-3, 1e-3])
    assert pt == 0


def test_rejects_bad_arguments(ctx):
    from paper_2505_00227_gb300 import binding
    a = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(binding.HpmdrError):
        ctx.vtotal_bound(a, a, a, [1e-3, -1.0, 0.0])
    with pytest.raises(binding.HpmdrError):
        ctx.vtotal_bound(a[:0], a[:0], a[:0], [0.0, 0.0, 0.0])
