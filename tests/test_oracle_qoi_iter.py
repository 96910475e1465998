"""Pins of the oracle's iterated QoI retrieval (Sec. 6.2, Algorithm 3) for
V = vx^2 + vy^2 + vz^2: the pointwise bound against exact rational error, the
maximum against brute force, every result against the exact error, and the
behaviour of the three next-bound estimators (MA adds exactly one group per
variable per iteration, MAPE without a threshold is MA, CP stops early)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import pyoracle as O


def _fields(shape=(12, 13, 14), seed=70):
    from paper_2505_00227_gb300 import synthetic as S
    return [S.spectral(shape, seed=seed + c).numpy() for c in range(3)]


def _exact_err(q, v):
    """max |q - (vx^2 + vy^2 + vz^2)| in exact rationals"""
    worst = Fraction(0)
    for i in range(q.size):
        V = sum(Fraction(float(x.flat[i])) ** 2 for x in v)
        worst = max(worst, abs(Fraction(float(q.flat[i])) - V))
    return worst


def test_vtotal_is_the_sum_of_squares():
    rng = np.random.default_rng(0)
    for _ in range(200):
        x, y, z = rng.standard_normal(3).astype(np.float32)
        ref = (np.float64(x) * np.float64(x) + np.float64(y) * np.float64(y)) + \
            np.float64(z) * np.float64(z)
        assert O.vtotal(x, y, z) == ref
    assert O.vtotal(3, 4, 12) == 169.0


def test_point_bound_covers_the_exact_error():
    rng = np.random.default_rng(1)
    for _ in range(3000):
        scale = 10.0 ** rng.uniform(-20, 15)
        xh = (rng.standard_normal(3) * scale).astype(np.float32)
        e = np.abs(rng.standard_normal(3)) * scale * 10.0 ** rng.uniform(-8, 0)
        # a true value within e of the reconstruction (as floats, then exact)
        x = [Fraction(float(xh[i])) + Fraction(float(e[i])) * Fraction(float(rng.uniform(-1, 1)))
             for i in range(3)]
        V = sum(t * t for t in x)
        Vh = float(np.float32(O.vtotal(*xh)))
        b = O.vtotal_point_bound(*xh, e) * (1.0 + 2.0 ** -40)
        assert abs(Fraction(Vh) - V) <= Fraction(b)


def test_bound_is_the_maximum_and_its_first_point():
    rng = np.random.default_rng(2)
    x, y, z = (rng.standard_normal(500).astype(np.float32) for _ in range(3))
    x[77] = x[311] = 40.0  # a tie: the first one is reported
    y[77] = y[311] = 0.0
    z[77] = z[311] = 0.0
    e = [1e-3, 2e-3, 5e-4]
    b, arg = O.vtotal_bound(x, y, z, e)
    pts = [O.vtotal_point_bound(x[i], y[i], z[i], e) for i in range(500)]
    assert arg == 77 and b == max(pts) * (1.0 + 2.0 ** -40)


@pytest.mark.parametrize("est", [O.EST_CP, O.EST_MA, O.EST_MAPE])
@pytest.mark.parametrize("tau", [1e-1, 1e-3, 1e-5])
def test_loop_meets_the_bound(est, tau):
    v = _fields()
    lo, hi = O.vtotal_range(*v)
    Fs = [O.Field(x) for x in v]
    st, outs, q, rep = O.qoi_vtotal(Fs, lo, hi, tau, est)
    assert st == 0 and rep.status == 0
    assert rep.tau_abs == tau * (hi - lo)
    assert rep.est <= rep.tau_abs
    assert _exact_err(q, v) <= Fraction(rep.est)
    # each variable is the plain retrieval at its final bound
    for F, o, E in zip(Fs, outs, rep.eps):
        rc, ref, g, Eref = F.retrieve(E)
        assert np.array_equal(o.view(np.uint32), ref.view(np.uint32))


def test_ma_adds_one_group_per_variable_per_iteration():
    v = _fields(seed=80)
    lo, hi = O.vtotal_range(*v)
    Fs = [O.Field(x) for x in v]
    tau = 1e-4
    st, outs, q, rep = O.qoi_vtotal(Fs, lo, hi, tau, O.EST_MA)
    tau_abs = tau * (hi - lo)
    for i, F in enumerate(Fs):
        eps0 = (tau_abs / hi) * F.range
        rc, g0, E0, _ = F.select(eps0)
        p0 = int(np.sum(g0))
        n = len(F.sequence())
        assert rep.prefix[i] == min(p0 + rep.iterations - 1, n)
    # MAPE whose threshold is never passed is MA
    st2, outs2, q2, rep2 = O.qoi_vtotal(Fs, lo, hi, tau, O.EST_MAPE, c=math.inf)
    assert rep2.iterations == rep.iterations and list(rep2.prefix) == list(rep.prefix)
    assert np.array_equal(q2.view(np.uint32), q.view(np.uint32))


def test_cp_needs_no_more_iterations_than_ma_but_fetches_at_least_as_much():
    v = _fields(seed=90)
    lo, hi = O.vtotal_range(*v)
    Fs = [O.Field(x) for x in v]
    _, _, _, cp = O.qoi_vtotal(Fs, lo, hi, 1e-4, O.EST_CP)
    _, _, _, ma = O.qoi_vtotal(Fs, lo, hi, 1e-4, O.EST_MA)
    assert cp.iterations <= ma.iterations
    assert sum(cp.prefix) >= sum(ma.prefix)


def test_unattainable_and_zero_fields():
    v = _fields(shape=(6, 7, 8), seed=95)
    lo, hi = O.vtotal_range(*v)
    Fs = [O.Field(x) for x in v]
    st, outs, q, rep = O.qoi_vtotal(Fs, lo, hi, 0.0, O.EST_MA)
    assert st == -5
    assert all(rep.prefix[i] == len(F.sequence()) for i, F in enumerate(Fs))
    z = [np.zeros((4, 5, 6), dtype=np.float32) for _ in range(3)]
    Fz = [O.Field(x) for x in z]
    st, outs, q, rep = O.qoi_vtotal(Fz, 0.0, 0.0, 1e-3, O.EST_MAPE)
    assert st == 0 and rep.iterations == 1 and rep.est == 0.0 and not q.any()
