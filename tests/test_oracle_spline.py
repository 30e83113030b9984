"""Pins of the ZBL-correction spline of the oracle (the reading of the
adjoint workload's six knot parameters: phi -> phi_ZBL exp(sum_i c_i
B_i(ln r)), cubic B-splines centred on ln of the knots {0.2, 0.35, 0.6, 1.0,
1.7, 3.0} A, width the mean knot spacing in ln r).

The basis is pinned against what the mathematics fixes for the cardinal cubic
B-spline -- its values at the knots, partition of unity and linear
reproduction over integer shifts -- and against an independent library
construction (scipy's B-spline basis element on the knots -2..2).  The
correction is then pinned against the same library basis evaluated at the
documented centres and width, so a wrong knot, centre, width or derivative
factor in the oracle fails here.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

KNOTS = [0.2, 0.35, 0.6, 1.0, 1.7, 3.0]


def test_cardinal_cubic_values_at_the_knots(O):
    for u, want in [(0.0, 2.0 / 3.0), (1.0, 1.0 / 6.0), (-1.0, 1.0 / 6.0), (2.0, 0.0), (-2.0, 0.0),
                    (2.5, 0.0), (-3.0, 0.0)]:
        b, _ = O.bspline3(u)
        assert b == pytest.approx(want, abs=1e-15), (u, b)
    # slope at the knots: 0 at the centre, -+1/2 at +-1, 0 at the support's ends
    for u, want in [(0.0, 0.0), (1.0, -0.5), (-1.0, 0.5), (2.0, 0.0), (-2.0, 0.0)]:
        assert O.bspline3(u)[1] == pytest.approx(want, abs=1e-15), u


def test_partition_of_unity_and_linear_reproduction(O):
    for u in np.linspace(-3.0, 3.0, 61) + 0.0137:
        ks = range(int(math.floor(u)) - 3, int(math.floor(u)) + 4)
        s = sum(O.bspline3(u - k)[0] for k in ks)
        s1 = sum(k * O.bspline3(u - k)[0] for k in ks)
        ds = sum(O.bspline3(u - k)[1] for k in ks)
        assert s == pytest.approx(1.0, abs=1e-14), u
        assert s1 == pytest.approx(u, abs=1e-13), u
        assert ds == pytest.approx(0.0, abs=1e-14), u


def test_basis_equals_the_library_b_spline(O):
    ref = BSpline.basis_element([-2.0, -1.0, 0.0, 1.0, 2.0], extrapolate=False)
    dref = ref.derivative()
    for u in np.linspace(-1.999, 1.999, 203):
        b, db = O.bspline3(u)
        assert b == pytest.approx(float(ref(u)), abs=1e-14), u
        assert db == pytest.approx(float(dref(u)), abs=1e-13), u


def test_correction_is_the_documented_combination(O):
    ref = BSpline.basis_element([-2.0, -1.0, 0.0, 1.0, 2.0], extrapolate=False)
    dref = ref.derivative()
    h = (math.log(KNOTS[-1]) - math.log(KNOTS[0])) / 5.0
    rng = np.random.default_rng(3)
    for _ in range(4):
        c = rng.normal(0.0, 0.1, 6)
        for r in np.geomspace(0.08, 6.0, 157):
            v, d = O.spline_corr(c, r)
            us = [(math.log(r) - math.log(k)) / h for k in KNOTS]
            want = sum(ci * (float(np.nan_to_num(ref(u))) if abs(u) < 2 else 0.0) for ci, u in zip(c, us))
            dwant = sum(ci * (float(np.nan_to_num(dref(u))) if abs(u) < 2 else 0.0) for ci, u in zip(c, us)) / (h * r)
            assert v == pytest.approx(want, abs=1e-14), r
            assert d == pytest.approx(dwant, rel=1e-12, abs=1e-13), r
    # a single knot: the correction is that knot's bump, 2/3 c_i at r = knot_i
    for i, k in enumerate(KNOTS):
        c = np.zeros(6)
        c[i] = 0.3
        assert O.spline_corr(c, k)[0] == pytest.approx(0.2, abs=1e-15)
        # and its neighbours' centres see 1/6 of it only where the spacing is h
        # (the knots are not exactly uniform in ln r): bounded by the support
        for j, kj in enumerate(KNOTS):
            if abs(i - j) >= 3:
                assert O.spline_corr(c, kj)[0] == 0.0


def test_correction_vanishes_outside_the_knots(O):
    c = np.full(6, 0.25)
    h = (math.log(KNOTS[-1]) - math.log(KNOTS[0])) / 5.0
    lo, hi = KNOTS[0] * math.exp(-2 * h), KNOTS[-1] * math.exp(2 * h)
    for r in [0.5 * lo, 0.999 * lo, 1.001 * hi, 2 * hi, 10.0]:
        v, d = O.spline_corr(c, r)
        assert v == 0.0 and d == 0.0, r
