"""Pins of the oracle's truncated-segment sensitivities (the adjoint workload).

* the pair function's second derivative and its derivatives with respect to
  the ZBL-correction coefficients agree with central finite differences;
* forward-mode tangents dz_T/dtheta through the frozen last segment agree
  with central finite differences of the same frozen replay (h = 1e-4,
  relative to max(|theta|, 1)) for all eight parameters.
"""
import numpy as np
import pytest

from paper_0810_4737_gb300.workloads import workload


def test_pair_second_derivative_and_coefficient_derivatives(O):
    c = [0.05, -0.03, 0.02, 0.04, -0.05, 0.01]
    p = O.params(workload("b10kev_si_300k_adjoint", spline_c=c))
    # (a grid that avoids the taper's end points, where the third derivative
    # jumps and central differences lose accuracy)
    for r in np.linspace(0.15, 4.95, 97) + 0.0123:
        U, dU, d2U, dc = O.pair_full(p, 14.0, r)
        h = 1e-6 * r
        fd2 = (O.pair_full(p, 14.0, r + h)[1] - O.pair_full(p, 14.0, r - h)[1]) / (2 * h)
        assert abs(fd2 - d2U) <= 1e-6 * max(abs(d2U), 1e-2), (r, fd2, d2U)
        # the plain ion-pair routine agrees on U and dU
        U0, dU0 = O.ion_pair(p, 14.0, r)
        assert abs(U0 - U) <= 1e-12 * max(abs(U), 1) and abs(dU0 - dU) <= 1e-12 * max(abs(dU), 1)
        for k in range(6):
            cp, cm = list(c), list(c)
            cp[k] += 1e-6
            cm[k] -= 1e-6
            pp = O.params(workload("b10kev_si_300k_adjoint", spline_c=cp))
            pm = O.params(workload("b10kev_si_300k_adjoint", spline_c=cm))
            fd = (O.pair_full(pp, 14.0, r)[1] - O.pair_full(pm, 14.0, r)[1]) / 2e-6
            assert abs(fd - dc[k]) <= 1e-6 * max(abs(dc[k]), 1e-3), (r, k, fd, dc[k])


@pytest.mark.parametrize("name,kw,tid", [
    ("b10kev_si_300k_adjoint", dict(energy=600.0, sigma=0.0), 0),
    ("b10kev_si_300k_adjoint", dict(energy=2000.0, s_loc=0.2, spline_c=[0.02, -0.01, 0.03, 0.0, 0.01, -0.02]), 1),
])
def test_segment_tangent_matches_finite_differences(O, name, kw, tid):
    w = workload(name, **kw)
    p = O.params(w)
    t = O.segment_tangent(p, 0, tid)
    assert t["T"] > 0 and t["s0"] == (0 if t["T"] <= 200 else 20 * ((t["T"] - 200) // 20))
    theta = [w["s_e"], w["s_loc"]] + list(w["spline_c"])
    for d in range(8):
        h = 1e-4 * max(abs(theta[d]), 1.0)
        zp, Tp, _ = O.segment_z(p, 0, tid, d, +h)
        zm, Tm, _ = O.segment_z(p, 0, tid, d, -h)
        assert Tp == Tm == t["T"]
        fd = (zp - zm) / (2 * h)
        g = t["grad"][d]
        assert abs(fd - g) <= 2e-4 * max(abs(g), 1e-3 * np.max(np.abs(t["grad"]))), (d, fd, g)
