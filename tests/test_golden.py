"""Hand-derived values of the three-circle product-space example of the
Introduction (Figs. 1-3) against the oracle.  Three unit circles centred at
(1, 0), (0, 1) and (-1, 0) all pass through the origin; divide projects each
copy onto its own circle, concur replaces every copy by the copies' average.
The expected values are worked out by hand in the comments, not by the
oracle."""
import math

import numpy as np

from oracle import abc, toy

CENTRES = [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0)]
RADII = [1.0, 1.0, 1.0]


def _tc():
    return toy.ThreeCircles(CENTRES, RADII)


def test_copies_already_on_their_circles():
    # (2, 0), (0, 2), (-2, 0) lie on their circles, so P_D x0 = x0.  Their
    # average is (0, 2/3): DC = P_C P_D gives three copies of (0, 2/3).  DR =
    # (1/2, 2, 2) = (R_C R_D + I)/2 with R_D x0 = x0 and R_C x0 = 2 P_C x0 - x0
    # gives (2 P_C x0 - x0 + x0)/2 = P_C x0 as well.
    tc = _tc()
    x0 = np.array([[2.0, 0.0], [0.0, 2.0], [-2.0, 0.0]])
    np.testing.assert_allclose(tc.project_D(x0), x0, atol=1e-15)
    want = np.array([[0.0, 2.0 / 3.0]] * 3)
    for name in ("DC", "DR"):
        out = abc.abc_step(x0, tc.project_D, tc.project_C, *abc.preset(name))
        np.testing.assert_allclose(out, want, atol=1e-15, err_msg=name)


def test_one_point_three_projections():
    # (1, 1) is at distance 1 from (1, 0) and from (0, 1): on the first two
    # circles.  From (-1, 0) it is at (2, 1), length sqrt(5), so its projection
    # onto the third circle is (-1, 0) + (2, 1)/sqrt(5).  DC averages the three
    # projections: ((1 + 1 - 1 + 2/sqrt5)/3, (1 + 1 + 1/sqrt5)/3).
    tc = _tc()
    s5 = math.sqrt(5.0)
    x0 = np.array([[1.0, 1.0]] * 3)
    pd = np.array([[1.0, 1.0], [1.0, 1.0], [-1.0 + 2.0 / s5, 1.0 / s5]])
    np.testing.assert_allclose(tc.project_D(x0), pd, atol=1e-15)
    out = abc.abc_step(x0, tc.project_D, tc.project_C, *abc.preset("DC"))
    np.testing.assert_allclose(out, np.array([[(1.0 + 2.0 / s5) / 3.0, (2.0 + 1.0 / s5) / 3.0]] * 3),
                               atol=1e-15)
