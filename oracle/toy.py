"""Three-circle product-space example (Introduction, Figs. 1-3; oracle).

Three circle constraint sets S, T, U in the plane.  The product space holds
three copies of the plane, x = [x^S, x^T, x^U] (array of shape (3, 2)); the
divide projection projects each copy onto its own circle, the concur
projection replaces every copy by their average (x^S + x^T + x^U) / 3.
"""
from __future__ import annotations

import numpy as np


def project_circle(p: np.ndarray, centre: np.ndarray, radius: float) -> np.ndarray:
    d = p - centre
    n = float(np.hypot(d[0], d[1]))
    if n == 0.0:
        return centre + np.array([radius, 0.0])
    return centre + radius * d / n


class ThreeCircles:
    def __init__(self, centres, radii):
        self.centres = [np.asarray(c, dtype=np.float64) for c in centres]
        self.radii = [float(r) for r in radii]

    def project_D(self, x: np.ndarray) -> np.ndarray:
        return np.stack([project_circle(x[i], self.centres[i], self.radii[i])
                         for i in range(len(self.centres))])

    def project_C(self, x: np.ndarray) -> np.ndarray:
        m = x.mean(axis=0)
        return np.stack([m] * x.shape[0])
