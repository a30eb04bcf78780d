"""Relaxed projections and the generic abc update (oracle, FP64).

* Relaxed projection (Introduction): P^a_S x = a P^1_S x + (1 - a) x;
  a = 1 is the standard projection, a = 2 the reflection R_S = 2 P^1_S - I.
* Generalised divide-and-concur (Introduction, the displayed update):
  x_{k+1} = a P^b_C P^c_D x_k + (1 - a) x_k.

``abc_step`` is written for any pair of projection callables so the same
driver serves the three-circle example (Fig. 3) and the ptychographic
product space (Fig. 4).

Presets.  The paper names DC, AR, DR, SF, RAAR, RRR (and T_lambda) but defines
only DC = P_C P_D, i.e. (a, b, c) = (1, 1, 1).  The other settings are the
readings obtained by expanding the abc update and matching the usual
published forms (P_C is applied exactly once to P^c_D x, so the matches hold
for a non-linear P_C as well):

  DR        (1/2, 2, 2)        = (R_C R_D + I) / 2
  RAAR(b)   (1/2, 2b, 2)       = (b/2)(R_C R_D + I) + (1 - b) P_D
  RRR(b)    (b/2, 2, 2)        = I + b (P_C R_D - P_D)
  SF        (1, 2, 1)          = R_C P_D
  AR        (1, 2, 2)          = R_C R_D   (alternating reflections)

The tests check each against its published form built from separate P_D and
P_C calls.
"""
from __future__ import annotations

from typing import Callable


def relax(proj: Callable, a: float) -> Callable:
    """Return x -> a * proj(x) + (1 - a) * x (relaxed projection)."""
    def P(x):
        return a * proj(x) + (1.0 - a) * x
    return P


def abc_step(x, proj_D: Callable, proj_C: Callable, a: float, b: float, c: float):
    """One generalised update x -> a P^b_C P^c_D x + (1 - a) x."""
    y = relax(proj_D, c)(x)
    return a * relax(proj_C, b)(y) + (1.0 - a) * x


def preset(name: str, beta: float | None = None) -> tuple[float, float, float]:
    """(a, b, c) of a named algorithm (readings listed in the module doc)."""
    n = name.upper()
    if n == "DC":
        return (1.0, 1.0, 1.0)
    if n == "AR":
        return (1.0, 2.0, 2.0)
    if n == "DR":
        return (0.5, 2.0, 2.0)
    if n == "SF":
        return (1.0, 2.0, 1.0)
    if n == "RAAR":
        b = 0.9 if beta is None else beta
        return (0.5, 2.0 * b, 2.0)
    if n == "RRR":
        b = 0.5 if beta is None else beta
        return (b / 2.0, 2.0, 2.0)
    raise ValueError(f"unknown preset {name!r}")
