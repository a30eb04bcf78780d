"""Ptychographic divide and concur projections and one abc iteration (oracle, FP64).

Product space (Introduction, Fig. 3): the point x is the stack of J exit waves
x = [x_0 .. x_{J-1}], one N x N complex array per scan position.  The flow of
Fig. 4 is: initial probe and object -> exit waves for all scan positions ->
projections -> updated probe and object.

Notation: positions s_j = (row, col) are integer top-left corners, the
object window is O_j(r) = O(s_j + r) for r in [0, N)^2; I_j are the measured
intensities (unshifted); F is the unnormalised 2-D DFT of ``oracle.dft``.

Divide projection P^1_D (Fig. 3(a), per-component projection): for every j,
Psi = F x_j; Psi' = sqrt(I_j) Psi / |Psi| (sqrt(I_j) where |Psi| = 0);
(P_D x)_j = F^{-1} Psi'.

Concur projection P^1_C (Fig. 3(b): reach one consensus from the divided
copies).  With an unknown probe the consensus set is the set of stacks of the
form {P * O_j}; the paper does not spell out the projection, and the reading
used here is one least-squares sweep per application: first the object with
the current probe,
    O(m) = sum_j conj(P(m - s_j)) y_j(m - s_j) / (sum_j |P(m - s_j)|^2 + alpha max),
then the probe with the new object,
    P(r) = sum_j conj(O(s_j + r)) y_j(r) / (sum_j |O(s_j + r)|^2 + alpha max),
where "max" is the maximum of that denominator over its array and a pixel
whose regularised denominator is exactly 0 is set to 0.  The result is the
re-split stack z_j = P * O_j.  Sums over j run in ascending j.

The paper does not say when the probe update begins.  The default reading
updates the object and then the probe from the first iteration; with
``probe_start = K`` the concur step of iterations k < K (k counted from 0)
updates the object only and keeps the probe as it is (the other reading).

One iteration is the displayed general update of the Introduction,
x_{k+1} = a P^b_C P^c_D x_k + (1 - a) x_k, evaluated by ``abc.abc_step`` with
the two projections above.  The Fourier error of the divide input,
E_F = sum_j sum_q (|F x_j| - sqrt(I_j))^2 / sum_j sum_q I_j, is recorded on
every call of P_D.
"""
from __future__ import annotations

import numpy as np

from . import abc as _abc
from .dft import fft2, ifft2


def exit_waves(P: np.ndarray, O: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """x_j = P * O(s_j + .) for every position (Fig. 4, forming exit waves)."""
    N = P.shape[0]
    out = np.empty((pos.shape[0], N, N), dtype=np.complex128)
    for j in range(pos.shape[0]):
        r, c = int(pos[j, 0]), int(pos[j, 1])
        out[j] = P * O[r:r + N, c:c + N]
    return out


def modulus_projection(Psi: np.ndarray, sqrtI: np.ndarray) -> np.ndarray:
    """Replace the modulus of Psi by sqrtI, keeping its phase (phase 0 where Psi = 0)."""
    mag = np.abs(Psi)
    out = np.empty_like(Psi)
    nz = mag > 0
    out[nz] = sqrtI[nz] * Psi[nz] / mag[nz]
    out[~nz] = sqrtI[~nz]
    return out


def project_D(x: np.ndarray, sqrtI: np.ndarray) -> tuple[np.ndarray, float]:
    """Divide projection P^1_D over all positions; also sum_j sum_q (|Psi| - sqrtI)^2."""
    y = np.empty_like(x, dtype=np.complex128)
    err = 0.0
    for j in range(x.shape[0]):
        Psi = fft2(x[j])
        err += float(((np.abs(Psi) - sqrtI[j]) ** 2).sum())
        y[j] = ifft2(modulus_projection(Psi, sqrtI[j]))
    return y, err


def regularised_ratio(num: np.ndarray, den: np.ndarray, alpha: float) -> np.ndarray:
    """num / (den + alpha * max(den)); exactly-zero regularised denominators give 0."""
    d = den + alpha * (den.max() if den.size else 0.0)
    out = np.zeros_like(num)
    nz = d > 0
    out[nz] = num[nz] / d[nz]
    return out


def concur_object(y: np.ndarray, P: np.ndarray, pos: np.ndarray,
                  M_shape: tuple[int, int], alpha: float) -> np.ndarray:
    """Least-squares object for the stack y with probe P held fixed."""
    N = P.shape[0]
    num = np.zeros(M_shape, dtype=np.complex128)
    den = np.zeros(M_shape, dtype=np.float64)
    Pc = np.conj(P)
    P2 = np.abs(P) ** 2
    for j in range(pos.shape[0]):
        r, c = int(pos[j, 0]), int(pos[j, 1])
        num[r:r + N, c:c + N] += Pc * y[j]
        den[r:r + N, c:c + N] += P2
    return regularised_ratio(num, den, alpha)


def concur_probe(y: np.ndarray, O: np.ndarray, pos: np.ndarray, alpha: float) -> np.ndarray:
    """Least-squares probe for the stack y with object O held fixed."""
    N = y.shape[-1]
    num = np.zeros((N, N), dtype=np.complex128)
    den = np.zeros((N, N), dtype=np.float64)
    for j in range(pos.shape[0]):
        r, c = int(pos[j, 0]), int(pos[j, 1])
        Oj = O[r:r + N, c:c + N]
        num += np.conj(Oj) * y[j]
        den += np.abs(Oj) ** 2
    return regularised_ratio(num, den, alpha)


class Problem:
    """A blind ptychographic problem with its current object/probe estimate.

    ``project_C`` updates the estimate (object sweep, then probe sweep) and
    returns the consensus stack; ``project_D`` records the Fourier error of its
    input in ``last_error``.  ``iterate`` counts the iterations it has run; in
    those with index below ``probe_start`` the probe sweep is skipped.
    """

    def __init__(self, intensity: np.ndarray, pos: np.ndarray,
                 O: np.ndarray, P: np.ndarray, alpha: float = 1e-6, probe_start: int = 0):
        self.I = np.asarray(intensity, dtype=np.float64)
        self.sqrtI = np.sqrt(self.I)
        self.sumI = float(self.I.sum())
        self.pos = np.asarray(pos, dtype=np.int64)
        self.O = np.array(O, dtype=np.complex128)
        self.P = np.array(P, dtype=np.complex128)
        self.alpha = float(alpha)
        self.last_error = float("nan")
        self.probe_start = int(probe_start)
        self.k = 0                      # iterations run so far
        self._hold_probe = False

    def project_D(self, x: np.ndarray) -> np.ndarray:
        y, err = project_D(x, self.sqrtI)
        self.last_error = err / self.sumI if self.sumI > 0 else err
        return y

    def project_C(self, y: np.ndarray) -> np.ndarray:
        self.O = concur_object(y, self.P, self.pos, self.O.shape, self.alpha)
        if not self._hold_probe:
            self.P = concur_probe(y, self.O, self.pos, self.alpha)
        return exit_waves(self.P, self.O, self.pos)

    def iterate(self, x: np.ndarray, a: float, b: float, c: float) -> np.ndarray:
        """x_{k+1} = a P^b_C P^c_D x_k + (1 - a) x_k."""
        self._hold_probe = self.k < self.probe_start
        out = _abc.abc_step(x, self.project_D, self.project_C, a, b, c)
        self.k += 1
        return out

    def run(self, x: np.ndarray, a: float, b: float, c: float, n: int):
        """n iterations; returns (x_n, [E_F of x_0 .. x_{n-1}])."""
        errs = []
        for _ in range(n):
            x = self.iterate(x, a, b, c)
            errs.append(self.last_error)
        return x, errs
