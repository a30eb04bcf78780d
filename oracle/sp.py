"""Sequential projections for blind ptychography (oracle, FP64).

The paper's alternative to the product space (Introduction, Fig. 2): one
estimate visits the constraint sets one after another, in a fixed order or
shuffled between iterations, with a relaxation per projection.  For
ptychography the constraint sets are the per-position Fourier-modulus sets
S_j = {exit wave psi : |F psi| = sqrt(I_j)}, and the estimate is the pair
(object, probe).  The paper does not spell out how (O, P) follows a projected
exit wave; the reading used here is the usual sequential form: at position j

    psi   = P * O_j
    psi'  = lam * P_{S_j}(psi) + (1 - lam) * psi        (relaxed projection)
    d     = psi' - psi
    O_j  <- O_j + conj(P)   * d / max|P|^2
    P    <- P   + conj(O_j) * d / max|O_j|^2            (O_j before its update)

(the maxima over the probe array and over the window).  One iteration visits
every position once, in the order given.
"""
from __future__ import annotations

import numpy as np

from .dft import fft2, ifft2
from .ptycho import modulus_projection


def sp_step(O: np.ndarray, P: np.ndarray, pos_j, sqrtI_j: np.ndarray, lam: float) -> float:
    """Update O (window at pos_j) and P in place; returns sum (|F psi| - sqrtI)^2."""
    N = P.shape[0]
    r, c = int(pos_j[0]), int(pos_j[1])
    Oj = O[r:r + N, c:c + N].copy()
    psi = P * Oj
    Psi = fft2(psi)
    err = float(((np.abs(Psi) - sqrtI_j) ** 2).sum())
    target = lam * ifft2(modulus_projection(Psi, sqrtI_j)) + (1.0 - lam) * psi
    d = target - psi
    mp = float((np.abs(P) ** 2).max())
    mo = float((np.abs(Oj) ** 2).max())
    if mp > 0:
        O[r:r + N, c:c + N] = Oj + np.conj(P) * d / mp
    if mo > 0:
        P += np.conj(Oj) * d / mo
    return err


def sp_iterate(O: np.ndarray, P: np.ndarray, pos: np.ndarray, intensity: np.ndarray,
               lam: float, order=None) -> float:
    """One pass over all positions (ascending, or the given order); O and P are
    updated in place; returns the Fourier error sum / sum I over the pass."""
    I = np.asarray(intensity, dtype=np.float64)
    sq = np.sqrt(I)
    idx = range(pos.shape[0]) if order is None else order
    err = 0.0
    for j in idx:
        err += sp_step(O, P, pos[j], sq[j], lam)
    tot = float(I.sum())
    return err / tot if tot > 0 else err
