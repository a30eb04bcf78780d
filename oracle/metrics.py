"""Error metrics (oracle, FP64).

The paper reports error curves per algorithm (Figs. 7 and 8) and marks an
error-metric box inside the reconstruction area (Fig. 5) without defining
either metric.  Readings used here:

* Fourier error of a stack x:
  E_F(x) = sum_j sum_q (|F x_j|(q) - sqrt(I_j(q)))^2 / sum_j sum_q I_j(q).
* Object error in the box [N/2, M - N/2) on both axes, with the ambiguities
  of blind ptychography (global complex scale and a linear phase ramp)
  removed: min over gamma, k of sum |O_true - gamma e^{i k.r} O|^2 / sum |O_true|^2.
  k is taken at the peak of an 8x zero-padded DFT of O_true conj(O) over the
  box; gamma then has the closed form DFT(peak) / sum |O|^2.
"""
from __future__ import annotations

import numpy as np

from .dft import fft2


def fourier_error(x: np.ndarray, intensity: np.ndarray) -> float:
    I = np.asarray(intensity, dtype=np.float64)
    s = 0.0
    for j in range(x.shape[0]):
        s += float(((np.abs(fft2(x[j])) - np.sqrt(I[j])) ** 2).sum())
    tot = float(I.sum())
    return s / tot if tot > 0 else s


def error_box(M_shape: tuple[int, int], N: int) -> tuple[slice, slice]:
    h = N // 2
    return slice(h, M_shape[0] - h), slice(h, M_shape[1] - h)


def object_error(O: np.ndarray, O_true: np.ndarray, N: int, pad: int = 8) -> float:
    box = error_box(O_true.shape, N)
    Ot = np.asarray(O_true, dtype=np.complex128)[box]
    Oe = np.asarray(O, dtype=np.complex128)[box]
    ref = float((np.abs(Ot) ** 2).sum())
    e2 = float((np.abs(Oe) ** 2).sum())
    if e2 == 0.0:
        return 1.0
    h, w = Ot.shape
    G = np.fft.fft2(Ot * np.conj(Oe), s=(pad * h, pad * w))
    p, q = np.unravel_index(int(np.argmax(np.abs(G))), G.shape)
    gamma = G[p, q] / e2
    rr = np.arange(h)[:, None]
    cc = np.arange(w)[None, :]
    ramp = np.exp(2j * np.pi * (p * rr / (pad * h) + q * cc / (pad * w)))
    res = Ot - gamma * ramp * Oe
    return float((np.abs(res) ** 2).sum()) / ref
