"""Host-side evaluation of a reconstruction's object (FP64, numpy).

The paper's error curves (Figs. 7 and 8) compare reconstructions inside an
error-metric box of the object (Fig. 5) without defining the metric.  This
module is the library's own reading, used by the benchmark's comparison mode:
inside the box [N/2, M - N/2) on both axes, the blind ambiguities (a global
complex factor and a linear phase ramp) are removed before comparing with the
true object:

    err = min over g, k of  sum |O_true - g exp(i k.r) O|^2 / sum |O_true|^2.

The ramp k is located at the peak of an 8x zero-padded 2-D FFT of
O_true * conj(O) over the box; g then follows in closed form.
"""
from __future__ import annotations

import numpy as np


def object_error(O: np.ndarray, O_true: np.ndarray, N: int, pad: int = 8) -> float:
    h0 = N // 2
    rows = slice(h0, O_true.shape[0] - h0)
    cols = slice(h0, O_true.shape[1] - h0)
    t = np.asarray(O_true, dtype=np.complex128)[rows, cols]
    o = np.asarray(O, dtype=np.complex128)[rows, cols]
    norm_o = float(np.vdot(o, o).real)
    if norm_o == 0.0:
        return 1.0
    h, w = t.shape
    spec = np.fft.fft2(t * o.conj(), s=(pad * h, pad * w))
    p, q = np.unravel_index(int(np.argmax(np.abs(spec))), spec.shape)
    g = spec[p, q] / norm_o
    phase = np.exp(2j * np.pi * (np.outer(np.arange(h), np.ones(w)) * (p / (pad * h)) +
                                 np.outer(np.ones(h), np.arange(w)) * (q / (pad * w))))
    resid = t - g * phase * o
    return float(np.vdot(resid, resid).real / np.vdot(t, t).real)
