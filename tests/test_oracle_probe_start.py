"""Pins of the oracle's probe-start reading (the concur step keeps the probe
fixed in iterations k < probe_start).

1. The probe is bitwise unchanged through iteration probe_start - 1 and
   changes in the next one; probe_start = 0 is the default behaviour.
2. With the probe held at the true probe and alpha = 0, the consensus set
   {P * O_j : O} is a linear subspace of the product space and the object
   sweep is the orthogonal (least-squares) projection onto it, so DC =
   P_C P_D is alternating projections between that subspace and the
   Fourier-modulus set; its error E_F(x_k) = ||F x_k - P_D-part||^2, by
   Parseval N^2 ||x_k - P_D x_k||^2, cannot increase from one iteration to
   the next (the error-reduction property of alternating projections).
"""
import numpy as np

from oracle import ptycho as optycho
from paper_2311_11466_gb300 import synth


def _tiny():
    return synth.make_scan(synth.named_spec("tiny"))


def test_probe_held_until_start_then_updated():
    s = _tiny()
    prob = optycho.Problem(s.intensity64, s.pos, s.obj0.astype(np.complex128),
                           s.probe0.astype(np.complex128), probe_start=2)
    P0 = prob.P.copy()
    x = optycho.exit_waves(prob.P, prob.O, s.pos)
    for k in range(2):
        x = prob.iterate(x, 0.5, 1.8, 2.0)
        assert np.array_equal(prob.P, P0), k
    x = prob.iterate(x, 0.5, 1.8, 2.0)
    assert not np.allclose(prob.P, P0)
    # probe_start = 0 is the default reading
    a = optycho.Problem(s.intensity64, s.pos, s.obj0.astype(np.complex128),
                        s.probe0.astype(np.complex128))
    b = optycho.Problem(s.intensity64, s.pos, s.obj0.astype(np.complex128),
                        s.probe0.astype(np.complex128), probe_start=0)
    xa = xb = optycho.exit_waves(a.P, a.O, s.pos)
    for _ in range(2):
        xa = a.iterate(xa, 0.5, 1.8, 2.0)
        xb = b.iterate(xb, 0.5, 1.8, 2.0)
    assert np.array_equal(xa, xb) and np.array_equal(a.P, b.P)


def test_known_probe_dc_is_error_reduction():
    s = _tiny()
    prob = optycho.Problem(s.intensity64, s.pos, np.ones(s.M_shape, dtype=np.complex128),
                           s.probe_true.astype(np.complex128), alpha=0.0, probe_start=10 ** 6)
    x = optycho.exit_waves(prob.P, prob.O, s.pos)
    errs = []
    for _ in range(20):
        x = prob.iterate(x, 1.0, 1.0, 1.0)
        errs.append(prob.last_error)
    errs = np.array(errs)
    assert np.all(np.diff(errs) <= 1e-12 * errs[:-1]), errs
    assert errs[-1] < 0.5 * errs[0]
    assert np.array_equal(prob.P, s.probe_true.astype(np.complex128))
