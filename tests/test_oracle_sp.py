"""Pins of the sequential-projections oracle: the noiseless truth is a fixed
point, lam = 0 changes nothing, a step with lam = 1 and the probe held fixed
makes the window's exit wave exactly the projected one when |P| is flat,
and the visiting order does not matter for windows that do not overlap."""
import numpy as np

from oracle import ptycho, sp
from paper_2311_11466_gb300 import synth


def test_truth_is_fixed_point():
    s = synth.make_scan(synth.named_spec("tiny"))
    O, P = s.obj_true.copy(), s.probe_true.copy()
    e = sp.sp_iterate(O, P, s.pos, s.intensity64, 1.0)
    assert e < 1e-24
    np.testing.assert_allclose(O, s.obj_true, atol=1e-12)
    np.testing.assert_allclose(P, s.probe_true, atol=1e-12)


def test_lambda_zero_is_identity():
    s = synth.make_scan(synth.named_spec("tiny"))
    O, P = s.obj0.astype(np.complex128), s.probe0.astype(np.complex128)
    O0, P0 = O.copy(), P.copy()
    sp.sp_iterate(O, P, s.pos, s.intensity, 0.0)
    np.testing.assert_array_equal(O, O0)
    np.testing.assert_array_equal(P, P0)


def test_flat_probe_step_projects_the_window():
    # |P| constant: conj(P) d / max|P|^2 = d / P, so P * O_new = psi' exactly
    rng = np.random.default_rng(0)
    N = 8
    P = 1.7 * np.exp(1j * rng.uniform(-3, 3, (N, N)))
    O = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    sqI = rng.uniform(0.5, 2.0, (N, N))
    Pc = P.copy()
    psi = P * O[2:2 + N, 3:3 + N]
    target = ptycho.project_D(psi[None], sqI[None])[0][0]
    sp.sp_step(O, Pc, (2, 3), sqI, 1.0)
    np.testing.assert_allclose(P * O[2:2 + N, 3:3 + N], target, atol=1e-12)


def test_order_free_for_disjoint_windows():
    rng = np.random.default_rng(1)
    N = 8
    pos = np.array([[0, 0], [0, 8], [8, 0], [8, 8]])
    O = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    P = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    I = rng.uniform(0.5, 3.0, (4, N, N))
    # with P updated between steps the order matters; hold P by giving each
    # window its own copy of the problem: compare O only through one step each
    O1, P1 = O.copy(), P.copy()
    O2, P2 = O.copy(), P.copy()
    for j in [0, 1, 2, 3]:
        sp.sp_step(O1, P.copy(), pos[j], np.sqrt(I[j]), 0.8)
    for j in [3, 1, 0, 2]:
        sp.sp_step(O2, P.copy(), pos[j], np.sqrt(I[j]), 0.8)
    np.testing.assert_allclose(O1, O2, atol=1e-14)
