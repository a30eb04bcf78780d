"""Pins of the sequential-projections oracle: the noiseless truth is a fixed
point, lam = 0 changes nothing, a step with lam = 1 and the probe held fixed
makes the window's exit wave exactly the projected one when |P| is flat (the
object half), the mirror of that with the object held fixed and |O_j| flat
(the probe half), a hand-derived 2 x 2 step (conjugates, the normalising
maxima and the use of O_j before its update), and the visiting order does not
matter for windows that do not overlap.

Each of the plausible slips in the probe half -- O_j without the conjugate,
the updated window O_j in place of the one the step started from, max|P|^2
in place of max|O_j|^2 -- changes the result of the mirror pin and of the
2 x 2 case (the planted-mistake test below checks that for each)."""
import numpy as np
import pytest

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


def test_flat_object_step_projects_the_window_through_the_probe():
    # |O_j| constant: conj(O_j) d / max|O_j|^2 = d / O_j, so P_new * O_j = psi'
    # exactly, where O_j is the window the step started from.  The object the
    # step updates is a copy, so O itself is held fixed.
    rng = np.random.default_rng(2)
    N = 8
    O = 1.3 * np.exp(1j * rng.uniform(-3, 3, (12, 12)))
    P = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    assert abs((np.abs(P) ** 2).max() - 1.69) > 0.1  # max|P|^2 differs from |O|^2
    sqI = rng.uniform(0.5, 2.0, (N, N))
    Oj = O[2:2 + N, 3:3 + N].copy()
    psi = P * Oj
    target = ptycho.project_D(psi[None], sqI[None])[0][0]
    Pn = P.copy()
    sp.sp_step(O.copy(), Pn, (2, 3), sqI, 1.0)
    np.testing.assert_allclose(Pn * Oj, target, atol=1e-12)


# Hand-derived step on a 2 x 2 problem (one position at (0, 0), N = 2):
#   P = 1 (all four pixels), O = 2i, sqrt(I) = [[2, 0], [0, 0]], lam = 1.
#   psi = P O = 2i everywhere; the 2 x 2 DFT (entries +-1) gives
#   Psi = [[8i, 0], [0, 0]].  Modulus projection: Psi' = [[2 * 8i/8, 0], [0, 0]]
#   = [[2i, 0], [0, 0]] (sqrt(I) = 0 where Psi = 0); inverse DFT with 1/4:
#   psi' = 0.5i everywhere, so d = psi' - psi = -1.5i.
#   max|P|^2 = 1, max|O_j|^2 = 4.
#   O_new = O + conj(P) d / 1     = 2i - 1.5i                 = 0.5i
#   P_new = P + conj(O_j) d / 4   = 1 + (-2i)(-1.5i)/4 = 1 - 0.75 = 0.25
#   error sum (|Psi| - sqrt I)^2  = (8 - 2)^2                 = 36
# The slips give other values: without the conjugate P_new = 1.75; with the
# updated window conj(0.5i)(-1.5i)/0.25 = -3, P_new = -2; with max|P|^2 in the
# probe step P_new = 1 - 3 = -2; with max|O_j|^2 in the object step
# O_new = 2i - 1.5i/4 = 1.625i.
def test_hand_derived_two_by_two_step():
    O = np.full((2, 2), 2j)
    P = np.ones((2, 2), dtype=np.complex128)
    sqI = np.array([[2.0, 0.0], [0.0, 0.0]])
    err = sp.sp_step(O, P, (0, 0), sqI, 1.0)
    assert err == pytest.approx(36.0, abs=1e-12)
    np.testing.assert_allclose(O, np.full((2, 2), 0.5j), atol=1e-14)
    np.testing.assert_allclose(P, np.full((2, 2), 0.25 + 0j), atol=1e-14)


def _sp_step_with_slip(slip, O, P, pos_j, sqrtI_j, lam):
    """sp.sp_step with one plausible slip planted in the probe half (test-only
    copy, so the planted mistake lives here on the CPU, not in the oracle)."""
    N = P.shape[0]
    r, c = int(pos_j[0]), int(pos_j[1])
    Oj = O[r:r + N, c:c + N].copy()
    psi = P * Oj
    Psi = np.fft.fft2(psi)
    target = lam * np.fft.ifft2(ptycho.modulus_projection(Psi, sqrtI_j)) + (1.0 - lam) * psi
    d = target - psi
    mp = float((np.abs(P) ** 2).max())
    mo = float((np.abs(Oj) ** 2).max())
    O[r:r + N, c:c + N] = Oj + np.conj(P) * d / mp
    if slip == "no_conj":
        P += Oj * d / mo
    elif slip == "updated_window":
        On = O[r:r + N, c:c + N]
        P += np.conj(On) * d / float((np.abs(On) ** 2).max())
    elif slip == "max_P":
        P += np.conj(Oj) * d / mp


@pytest.mark.parametrize("slip", ["no_conj", "updated_window", "max_P"])
def test_pins_catch_each_probe_slip(slip):
    # the 2 x 2 case
    O = np.full((2, 2), 2j)
    P = np.ones((2, 2), dtype=np.complex128)
    _sp_step_with_slip(slip, O, P, (0, 0), np.array([[2.0, 0.0], [0.0, 0.0]]), 1.0)
    assert not np.allclose(P, 0.25, atol=1e-6)
    # the mirror pin
    rng = np.random.default_rng(2)
    N = 8
    O = 1.3 * np.exp(1j * rng.uniform(-3, 3, (12, 12)))
    P = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    sqI = rng.uniform(0.5, 2.0, (N, N))
    Oj = O[2:2 + N, 3:3 + N].copy()
    target = ptycho.project_D((P * Oj)[None], sqI[None])[0][0]
    _sp_step_with_slip(slip, O.copy(), P, (2, 3), sqI, 1.0)
    assert not np.allclose(P * Oj, target, atol=1e-6)
