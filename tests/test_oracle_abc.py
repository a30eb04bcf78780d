"""Pins of the abc driver: relaxation identities, a = 0, DC = P_C P_D, every
preset against its published form, the three-circle example, and the
noiseless ground truth as a fixed point of every setting."""
import copy

import numpy as np
import pytest

from oracle import abc, ptycho, toy
from paper_2311_11466_gb300 import synth


def test_relax_identities():
    proj = lambda v: np.array([3.0, -1.0])  # any map
    x = np.array([0.5, 2.0])
    np.testing.assert_allclose(abc.relax(proj, 1.0)(x), proj(x))
    np.testing.assert_allclose(abc.relax(proj, 2.0)(x), 2 * proj(x) - x)
    np.testing.assert_allclose(abc.relax(proj, 0.0)(x), x)
    np.testing.assert_allclose(abc.relax(proj, 0.5)(x), (proj(x) + x) / 2)


def _blind(seed=0, N=8, M=(22, 25), J=7):
    rng = np.random.default_rng(seed)
    O = (0.8 + 0.2 * rng.uniform(size=M)) * np.exp(1j * rng.uniform(-1, 1, size=M))
    P = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    pos = np.stack([rng.integers(0, M[0] - N + 1, size=J),
                    rng.integers(0, M[1] - N + 1, size=J)], axis=1)
    I = np.stack([np.abs(np.fft.fft2(e)) ** 2 for e in ptycho.exit_waves(P, O, pos)])
    prob = ptycho.Problem(I, pos, np.ones(M), P + 0.3 * rng.standard_normal((N, N)), alpha=1e-6)
    x = rng.standard_normal((J, N, N)) + 1j * rng.standard_normal((J, N, N))
    return prob, x


def _abc(prob, x, a, b, c):
    p = copy.deepcopy(prob)
    return p.iterate(x, a, b, c), p


def test_a_zero_is_identity():
    prob, x = _blind(1)
    out, _ = _abc(prob, x, 0.0, 1.3, 0.7)
    np.testing.assert_array_equal(out, x)


def test_dc_is_concur_after_divide():
    prob, x = _blind(2)
    out, _ = _abc(prob, x, *abc.preset("DC"))
    p = copy.deepcopy(prob)
    ref = p.project_C(p.project_D(x))
    np.testing.assert_allclose(out, ref, atol=1e-12)


def _published(name, prob, x, beta=None):
    p = copy.deepcopy(prob)
    pd = p.project_D(x)
    if name == "DC":
        return p.project_C(pd)
    if name == "AR":          # R_C R_D x
        rd = 2 * pd - x
        return 2 * p.project_C(rd) - rd
    if name == "DR":          # x + P_C(2 P_D x - x) - P_D x
        return x + p.project_C(2 * pd - x) - pd
    if name == "SF":          # R_C P_D x
        return 2 * p.project_C(pd) - pd
    if name == "RAAR":        # (beta/2)(R_C R_D + I) x + (1 - beta) P_D x
        rd = 2 * pd - x
        return beta / 2 * (2 * p.project_C(rd) - rd + x) + (1 - beta) * pd
    if name == "RRR":         # x + beta (P_C(2 P_D x - x) - P_D x)
        return x + beta * (p.project_C(2 * pd - x) - pd)
    raise KeyError(name)


@pytest.mark.parametrize("name,beta", [("DC", None), ("AR", None), ("DR", None), ("SF", None),
                                       ("RAAR", 0.9), ("RAAR", 0.75), ("RRR", 0.5), ("RRR", 1.0)])
def test_preset_matches_published_form(name, beta):
    prob, x = _blind(3)
    out, _ = _abc(prob, x, *abc.preset(name, beta))
    ref = _published(name, prob, x, beta)
    np.testing.assert_allclose(out, ref, atol=1e-11 * np.abs(ref).max())


def test_three_circles_fixed_point_and_dc():
    rng = np.random.default_rng(0)
    p_star = np.array([0.3, -0.2])
    centres = [p_star + 2.0 * np.array([np.cos(t), np.sin(t)]) for t in (0.1, 2.2, 4.1)]
    tc = toy.ThreeCircles(centres, [2.0, 2.0, 2.0])
    xs = np.stack([p_star] * 3)
    for name in ["DC", "AR", "DR", "SF", "RAAR", "RRR"]:
        out = abc.abc_step(xs, tc.project_D, tc.project_C, *abc.preset(name))
        np.testing.assert_allclose(out, xs, atol=1e-14)
    x = xs + 0.05 * rng.standard_normal((3, 2))
    for _ in range(500):
        x = abc.abc_step(x, tc.project_D, tc.project_C, *abc.preset("DC"))
    np.testing.assert_allclose(x, xs, atol=1e-6)
    # divide output lies on the circles; concur output is a consensus
    d = tc.project_D(xs + rng.standard_normal((3, 2)))
    for i in range(3):
        assert abs(np.hypot(*(d[i] - centres[i])) - 2.0) < 1e-12
    c = tc.project_C(d)
    np.testing.assert_allclose(tc.project_C(c), c)
    np.testing.assert_allclose(c[0], c[1])


def test_three_circles_dr_finds_intersection():
    p_star = np.array([1.0, 0.5])
    centres = [p_star + np.array([1.5, 0.0]), p_star + np.array([-0.5, 1.2]),
               p_star + np.array([0.2, -1.7])]
    radii = [float(np.hypot(*(p_star - c))) for c in centres]
    tc = toy.ThreeCircles(centres, radii)
    x = np.stack([p_star + np.array([0.1, -0.05])] * 3)
    for _ in range(2000):
        x = abc.abc_step(x, tc.project_D, tc.project_C, *abc.preset("DR"))
    sol = tc.project_D(x)   # the shadow sequence P_D x carries the solution
    np.testing.assert_allclose(sol, np.stack([p_star] * 3), atol=1e-6)


@pytest.mark.parametrize("name", ["DC", "AR", "DR", "SF", "RAAR", "RRR"])
def test_noiseless_truth_is_fixed_point(name):
    scan = synth.make_scan(synth.named_spec("tiny"))
    x_true = ptycho.exit_waves(scan.probe_true, scan.obj_true, scan.pos)
    prob = ptycho.Problem(scan.intensity64, scan.pos, scan.obj_true, scan.probe_true, alpha=0.0)
    out = prob.iterate(x_true, *abc.preset(name))
    assert np.abs(out - x_true).max() <= 1e-11 * np.abs(x_true).max()
    assert prob.last_error < 1e-24
    prob = ptycho.Problem(scan.intensity64, scan.pos, scan.obj_true, scan.probe_true, alpha=1e-6)
    out = prob.iterate(x_true, *abc.preset(name))
    assert np.abs(out - x_true).max() <= 1e-5 * np.abs(x_true).max()


def test_fixed_point_up_to_global_phase():
    # the truth with a global phase on the object (and the inverse on nothing) is
    # still a fixed point: every exit wave carries the same phase factor
    scan = synth.make_scan(synth.named_spec("tiny"))
    ph = np.exp(0.7j)
    x = ptycho.exit_waves(scan.probe_true, scan.obj_true * ph, scan.pos)
    prob = ptycho.Problem(scan.intensity64, scan.pos, scan.obj_true * ph, scan.probe_true, alpha=0.0)
    out = prob.iterate(x, *abc.preset("RAAR"))
    assert np.abs(out - x).max() <= 1e-11 * np.abs(x).max()
