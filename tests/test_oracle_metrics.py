"""Pins of the error metrics: closed-form values of the Fourier error and of
the ambiguity-corrected object error."""
import numpy as np
import pytest

from oracle import metrics, ptycho
from paper_2311_11466_gb300 import synth


@pytest.fixture(scope="module")
def tiny():
    return synth.make_scan(synth.named_spec("tiny"))


def test_fourier_error_closed_forms(tiny):
    x = ptycho.exit_waves(tiny.probe_true, tiny.obj_true, tiny.pos)
    I = tiny.intensity64
    assert metrics.fourier_error(x, I) < 1e-24
    # |F 2x| = 2 sqrt(I): sum (2s - s)^2 / sum s^2 = 1
    assert abs(metrics.fourier_error(2 * x, I) - 1.0) < 1e-12
    assert abs(metrics.fourier_error(0 * x, I) - 1.0) < 1e-12
    # a global phase and a shift of the exit wave do not change |F x|
    xs = np.roll(x, (3, 5), axis=(1, 2)) * np.exp(0.4j)
    assert metrics.fourier_error(xs, I) < 1e-24


def test_divide_error_equals_metric(tiny):
    rng = np.random.default_rng(0)
    x = ptycho.exit_waves(tiny.probe_true, tiny.obj_true, tiny.pos) * (1 + 0.1 * rng.standard_normal())
    prob = ptycho.Problem(tiny.intensity64, tiny.pos, tiny.obj0, tiny.probe0)
    prob.project_D(x)
    assert abs(prob.last_error - metrics.fourier_error(x, tiny.intensity64)) < 1e-12


def test_object_error_ambiguities(tiny):
    Ot, N = tiny.obj_true, tiny.N
    assert metrics.object_error(Ot, Ot, N) < 1e-24
    assert metrics.object_error(0 * Ot, Ot, N) == 1.0
    h, w = Ot.shape
    rr, cc = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    # ramp on the 8x-padded grid of the error box, plus a complex scale
    bh, bw = h - N, w - N
    ramp = np.exp(2j * np.pi * (3 * rr / (8 * bh) - 5 * cc / (8 * bw)))
    O = (0.5 - 0.2j) * ramp * Ot
    assert metrics.object_error(O, Ot, N) < 1e-20
    # outside the box nothing counts
    O2 = Ot.copy()
    O2[:N // 2] = 0
    assert metrics.object_error(O2, Ot, N) < 1e-24


def test_object_error_of_noise(tiny):
    rng = np.random.default_rng(1)
    Ot, N = tiny.obj_true, tiny.N
    noise = 0.05 * (rng.standard_normal(Ot.shape) + 1j * rng.standard_normal(Ot.shape))
    e = metrics.object_error(Ot + noise, Ot, N)
    box = metrics.error_box(Ot.shape, N)
    ratio = (np.abs(noise[box]) ** 2).sum() / (np.abs(Ot[box]) ** 2).sum()
    # the fitted scale absorbs a little of the noise: e is just below the raw ratio
    assert 0.9 * ratio < e <= ratio * (1 + 1e-9)
