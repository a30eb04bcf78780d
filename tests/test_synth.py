"""The shared input generator: geometry, normalisation and determinism."""
import numpy as np
import pytest

from paper_2311_11466_gb300 import synth


def test_tiny_geometry():
    s = synth.make_scan(synth.named_spec("tiny"))
    assert s.pos.dtype == np.int32 and s.pos.shape == (64, 2)
    assert s.obj_true.shape == (176, 176)
    assert s.pos.min() >= 0 and s.pos.max() <= 176 - 64
    amp = np.abs(s.obj_true)
    assert 0.8 <= amp.min() and amp.max() <= 1.0
    ph = np.angle(s.obj_true)
    assert abs(ph.min() + np.pi / 2) < 1e-9 and abs(ph.max() - np.pi / 2) < 1e-9
    # raster step 16 with jitter at most 2 (before clamping)
    d = np.diff(s.pos[:8, 1].astype(int))
    assert np.all(np.abs(d - 16) <= 4)


def test_probe_start_normalisation():
    s = synth.make_scan(synth.named_spec("tiny"))
    N = s.N
    lhs = N * N * (np.abs(s.probe0.astype(np.complex128)) ** 2).sum()
    rhs = s.intensity.astype(np.float64).sum(axis=(1, 2)).mean()
    assert abs(lhs / rhs - 1) < 1e-6
    np.testing.assert_array_equal(s.obj0, np.ones_like(s.obj0))


def test_deterministic():
    a = synth.make_scan(synth.named_spec("tiny"))
    b = synth.make_scan(synth.named_spec("tiny"))
    np.testing.assert_array_equal(a.intensity, b.intensity)
    np.testing.assert_array_equal(a.pos, b.pos)


def test_poisson_scaling():
    spec = synth.named_spec("tiny", photons=1e5)
    s = synth.make_scan(spec)
    tot = s.intensity.astype(np.float64).sum(axis=(1, 2)).mean()
    assert abs(tot / 1e5 - 1) < 0.02
    assert np.all(s.intensity == np.round(s.intensity))


def test_fermat_and_batch_specs():
    specs = synth.batch_specs(16)
    assert len(specs) == 16
    assert {sp.N for sp in specs} <= {128, 256}
    for sp in specs:
        assert 100 <= sp.J <= 2000
    fs = synth.ScanSpec(N=64, step=8, radius=16, geometry="fermat", n_fermat=200, seed=3)
    s = synth.make_scan(fs, with_data=False)
    M = s.M_shape
    assert s.pos.min() >= 0
    assert s.pos[:, 0].max() <= M[0] - 64 and s.pos[:, 1].max() <= M[1] - 64
    # mean nearest-neighbour spacing is of the order of the step
    p = s.pos.astype(float)
    d = np.sqrt(((p[:, None] - p[None]) ** 2).sum(-1)) + np.eye(len(p)) * 1e9
    assert 4 < d.min(axis=1).mean() < 12


def test_product_object_error_matches_oracle():
    # the library's own object-error metric (used by the benchmark) against the
    # oracle's independent implementation of the same reading
    from oracle import metrics as om
    from paper_2311_11466_gb300 import metrics as pm
    s = synth.make_scan(synth.named_spec("tiny"))
    rng = np.random.default_rng(3)
    rr, cc = np.meshgrid(np.arange(176), np.arange(176), indexing="ij")
    for trial in range(3):
        O = (0.7 - 0.3j) * np.exp(2j * np.pi * (rr * 5 / 896 + cc * 2 / 896)) * s.obj_true
        O = O + 0.05 * trial * (rng.standard_normal(O.shape) + 1j * rng.standard_normal(O.shape))
        a, b = pm.object_error(O, s.obj_true, s.N), om.object_error(O, s.obj_true, s.N)
        assert abs(a - b) <= 1e-12 + 1e-9 * b
    assert pm.object_error(0 * s.obj_true, s.obj_true, s.N) == 1.0
