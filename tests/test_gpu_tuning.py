"""The autotuner of launch shapes (ptycho_tuning, ptycho_set_tuning,
ptycho_set_launch_shapes) changes no arithmetic: every candidate -- the four
object-gather tiles, one or two probe pixels per thread, and at 128 x 128 the
two cluster shapes of the divide kernel -- gives bit-identical exit waves,
object, probe and error history, so the tuner's choice cannot move a
result.  The tuner reports what it measured and picks the fastest candidate.
"""
import numpy as np
import pytest

from paper_2311_11466_gb300 import native, synth

from gpu_cases import small_spec

pytestmark = pytest.mark.gpu

TILES = [(16, 32), (8, 32), (32, 32), (8, 64)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


def _run(scan, shapes=None, tune=False, n=3):
    abc = native.PRESETS["RAAR"]
    with native.Reconstruction() as r:
        r.set_tuning(tune)
        r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
        if shapes is not None:
            r.set_launch_shapes(*shapes)
        r.iterate(*abc, n)
        O, P = r.object_probe()
        return (r.exit_waves(), O, P, r.errors()), r.tuning()


@pytest.mark.parametrize("N", [128, 256])
def test_every_launch_shape_gives_identical_bits(N):
    scan = synth.make_scan(small_spec(N, ny=3, nx=5, photons=1e6, seed=50 + N))
    ref, _ = _run(scan, shapes=(16, 32, 1, 8 if N == 128 else 0))
    clusters = [8, 16] if N == 128 else [0]
    for (tr, tc) in TILES:
        for ppt in (1, 2):
            for cs in clusters:
                got, info = _run(scan, shapes=(tr, tc, ppt, cs))
                assert info["gather_tile"] == (tr, tc) and info["probe_pixels_per_thread"] == ppt
                if cs:
                    assert info["cluster_size"] == cs
                for a, b in zip(got, ref):
                    np.testing.assert_array_equal(a, b, err_msg=f"{(tr, tc, ppt, cs)}")


def test_tuner_reports_and_picks_the_fastest():
    scan = synth.make_scan(small_spec(128, ny=4, nx=5, photons=1e6, seed=61))
    ref, _ = _run(scan, shapes=(16, 32, 1, 8))
    got, info = _run(scan, tune=True)
    assert info["tuned"]
    ms = info["gather_ms"]
    assert all(v > 0 for v in ms.values()), ms
    best = min(ms, key=ms.get)
    assert f"{info['gather_tile'][0]}x{info['gather_tile'][1]}" == best
    pm = info["probe_ms"]
    assert pm["1"] > 0 and pm["2"] > 0
    assert info["probe_pixels_per_thread"] == (2 if pm["2"] < pm["1"] else 1)
    dm = info["divide128_ms"]
    assert dm["8x128"] > 0 and dm["16x64"] > 0
    assert info["cluster_size"] == (16 if dm["16x64"] < dm["8x128"] else 8)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_pinning_rejects_non_candidates():
    scan = synth.make_scan(small_spec(64, ny=2, nx=2, seed=62))
    with native.Reconstruction() as r:
        r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
        with pytest.raises(native.PtychoError):
            r.set_launch_shapes(12, 32, 1)
        with pytest.raises(native.PtychoError):
            r.set_launch_shapes(16, 32, 3)
        with pytest.raises(native.PtychoError):
            r.set_launch_shapes(16, 32, 1, 16)   # cluster size only at N = 128
