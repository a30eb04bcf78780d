"""Batching and serving: several reconstructions of different sizes and
settings share the GPU; each result must equal (bitwise: the kernels are
deterministic and the reconstructions independent) the result of the same
reconstruction run alone through ptycho_iterate."""
import numpy as np
import pytest

from paper_2311_11466_gb300 import native, serve, synth

from gpu_cases import small_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def scans():
    return [synth.make_scan(small_spec(64, 3, 4, seed=21, photons=1e5)),
            synth.make_scan(small_spec(128, 3, 5, seed=22, photons=1e6)),
            synth.make_scan(small_spec(64, 4, 4, seed=23, photons=None)),
            synth.make_scan(small_spec(256, 2, 3, seed=24, photons=1e7))]


SETTINGS = [native.PRESETS["RAAR"], native.PRESETS["DC"], native.PRESETS["DR"], native.PRESETS["SF"]]


def _alone(scan, abc, n):
    with native.Reconstruction() as r:
        r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
        r.iterate(*abc, n)
        O, P = r.object_probe()
        return r.exit_waves(), O, P, r.errors()


def test_batch_graph_equals_alone(scans):
    n = 6
    recons = []
    for sc in scans:
        r = native.Reconstruction()
        r.load_scan(sc.pos, sc.intensity, sc.obj0, sc.probe0)
        recons.append(r)
    serve.run_batch(recons, SETTINGS, n)
    for r, sc, abc in zip(recons, scans, SETTINGS):
        x, O, P, e = _alone(sc, abc, n)
        Ob, Pb = r.object_probe()
        np.testing.assert_array_equal(Ob, O)
        np.testing.assert_array_equal(Pb, P)
        np.testing.assert_array_equal(r.exit_waves(), x)
        np.testing.assert_array_equal(r.errors(), e)
        assert r.iteration_count == n
        r.close()


def test_server_results_equal_alone(scans):
    n = 7
    arrivals = [0.0, 0.0, 0.02, 0.05]
    recs, wall = serve.run_stream(scans, SETTINGS, n, arrivals, budget_bytes=8 << 30,
                                  max_active=2, iters_per_round=3, keep_results=True)
    for rec, sc, abc in zip(recs, scans, SETTINGS):
        assert rec["state"] == serve.PTYCHO_REQ_DONE
        _, O, P, _ = _alone(sc, abc, n)
        np.testing.assert_array_equal(rec["O"], O)
        np.testing.assert_array_equal(rec["P"], P)
        assert 0 <= rec["queue_s"] <= rec["latency_s"] <= wall + 1e-3
        assert rec["final_error"] > 0


def test_server_rejects_scan_beyond_budget(scans):
    s = serve.ptycho_server_create(1 << 20, 2)
    try:
        sc = scans[1]
        with pytest.raises(native.PtychoError):
            serve.ptycho_server_submit(s, sc.pos, sc.intensity, sc.obj0, sc.probe0, 1, 1, 1, 5)
    finally:
        serve.ptycho_server_destroy(s)
