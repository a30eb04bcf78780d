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


@pytest.mark.parametrize("mode", [serve.PTYCHO_BATCH_GROUPS, serve.PTYCHO_BATCH_BRANCHES,
                                  serve.PTYCHO_BATCH_AUTO])
def test_batch_graph_equals_alone(scans, mode):
    n = 6
    recons = []
    for sc in scans:
        r = native.Reconstruction()
        r.load_scan(sc.pos, sc.intensity, sc.obj0, sc.probe0)
        recons.append(r)
    info = serve.run_batch(recons, SETTINGS, n, mode=mode)
    # every context is an FP32 cluster-design context: with launch groups, all
    # of them run in the groups, one per pattern side (64, 128, 256)
    if mode == serve.PTYCHO_BATCH_GROUPS:
        assert (info["groups"], info["in_groups"], info["used"]) == (3, len(scans), "groups")
    elif mode == serve.PTYCHO_BATCH_BRANCHES:
        assert (info["groups"], info["used"]) == (0, "branches")
    else:
        assert info["groups_ms"] > 0 and info["branches_ms"] > 0
        assert info["used"] == ("groups" if info["groups_ms"] <= info["branches_ms"] else "branches")
    for r, sc, abc in zip(recons, scans, SETTINGS):
        x, O, P, e = _alone(sc, abc, n)
        Ob, Pb = r.object_probe()
        np.testing.assert_array_equal(Ob, O)
        np.testing.assert_array_equal(Pb, P)
        np.testing.assert_array_equal(r.exit_waves(), x)
        np.testing.assert_array_equal(r.errors(), e)
        assert r.iteration_count == n
        r.close()


def test_batch_with_tensor_core_context(scans):
    """A batch mixing an FP32 context and a tensor-core (BF16 x 3) context:
    the captured graph replays both, each bitwise equal to its run alone."""
    n = 4
    sc32, sc16 = scans[0], scans[1]
    r32 = native.Reconstruction()
    r32.load_scan(sc32.pos, sc32.intensity, sc32.obj0, sc32.probe0)
    r16 = native.Reconstruction(precision="bf16x3")
    r16.load_scan(sc16.pos, sc16.intensity, sc16.obj0, sc16.probe0)
    abc = native.PRESETS["RAAR"]
    serve.run_batch([r32, r16], [abc, abc], n)
    for r, sc, prec in ((r32, sc32, "fp32"), (r16, sc16, "bf16x3")):
        with native.Reconstruction(precision=prec) as ra:
            ra.load_scan(sc.pos, sc.intensity, sc.obj0, sc.probe0)
            ra.iterate(*abc, n)
            O, P = ra.object_probe()
            e = ra.errors()
        Ob, Pb = r.object_probe()
        np.testing.assert_array_equal(Ob, O)
        np.testing.assert_array_equal(Pb, P)
        np.testing.assert_array_equal(r.errors(), e)
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


def test_server_tensor_core_requests(scans):
    """A server whose contexts use the tensor-core path (server options carry
    the precision): two requests (128^2 and 256^2) served in interleaved
    rounds, each bitwise equal to the same reconstruction run alone."""
    n = 5
    abc = native.PRESETS["DR"]
    o = native.ptycho_default_opts()
    o.precision = native.PTYCHO_PREC_BF16X3
    s = serve.ptycho_server_create(8 << 30, 2, o)
    try:
        picks = [scans[1], scans[3]]
        ids = [serve.ptycho_server_submit(s, sc.pos, sc.intensity, sc.obj0, sc.probe0, *abc, n)
               for sc in picks]
        for _ in range(100):
            na, nq = serve.ptycho_server_step(s, 2)
            if na == 0 and nq == 0:
                break
        for rid, sc in zip(ids, picks):
            O = np.empty(sc.M_shape, dtype=np.complex64)
            P = np.empty((sc.N, sc.N), dtype=np.complex64)
            st, _ = serve.ptycho_server_poll(s, rid, O, P)
            assert st == serve.PTYCHO_REQ_DONE
            with native.Reconstruction(precision="bf16x3") as r:
                r.load_scan(sc.pos, sc.intensity, sc.obj0, sc.probe0)
                r.iterate(*abc, n)
                Oa, Pa = r.object_probe()
            np.testing.assert_array_equal(O, Oa)
            np.testing.assert_array_equal(P, Pa)
    finally:
        serve.ptycho_server_destroy(s)
