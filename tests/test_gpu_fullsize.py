"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (one context, FP32, 1024 exit waves of 256 x 256 on a 1300 x 1300
object, with either concur mode; the 4096-wave precision workload on the tensor-core path; and the
4096-wave 128 x 128 workload on the FP32 path).

The FP64 oracle runs one whole RAAR iteration of the 1024-wave scan (about
half a minute on the host), so exit waves, object and probe are compared in
full; on the 4096-wave scans the oracle computes the divided exit waves of a
sample of positions one by one.  Tolerances as in the small-size parity
tests: relative L2 <= 1e-5 (FP32) and <= 5e-3 (BF16 x 3).
"""
import numpy as np
import pytest

from oracle import abc as oabc, ptycho as optycho
from paper_2311_11466_gb300 import native, synth

from gpu_cases import gpu_recon, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def large():
    return synth.make_scan(synth.named_spec("large"))


@pytest.fixture(scope="module")
def large_ref(large):
    """One FP64 RAAR iteration of the whole 1024-wave scan: x_1, O_1, P_1, E_F."""
    prob, x0 = oracle_problem(large)
    x1 = prob.iterate(x0, *native.PRESETS["RAAR"])
    return x1, prob.O, prob.P, prob.last_error


@pytest.mark.parametrize("name", ["DC", "SF", "RRR"])
def test_large_two_iterations_other_presets(large, name):
    """The divide kernel's other input paths at full size, two iterations so
    the second forms x_k from the lazy re-split: DC (no y_{k-1}, no x_{k-1}),
    SF (a = 1: y_{k-1} but no x_{k-1}), RRR (both).  Exit waves, object, probe
    and both Fourier errors against the FP64 oracle, 2e-5 (two iterations)."""
    abc = native.PRESETS[name]
    prob, x = oracle_problem(large)
    errs = []
    for _ in range(2):
        x = prob.iterate(x, *abc)
        errs.append(prob.last_error)
    with gpu_recon(large) as r:
        r.iterate(*abc, 2)
        O, P = r.object_probe()
        e = r.errors()
        xg = r.exit_waves()
    assert rel_l2(xg, x) <= 2e-5
    assert rel_l2(O, prob.O) <= 2e-5
    assert rel_l2(P, prob.P) <= 2e-5
    np.testing.assert_allclose(e, errs, rtol=2e-5)


@pytest.mark.parametrize("concur", ["deterministic", "atomic"])
def test_large_raar_iteration_in_full(large, large_ref, concur):
    x1, O_ref, P_ref, e_ref = large_ref
    with gpu_recon(large, concur=concur) as r:
        r.iterate(*native.PRESETS["RAAR"], 1)
        O, P = r.object_probe()
        e = r.errors()
        x = r.exit_waves()
    assert rel_l2(x, x1) <= 1e-5
    assert rel_l2(O, O_ref) <= 1e-5
    assert rel_l2(P, P_ref) <= 1e-5
    assert abs(e[0] - e_ref) <= 1e-5 * e_ref
    # worst single exit wave, not only the aggregate
    worst = max(rel_l2(x[j], x1[j]) for j in range(0, large.J, 37))
    assert worst <= 1e-5


def test_precision_workload_sampled_divide():
    scan = synth.make_scan(synth.named_spec("precision"))
    sample = [0, 1, 63, 64, 2047, 2048, 4031, 4095]
    with gpu_recon(scan, precision="bf16x3") as r:
        r.iterate(1.0, 0.0, 2.0, 1)   # x_1 = y_0 = P^2_D x_0
        y = r.exit_waves()
    P0 = scan.probe0.astype(np.complex128)
    O0 = scan.obj0.astype(np.complex128)
    for j in sample:
        xj = optycho.exit_waves(P0, O0, scan.pos[j:j + 1])
        sq = np.sqrt(scan.intensity[j:j + 1].astype(np.float64))
        yj = oabc.relax(lambda v: optycho.project_D(v, sq)[0], 2.0)(xj)
        assert rel_l2(y[j], yj[0]) <= 5e-3
        assert rel_l2(y[j], yj[0]) <= 1e-4


def test_large128_sampled_divide():
    """4096 exit waves of 128 x 128 (the 128^2 bench workload, clusters of 8
    CTAs): the divided exit waves of sampled positions against the oracle,
    FP32 tolerance."""
    scan = synth.make_scan(synth.named_spec("large128"))
    sample = [0, 1, 7, 8, 63, 64, 2047, 2048, 4031, 4095]
    with gpu_recon(scan) as r:
        r.iterate(1.0, 0.0, 2.0, 1)   # x_1 = y_0 = P^2_D x_0
        y = r.exit_waves()
    P0 = scan.probe0.astype(np.complex128)
    O0 = scan.obj0.astype(np.complex128)
    for j in sample:
        xj = optycho.exit_waves(P0, O0, scan.pos[j:j + 1])
        sq = np.sqrt(scan.intensity[j:j + 1].astype(np.float64))
        yj = oabc.relax(lambda v: optycho.project_D(v, sq)[0], 2.0)(xj)
        assert rel_l2(y[j], yj[0]) <= 1e-5
