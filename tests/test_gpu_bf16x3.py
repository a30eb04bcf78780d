"""Tensor-core precision path (PTYCHO_PREC_BF16X3): the divide step's DFTs as
dense GEMMs with BF16 hi/lo operands (three products, FP32 accumulation),
against the FP64 oracle.  Tolerance: relative L2 <= 5e-3 after one iteration
(exit waves, object, probe) and on the per-iteration Fourier error; measured
errors are far below (about 1e-5), and the test also bounds them against the
FP32 path's."""
import numpy as np
import pytest

from oracle import abc as oabc, metrics, ptycho as optycho
from paper_2311_11466_gb300 import native, synth

from gpu_cases import gpu_recon, oracle_problem, rel_l2, small_spec

pytestmark = pytest.mark.gpu

TOL = 5e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


@pytest.fixture(scope="module", params=[128, 256])
def scan(request):
    N = request.param
    return synth.make_scan(small_spec(N, 3, 4, seed=100 + N, photons=1e6))


@pytest.mark.parametrize("c", [1.0, 2.0])
def test_divide_step(scan, c):
    prob, x0 = oracle_problem(scan)
    y_ref = oabc.relax(prob.project_D, c)(x0)
    with gpu_recon(scan, precision="bf16x3") as r:
        r.iterate(1.0, 0.0, c, 1)
        y = r.exit_waves()
        e = r.errors()
    err = rel_l2(y, y_ref)
    print(f"N={scan.N} c={c}: divide rel L2 {err:.2e}")
    assert err <= TOL
    assert err <= 1e-4        # three-product BF16 is near FP32 quality
    assert abs(e[0] - prob.last_error) <= TOL * prob.last_error


@pytest.mark.parametrize("name", ["DC", "DR", "RAAR", "RRR"])
def test_one_iteration(scan, name):
    abc = native.PRESETS[name]
    prob, x0 = oracle_problem(scan)
    x1 = prob.iterate(x0, *abc)
    with gpu_recon(scan, precision="bf16x3") as r:
        r.iterate(*abc, 1)
        x = r.exit_waves()
        O, P = r.object_probe()
    for got, ref in ((x, x1), (O, prob.O), (P, prob.P)):
        assert rel_l2(got, ref) <= TOL


def test_iterations_track_the_fp32_path(scan):
    abc = native.PRESETS["DC"]
    with gpu_recon(scan, precision="bf16x3") as r:
        r.iterate(*abc, 20)
        e16 = r.errors()
        O16, _ = r.object_probe()
    with gpu_recon(scan) as r:
        r.iterate(*abc, 20)
        e32 = r.errors()
        O32, _ = r.object_probe()
    np.testing.assert_allclose(e16, e32, rtol=TOL)
    assert rel_l2(O16, O32) <= TOL


def test_odd_row_block_count():
    """J = 9 waves of 128 x 128: an odd number of 128-row blocks, so one CTA
    pair of the GEMM has a block beyond the last wave (loaded as zeros, no
    output)."""
    sc = synth.make_scan(small_spec(128, 3, 3, seed=77, photons=1e6))
    assert sc.J == 9
    prob, x0 = oracle_problem(sc)
    y_ref = oabc.relax(prob.project_D, 2.0)(x0)
    with gpu_recon(sc, precision="bf16x3") as r:
        r.iterate(1.0, 0.0, 2.0, 1)
        y = r.exit_waves()
        e = r.errors()
    assert rel_l2(y, y_ref) <= 1e-4
    assert abs(e[0] - prob.last_error) <= TOL * prob.last_error


def test_sp_and_model_error_on_tensor_core_context(scan):
    """Sequential projections and the model error run the FP32 kernels in
    either kind of context: from the same start a tensor-core context gives
    bitwise the FP32 context's object, probe and model error."""
    out = []
    for prec in ("fp32", "bf16x3"):
        with gpu_recon(scan, precision=prec) as r:
            r.sp_iterate(0.8, 1)
            O, P = r.object_probe()
            out.append((O, P, r.model_error()))
    (O32, P32, m32), (O16, P16, m16) = out
    np.testing.assert_array_equal(O16, O32)
    np.testing.assert_array_equal(P16, P32)
    assert m16 == m32


def test_bf16x3_rejects_other_sizes():
    sc = synth.make_scan(small_spec(64, 2, 2, seed=3))
    with native.Reconstruction(precision="bf16x3") as r:
        with pytest.raises(native.PtychoError) as ei:
            r.load_scan(sc.pos, sc.intensity, sc.obj0, sc.probe0)
        assert ei.value.code == native.PTYCHO_EINVAL
