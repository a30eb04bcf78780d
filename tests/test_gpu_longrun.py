"""Long-run parity: 100 iterations of the tiny scan (64 patterns of 64 x 64,
blind start) for DC, DR and RAAR(0.9); the final Fourier error of the model
and the phase-ramp-corrected object error agree with the FP64 oracle's within
1e-3 relative, and the per-iteration error curve tracks the oracle's."""
import numpy as np
import pytest

from oracle import metrics, ptycho as optycho
from paper_2311_11466_gb300 import native, synth

from gpu_cases import gpu_recon, oracle_problem

pytestmark = pytest.mark.gpu

ITERS = 100


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


@pytest.mark.parametrize("name", ["DC", "DR", "RAAR"])
def test_tiny_scan_long_run(name):
    scan = synth.make_scan(synth.named_spec("tiny"))
    abc = native.PRESETS[name]
    prob, x = oracle_problem(scan)
    x, errs = prob.run(x, *abc, ITERS)
    z = optycho.exit_waves(prob.P, prob.O, scan.pos)
    ef_ref = metrics.fourier_error(z, prob.I)
    eo_ref = metrics.object_error(prob.O, scan.obj_true, scan.N)
    with gpu_recon(scan) as r:
        r.iterate(*abc, ITERS)
        e = r.errors()
        ef = r.model_error()
        O, P = r.object_probe()
    eo = metrics.object_error(O, scan.obj_true, scan.N)
    assert abs(ef - ef_ref) <= 1e-3 * ef_ref, (ef, ef_ref)
    assert abs(eo - eo_ref) <= 1e-3 * eo_ref, (eo, eo_ref)
    np.testing.assert_allclose(e, errs, rtol=1e-3)
    assert errs[-1] < errs[0]   # the reconstruction makes progress
