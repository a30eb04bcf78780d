"""Long-run parity: 200 iterations of the tiny scan (64 patterns of 64 x 64,
blind start, noiseless) for every preset.

DC is not sensitive to rounding: FP64 oracle runs whose start differs by a
relative 1e-7 (the size of FP32 rounding) end within 2e-4 of each other, so
the GPU must match the oracle's final model Fourier error and phase-ramp-
corrected object error within 1e-3 relative.

AR, DR, SF, RAAR and RRR are chaotic on this blind problem: the same 1e-7
start perturbation of the FP64 oracle changes the 200-iteration errors by
0.6% (AR) up to more than 100% (RRR), with error curves that separate past
1e-3 after about 16 iterations.  No FP32 (or reordered FP64) evaluation can
track one trajectory that long, so for these settings the test checks
(i) the per-iteration error curve within 1e-3 for the first 10 iterations, and
(ii) the final errors within three times the spread of an ensemble of FP64
oracle runs started from rounding-size perturbations of x_0.
"""
import numpy as np
import pytest

from oracle import metrics, ptycho as optycho
from paper_2311_11466_gb300 import native, synth

from gpu_cases import gpu_recon, oracle_problem

pytestmark = pytest.mark.gpu

ITERS = 200


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def scan():
    return synth.make_scan(synth.named_spec("tiny"))


def _oracle(scan, abc, eps=0.0, seed=0):
    prob, x = oracle_problem(scan)
    if eps > 0:
        rng = np.random.default_rng(seed)
        x = x * (1 + eps * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)))
    x, errs = prob.run(x, *abc, ITERS)
    z = optycho.exit_waves(prob.P, prob.O, scan.pos)
    return (metrics.fourier_error(z, prob.I), metrics.object_error(prob.O, scan.obj_true, scan.N),
            np.array(errs))


def _gpu(scan, abc):
    with gpu_recon(scan) as r:
        r.iterate(*abc, ITERS)
        e = r.errors()
        ef = r.model_error()
        O, _ = r.object_probe()
    return ef, metrics.object_error(O, scan.obj_true, scan.N), e


def test_dc_200_iterations(scan):
    abc = native.PRESETS["DC"]
    ef_ref, eo_ref, curve_ref = _oracle(scan, abc)
    ef, eo, curve = _gpu(scan, abc)
    assert abs(ef - ef_ref) <= 1e-3 * ef_ref, (ef, ef_ref)
    assert abs(eo - eo_ref) <= 1e-3 * eo_ref, (eo, eo_ref)
    np.testing.assert_allclose(curve[:100], curve_ref[:100], rtol=1e-3)
    assert curve[-1] < 0.1 * curve[0]


@pytest.mark.parametrize("name", ["AR", "DR", "SF", "RAAR", "RRR"])
def test_chaotic_presets_200_iterations(scan, name):
    abc = native.PRESETS[name]
    ef_ref, eo_ref, curve_ref = _oracle(scan, abc)
    ens = [_oracle(scan, abc, eps=1e-7, seed=s) for s in (1, 2, 3)]
    spread_f = max(abs(e[0] - ef_ref) for e in ens)
    spread_o = max(abs(e[1] - eo_ref) for e in ens)
    ef, eo, curve = _gpu(scan, abc)
    np.testing.assert_allclose(curve[:10], curve_ref[:10], rtol=1e-3)
    assert abs(ef - ef_ref) <= 3 * spread_f + 1e-3 * ef_ref, (ef, ef_ref, spread_f)
    assert abs(eo - eo_ref) <= 3 * spread_o + 1e-3 * eo_ref, (eo, eo_ref, spread_o)
