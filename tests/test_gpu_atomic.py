"""The atomic concur mode (PTYCHO_CONCUR_ATOMIC) against the FP64 oracle.

The object numerator and denominator are built by shared-memory-staged
atomics (position groups accumulated band by band in a shared-memory box,
then added to the global sums with FP32 / FP64 atomics), the probe's by
register-staged FP64 atomics.  The order of the global additions depends on
timing, so the results are compared with the oracle at the FP32 bar (exit
waves, object and probe relative L2 <= 1e-5, Fourier error within 1e-5
relative), not bitwise; against the deterministic gather the two FP32 paths
differ only by the order of additions."""
import numpy as np
import pytest

from oracle import ptycho as optycho
from paper_2311_11466_gb300 import native, synth

from gpu_cases import conditioned_tol, gpu_recon, oracle_problem, oracle_sensitivity, rel_l2, small_spec

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


def _concur_refs(scan):
    prob, x0 = oracle_problem(scan)
    y = prob.project_D(x0)
    O_ref = optycho.concur_object(y, prob.P, scan.pos, prob.O.shape, prob.alpha)
    P_ref = optycho.concur_probe(y, O_ref, scan.pos, prob.alpha)
    return O_ref, P_ref


@pytest.mark.parametrize("N,ny,nx", [(8, 3, 5), (16, 3, 5), (32, 2, 3), (64, 3, 4), (128, 3, 5),
                                     (256, 3, 5), (256, 1, 1), (256, 1, 2)])
@pytest.mark.parametrize("ppt", [1, 2])
def test_staged_concur_step(N, ny, nx, ppt):
    # DC's first iteration leaves O and P = P_C(P_D x_0) (the concur step)
    scan = synth.make_scan(small_spec(N, ny, nx, seed=70 + N + nx))
    O_ref, P_ref = _concur_refs(scan)
    with gpu_recon(scan, concur="atomic") as r:
        r.set_tuning(False)
        r.set_launch_shapes(16, 32, ppt)
        r.iterate(1.0, 1.0, 1.0, 1)
        O, P = r.object_probe()
    # 1e-5, or three times the oracle's own response to a 1e-7 input
    # perturbation where that is larger (one or two positions at 256^2)
    tol = conditioned_tol(TOL, oracle_sensitivity(scan, (1.0, 1.0, 1.0), 1))
    assert rel_l2(O, O_ref) <= tol["O"]
    assert rel_l2(P, P_ref) <= tol["P"]


@pytest.mark.parametrize("name", ["DC", "AR", "DR", "SF", "RAAR", "RRR"])
def test_one_iteration_every_preset(name):
    scan = synth.make_scan(synth.named_spec("tiny"))
    abc = native.PRESETS[name]
    prob, x0 = oracle_problem(scan)
    x1 = prob.iterate(x0, *abc)
    with gpu_recon(scan, concur="atomic") as r:
        r.iterate(*abc, 1)
        x = r.exit_waves()
        O, P = r.object_probe()
        e = r.errors()
    assert rel_l2(x, x1) <= TOL
    assert rel_l2(O, prob.O) <= TOL
    assert rel_l2(P, prob.P) <= TOL
    assert abs(e[0] - prob.last_error) <= TOL * prob.last_error


def test_fermat_scan_and_held_probe():
    """A spiral scan (positions not in raster order, so the groups follow the
    spatial sort, not the position index) with the probe held for the first
    iteration: the held iteration takes the object-only path of the atomic
    mode, the next one the probe atomics."""
    spec = synth.ScanSpec(N=64, step=12, radius=16.0, defocus=0.02, geometry="fermat",
                          n_fermat=40, seed=81)
    scan = synth.make_scan(spec)
    abc = native.PRESETS["RAAR"]
    prob = optycho.Problem(scan.intensity.astype(np.float64), scan.pos,
                           scan.obj0.astype(np.complex128), scan.probe0.astype(np.complex128),
                           probe_start=1)
    x = optycho.exit_waves(prob.P, prob.O, scan.pos)
    errs = []
    for _ in range(2):
        x = prob.iterate(x, *abc)
        errs.append(prob.last_error)
    with native.Reconstruction(concur="atomic") as r:
        r.set_probe_start(1)
        r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
        r.iterate(*abc, 1)
        _, P_held = r.object_probe()
        assert np.array_equal(P_held, scan.probe0)
        r.iterate(*abc, 1)
        xg = r.exit_waves()
        O, P = r.object_probe()
        e = r.errors()
    # two iterations: 2e-5, or three times the oracle's own response to a 1e-7
    # input perturbation where that is larger
    tol = conditioned_tol(2 * TOL, oracle_sensitivity(scan, abc, 2, probe_start=1))
    assert rel_l2(xg, x) <= tol["x"]
    assert rel_l2(O, prob.O) <= tol["O"]
    assert rel_l2(P, prob.P) <= tol["P"]
    np.testing.assert_allclose(e, errs, rtol=2 * TOL)


def test_atomic_and_gather_agree():
    """Both FP32 paths on a 256^2 scan after one iteration: the same sums in
    another order (one iteration only: later iterations of a sparse scan
    amplify rounding differences, see the conditioning bars)."""
    scan = synth.make_scan(small_spec(256, 3, 4, seed=83, photons=1e6))
    abc = native.PRESETS["RAAR"]
    out = {}
    for mode in ("deterministic", "atomic"):
        with gpu_recon(scan, concur=mode) as r:
            r.iterate(*abc, 1)
            out[mode] = (r.exit_waves(), *r.object_probe(), r.errors())
    d, a = out["deterministic"], out["atomic"]
    for u, v in zip(d[:3], a[:3]):
        assert rel_l2(v, u) <= 1e-6
    np.testing.assert_array_equal(a[3], d[3])   # E_F of iteration 1 precedes the concur step
