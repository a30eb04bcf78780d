"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance: exit-wave relative L2 <= 1e-5 after one FP32 iteration (object and
probe likewise); Fourier errors within 1e-5 relative; after 100 iterations of
the tiny scan the Fourier error and the ambiguity-corrected object error
within 1e-3 relative of the oracle's.
"""
import numpy as np
import pytest

from oracle import abc as oabc, metrics, ptycho as optycho
from paper_2311_11466_gb300 import native, synth

from gpu_cases import gpu_recon, oracle_problem, rel_l2, small_spec

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def tiny():
    return synth.make_scan(synth.named_spec("tiny"))


@pytest.mark.parametrize("c", [1.0, 2.0, 0.7, 0.0])
def test_divide_step(tiny, c):
    # (a, b) = (1, 0) makes x_1 = y = P^c_D x_0 exactly; c = 0 makes it the
    # identity up to the FFT round trip
    prob, x0 = oracle_problem(tiny)
    y_ref = oabc.relax(prob.project_D, c)(x0)
    with gpu_recon(tiny) as r:
        r.iterate(1.0, 0.0, c, 1)
        y = r.exit_waves()
        e = r.errors()
    assert rel_l2(y, y_ref) <= TOL
    assert e.shape == (1,)
    assert abs(e[0] - prob.last_error) <= TOL * max(prob.last_error, 1e-30) + 1e-12


def test_concur_step(tiny):
    prob, x0 = oracle_problem(tiny)
    y = prob.project_D(x0)
    O_ref = optycho.concur_object(y, prob.P, tiny.pos, prob.O.shape, prob.alpha)
    P_ref = optycho.concur_probe(y, O_ref, tiny.pos, prob.alpha)
    with gpu_recon(tiny) as r:
        r.iterate(1.0, 1.0, 1.0, 1)
        O, P = r.object_probe()
    assert rel_l2(O, O_ref) <= TOL
    assert rel_l2(P, P_ref) <= TOL


@pytest.mark.parametrize("name", ["DC", "AR", "DR", "SF", "RAAR", "RRR"])
def test_one_iteration_every_preset(tiny, name):
    abc = native.PRESETS[name]
    prob, x0 = oracle_problem(tiny)
    x1 = prob.iterate(x0, *abc)
    with gpu_recon(tiny) as r:
        r.iterate(*abc, 1)
        x = r.exit_waves()
        O, P = r.object_probe()
    assert rel_l2(x, x1) <= TOL
    assert rel_l2(O, prob.O) <= TOL
    assert rel_l2(P, prob.P) <= TOL


@pytest.mark.parametrize("name", ["DC", "DR", "RAAR"])
def test_three_iterations_mixed_state(tiny, name):
    # exercises the lazy re-split (x_prev and y_prev reads) across iterations
    abc = native.PRESETS[name]
    prob, x = oracle_problem(tiny)
    errs = []
    for _ in range(3):
        x = prob.iterate(x, *abc)
        errs.append(prob.last_error)
    with gpu_recon(tiny) as r:
        r.iterate(*abc, 3)
        xg = r.exit_waves()
        e = r.errors()
    assert rel_l2(xg, x) <= 3 * TOL
    np.testing.assert_allclose(e, errs, rtol=3 * TOL)


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128, 256])
def test_pattern_sizes_and_ragged_scans(N):
    # ragged J (3 x 4 = 12, not a multiple of anything), non-square object
    spec = small_spec(N, ny=3, nx=4, seed=N)
    scan = synth.make_scan(spec)
    abc = native.PRESETS["RAAR"]
    prob, x0 = oracle_problem(scan)
    x1 = prob.iterate(x0, *abc)
    with gpu_recon(scan) as r:
        r.iterate(*abc, 1)
        x = r.exit_waves()
        O, P = r.object_probe()
    assert rel_l2(x, x1) <= TOL
    assert rel_l2(O, prob.O) <= TOL
    assert rel_l2(P, prob.P) <= TOL


def test_single_position_at_object_corner():
    spec = synth.ScanSpec(N=64, ny=1, nx=1, step=16, jitter=0, M_rows=64, M_cols=80, radius=16,
                          defocus=0.02, photons=1e4, seed=5)
    scan = synth.make_scan(spec)
    scan.pos[:] = [[0, 16]]   # flush with the bottom-right edge
    from paper_2311_11466_gb300.synth import forward_intensity
    scan.intensity = forward_intensity(scan.probe_true, scan.obj_true, scan.pos).astype(np.float32)
    prob, x0 = oracle_problem(scan)
    x1 = prob.iterate(x0, *native.PRESETS["DR"])
    with gpu_recon(scan) as r:
        r.iterate(*native.PRESETS["DR"], 1)
        x = r.exit_waves()
        O, _ = r.object_probe()
    assert rel_l2(x, x1) <= TOL
    assert rel_l2(O, prob.O) <= TOL
    assert np.all(O[:, :16] == 0)   # never covered: the guard gives exactly 0


def test_model_error_matches_oracle(tiny):
    prob, x0 = oracle_problem(tiny)
    prob.iterate(x0, *native.PRESETS["RAAR"])
    z = optycho.exit_waves(prob.P, prob.O, tiny.pos)
    ref = metrics.fourier_error(z, prob.I)
    with gpu_recon(tiny) as r:
        r.iterate(*native.PRESETS["RAAR"], 1)
        got = r.model_error()
    assert abs(got - ref) <= 1e-4 * ref


def test_noiseless_truth_is_a_fixed_point():
    scan = synth.make_scan(synth.named_spec("tiny"))
    x_true = optycho.exit_waves(scan.probe_true, scan.obj_true, scan.pos).astype(np.complex64)
    with gpu_recon(scan, alpha=0.0) as r:
        r.set_object_probe(scan.obj_true.astype(np.complex64), scan.probe_true.astype(np.complex64))
        r.set_exit_waves(x_true)
        for name in ["DC", "DR", "RAAR"]:
            r.iterate(*native.PRESETS[name], 1)
        x = r.exit_waves()
        e = r.errors()
    assert rel_l2(x, x_true) <= 1e-5
    assert np.all(e < 1e-10)


def test_deterministic_bitwise(tiny):
    outs = []
    for _ in range(2):
        with gpu_recon(tiny) as r:
            r.iterate(*native.PRESETS["RAAR"], 5)
            O, P = r.object_probe()
            outs.append((O, P, r.exit_waves(), r.errors()))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)


def test_checkpoint_resume_bitwise(tiny):
    abc = native.PRESETS["RAAR"]
    with gpu_recon(tiny) as r:
        r.iterate(*abc, 6)
        ref = r.exit_waves(), *r.object_probe()
    with gpu_recon(tiny) as r:
        r.iterate(*abc, 3)
        x, (O, P) = r.exit_waves(), r.object_probe()
    with gpu_recon(tiny) as r:
        r.set_object_probe(O, P)
        r.set_exit_waves(x)
        r.iterate(*abc, 3)
        got = r.exit_waves(), *r.object_probe()
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_atomic_concur_within_tolerance(tiny):
    prob, x0 = oracle_problem(tiny)
    x1 = prob.iterate(x0, *native.PRESETS["RAAR"])
    with gpu_recon(tiny, concur="atomic") as r:
        r.iterate(*native.PRESETS["RAAR"], 1)
        x = r.exit_waves()
        O, P = r.object_probe()
    assert rel_l2(x, x1) <= TOL
    assert rel_l2(O, prob.O) <= TOL


def test_zero_exit_waves_take_sqrt_I(tiny):
    """Where Psi = 0 the modulus projection returns sqrt(I) with phase 0. A zero
    object makes every exit wave and every Psi zero, so the divide step is
    y = c F^-1(sqrt I) (a closed form, checked here against numpy's inverse
    FFT as well) and the Fourier error is exactly 1."""
    c = 2.0
    obj0 = np.zeros_like(tiny.obj0)
    prob = optycho.Problem(tiny.intensity.astype(np.float64), tiny.pos, obj0.astype(np.complex128),
                           tiny.probe0.astype(np.complex128))
    x0 = optycho.exit_waves(prob.P, prob.O, tiny.pos)
    assert not np.any(x0)
    y_ref = oabc.relax(prob.project_D, c)(x0)
    closed = c * np.fft.ifft2(np.sqrt(tiny.intensity.astype(np.float64)))
    assert rel_l2(y_ref, closed) <= 1e-12
    r = native.Reconstruction()
    with r:
        r.load_scan(tiny.pos, tiny.intensity, obj0, tiny.probe0)
        r.iterate(1.0, 0.0, c, 1)
        y = r.exit_waves()
        e = r.errors()
    assert rel_l2(y, y_ref) <= TOL
    assert abs(e[0] - 1.0) <= TOL


def test_device_intensity_equals_host_intensity(tiny):
    """Intensities given as a device buffer (PTYCHO_LOAD_INTENSITY_DEVICE)
    give bitwise the same run as the host copy; a non-contiguous or
    non-float32 device tensor is refused before the call."""
    torch = pytest.importorskip("torch")
    abc = native.PRESETS["RAAR"]
    with gpu_recon(tiny) as r:
        r.iterate(*abc, 3)
        O_h, P_h = r.object_probe()
        e_h = r.errors()
    dev = torch.from_numpy(tiny.intensity).cuda()
    with native.Reconstruction() as r:
        r.load_scan(tiny.pos, dev, tiny.obj0, tiny.probe0)
        r.iterate(*abc, 3)
        O_d, P_d = r.object_probe()
        e_d = r.errors()
    assert np.array_equal(O_h, O_d) and np.array_equal(P_h, P_d) and np.array_equal(e_h, e_d)
    with native.Reconstruction() as r:
        with pytest.raises(ValueError):
            r.load_scan(tiny.pos, dev.transpose(1, 2), tiny.obj0, tiny.probe0)
        with pytest.raises(ValueError):
            r.load_scan(tiny.pos, dev.double(), tiny.obj0, tiny.probe0)


def test_external_stream_profile_and_device_bytes(tiny):
    """A caller-provided stream gives bitwise the same run as the private one;
    the event hook records one divide and one concur duration per iteration;
    the device bytes of a loaded scan stay within the admission estimate
    (ptycho_scan_bytes, an upper bound) and within 5 % of it."""
    torch = pytest.importorskip("torch")
    abc = native.PRESETS["DR"]
    with gpu_recon(tiny) as r:
        r.iterate(*abc, 4)
        O_a, P_a = r.object_probe()
    st = torch.cuda.Stream()
    with native.Reconstruction(stream=st.cuda_stream) as r:
        r.load_scan(tiny.pos, tiny.intensity, tiny.obj0, tiny.probe0)
        native.ptycho_profile_enable(r.h, True)
        r.iterate(*abc, 4)
        div_ms, con_ms, n = native.ptycho_profile_read(r.h)
        native.ptycho_profile_enable(r.h, False)
        O_b, P_b = r.object_probe()
        used = native.ptycho_device_bytes(r.h)
    assert np.array_equal(O_a, O_b) and np.array_equal(P_a, P_b)
    assert n == 4 and div_ms > 0.0 and con_ms > 0.0
    est = native.ptycho_scan_bytes(tiny.J, tiny.N, *tiny.M_shape)
    assert 0.95 * est <= used <= est


def test_empty_scan_rejected(tiny):
    N = tiny.N
    with native.Reconstruction() as r:
        with pytest.raises(native.PtychoError) as ei:
            r.load_scan(np.zeros((0, 2), np.int32), np.zeros((0, N, N), np.float32), tiny.obj0,
                        tiny.probe0)
        assert ei.value.code == native.PTYCHO_EINVAL
        # the context stays usable
        r.load_scan(tiny.pos, tiny.intensity, tiny.obj0, tiny.probe0)
        r.iterate(*native.PRESETS["DC"], 1)
        assert r.iteration_count == 1


def test_validation_errors(tiny):
    with native.Reconstruction() as r:
        with pytest.raises(native.PtychoError) as ei:
            r.iterate(1, 1, 1, 1)
        assert ei.value.code == native.PTYCHO_ESTATE
        bad = tiny.pos.copy()
        bad[3, 0] = 176 - 64 + 1
        with pytest.raises(native.PtychoError) as ei:
            r.load_scan(bad, tiny.intensity, tiny.obj0, tiny.probe0)
        assert ei.value.code == native.PTYCHO_EINVAL
        I = tiny.intensity.copy()
        I[5, 3, 3] = -1.0
        with pytest.raises(native.PtychoError) as ei:
            r.load_scan(tiny.pos, I, tiny.obj0, tiny.probe0)
        assert ei.value.code == native.PTYCHO_EINVAL
        I[5, 3, 3] = np.nan
        with pytest.raises(native.PtychoError):
            r.load_scan(tiny.pos, I, tiny.obj0, tiny.probe0)
        r.load_scan(tiny.pos, tiny.intensity, tiny.obj0, tiny.probe0)
        with pytest.raises(native.PtychoError) as ei:
            r.iterate(float("nan"), 1, 1, 1)
        assert ei.value.code == native.PTYCHO_EINVAL
        with pytest.raises(native.PtychoError):
            r.iterate(1, 1, 1, -1)
        r.iterate(1, 1, 1, 0)
        assert r.iteration_count == 0


def test_scan_beyond_device_memory_is_enomem(tiny):
    """A scan whose footprint (ptycho_scan_bytes, about 1.8 TB here) exceeds
    the device fails with ENOMEM before its intensities are read -- the buffer
    passed is a small stand-in that is never touched -- and the context still
    loads and runs a scan that fits."""
    import ctypes
    J, N = 1 << 20, 256
    assert native.ptycho_scan_bytes(J, N, N, N) > (1 << 40)
    pos = np.zeros((J, 2), dtype=np.int32)
    stand_in = np.zeros(16, dtype=np.float32)
    obj = np.ones((N, N), dtype=np.complex64)
    probe = np.ones((N, N), dtype=np.complex64)
    with native.Reconstruction() as r:
        rc = native.lib().ptycho_load_scan(r.h, J, N, pos.ctypes.data_as(ctypes.c_void_p),
                                           stand_in.ctypes.data_as(ctypes.c_void_p), N, N,
                                           obj.ctypes.data_as(ctypes.c_void_p),
                                           probe.ctypes.data_as(ctypes.c_void_p), 0)
        assert rc == native.PTYCHO_ENOMEM
        assert "device memory" in native.ptycho_last_error(r.h)
        r.load_scan(tiny.pos, tiny.intensity, tiny.obj0, tiny.probe0)
        r.iterate(*native.PRESETS["DC"], 2)
        assert np.all(np.isfinite(r.errors()))


def test_a_zero_is_the_identity(tiny):
    """a = 0 makes the update the identity on the exit waves (Introduction:
    x_{k+1} = a (...) + (1 - a) x_k): after any number of iterations with
    a = 0 the exit waves are the initial ones, bit for bit, while the
    concur step still runs (the object and probe move)."""
    with gpu_recon(tiny) as r:
        x0 = r.exit_waves()
        O0, P0 = r.object_probe()
        r.iterate(0.0, 1.8, 2.0, 3)
        x3 = r.exit_waves()
        O3, P3 = r.object_probe()
    np.testing.assert_array_equal(x3, x0)
    assert not np.array_equal(O3, O0) and not np.array_equal(P3, P0)
