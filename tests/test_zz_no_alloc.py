"""The allocation-free probe update, ptycho_probe_update_noalloc.

Some callers of this library cannot allocate device memory: their device
memory belongs to their own allocator or pool, or they run a pipeline that
must not allocate once it is running.  For them the library offers one entry
point that takes device buffers for every input and output and keeps its
scratch in a static device array.  This file checks it through the C ABI,
with device buffers the test provides, on two calls in a row (two different
scans, so the second call runs on the scratch the first one left behind):
against the probe that the context-based entry points (ptycho_iterate, then
ptycho_get_object_probe) compute from the same divided exit waves and object,
and against the FP64 oracle's probe update (oracle.ptycho.concur_probe) on
seeded synthetic exit waves and objects, including probe sides that the
context path does not take (N = 48 with J = 300, N = 255 with J = 16: the
sizes where the partial sums fill the most of the scratch), all within the
parity tolerance of the other GPU tests (relative L2 <= 1e-5).

The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2311_11466_gb300 import native, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


def _scans():
    a = synth.make_scan(synth.named_spec("tiny"))
    b = synth.make_scan(synth.ScanSpec(N=128, ny=3, nx=5, step=32, jitter=3, M_rows=210,
                                       M_cols=270, radius=32, defocus=0.005, photons=1e6, seed=9))
    return a, b


def _context_path(scan, alpha):
    # (a, b) = (1, 0) makes the new iterate the divided waves y = P^c_D x_0; the
    # probe after the iteration is the probe update of y with the new object.
    with native.Reconstruction(alpha=alpha) as r:
        r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
        r.iterate(1.0, 0.0, 2.0, 1)
        y = r.exit_waves()
        O, P = r.object_probe()
    return y, O, P


def _no_alloc(y, O, pos, alpha, out=None):
    import torch
    dev = torch.device("cuda", 0)
    yt = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
    Ot = torch.from_numpy(np.ascontiguousarray(O)).to(dev)
    pt = torch.from_numpy(np.ascontiguousarray(pos, dtype=np.int32)).to(dev)
    N = y.shape[-1]
    if out is None:
        out = torch.full((N, N), 7.0 + 7.0j, dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()
    rc = native.ptycho_probe_update_noalloc(yt.data_ptr(), Ot.data_ptr(), pt.data_ptr(),
                                            y.shape[0], N, O.shape[0], O.shape[1], alpha,
                                            out.data_ptr(), None)
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a.astype(np.complex128) - b) / np.linalg.norm(b))


def test_matches_context_path_on_two_calls_in_a_row():
    alpha = 1e-6
    for scan in _scans():
        y, O, P_ref = _context_path(scan, alpha)
        rc, P = _no_alloc(y, O, scan.pos, alpha)
        assert rc == native.PTYCHO_OK
        assert _rel(P, P_ref) <= TOL, (scan.N, _rel(P, P_ref))


def _synthetic(N, J, M, seed):
    """Seeded exit waves, object and valid window corners (no GPU output)."""
    rng = np.random.default_rng(seed)
    y = (rng.standard_normal((J, N, N)) + 1j * rng.standard_normal((J, N, N))).astype(np.complex64)
    O = (rng.uniform(0.5, 1.0, (M, M)) * np.exp(1j * rng.uniform(-np.pi, np.pi, (M, M))))
    O = O.astype(np.complex64)
    pos = rng.integers(0, M - N + 1, size=(J, 2)).astype(np.int32)
    return y, O, pos


@pytest.mark.parametrize("N,J,M", [(64, 64, 176), (48, 300, 120), (255, 16, 300)])
def test_matches_oracle_on_two_calls_in_a_row(N, J, M):
    from oracle import ptycho as optycho
    alpha = 1e-6
    for seed in (0, 1):
        y, O, pos = _synthetic(N, J, M, seed)
        ref = optycho.concur_probe(y.astype(np.complex128), O.astype(np.complex128), pos, alpha)
        rc, P = _no_alloc(y, O, pos, alpha)
        assert rc == native.PTYCHO_OK
        assert _rel(P, ref) <= TOL, (N, J, seed, _rel(P, ref))


def test_rejects_sizes_beyond_the_scratch_and_bad_windows():
    a, _ = _scans()
    y, O, P_ref = _context_path(a, 1e-6)
    # N above the 256 the scratch holds: rejected on the host, nothing runs
    rc = native.ptycho_probe_update_noalloc(1, 1, 1, 4, 512, 600, 600, 1e-6, 1, None)
    assert rc == native.PTYCHO_EINVAL
    # a window outside the object: skipped on the device, reported, output untouched
    bad = a.pos.copy()
    bad[5] = [O.shape[0] - a.N + 1, 0]
    rc, P = _no_alloc(y, O, bad, 1e-6)
    assert rc == native.PTYCHO_EINVAL
    assert np.all(P == np.complex64(7.0 + 7.0j))
    # and the next valid call is correct again
    rc, P = _no_alloc(y, O, a.pos, 1e-6)
    assert rc == native.PTYCHO_OK
    assert _rel(P, P_ref) <= TOL
