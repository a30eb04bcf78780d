"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs."""
import numpy as np

from oracle import ptycho as optycho
from paper_2311_11466_gb300 import native, synth


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_problem(scan, alpha=1e-6):
    """Oracle problem on exactly the inputs the GPU receives."""
    I = scan.intensity.astype(np.float64)
    prob = optycho.Problem(I, scan.pos, scan.obj0.astype(np.complex128),
                           scan.probe0.astype(np.complex128), alpha=alpha)
    x0 = optycho.exit_waves(prob.P, prob.O, scan.pos)
    return prob, x0


def gpu_recon(scan, **kw):
    r = native.Reconstruction(**kw)
    r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
    return r


def small_spec(N, ny=3, nx=4, seed=11, photons=None, jitter=2, M=None):
    step = max(2, N // 4)
    if M is None:
        M = (step * (ny - 1) + N + 6, step * (nx - 1) + N + 9)
    return synth.ScanSpec(N=N, ny=ny, nx=nx, step=step, jitter=jitter, M_rows=M[0], M_cols=M[1],
                          radius=N / 4, defocus=0.02 * (16 / (N / 4)) ** 2, photons=photons,
                          seed=seed)
