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


def oracle_sensitivity(scan, abc, n_iter, eps=1e-7, seeds=(1, 2), probe_start=0):
    """How far the FP64 oracle itself moves (relative L2 of x, O, P after
    n_iter iterations) when x_0 is perturbed by a relative eps, the size of
    the FP32 rounding of the inputs; the largest over a few seeds.  On
    ill-conditioned scans (very few positions, scan edges covered only by the
    blind probe's tail) this exceeds the flat 1e-5 bar, and no FP32
    evaluation can be held to less than this response."""
    def run(e, seed):
        prob, x = oracle_problem(scan)
        prob.probe_start = probe_start
        if e > 0:
            rng = np.random.default_rng(seed)
            x = x * (1 + e * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)))
        for _ in range(n_iter):
            x = prob.iterate(x, *abc)
        return x, prob.O, prob.P
    ref = run(0.0, 0)
    out = [0.0, 0.0, 0.0]
    for sd in seeds:
        got = run(eps, sd)
        for i in range(3):
            out[i] = max(out[i], rel_l2(got[i], ref[i]))
    return {"x": out[0], "O": out[1], "P": out[2]}


def conditioned_tol(base, sens, factor=3.0):
    """The parity bar of each of x, O, P: the flat base, or factor times the
    oracle's own response to FP32-sized input perturbations where that is
    larger."""
    return {k: max(base, factor * v) for k, v in sens.items()}
