"""Seeded synthetic ptychographic scans (the simulated experiment).

This module is the one input generator shared by the CUDA path's tests and
benchmarks and by the FP64 oracle's tests.  It holds none of the
reconstruction's arithmetic: it draws an object, a probe and scan positions,
simulates far-field intensities I_j = |F(P * O_j)|^2 (the forward model of the
experiment, computed with scipy's FFT in FP64), optionally adds Poisson noise,
and builds the blind start (flat object, disk probe).

The paper's simulation (Introduction, blood-cell object of Fig. 5 and the two
probes of Fig. 6) ships no data, so every workload here is a synthetic stand-in
with the same structure:

* object: amplitude U[0.8, 1]; phase = normal noise smoothed by a separable
  Gaussian (sigma = 4 px, truncated at 4 sigma, reflect boundary), then
  min-max scaled to [-pi/2, pi/2];
* probe: a disk of radius R (r measured from (N/2, N/2), r <= R inclusive)
  with a quadratic defocus phase coef * r^2 rad;
* positions: integer top-left window corners (row, col); raster with integer
  jitter U{-jit..jit} per axis clamped to [0, M - N], or a Fermat spiral;
* data: noiseless I_j, or Poisson counts of s * I_j with
  s = photons / mean_j sum_q I_j;
* blind start: O_0 = 1 everywhere, P_0 = the disk of the true radius with a
  flat phase, scaled so that N^2 * sum |P_0|^2 = mean_j sum_q I_j.

Conventions: F is the unnormalised forward DFT (exp(-2 pi i q.r / N)),
intensities are stored unshifted (zero frequency at [0, 0]).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.fft
import scipy.ndimage

__all__ = ["ScanSpec", "Scan", "make_scan", "named_spec", "batch_specs",
           "serving_specs", "NAMED"]


@dataclasses.dataclass(frozen=True)
class ScanSpec:
    """Recipe of one synthetic scan."""
    N: int                      # pattern (and probe) side
    ny: int = 1                 # raster rows (ignored for fermat)
    nx: int = 1                 # raster cols (ignored for fermat)
    step: int = 16              # raster step / spiral spacing, px
    jitter: int = 0             # raster jitter amplitude, px
    M_rows: int = 0             # object rows (0: from geometry)
    M_cols: int = 0             # object cols (0: from geometry)
    radius: float = 16.0        # probe disk radius, px
    defocus: float = 0.0        # probe phase coefficient, rad / px^2
    photons: float | None = None  # photons per pattern (None: noiseless)
    geometry: str = "raster"    # "raster" or "fermat"
    n_fermat: int = 0           # number of spiral points (fermat only)
    margin: int = 16            # object margin when M comes from geometry
    seed: int = 0

    @property
    def J(self) -> int:
        return self.n_fermat if self.geometry == "fermat" else self.ny * self.nx


@dataclasses.dataclass
class Scan:
    spec: ScanSpec
    obj_true: np.ndarray        # complex128 [M_rows, M_cols]
    probe_true: np.ndarray      # complex128 [N, N]
    pos: np.ndarray             # int32 [J, 2], (row, col) top-left
    intensity: np.ndarray       # float32 [J, N, N], the stored data
    intensity64: np.ndarray     # float64 [J, N, N], noiseless exact forward model
    obj0: np.ndarray            # complex64 [M_rows, M_cols], blind start
    probe0: np.ndarray          # complex64 [N, N], blind start

    @property
    def J(self) -> int:
        return int(self.pos.shape[0])

    @property
    def N(self) -> int:
        return int(self.probe_true.shape[0])

    @property
    def M_shape(self) -> tuple[int, int]:
        return tuple(self.obj_true.shape)


def _phase_screen(rng: np.random.Generator, shape) -> np.ndarray:
    noise = rng.standard_normal(shape)
    sm = scipy.ndimage.gaussian_filter(noise, sigma=4.0, mode="reflect", truncate=4.0)
    lo, hi = sm.min(), sm.max()
    if hi == lo:
        return np.zeros(shape)
    return (sm - lo) / (hi - lo) * math.pi - math.pi / 2


def _disk(N: int, radius: float, defocus: float) -> np.ndarray:
    r = np.arange(N, dtype=np.float64) - N / 2
    rr = r[:, None] ** 2 + r[None, :] ** 2
    amp = (rr <= radius * radius).astype(np.float64)
    return amp * np.exp(1j * defocus * rr)


def _raster_positions(spec: ScanSpec, rng, M_rows, M_cols):
    span_r = spec.step * (spec.ny - 1) + spec.N
    span_c = spec.step * (spec.nx - 1) + spec.N
    org_r = (M_rows - span_r) // 2
    org_c = (M_cols - span_c) // 2
    iy, ix = np.meshgrid(np.arange(spec.ny), np.arange(spec.nx), indexing="ij")
    jit = rng.integers(-spec.jitter, spec.jitter + 1, size=(spec.ny * spec.nx, 2)) \
        if spec.jitter > 0 else np.zeros((spec.ny * spec.nx, 2), dtype=np.int64)
    r = org_r + spec.step * iy.reshape(-1) + jit[:, 0]
    c = org_c + spec.step * ix.reshape(-1) + jit[:, 1]
    r = np.clip(r, 0, M_rows - spec.N)
    c = np.clip(c, 0, M_cols - spec.N)
    return np.stack([r, c], axis=1).astype(np.int32)


def _fermat_relative(spec: ScanSpec) -> np.ndarray:
    k = np.arange(spec.n_fermat, dtype=np.float64)
    cst = spec.step / math.sqrt(math.pi)
    th = np.deg2rad(137.508) * k
    rad = cst * np.sqrt(k)
    p = np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1)
    return np.rint(p).astype(np.int64)   # round half to even


def _object_shape(spec: ScanSpec) -> tuple[int, int]:
    if spec.M_rows > 0 and spec.M_cols > 0:
        return spec.M_rows, spec.M_cols
    if spec.geometry == "fermat":
        rel = _fermat_relative(spec)
        ext = rel.max(axis=0) - rel.min(axis=0)
        return (int(ext[0]) + spec.N + 2 * spec.margin,
                int(ext[1]) + spec.N + 2 * spec.margin)
    return (spec.step * (spec.ny - 1) + spec.N + 2 * spec.jitter + 2 * spec.margin,
            spec.step * (spec.nx - 1) + spec.N + 2 * spec.jitter + 2 * spec.margin)


def forward_intensity(probe: np.ndarray, obj: np.ndarray, pos: np.ndarray,
                      workers: int = -1) -> np.ndarray:
    """Noiseless far-field data |FFT2(P * O_j)|^2, FP64 (the simulated experiment)."""
    N = probe.shape[0]
    out = np.empty((pos.shape[0], N, N), dtype=np.float64)
    chunk = 64
    for j0 in range(0, pos.shape[0], chunk):
        j1 = min(pos.shape[0], j0 + chunk)
        ex = np.stack([probe * obj[r:r + N, c:c + N] for r, c in pos[j0:j1]])
        f = scipy.fft.fft2(ex, axes=(-2, -1), workers=workers)
        out[j0:j1] = f.real ** 2 + f.imag ** 2
    return out


def make_scan(spec: ScanSpec, with_data: bool = True) -> Scan:
    """Draw one synthetic scan from its recipe (deterministic in spec.seed)."""
    rng = np.random.default_rng(spec.seed)
    M_rows, M_cols = _object_shape(spec)
    if M_rows < spec.N or M_cols < spec.N:
        raise ValueError("object smaller than the probe window")
    amp = rng.uniform(0.8, 1.0, size=(M_rows, M_cols))
    obj = amp * np.exp(1j * _phase_screen(rng, (M_rows, M_cols)))
    probe = _disk(spec.N, spec.radius, spec.defocus)
    if spec.geometry == "fermat":
        rel = _fermat_relative(spec)
        pos = (rel - rel.min(axis=0) + spec.margin).astype(np.int32)
        if pos.max(axis=0)[0] > M_rows - spec.N or pos.max(axis=0)[1] > M_cols - spec.N:
            raise ValueError("fermat positions exceed the object")
    else:
        pos = _raster_positions(spec, rng, M_rows, M_cols)
    J = pos.shape[0]
    N = spec.N
    if with_data:
        I64 = forward_intensity(probe, obj, pos)
        if spec.photons is not None:
            s = spec.photons / float(I64.sum(axis=(1, 2)).mean())
            I = rng.poisson(s * I64).astype(np.float32)
        else:
            I = I64.astype(np.float32)
        mean_tot = float(I.astype(np.float64).sum(axis=(1, 2)).mean())
    else:
        I64 = np.zeros((0, N, N))
        I = np.zeros((0, N, N), dtype=np.float32)
        mean_tot = float(N * N * (np.abs(probe) ** 2).sum())
    p0 = np.abs(_disk(N, spec.radius, 0.0))
    p0_norm = (p0 ** 2).sum()
    scale = math.sqrt(mean_tot / (N * N * p0_norm)) if p0_norm > 0 else 1.0
    probe0 = (p0 * scale).astype(np.complex64)
    obj0 = np.ones((M_rows, M_cols), dtype=np.complex64)
    return Scan(spec=spec, obj_true=obj, probe_true=probe, pos=pos,
                intensity=I, intensity64=I64, obj0=obj0, probe0=probe0)


# Named workloads.  "tiny": 8x8 raster of 64x64 patterns on a 176x176 object,
# noiseless; "large": 32x32 raster of 256x256 patterns on a 1300x1300 object,
# Poisson 1e6 photons; "precision": 64x64 raster of 256x256 patterns on a
# 2296x2296 object, same probe and noise as "large"; "medium": the 16x16
# raster version of "large" (a small case of the same kernels for profiling).
NAMED = {
    "tiny": ScanSpec(N=64, ny=8, nx=8, step=16, jitter=2, M_rows=176, M_cols=176,
                     radius=16.0, defocus=0.02, photons=None, seed=0),
    "large": ScanSpec(N=256, ny=32, nx=32, step=32, jitter=4, M_rows=1300, M_cols=1300,
                      radius=64.0, defocus=0.00125, photons=1e6, seed=1),
    "precision": ScanSpec(N=256, ny=64, nx=64, step=32, jitter=4, M_rows=2296, M_cols=2296,
                          radius=64.0, defocus=0.00125, photons=1e6, seed=3),
    "medium": ScanSpec(N=256, ny=16, nx=16, step=32, jitter=4, M_rows=780, M_cols=780,
                       radius=64.0, defocus=0.00125, photons=1e6, seed=5),
    # the 128^2 half of the uneven-scan mix at the large workload's pixel count
    "large128": ScanSpec(N=128, ny=64, nx=64, step=16, jitter=2, M_rows=1160, M_cols=1160,
                         radius=32.0, defocus=0.005, photons=1e6, seed=7),
}


def named_spec(name: str, **overrides) -> ScanSpec:
    return dataclasses.replace(NAMED[name], **overrides)


def _uneven_spec(rng: np.random.Generator, seed: int, j_lo: int, j_hi: int) -> ScanSpec:
    N = int(rng.choice([128, 256]))
    J = int(round(math.exp(rng.uniform(math.log(j_lo), math.log(j_hi)))))
    photons = float(math.exp(rng.uniform(math.log(1e5), math.log(1e7))))
    step = N // 8
    if rng.uniform() < 0.5:
        ny = max(1, int(math.floor(math.sqrt(J))))
        nx = max(1, int(math.ceil(J / ny)))
        return ScanSpec(N=N, ny=ny, nx=nx, step=step, jitter=step // 8, radius=N / 4,
                        defocus=0.02 * (16.0 / (N / 4)) ** 2, photons=photons,
                        geometry="raster", seed=seed)
    return ScanSpec(N=N, step=step, radius=N / 4, defocus=0.02 * (16.0 / (N / 4)) ** 2,
                    photons=photons, geometry="fermat", n_fermat=J, seed=seed)


def batch_specs(n_scans: int = 16, base_seed: int = 2) -> list[ScanSpec]:
    """Uneven batch: N in {128, 256} 50/50, J log-uniform in [100, 2000],
    raster or Fermat 50/50, step N/8, photons log-uniform in [1e5, 1e7]."""
    out = []
    for i in range(n_scans):
        ss = np.random.SeedSequence([base_seed, i])
        rng = np.random.default_rng(ss)
        out.append(_uneven_spec(rng, int(ss.generate_state(1)[0]), 100, 2000))
    return out


def serving_specs(n_requests: int, base_seed: int = 4) -> list[ScanSpec]:
    """Serving stream: as the batch recipe with J log-uniform in [100, 4096]."""
    out = []
    for i in range(n_requests):
        ss = np.random.SeedSequence([base_seed, i])
        rng = np.random.default_rng(ss)
        out.append(_uneven_spec(rng, int(ss.generate_state(1)[0]), 100, 4096))
    return out
