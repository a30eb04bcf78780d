"""Unnormalised 2-D DFT as dense matrix products, FP64 (oracle).

Convention (the paper fixes none; this is the reading used throughout):
forward F x(q) = sum_r x(r) exp(-2 pi i q.r / N), no normalisation, no shift;
inverse includes 1/N^2.  The divide step of the paper (Introduction, Fig. 3(a)
"divide": per-component projection) applies the Fourier-modulus constraint in
this transform domain.

The exponent q*n is reduced mod N in exact integer arithmetic before the
exponential, so every matrix entry is a correctly rounded root of unity.
"""
from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=16)
def dft_matrix(N: int) -> np.ndarray:
    """F_N[q, n] = exp(-2 pi i ((q n) mod N) / N), complex128, read-only."""
    q = np.arange(N, dtype=np.int64)
    k = np.outer(q, q) % N
    F = np.exp(-2j * np.pi * k.astype(np.float64) / N)
    F.setflags(write=False)
    return F


def fft2(x: np.ndarray) -> np.ndarray:
    """Forward unnormalised 2-D DFT of one N x N array: F_N @ x @ F_N^T."""
    N = x.shape[-1]
    F = dft_matrix(N)
    return F @ x @ F.T


def ifft2(X: np.ndarray) -> np.ndarray:
    """Inverse 2-D DFT: conj(F_N) @ X @ conj(F_N)^T / N^2."""
    N = X.shape[-1]
    Fc = dft_matrix(N).conj()
    return Fc @ X @ Fc.T / (N * N)
