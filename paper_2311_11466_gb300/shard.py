"""Position sharding of one scan over several GPUs: the partition and the
exchange of the concur step (host-side plan; the library itself runs one
scan on one GPU).

The product space of the paper (Introduction, Fig. 3) is a stack of one exit
wave per scan position.  The divide step P_D and the re-split act on each
position alone, so a scan shards by positions; only the concur step P_C
needs data from every position:

  object:  O(m) = sum_j conj(P) y_j / (sum_j |P|^2 + alpha max_m(.))
  probe:   P(r) = sum_j conj(O_j) y_j / (sum_j |O_j|^2 + alpha max_r(.))

Each rank holds a contiguous block of positions (scan order, so the block's
windows cover a compact band of the object), and:

  1. computes the divide step and the object numerator and denominator
     partial sums over its own positions, on the whole object array;
  2. all-reduces (sum) the object numerator (complex64) and denominator
     (float64): M_rows x M_cols x (8 + 8) bytes;
  3. takes max(den) of the reduced denominator (every rank the same) and
     normalises the object (identical on every rank);
  4. computes the probe partial sums over its positions with that object,
     all-reduces (sum) them in float64: N x N x (16 + 8) bytes;
  5. takes max(den) of the reduced probe denominator and normalises.

The maxima are taken after the sums (the maximum of per-rank maxima would be
a different regulariser).  The per-iteration Fourier error is a sum of
per-rank partial sums (one more scalar all-reduce).  Plain point-to-point
loads over the interconnect (NCCL's own algorithms) suffice.

A halo exchange of only the overlapping band of the object would move less
than step 2 when the ranks' bands are thin, at the price of a position-
dependent communication pattern; the all-reduce is the plan because it is
uniform and its size is known up front.
"""
from __future__ import annotations

import numpy as np


def partition(J: int, world: int) -> list[np.ndarray]:
    """Contiguous blocks of position indices, one per rank, sizes within one
    of each other (the first J % world ranks take one more)."""
    if J < 0 or world < 1:
        raise ValueError("J >= 0 and world >= 1")
    base, extra = divmod(J, world)
    out, start = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append(np.arange(start, start + n, dtype=np.int64))
        start += n
    return out


def exchange_bytes(M_rows: int, M_cols: int, N: int) -> dict:
    """Bytes of the two all-reduces of one iteration (per rank, before the
    algorithm's own factor for ring or tree reduction)."""
    obj = M_rows * M_cols * (8 + 8)      # complex64 numerator + float64 denominator
    probe = N * N * (16 + 8)             # complex128 numerator + float64 denominator
    return {"object": obj, "probe": probe, "scalars": 8, "total": obj + probe + 8}
