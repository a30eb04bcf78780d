"""Position sharding of the concur step (the multi-GPU plan), on CPU with two
gloo ranks: each rank sums the object and probe numerators and denominators
over its own contiguous block of positions (the definitions of the concur
step, written out here), the ranks all-reduce them, and the normalised
object and probe must equal the single-process FP64 oracle's concur step on
all positions, to rounding (the sums are only regrouped)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2311_11466_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_is_contiguous_and_balanced():
    for J, world in [(0, 1), (1, 2), (7, 3), (1024, 8), (1025, 8), (12, 12)]:
        parts = shard.partition(J, world)
        assert len(parts) == world
        assert np.array_equal(np.concatenate(parts) if J else np.array([], dtype=np.int64),
                              np.arange(J))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.partition(4, 0)


def test_exchange_bytes_of_the_bench_workload():
    b = shard.exchange_bytes(1300, 1300, 256)
    assert b["object"] == 1300 * 1300 * 16      # about 27 MB
    assert b["probe"] == 256 * 256 * 24         # 1.5 MiB


def _case():
    from paper_2311_11466_gb300 import synth
    scan = synth.make_scan(synth.ScanSpec(N=16, ny=3, nx=5, step=5, jitter=1, M_rows=40, M_cols=50,
                                          radius=5.0, defocus=0.02, photons=None, seed=12))
    rng = np.random.default_rng(3)
    y = rng.standard_normal((scan.J, 16, 16)) + 1j * rng.standard_normal((scan.J, 16, 16))
    return scan, y, scan.probe0.astype(np.complex128)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scan, y, P = _case()
    N = P.shape[0]
    M = scan.M_shape
    alpha = 1e-6
    mine = shard.partition(scan.J, world)[rank]
    # object partial sums over this rank's positions
    num = np.zeros(M, dtype=np.complex128)
    den = np.zeros(M, dtype=np.float64)
    for j in mine:
        r, c = scan.pos[j]
        num[r:r + N, c:c + N] += np.conj(P) * y[j]
        den[r:r + N, c:c + N] += np.abs(P) ** 2
    t = torch.from_numpy(np.stack([num.real, num.imag, den]))
    dist.all_reduce(t)
    num = t[0].numpy() + 1j * t[1].numpy()
    den = t[2].numpy()
    d = den + alpha * den.max()             # the maximum of the reduced denominator
    O = np.where(d > 0, num / np.where(d > 0, d, 1.0), 0.0)
    # probe partial sums with the new object
    nump = np.zeros((N, N), dtype=np.complex128)
    denp = np.zeros((N, N), dtype=np.float64)
    for j in mine:
        r, c = scan.pos[j]
        Oj = O[r:r + N, c:c + N]
        nump += np.conj(Oj) * y[j]
        denp += np.abs(Oj) ** 2
    t = torch.from_numpy(np.stack([nump.real, nump.imag, denp]))
    dist.all_reduce(t)
    nump = t[0].numpy() + 1j * t[1].numpy()
    denp = t[2].numpy()
    dp = denp + alpha * denp.max()
    Pn = np.where(dp > 0, nump / np.where(dp > 0, dp, 1.0), 0.0)
    out[rank] = (O, Pn, len(mine))
    dist.destroy_process_group()


def test_sharded_concur_equals_single_rank_oracle():
    from oracle import ptycho as optycho
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    scan, y, P = _case()
    O_ref = optycho.concur_object(y, P, scan.pos, scan.M_shape, 1e-6)
    P_ref = optycho.concur_probe(y, O_ref, scan.pos, 1e-6)
    assert sum(res[r][2] for r in range(world)) == scan.J
    for r in range(world):
        O, Pn, _ = res[r]
        np.testing.assert_allclose(O, O_ref, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(Pn, P_ref, rtol=1e-12, atol=1e-14)
