"""Sequential projections (ptycho_sp_iterate) against the FP64 oracle's
sp_iterate on the same inputs: object and probe after one and three passes,
ascending and shuffled order, lam = 1 and 0.7, and the per-pass Fourier error.

Tolerance: the probe is updated at every one of the J positions of a pass,
so FP32 rounding compounds along a chain of J sequential steps (about J
single-step errors of ~1e-6 at worst): relative L2 <= 1e-4 after one pass of
the 64-position scan.  Over several passes sequential projections amplify
perturbations: FP64 oracle runs whose probe starts 1e-7 apart (relative) end
1e-5, 3e-4 and 6e-3 apart after one, two and three passes.  The three-pass
case is therefore checked against three times the spread of two such
perturbed oracle runs."""
import numpy as np
import pytest

from oracle import sp as osp
from paper_2311_11466_gb300 import native, synth

from gpu_cases import gpu_recon, rel_l2, small_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def tiny():
    return synth.make_scan(synth.named_spec("tiny"))


def _oracle_sp(scan, lam, order, passes, eps=0.0, seed=0):
    O = scan.obj0.astype(np.complex128)
    P = scan.probe0.astype(np.complex128)
    if eps:
        rng = np.random.default_rng(seed)
        P = P * (1 + eps * (rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape)))
    errs = [osp.sp_iterate(O, P, scan.pos, scan.intensity.astype(np.float64), lam, order)
            for _ in range(passes)]
    return O, P, errs


@pytest.mark.parametrize("lam,shuffle", [(1.0, False), (0.7, True)])
def test_sp_one_pass_matches_oracle(tiny, lam, shuffle):
    order = np.random.default_rng(5).permutation(tiny.J) if shuffle else None
    O, P, errs = _oracle_sp(tiny, lam, order, 1)
    with gpu_recon(tiny) as r:
        r.sp_iterate(lam, 1, order)
        Og, Pg = r.object_probe()
        e = r.errors()
    assert rel_l2(Og, O) <= 1e-4
    assert rel_l2(Pg, P) <= 1e-4
    np.testing.assert_allclose(e, errs, rtol=1e-4)


def test_sp_three_passes_within_oracle_sensitivity(tiny):
    order = np.random.default_rng(5).permutation(tiny.J)
    O, P, errs = _oracle_sp(tiny, 1.0, order, 3)
    ens = [_oracle_sp(tiny, 1.0, order, 3, eps=1e-7, seed=s) for s in (1, 2)]
    spread_o = max(rel_l2(e[0], O) for e in ens)
    spread_p = max(rel_l2(e[1], P) for e in ens)
    with gpu_recon(tiny) as r:
        r.sp_iterate(1.0, 3, order)
        Og, Pg = r.object_probe()
        e = r.errors()
    assert rel_l2(Og, O) <= 3 * spread_o + 1e-4
    assert rel_l2(Pg, P) <= 3 * spread_p + 1e-4
    np.testing.assert_allclose(e[0], errs[0], rtol=1e-4)


@pytest.mark.parametrize("N", [128, 256])
def test_sp_then_abc_and_other_sizes(N):
    sc = synth.make_scan(small_spec(N, 2, 3, seed=31, photons=1e6))
    O = sc.obj0.astype(np.complex128)
    P = sc.probe0.astype(np.complex128)
    osp.sp_iterate(O, P, sc.pos, sc.intensity.astype(np.float64), 1.0)
    with gpu_recon(sc) as r:
        r.sp_iterate(1.0, 1)
        Og, Pg = r.object_probe()
        x = r.exit_waves()           # the iterate follows the SP result
        r.iterate(*native.PRESETS["DC"], 1)
    assert rel_l2(Og, O) <= 1e-4
    assert rel_l2(Pg, P) <= 1e-4
    ref = np.stack([P * O[a:a + N, b:b + N] for a, b in sc.pos])
    assert rel_l2(x, ref) <= 1e-5


def test_sp_rejects_bad_order(tiny):
    with gpu_recon(tiny) as r:
        with pytest.raises(native.PtychoError) as ei:
            r.sp_iterate(1.0, 1, np.zeros(tiny.J, dtype=np.int32))
        assert ei.value.code == native.PTYCHO_EINVAL
