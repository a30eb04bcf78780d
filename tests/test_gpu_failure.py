"""Failure detection without a GPU fault: a device wait on a flag that nothing
sets is bounded; the bound fires, the host sees PTYCHO_ETIMEOUT, and the
device and a fresh context keep working afterwards."""
import numpy as np
import pytest

from paper_2311_11466_gb300 import native, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2311_11466_gb300 import build
    build.build()


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    assert native.ptycho_check_bounded_wait(0, 200) == native.PTYCHO_ETIMEOUT
    s = synth.make_scan(synth.named_spec("tiny"))
    with native.Reconstruction() as r:
        r.load_scan(s.pos, s.intensity, s.obj0, s.probe0)
        r.iterate(*native.PRESETS["DC"], 2)
        e = r.errors()
    assert e.shape == (2,) and np.all(np.isfinite(e))


def test_bounded_wait_rejects_bad_arguments():
    assert native.ptycho_check_bounded_wait(0, 0) == native.PTYCHO_EINVAL
    assert native.ptycho_check_bounded_wait(0, 60000) == native.PTYCHO_EINVAL
