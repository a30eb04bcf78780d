"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/*.h; host-side validation that needs no GPU."""
import glob
import os
import re

import numpy as np
import pytest

from oracle import abc as oabc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2311_11466_gb300 import build, native
    build.build()
    native.lib()
    return native


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(ptycho\w*)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(native):
    import ctypes
    L = ctypes.CDLL(native.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert _declared(), "no declarations found"
    assert not missing, missing


def test_binding_covers_the_abi(native):
    from paper_2311_11466_gb300 import serve
    for n in _declared():
        assert hasattr(native, n) or hasattr(serve, n), n


def test_presets_match_oracle_readings(native):
    for name, abc in native.PRESETS.items():
        assert abc == pytest.approx(oabc.preset(name)), name


def test_scan_bytes_scales_with_positions(native):
    a = native.ptycho_scan_bytes(1024, 256, 1300, 1300)
    b = native.ptycho_scan_bytes(2048, 256, 1300, 1300)
    # x, y, sqrt(I): 20 bytes per pixel per position at least
    assert b - a >= 1024 * 256 * 256 * 20
    assert native.ptycho_scan_bytes(0, 256, 1300, 1300) == 0


def test_create_without_gpu_fails_loudly(native):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(native.PtychoError):
        native.ptycho_create()
    assert native.ptycho_last_error(None) != ""
