"""The checked build (libptycho_debug.so, the library compiled with
-DPTYCHO_DEBUG): it compiles for sm_103a, exports the same ABI, and reports
itself as the checked build; the normal build reports 0.  The GPU half
(J = 1..4 scans run through every kernel with no check firing) is in
tests/test_gpu_debug_build.py."""
import ctypes
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_compiles_and_reports_itself():
    from paper_2311_11466_gb300 import build
    from test_abi import _declared
    path = build.build(debug=True)
    assert path.endswith("libptycho_debug.so") and os.path.exists(path)
    L = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert L.ptycho_debug_build() == 1
    N = ctypes.CDLL(build.build())
    assert N.ptycho_debug_build() == 0


def test_binding_selects_the_checked_build():
    code = ("import sys; sys.path.insert(0, %r); from paper_2311_11466_gb300 import native; "
            "print(native.LIB_PATH.endswith('libptycho_debug.so'), native.ptycho_debug_build())" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], env={**os.environ, "PTYCHO_LIB": "debug"},
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split() == ["True", "True"]
