"""The checked build on the GPU: scans of J = 1, 2, 3 and 4 positions (N = 64
and 256, both divide designs at 256) through the divide step, the concur
step, the model error and sequential projections in libptycho_debug.so.  On
valid input no check may fire (ptycho_debug_flags returns 0) and the results
match the FP64 oracle at the FP32 bar (relative L2 <= 1e-5 after one
iteration, or three times the FP64 oracle's own response to a 1e-7 input
perturbation where that is larger: with one to four positions the scan is
ill-conditioned, and at J = 1, N = 256 that response is 3e-5).  The checked
library is loaded in a child process (PTYCHO_LIB=debug), so the rest of the
suite keeps the normal build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import numpy as np
from paper_2311_11466_gb300 import native, synth
from gpu_cases import conditioned_tol, oracle_problem, oracle_sensitivity, rel_l2, small_spec
assert native.ptycho_debug_build()
out = []
for N, design in ((64, "auto"), (256, "cluster"), (256, "twopass")):
    for J in (1, 2, 3, 4):
        scan = synth.make_scan(small_spec(N, ny=1, nx=J, photons=1e6, seed=40 + J))
        abc = native.PRESETS["RAAR"]
        prob, x0 = oracle_problem(scan)
        x1 = prob.iterate(x0, *abc)
        tol = conditioned_tol(1e-5, oracle_sensitivity(scan, abc, 1))
        with native.Reconstruction(divide=design) as r:
            r.load_scan(scan.pos, scan.intensity, scan.obj0, scan.probe0)
            r.iterate(*abc, 1)
            x = r.exit_waves()
            O, P = r.object_probe()
            r.model_error()
            r.sp_iterate(1.0, 1)
            f = native.ptycho_debug_flags(0)
        out.append({"N": N, "J": J, "design": design, "flags": f,
                    "x": rel_l2(x, x1) / tol["x"], "O": rel_l2(O, prob.O) / tol["O"],
                    "P": rel_l2(P, prob.P) / tol["P"]})
print(json.dumps(out))
'''


def test_checked_build_on_small_scans():
    from paper_2311_11466_gb300 import build
    build.build(debug=True)
    code = CHILD.replace("ROOT", repr(ROOT))
    res = subprocess.run([sys.executable, "-c", code], env={**os.environ, "PTYCHO_LIB": "debug"},
                         capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    rows = json.loads(res.stdout.strip().splitlines()[-1])
    assert len(rows) == 12
    for row in rows:
        assert row["flags"] == 0, row
        # each entry is the error over its bar
        assert row["x"] <= 1 and row["O"] <= 1 and row["P"] <= 1, row
