"""The index-checked build (librexi_debug.so, REXI_DEBUG): the Lanczos kernel
with every indexed access checked against its buffer's extent runs the parity
cases clean and reports a failed check as REXI_EBOUNDS with its site.

The checks stand in for a memory checker: a failed check records the site,
index and extent, skips the access and ends the launch at its next grid
barrier, so no case touches memory outside a buffer; the failing path is
exercised by making each site's check fail on purpose (no bad index exists).
The cases run in a child process with REXI_DEBUG=1 (tests/debug_checks_run.py),
since the binding loads one library per process.
"""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_runs_clean_and_reports_every_site():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03312_gb300 import _native as N
    from paper_1912_03312_gb300 import build
    build.build()
    env = dict(os.environ, REXI_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_checks_run.py")], env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(out["steps"]) >= 10 and all(c["record"] == [0, 0, 0, 0] for c in out["steps"])
    assert out["batched"]["records"] == "clean"
    assert {t["site"] for t in out["trips"]} == set(N.LZ_SITES)
    assert all(t["status"] == N.REXI_EBOUNDS and t["recovered"] for t in out["trips"])
