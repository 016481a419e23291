"""The checked build of libygs (YGS_DEBUG_BOUNDS=1: every per-solve kernel
checks the global index of its main loads and stores against the extent of
the buffer it addresses and, outside it, skips the access and records the
event for ygs_get_status as YGS_ERR_BOUNDS instead of faulting).

The build is compiled here (its own directory) and exercised in a child
process that loads it through YGS_LIB (a process holds one build): forward
solves, adjoints and a grouped batch of every precision on ragged Yin-Yang,
three-patch and polar grids agree with the CPU FP64 oracle with no index
reported out of range; and with the field extent the checks use shortened
by one shell, a solve's checks report the accesses past it (which they
skip, so nothing leaves the buffers)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_every_precision_clean_and_reports(cuda):
    from paper_1903_08475_gb300 import build as B
    lib = B.build(checked=True)
    env = dict(os.environ, YGS_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_checked_run.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "all ok" in r.stdout, out[-4000:]
    for prec in ("fp64", "fp16x3", "bf16x6", "fp64emu"):
        assert f"ok reported {prec}" in r.stdout, out[-4000:]
