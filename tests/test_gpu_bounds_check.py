"""The bounds-checking build (-DGBSZ_BOUNDS_CHECK) compiles an index check
into the kernels at every access whose index a kernel computes (codes,
residuals, histogram bins, chunk table, stream and outlier entries, carries,
values, the warp decoder's chunk buffer); a failed check records
GBSZ_ERR_BOUNDS and skips the access.  Built here, then every library path
runs with it in a child process on fields of each kind, valid and corrupt,
and must give the oracle's bytes and floats with no check failing."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checking_build_passes_every_path():
    sys.path.insert(0, ROOT)
    from paper_2007_09625_gb300 import build
    lib = build.build(check=True)
    env = dict(os.environ, GBSZ_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_check_child.py")], env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=900)
    out = r.stdout.decode()
    assert r.returncode == 0, out[-3000:]
    lines = [ln for ln in out.splitlines() if ln.startswith(("ok ", "FAIL"))]
    assert len(lines) >= 19, out[-3000:]
    fails = [ln for ln in lines if ln.startswith("FAIL")]
    assert not fails, "\n".join(fails)
