"""The bounds-checked build (libakra_debug.so, -DAKRA_DEBUG) run on every operator family and
solver at small sizes, in a child process whose AKRA_LIBRARY names it (the release build stays
loaded in this process).  Its results must match the oracle and it must record no out-of-bounds
index; the release library must report that it carries no checks (count -1).  With no device
memory checker available, these bounds checks and the workspace-poisoning test stand in for one.
"""
import json
import os
import subprocess
import sys

import pytest

from paper_2606_06175_gb300 import akra as A
from paper_2606_06175_gb300 import build as B

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_release_library_has_no_bounds_checks():
    assert A.akra_debug_violations()["count"] == -1


def test_debug_build_records_no_out_of_bounds_access():
    B.build()
    assert os.path.exists(B.OUT_DEBUG)
    env = dict(os.environ, AKRA_LIBRARY=B.OUT_DEBUG)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"] == "libakra_debug.so"
    assert out["violations"]["count"] == 0, out["violations"]
