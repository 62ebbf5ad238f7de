"""The bounds-checked build (a stand-in for a device memory checker): the
parity suite's small cases run through libcp_gb300_checked.so in a fresh
process and must equal the oracle with no call flagged for an out-of-range
index (CP_ERR_INTERNAL would fail them)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


def test_parity_cases_under_the_bounds_checked_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_04801_gb300 import build

    build.build(checked=True)
    env = dict(os.environ, CP_LIB_VARIANT="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
