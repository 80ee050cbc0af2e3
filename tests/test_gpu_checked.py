"""The engine built with invariant checks after every message
(liblob_checked.so, -DLOB_CHECKS): side counts within capacity, sides in
priority order, resting quantities > 0, no crossed book.  A failed check sets
LOB_STATUS_CHECK instead of trapping; the cases in checked_cases.py must
leave the status word at 0 and match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_finds_no_invariant_failure():
    from paper_2308_13289_b300 import build
    build.build(checked=True)
    env = dict(os.environ, LOB_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked-ok" in r.stdout
