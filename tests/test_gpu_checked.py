"""The checked build: no workload indexes outside a buffer.

libgbrt_checked.so (built beside libgbrt.so) tests every index that comes
from data against its buffer; tests/checked_workloads.py renders a spread of
workloads through it in a process of its own, syncing after each, and any
stray index surfaces there as GBRT_EBOUNDS.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_index_outside_its_buffer():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, GBRT_LIB_VARIANT="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workloads.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
