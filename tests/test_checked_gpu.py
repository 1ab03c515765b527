"""Sanitizer stand-in: every configuration run through the checked build of
the library (-DDD_CHECKED: each staged span, shared-memory row read and Tensor
Memory window and column is range-checked on the device; a miss is recorded in
the status word and the access skipped), on small, ragged and edge shapes."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_every_configuration_in_range():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_01165_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, DD_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "in range and equal to the oracle" in r.stdout
