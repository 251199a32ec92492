"""The checked build (GEODOCK_CHECKED: every kernel tests the indices it derives from its inputs and reports a
failure as an error of the call): on the parity workloads' shapes, through every entry point that launches
kernels, it reports no failed check and returns the results of the library bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_matches_and_reports_nothing(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import checked_worker
    from paper_1901_06363_gb300 import build
    assert os.path.exists(build.OUT_CHECKED), "the checked build is missing"
    f = str(tmp_path / "checked.npz")
    env = dict(os.environ, GEODOCK_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_worker.py"), f], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]  # a failed check raises DockError there
    got = np.load(f)
    want = checked_worker.run_cases()
    assert set(got.files) == set(want)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
