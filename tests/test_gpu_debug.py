"""The debug build's index checks (-DSCS_DEBUG, scs_debug_error) on the GPU:
over every evaluation path, both segmentations, a batch with a three-channel
stream and swarm iterations, no check fails, and the results are the same
bits as the normal build's (a check only skips an access that would be out
of bounds).  The debug library is built in the child process that loads it."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def scstat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_13170_gb300 import scstat as m
    return m


def test_debug_build_checks_pass_and_change_nothing(scstat, tmp_path):
    sys.path.insert(0, HERE)
    import debug_cases
    ref, dbg = debug_cases.run()
    assert dbg == (False, 0, -1)   # the normal build has no checks
    out = tmp_path / "debug.npz"
    env = dict(os.environ, SCS_DEBUG="1", PYTHONPATH=os.pathsep.join([ROOT, HERE]))
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_cases.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(out)
    is_debug, check, index = got["dbg"]
    assert is_debug == 1, "the child did not load the debug build"
    assert (check, index) == (0, -1), f"index check {check} failed at {index}"
    for k, v in ref.items():
        np.testing.assert_array_equal(got[k], v, err_msg=k)
