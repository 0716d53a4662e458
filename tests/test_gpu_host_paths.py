"""Host-buffer inputs take two paths: read in place by the kernels (page-locked
memory, or pageable memory on a device with coherent access) or copied to
the device.  Both must give the oracle's answers; the environment switch
GCONN_HOST_STAGE=1 forces the copies, and is read once per process, so each
path runs in a child process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("stage", ["0", "1"])
def test_host_inputs_in_place_and_staged(stage):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, GCONN_HOST_STAGE=stage)
    r = subprocess.run([sys.executable, os.path.join(HERE, "host_paths_check.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "host paths ok" in r.stdout
