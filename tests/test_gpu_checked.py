"""The checked build (device-side index checks compiled in, failures counted
in a status word instead of faulting): C1 in every form, C2 at every grain
and the C3 wordcount give the oracle's results with all status words zero.
Then, with every pread the service makes capped at 1,000 bytes (a host-side
knob of the checked build: short reads in the middle of files, which Linux
allows), C1 in every form, C3 in both forms and C5's preads still equal the
oracle, whose reader loops until it has what it asked for or the file ends."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_checked_build_runs_clean(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_06965_b300 import build
    lib = build.build(device_checks=True)
    assert os.path.exists(lib)
    env = dict(os.environ, GENESYS_LIBRARY="checked")
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, os.path.join(here, "checked_run.py"), str(tmp_path)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked ok" in r.stdout
