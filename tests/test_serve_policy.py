"""Host logic of the serving loop: how the idle streams share the admitted
requests (csrc/serve_policy.h, the header canny_serve includes). Property checks
compiled from tests/native/serve_policy_check.cpp against that header: every
idle stream takes at least one request, batches keep to their image and pixel
limits, a batch of several requests stays within its share, no batch stops
short of both its limits and its share, a lone idle stream takes a whole
batch, and the idle streams together leave nothing waiting when the limits do
not bind."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1710_07745_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="no C++ compiler")
def test_serving_batch_policy_properties(tmp_path):
    exe = str(tmp_path / "serve_policy_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(HERE, "native", "serve_policy_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("0 failures")
