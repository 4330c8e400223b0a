"""Host checks of the device arithmetic (no GPU): the NTT building blocks of
csrc/device.cuh compiled by g++ and run with the pass structure of the
library's NTT kernels (tests/host/ntt_check.cpp): forward values against
direct evaluation at psi^(2 brev(c) + 1), inverse(forward) == identity, the
scaled inverse, the lazy-reduction bounds, and the approximate-quotient
Shoup product and narrow centred lift on random and extreme inputs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ntt_building_blocks_on_the_host(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    exe = str(tmp_path / "ntt_check")
    src = os.path.join(ROOT, "tests", "host", "ntt_check.cpp")
    inc = os.path.join(ROOT, "paper_2405_02238_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", inc, src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
