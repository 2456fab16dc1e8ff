"""CPU tests of the served form's host-only logic (csrc/dfr_tickets.h): a
small C++ program (tests/host/server_tickets_check.cpp) is compiled with g++
under AddressSanitizer and run.

* Several threads waiting on and polling one ticket while it completes: one of
  them takes the request, the others are told the ticket is gone, and none of
  them reads the request after it was freed (a use-after-free would stop the
  sanitized program).
* A dispatcher-thread start that the system refuses comes back as a failure
  (dfr_server_create turns it into DFR_ERR_HOST), not as an exception thrown
  through the C boundary.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "server_tickets_check.cpp")
CSRC = os.path.join(ROOT, "paper_2207_14334_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("srvhost") / "server_tickets_check")
    base = [gxx, "-std=c++17", "-O1", "-g", "-pthread", "-I" + CSRC, SRC, "-o", exe]
    r = subprocess.run(base[:1] + ["-fsanitize=address"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:  # no sanitizer runtime on this machine: plain build
        r = subprocess.run(base, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("what", ["tickets", "refused"])
def test_server_host_logic(checker, what):
    r = subprocess.run([checker, what], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert ("%s ok" % what) in r.stdout
