"""The scheduler server under ThreadSanitizer on the CPU: its service thread,
eight client threads on the wire protocol, and a thread reading the
counters, over the test engine (no GPU)."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_server_has_no_data_race():
    d = tempfile.mkdtemp(prefix="sg_tsan_")
    exe = os.path.join(d, "tsan_main")
    src = os.path.join(ROOT, "tests", "server_harness", "tsan_main.cpp")
    try:
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-g", "-fsanitize=thread", "-o", exe, src,
                               "-lpthread"])
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("ThreadSanitizer is not available")
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 second_deadlock_stack=1")
    p = subprocess.run([exe, os.path.join(d, "sock")], capture_output=True, text=True, timeout=300, env=env)
    assert "ThreadSanitizer" not in p.stderr, p.stderr[-4000:]
    assert p.returncode == 0, (p.stdout, p.stderr[-2000:])
    assert "served 1200 of 1200" in p.stdout
