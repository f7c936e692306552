"""Build the CPU harness of the texture-window geometry (texwin.h)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def build(out_dir: str) -> str:
    so = os.path.join(out_dir, "texwin_host.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "paper_1712_04495_b300", "csrc"), "-o", so,
                           os.path.join(HERE, "texwin_host.cpp")])
    return so
