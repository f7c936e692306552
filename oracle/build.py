"""Compile the oracle's C sources into ``oracle/_des.so`` with plain gcc."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_des.so")


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "des.c")
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= os.path.getmtime(src):
        return SO
    tmp = SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
                           "-o", tmp, src])
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True))
