"""Compile the oracle's C sources with plain gcc: ``oracle/_des.so`` (the
admission simulator) and ``oracle/_omp.so`` (the job kinds' reference
results with OpenMP, for the CPU baseline)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_des.so")
OMP_SO = os.path.join(HERE, "_omp.so")


def _compile(src: str, so: str, extra, force: bool) -> str:
    src = os.path.join(HERE, src)
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(src):
        return so
    tmp = so + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared", *extra,
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, so)
    return so


def build(force: bool = False) -> str:
    return _compile("des.c", SO, [], force)


def build_omp(force: bool = False) -> str:
    # no contraction of the triad's product and sum into a fused multiply-add
    return _compile("omp.c", OMP_SO, ["-fopenmp", "-ffp-contract=off"], force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_omp(force=True))
