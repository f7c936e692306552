"""Build the host harness of the device engine: engine.cuh compiled by g++
with warp_shim.h standing in for the CUDA intrinsics (test harness only)."""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def build(out_dir: str) -> str:
    src = os.path.join(out_dir, "src")
    os.makedirs(src, exist_ok=True)
    with open(os.path.join(ROOT, "paper_1712_04495_b300", "csrc", "engine.cuh")) as f:
        text = f.read()
    # every state access through the shim's accessors, owned state included
    for old, new in (("return E.owned ? *p : ld_gpu(p);", "return ld_gpu(p);"),
                     ("if (E.owned) *p = v;\n  else st_gpu(p, v);", "st_gpu(p, v);")):
        assert text.count(old) == 1, old
        text = text.replace(old, new)
    with open(os.path.join(src, "engine.cuh"), "w") as f:
        f.write(text)
    with open(os.path.join(src, "common.cuh"), "w") as f:
        f.write('#pragma once\n#include "warp_shim.h"\n')
    so = os.path.join(out_dir, "engine_host.so")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", src, "-I", HERE,
                           "-I", os.path.join(ROOT, "include"), "-o", so,
                           os.path.join(HERE, "engine_host.cpp"), "-lpthread"])
    return so
