"""The C ABI library loads on a machine without a GPU and exports every
function that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1712_04495_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_life_cycle():
    names = _declared()
    for n in ("sg_init", "sg_declare", "sg_try", "sg_wait", "sg_release", "sg_launch", "sg_shutdown",
              "sg_run_trace", "sg_replay", "sg_triad", "sg_spmv", "sg_gemm_bf16"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1712_04495_b300 import abi
    assert sorted(abi.exported_symbols()) == _declared()


def test_host_only_calls(lib):
    lib.sg_strerror.restype = ctypes.c_char_p
    assert lib.sg_strerror(0) == b"ok"
    assert b"pool" in lib.sg_strerror(3)
    lib.sg_replay_workspace_bytes.restype = ctypes.c_uint64
    assert lib.sg_replay_workspace_bytes(1000) > 1000 * 48
    # argument checks happen before any device work
    assert lib.sg_init(None, None, ctypes.c_uint64(0), None) == 4
    # an unknown start-rule flag is refused before anything is allocated
    from paper_1712_04495_b300 import abi
    out = ctypes.c_void_p()
    cfg = abi.SgConfig(1, 0, 0, 0, 0, 0, 2, 0)
    assert lib.sg_init(ctypes.byref(out), ctypes.c_void_p(1 << 20), ctypes.c_uint64(1 << 20),
                       ctypes.byref(cfg)) == 4
    assert out.value is None
    assert lib.sg_gemm_bf16(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 100, 128, 63,
                            None) == 4


def test_gemm_tile_codes():
    from paper_1712_04495_b300 import abi
    assert abi.gemm_tile(256, 256) == (256 << 16) | 256
    assert abi.gemm_tile_name(abi.gemm_tile(128, 64)) == "128x64"
    assert abi.gemm_tile_name(128) == "128x128"          # a plain width names a 128-row tile
    assert len(set(abi.GEMM_TILES)) == 4


def test_config_struct_matches_the_header():
    """sg_config's fields, in order, as the header declares them."""
    import re
    from paper_1712_04495_b300 import abi
    text = open(os.path.join(ROOT, "include", "schedgpu.h")).read()
    body = re.search(r"typedef struct sg_config \{(.*?)\} sg_config;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b(\w+);", body)
    assert names == [n for n, _ in abi.SgConfig._fields_]
    assert ctypes.sizeof(abi.SgConfig) == 32


def test_binding_constants_match_the_header():
    # every #define SG_<NAME> <integer> of the header has the same value in abi.py
    from paper_1712_04495_b300 import abi
    text = open(os.path.join(ROOT, "include", "schedgpu.h")).read()
    checked = 0
    for m in re.finditer(r"^#define\s+(SG_[A-Z0-9_]+)\s+(\d+)u?\b", text, flags=re.M):
        name, val = m.group(1), int(m.group(2))
        if hasattr(abi, name):
            assert getattr(abi, name) == val, name
            checked += 1
    for name in ("SG_OK", "SG_ERR_DEVICE", "SG_POLICY_PRIO_FIRST_FIT", "SG_DEVERR_ITEM"):
        assert hasattr(abi, name), name
    assert checked >= 20


def test_no_alloc_workspace_holds_the_stated_limit():
    """The fixed array behind sg_replay_noalloc (2048 KiB) holds the workspace
    of a trace of exactly SG_REPLAY_NOALLOC_MAX_JOBS jobs; a larger trace is
    refused before any device work."""
    from paper_1712_04495_b300 import abi
    lib = abi.lib()
    n = abi.SG_REPLAY_NOALLOC_MAX_JOBS
    assert lib.sg_replay_workspace_bytes(n) <= 2048 * 1024
    assert lib.sg_replay_noalloc(None, n + 1, 1 << 20, 256, 0, 0, 0, None, None, None) == abi.SG_ERR_TOO_LARGE
