"""The C-ABI library without a GPU: it builds, loads, exports every function
include/crsh.h declares, its ctypes structs match the C layout, and argument
errors come back synchronously before any CUDA work."""
import ctypes
import glob
import os
import re
import subprocess
import tempfile

import pytest

from paper_2312_06538_gb300 import crsh as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "crsh.h")
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(crsh_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("crsh_hash_sort", "crsh_build", "crsh_traverse", "crsh_closest_hit", "crsh_prepare_scene",
              "crsh_bruteforce_closest_hit", "crsh_status_string", "crsh_version"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = C.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    bound = {s[0] for s in C.SIGNATURES}
    assert set(declared_functions()) <= bound, set(declared_functions()) - bound


def test_version_and_status_strings():
    assert C.crsh_version() >= 100
    lib = C.load()
    assert lib.crsh_status_string(C.ERR_CAPACITY) == b"capacity exceeded"
    assert lib.crsh_status_string(99) == b"unknown status"


STRUCTS = ["crsh_gbuffer", "crsh_rays_in", "crsh_hash_params", "crsh_rays", "crsh_counters", "crsh_scene",
           "crsh_build_params", "crsh_hierarchy", "crsh_traverse_params", "crsh_pairs", "crsh_hits", "crsh_camera",
           "crsh_gbuffer_out", "crsh_scene_out", "crsh_pair_words"]


def test_ctypes_layout_matches_header():
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"crsh.h\"\nint main(void){\n"
    for s in STRUCTS:
        src += f'printf("{s} %zu\\n", sizeof({s}));\n'
    src += 'printf("counters.status %zu\\n", offsetof(crsh_counters, status));\n'
    src += 'printf("hierarchy.count %zu\\n", offsetof(crsh_hierarchy, count));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = dict(line.split() for line in subprocess.check_output([exe], text=True).splitlines())
    for s in STRUCTS:
        assert int(out[s]) == ctypes.sizeof(getattr(C, s)), s
    assert int(out["counters.status"]) == C.crsh_counters.status.offset
    assert int(out["hierarchy.count"]) == C.crsh_hierarchy.count.offset


def test_argument_errors_are_synchronous():
    lib = C.load()
    P = ctypes.c_void_p
    hp = C.crsh_hash_params((C.F32 * 3)(0, 0, 0), (C.F32 * 3)(1, 1, 1), 13, 13, 5, 7, 8, 1, 1, 1)
    rays = C.crsh_rays()
    # neither or both inputs
    assert lib.crsh_hash_sort(None, None, None, 0, ctypes.byref(hp), ctypes.byref(rays), None, None, None, None, 0,
                              None) == C.ERR_INVALID_ARG
    # bad key layout
    hp2 = C.crsh_hash_params((C.F32 * 3)(0, 0, 0), (C.F32 * 3)(1, 1, 1), 20, 13, 5, 7, 8, 1, 1, 1)
    g = C.crsh_gbuffer()
    assert lib.crsh_hash_sort(ctypes.byref(g), None, None, 0, ctypes.byref(hp2), ctypes.byref(rays), P(1), P(1),
                              P(1), P(1), 0, None) == C.ERR_INVALID_ARG
    bp = C.crsh_build_params(12, 3, 0, 0, 0, 0)   # bundle not a power of two
    h = C.crsh_hierarchy()
    assert lib.crsh_build(ctypes.byref(rays), P(1), ctypes.byref(bp), ctypes.byref(h), None) == C.ERR_INVALID_ARG
    sc = C.crsh_scene()
    assert lib.crsh_prepare_scene(ctypes.byref(sc), None) == C.ERR_INVALID_ARG
    assert lib.crsh_traverse(ctypes.byref(h), ctypes.byref(sc), None, None, None, None, 0, None) == C.ERR_INVALID_ARG
    assert lib.crsh_closest_hit(ctypes.byref(h), ctypes.byref(rays), None, ctypes.byref(sc), None, None, None, None,
                                0, None) == C.ERR_INVALID_ARG
    # the look-back self-test: tile 0 has no predecessor, the spin limit must be in [1, 2^22]
    for tile, limit in ((0, 16), (3, 0), (3, (1 << 22) + 1)):
        assert lib.crsh_lookback_selftest(P(0x1000), P(0x1000), 1, tile, 1, limit, P(0x1000), P(0x1000),
                                          None) == C.ERR_INVALID_ARG


def test_misaligned_workspace_is_an_argument_error():
    """Workspaces are carved into 256-byte-aligned arrays read with 16-byte
    vector accesses; a base off that alignment is refused before any launch
    (only the refused case is called: the pointers here are not memory)."""
    lib = C.load()
    P = ctypes.c_void_p
    hp = C.crsh_hash_params((C.F32 * 3)(0, 0, 0), (C.F32 * 3)(1, 1, 1), 13, 13, 5, 7, 8, 1, 1, 1)
    g = C.crsh_gbuffer(*([P(0x1000)] * 11), 16)
    rays = C.crsh_rays(*([P(0x1000)] * 10), 64)
    for off in (16, 128, 255):
        assert lib.crsh_hash_sort(ctypes.byref(g), None, None, 0, ctypes.byref(hp), ctypes.byref(rays), P(0x1000),
                                  P(0x1000), P(0x1000), P(0x10000 + off), 1 << 20, None) == C.ERR_INVALID_ARG


def test_workspace_queries_are_monotone():
    assert C.crsh_hash_sort_workspace(1000, 100) < C.crsh_hash_sort_workspace(100000, 100)
    assert C.crsh_closest_hit_workspace(10) < C.crsh_closest_hit_workspace(1000)
    h = C.crsh_hierarchy()
    h.levels, h.bundle = 3, 8
    for l, c in enumerate((100, 13, 2)):
        h.capacity[l] = c
    assert 0 < C.crsh_traverse_workspace(h, 1000, 3, 1 << 10) < C.crsh_traverse_workspace(h, 1000, 3, 1 << 20)
    h.bundle = 12
    assert C.crsh_traverse_workspace(h, 1000, 3, 1 << 10) == 0


def test_oracle_and_library_share_nothing():
    """The oracle is built from its own C file and never includes the library header."""
    src = open(os.path.join(ROOT, "oracle", "crsh_oracle.c")).read()
    assert "crsh.h" not in src and "paper_2312_06538_gb300" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_2312_06538_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_2312_06538_gb300", "csrc", f)).read().lower()
    for f in ("crsh.py", "pipeline.py", "__init__.py", "_build.py"):
        txt = open(os.path.join(ROOT, "paper_2312_06538_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt
