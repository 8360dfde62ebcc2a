"""CPU-only checks of the boundary: the C-ABI library builds for sm_103a, loads without a GPU,
and exports every function include/gblod.h declares; the oracle and the library share nothing."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gblod.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(gblod_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_0811_2055_gb300 import build as B
    return B.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gblod_build_lod", "gblod_render", "gblod_render_bruteforce", "gblod_octree_free",
                 "gblod_octree_export", "gblod_renderer_create", "gblod_renderer_status"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gblod_[a-z0-9_]+)$", out, flags=re.M))
    assert set(_declared()) <= exported


def test_library_is_built_for_sm103a_only():
    from paper_0811_2055_gb300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-gencode" not in " ".join(B.flags()).replace(" ".join(B.ARCH), "")


def test_oracle_and_library_share_nothing(libpath):
    from oracle import oracle as O
    olib = O.build()
    lib_syms = subprocess.run(["nm", "-D", libpath], capture_output=True, text=True).stdout
    or_syms = subprocess.run(["nm", "-D", olib], capture_output=True, text=True).stdout
    assert "orc_" not in lib_syms and "liboracle" not in lib_syms
    assert "gblod_" not in or_syms
    ldd = subprocess.run(["ldd", libpath], capture_output=True, text=True).stdout
    assert "oracle" not in ldd
    # no source file of the library mentions the oracle
    csrc = os.path.join(ROOT, "paper_0811_2055_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "orc_" not in open(os.path.join(csrc, f)).read()
    for f in ("gblod.py", "build.py", "__init__.py"):
        assert "oracle" not in open(os.path.join(ROOT, "paper_0811_2055_gb300", f)).read()


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gblod_status_string.restype = ctypes.c_char_p
    assert lib.gblod_status_string(0) == b"ok"
    assert lib.gblod_status_string(2) == b"value out of range"
    lib.gblod_launch_count.restype = ctypes.c_uint64
    assert lib.gblod_launch_count() == 0
    # argument errors are caught on the host before any CUDA call
    lib.gblod_build_lod.restype = ctypes.c_int
    assert lib.gblod_build_lod(None, None, None, None, ctypes.c_uint64(0), None, None, None, None) == 1
