"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU, and exports
every function declared in include/huge.h."""
import ctypes
import os
import re

from paper_2103_14294_b300 import build, huge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(huge_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    assert lib is not None


def test_every_declared_symbol_is_exported():
    build.build()
    lib = ctypes.CDLL(huge.LIB_PATH)
    declared = declared_functions()
    assert len(declared) >= 14
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the same names
    assert set(huge.exported_names()) <= declared


def test_last_error_without_gpu_calls():
    build.build()
    lib = huge.load()
    assert lib.huge_last_error() in (b"",)
    # null arguments are rejected on the host, before any device work
    rc = lib.huge_graph_load(None, None, 0, 0, 0, None)
    assert rc == huge.EINVAL
    assert lib.huge_last_error()
