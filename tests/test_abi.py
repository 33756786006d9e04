"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/schwinger.h declares.  No compute calls (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?[\s\*]+(sm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_build_and_load():
    import paper_1512_03812_gb300 as P
    P.build()
    lib = P.load()
    assert lib.sm_version() == 1


def test_every_declared_symbol_is_exported_and_bound():
    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import binding
    lib = P.load()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(binding.exported_symbols())


def test_error_path_without_gpu_work():
    import ctypes
    import paper_1512_03812_gb300 as P
    lib = P.load()
    h = ctypes.c_void_p()
    rc = lib.sm_lattice_create(0, None, None, None, None, ctypes.byref(h))
    assert rc == 1 and b"nchains" in lib.sm_last_error()
    assert lib.sm_lattice_destroy(None) == 0
