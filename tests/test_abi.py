"""CPU checks of the boundary: the library builds, loads, and exports every entry point the
public header declares (no compute call: there may be no GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(whv_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2606_31842_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    decl = declared_functions()
    assert len(decl) >= 14
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_2606_31842_b300 import whv
    assert sorted(whv.EXPORTED) == declared_functions()
    assert whv.whv_version().startswith("whv")


def test_library_is_built_for_sm_103a():
    from paper_2606_31842_b300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2606_31842_b300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "from oracle" not in src, fn
