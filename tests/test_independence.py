"""Static checks of the separation between the product path and the oracle.

The CUDA library and its binding must not use the oracle (no CPU fallback, no shared
arithmetic), and the oracle must not use the library: the two share only the seeded input
generators, which hold none of the method's arithmetic."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1503_02564_gb300")


def _py_imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
    return names


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_import_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in _py_imports(f), f


def test_cuda_sources_do_not_include_oracle_code():
    for f in list(_files(PKG, (".cu", ".cuh", ".h", ".cpp"))) + list(
            _files(os.path.join(ROOT, "include"), (".h",))):
        src = open(f).read()
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', src):
            assert "oracle" not in inc, (f, inc)


def _package_modules(path):
    """Modules of the package a file imports (``from pkg import x`` counts as pkg.x)."""
    tree = ast.parse(open(path).read(), filename=path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name for a in node.names if a.name.startswith("paper_1503_02564_gb300"))
        elif isinstance(node, ast.ImportFrom) and node.module and \
                node.module.startswith("paper_1503_02564_gb300"):
            if node.module == "paper_1503_02564_gb300":
                mods.update(node.module + "." + a.name for a in node.names)
            else:
                mods.add(node.module)
    return mods


def test_oracle_does_not_use_the_library():
    """The oracle may read the shared input generators, nothing else of the package."""
    od = os.path.join(ROOT, "oracle")
    for f in _files(od, (".py",)):
        assert _package_modules(f) <= {"paper_1503_02564_gb300.workloads"}, f
    for f in _files(od, (".c", ".h")):
        src = open(f).read()
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', src):
            assert "swr" not in inc or "oracle" in inc, (f, inc)


def test_input_generators_hold_no_method_arithmetic():
    """workloads.py draws inputs; it imports neither side and calls no solver."""
    imps = _py_imports(os.path.join(PKG, "workloads.py"))
    assert "oracle" not in imps
    assert not (imps & {"torch", "ctypes"})
