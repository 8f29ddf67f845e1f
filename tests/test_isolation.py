"""The oracle and the CUDA path share no code, and the product path never reaches the oracle.

Checked on the sources and on the two built libraries: the package's Python imports neither
`oracle` nor the seeded input generators; the CUDA sources include no oracle file and the oracle no
header of the library; neither shared library references the other's symbols; and the only
committed code outside `tests/` that imports the oracle is the benchmark's CPU-baseline / reference
legs and `__graft_entry__` (its build and smoke check)."""
import ast
import glob
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1401_0838_gb300")


def _imports(path):
    """(top-level module, enclosing function or None) for every import in a Python file."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                out.extend((a.name.split(".")[0], func) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.module and child.level == 0:
                out.append((child.module.split(".")[0], func))
            visit(child, f)

    visit(tree, None)
    return out


def test_package_python_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        mods = {m for m, _ in _imports(path)}
        assert not mods & {"oracle", "synth", "tests"}, (path, mods)


def test_oracle_never_imports_the_package():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        mods = {m for m, _ in _imports(path)}
        assert "paper_1401_0838_gb300" not in mods and "synth" not in mods, (path, mods)


def test_sources_include_nothing_of_the_other_side():
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)
    for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(os.path.join(ROOT, "oracle", "oracle.c")).read()):
        assert "/" not in inc and not inc.startswith("pic") and inc.endswith(".h") and "common" not in inc, inc


def test_built_libraries_reference_no_symbol_of_the_other():
    nm = shutil.which("nm")
    lib = os.path.join(PKG, "libpic_gb300.so")
    orc = glob.glob(os.path.join(ROOT, "oracle", "_build", "liboracle.so"))
    if nm is None or not os.path.exists(lib) or not orc:
        pytest.skip("nm or a built library is missing")

    def symbols(path):
        res = subprocess.run([nm, "-D", path], capture_output=True, text=True, check=True)
        return {ln.split()[-1] for ln in res.stdout.splitlines() if ln.strip()}

    assert not {s for s in symbols(lib) if s.startswith("orc_")}
    assert not {s for s in symbols(orc[0]) if s.startswith("pic_")}


def test_only_the_baseline_legs_import_the_oracle():
    allowed = {
        "bench.py": {"oracle_sample", "oracle_sample_3d", "oracle_config1"},
        "__graft_entry__.py": {"build", "smoke"},
    }
    for name, funcs in allowed.items():
        for mod, func in _imports(os.path.join(ROOT, name)):
            if mod == "oracle":
                assert func in funcs, (name, func)
    # and nothing else committed outside tests/ and oracle/ imports it
    for path in glob.glob(os.path.join(ROOT, "*.py")):
        if os.path.basename(path) in allowed:
            continue
        assert "oracle" not in {m for m, _ in _imports(path)}, path
