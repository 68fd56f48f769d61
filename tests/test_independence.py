"""The oracle and the product path share no code: no Python module of one
imports the other, no C/CUDA source of one includes a file of the other,
and the product package never reaches the oracle (its only shared module,
the seeded input generators, imports neither side).  Static checks of the
sources; nothing is run."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2604_14435_gb300"


def py_files(sub):
    base = os.path.join(ROOT, sub)
    for dirpath, _, files in os.walk(base):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def imported_modules(path):
    tree = ast.parse(open(path).read(), filename=path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                mods.add(node.module)
    return mods


def top(mod):
    return mod.split(".")[0]


def c_includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path, errors="replace").read(), re.M)


def test_oracle_imports_nothing_of_the_package():
    files = list(py_files("oracle"))
    assert files
    for f in files:
        bad = [m for m in imported_modules(f) if top(m) == PKG]
        assert not bad, (f, bad)


def test_package_never_imports_the_oracle():
    files = list(py_files(PKG))
    assert files
    for f in files:
        bad = [m for m in imported_modules(f) if top(m) == "oracle"]
        assert not bad, (f, bad)


def test_input_generators_import_neither_side():
    mods = imported_modules(os.path.join(ROOT, PKG, "workloads.py"))
    assert not [m for m in mods if top(m) in ("oracle", PKG)], mods


def test_native_sources_include_nothing_of_the_other_side():
    csrc = os.path.join(ROOT, PKG, "csrc")
    ours = {f for f in os.listdir(csrc)} | {"dvqls.h"}
    oracle_dir = os.path.join(ROOT, "oracle")
    theirs = {f for f in os.listdir(oracle_dir) if f.endswith((".c", ".h"))}
    assert theirs
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh", ".h")):
            inc = {os.path.basename(i) for i in c_includes(os.path.join(csrc, f))}
            assert not (inc & theirs) and not any("oracle" in i for i in c_includes(os.path.join(csrc, f))), f
    for f in theirs:
        inc = {os.path.basename(i) for i in c_includes(os.path.join(oracle_dir, f))}
        assert not (inc & ours), (f, inc & ours)
