"""The oracle and the CUDA path share nothing, and only the test side runs the oracle (no GPU).

- Nothing under the package or the public header imports, includes or names `oracle/`.
- Nothing under `oracle/` or `workloads/` imports the package or includes its sources.
- bench.py imports the oracle only inside its CPU legs, and __graft_entry__ only inside smoke().
"""
import ast
import os
import re

from conftest import ROOT

PKG = os.path.join(ROOT, "paper_1704_02770_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or os.sep + "_build" in d or os.sep + "lib" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imported_modules(tree):
    """(module, enclosing function or None) for every import in a parsed file."""
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name, fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.module:
                out.append((child.module, fn))
            visit(child, f)

    visit(tree, None)
    return out


def test_the_cuda_path_never_reaches_the_oracle():
    for path in _files(PKG, (".py",)):
        for mod, _ in _imported_modules(ast.parse(open(path).read())):
            assert not mod.split(".")[0] == "oracle", f"{path} imports {mod}"
    for path in list(_files(PKG, (".cu", ".cuh", ".h"))) + [os.path.join(ROOT, "include", "kry.h")]:
        text = open(path).read()
        assert not re.search(r'#include\s*[<"][^>"]*oracle', text), path
        assert "orc_" not in text, f"{path} names an oracle C symbol"


def test_the_oracle_and_the_inputs_never_reach_the_cuda_path():
    for top in ("oracle", "workloads"):
        for path in _files(os.path.join(ROOT, top), (".py",)):
            for mod, _ in _imported_modules(ast.parse(open(path).read())):
                assert mod.split(".")[0] not in ("paper_1704_02770_gb300", "bench", "torch"), \
                    f"{path} imports {mod}"
        for path in _files(os.path.join(ROOT, top), (".c", ".h")):
            text = open(path).read()
            assert not re.search(r'#include\s*"[^"]*(csrc|kry)', text), path
    for path in _files(os.path.join(ROOT, "workloads"), (".py",)):
        for mod, _ in _imported_modules(ast.parse(open(path).read())):
            assert mod.split(".")[0] != "oracle", f"{path} imports {mod}"


def test_only_the_cpu_legs_and_smoke_run_the_oracle():
    allowed = {"bench.py": {"oracle_sample"}, "__graft_entry__.py": {"smoke", "build"}}
    for name, fns in allowed.items():
        tree = ast.parse(open(os.path.join(ROOT, name)).read())
        for mod, fn in _imported_modules(tree):
            if mod.split(".")[0] == "oracle":
                assert fn in fns, f"{name} imports {mod} in {fn}"
