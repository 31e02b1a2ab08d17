"""The oracle and the CUDA path share no code: the product package never imports the oracle,
the CUDA sources never include anything from it, the oracle never imports the product package,
and the binding refuses to run without the compiled library (no CPU fallback)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1301_5914_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def _files(root, exts):
    for d, _, fs in os.walk(root):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_package_never_imports_the_oracle():
    for path in _files(PKG, (".py",)):
        assert "oracle" not in _imports(path), path


def test_cuda_sources_include_nothing_from_the_oracle():
    for path in _files(PKG, (".cu", ".cuh", ".h")):
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)


def test_oracle_never_imports_the_product_package():
    for path in _files(os.path.join(ROOT, "oracle"), (".py",)):
        assert "paper_1301_5914_gb300" not in _imports(path), path
    src = open(os.path.join(ROOT, "oracle", "hobi_oracle.c")).read()
    assert not re.search(r'#include\s*"[^"]*(hobi\.h|csrc|hobi_internal)', src)


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_1301_5914_gb300 import hobi

    saved = hobi._lib
    hobi._lib = None  # as in a fresh process
    try:
        with pytest.raises(ImportError):
            hobi.load_library(str(tmp_path / "missing" / "libhobi.so"))
    finally:
        hobi._lib = saved


def _oracle_imports_by_function(path):
    """(enclosing top-level function or None, line) of every import of the oracle package."""
    tree = ast.parse(open(path).read(), path)
    found = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) and fn is None else fn
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.append((name, child.lineno))
            elif isinstance(child, ast.ImportFrom) and child.module and child.module.split(".")[0] == "oracle":
                found.append((name, child.lineno))
            visit(child, name)

    visit(tree, None)
    return found


def test_bench_touches_the_oracle_only_in_its_cpu_leg():
    # the CPU baseline and the reference arm both time the oracle through cpu_oracle_sample
    found = _oracle_imports_by_function(os.path.join(ROOT, "bench.py"))
    assert found and all(fn == "cpu_oracle_sample" for fn, _ in found), found


def test_graft_entry_runs_the_oracle_only_in_smoke():
    # build() compiles the oracle's C (building the checker, not using it); smoke() compares
    found = _oracle_imports_by_function(os.path.join(ROOT, "__graft_entry__.py"))
    assert {fn for fn, _ in found} <= {"build", "smoke"}, found
