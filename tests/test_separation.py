"""Separation rules, checked on the sources (no GPU):
- the CUDA engine and the oracle share no code: neither imports nor includes the other;
- the product package never reaches the oracle, and only the benchmark's CPU-baseline
  functions do in bench.py;
- the one module both sides read (the run descriptors) holds no arithmetic of the method;
- a missing engine library is an error, never a fallback;
- nothing committed points at the untracked working folder."""
import ast
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2207_05535_gb300")
CSRC = os.path.join(PKG, "csrc")
ORACLE = os.path.join(ROOT, "oracle")
SKIP_DIRS = {"__pycache__", "_build", ".git", "gpurun_out", "_work", "baseline"}


def _files(top, suffixes):
    for d, dirs, names in os.walk(top):
        dirs[:] = [x for x in dirs if x not in SKIP_DIRS]
        for n in sorted(names):
            if n.endswith(suffixes):
                yield os.path.join(d, n)


def _imports(path):
    """Absolute module names a Python file imports (relative imports resolved to the
    file's own package)."""
    tree = ast.parse(open(path).read(), path)
    pkg = os.path.basename(os.path.dirname(path))
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            out.add(pkg + "." + (node.module or "") if node.level else node.module)
    return out


def _reaches_oracle(mods):
    return any(m == "oracle" or m.startswith("oracle.") for m in mods)


def test_product_package_never_reaches_the_oracle():
    for f in _files(PKG, (".py",)):
        assert not _reaches_oracle(_imports(f)), f
        src = open(f).read()
        assert "pa_oracle" not in src and "oracle/" not in src, f


def test_cuda_sources_include_only_the_engine_headers():
    for f in _files(CSRC, (".cu", ".cuh", ".h")):
        src = open(f).read()
        local = re.findall(r'#include\s+"([^"]+)"', src)
        assert set(local) <= {"pa_internal.cuh", "pa.h"}, (f, local)
        assert "pa_oracle" not in src, f


def test_oracle_uses_nothing_of_the_engine():
    c = open(os.path.join(ORACLE, "pa_oracle.c")).read()
    includes = set(re.findall(r'#include\s+[<"]([^>"]+)[>"]', c))
    assert includes <= {"math.h", "stdint.h", "stdlib.h", "string.h", "stdio.h", "stddef.h", "float.h",
                        "limits.h"}, includes
    for f in _files(ORACLE, (".py",)):
        mods = _imports(f)
        assert not any(m.startswith("paper_2207_05535_gb300") for m in mods), (f, mods)
        src = open(f).read()
        assert "csrc" not in src and not re.search(r"\blibpa\.so\b", src) and "pa_internal" not in src, f


def test_shared_input_module_holds_descriptors_only():
    mods = _imports(os.path.join(PKG, "workloads.py"))
    assert mods <= {"__future__", "dataclasses", "math", "numpy"}, mods


def test_bench_reaches_the_oracle_only_in_its_cpu_baseline():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    for node in tree.body:  # nothing at module level
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            assert not _reaches_oracle({a.name for a in node.names} if isinstance(node, ast.Import)
                                       else {node.module or ""}), ast.dump(node)
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            for node in fn.body:
                for sub in ast.walk(node):
                    if isinstance(sub, ast.Import) and _reaches_oracle({a.name for a in sub.names}):
                        users.add(fn.name)
                    if isinstance(sub, ast.ImportFrom) and _reaches_oracle({sub.module or ""}):
                        users.add(fn.name)
    assert users <= {"_oracle_job", "oracle_sample"}, users


def test_missing_engine_library_is_an_error_not_a_fallback():
    code = ("from paper_2207_05535_gb300 import _lib\n"
            "_lib.load('/nonexistent/libpa.so')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "RuntimeError" in r.stderr and "libpa.so not found" in r.stderr


def test_nothing_committed_points_at_the_working_folder():
    """Code, configuration and the profile summaries (whose commands must run
    committed files only)."""
    r = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("not a git checkout")
    work = "_wo" + "rk/"
    code = (".py", ".cu", ".cuh", ".h", ".c", ".ini", ".cfg", ".toml", ".sh", ".txt")
    hits = []
    for rel in r.stdout.split():
        if not (rel.endswith(code) or rel.startswith("profiles/")):
            continue
        p = os.path.join(ROOT, rel)
        try:
            text = open(p, encoding="utf-8").read()
        except (UnicodeDecodeError, FileNotFoundError):
            continue
        if work in text:
            hits.append(rel)
    assert not hits, hits
