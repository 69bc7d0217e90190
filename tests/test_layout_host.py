"""Separation rules checked on the host.  The product package neither
imports nor reads the oracle, and the oracle neither imports nor reads the
package's compute path.  bench.py runs the oracle only from its CPU-baseline
leg and its reference arm.  The binding fails loudly, with no fallback, when
the compiled library is missing."""
import ast
import os

import pytest

from conftest import ROOT

PKG = os.path.join(ROOT, "paper_2302_07804_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(d, exts):
    for dp, _, fn in os.walk(d):
        if "__pycache__" in dp:
            continue
        for f in sorted(fn):
            if f.endswith(exts):
                yield os.path.join(dp, f)


def _imported_modules(path):
    """(module, enclosing function names) for every import in a Python file."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, funcs):
        for ch in ast.iter_child_nodes(node):
            f = funcs + (ch.name,) if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) else funcs
            if isinstance(ch, ast.Import):
                out.extend((a.name, f) for a in ch.names)
            elif isinstance(ch, ast.ImportFrom):
                mod = ("." * ch.level) + (ch.module or "")
                out.extend(((mod + "." + a.name) if not ch.module else mod, f) for a in ch.names)
            visit(ch, f)
    visit(tree, ())
    return out


def test_package_does_not_use_the_oracle():
    for p in _files(PKG, (".py",)):
        for mod, _ in _imported_modules(p):
            assert mod.split(".")[0] != "oracle", (p, mod)
    for p in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h")):
        src = open(p).read()
        assert "oracle" not in src, p
    assert "oracle" not in open(os.path.join(ROOT, "include", "henry.h")).read()


def test_oracle_does_not_use_the_compute_path():
    for p in _files(ORACLE, (".py", ".c", ".h")):
        src = open(p).read()
        for word in ("libhenry", "csrc", "henry.h", "ctypes", "torch.cuda"):
            assert word not in src, (p, word)
        if p.endswith(".py"):
            for mod, _ in _imported_modules(p):
                root = mod.split(".")[0]
                # the seeded input generators are the one module both sides share
                assert root != "paper_2302_07804_gb300" or mod.endswith("inputs"), (p, mod)
                assert root not in ("bench", "__graft_entry__"), (p, mod)


def test_bench_runs_the_oracle_only_in_its_cpu_legs():
    allowed = {"oracle_sample", "_oracle_job", "run_reference"}
    seen = set()
    for mod, funcs in _imported_modules(os.path.join(ROOT, "bench.py")):
        if mod.split(".")[0] == "oracle":
            assert funcs and funcs[0] in allowed, (mod, funcs)
            seen.add(funcs[0])
    assert seen, "bench.py has a CPU-baseline leg that times the oracle"


def test_binding_fails_loudly_without_the_library(monkeypatch):
    from paper_2302_07804_gb300 import henry
    monkeypatch.setattr(henry, "_lib", None)
    monkeypatch.setattr(henry, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libhenry.so"))
    with pytest.raises(RuntimeError) as e:
        henry.Solver()
    assert "not built" in str(e.value)
    with pytest.raises(RuntimeError):
        henry.mlmc_allocate([1.0], [1.0], 1.0)
