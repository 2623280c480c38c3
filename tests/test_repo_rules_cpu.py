"""Structural rules of the repository, checked on the sources:
* the product (the package and its CUDA/C++ sources) never imports or
  includes the oracle;
* the oracle imports nothing but numpy and the standard library;
* no committed file outside tests/ and bench.py runs the oracle;
* no product, test or profile file refers to the scratch folder.
"""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2606_00817_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield (node.module or "") if node.level == 0 else "." + (node.module or "")


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        for name in _imports(path):
            assert not name.split(".")[0] == "oracle", (path, name)
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        assert not re.search(r'#include\s*[<"][^>"]*oracle', open(path, errors="replace").read()), path


def test_oracle_imports_only_numpy_and_the_standard_library():
    allowed = {"__future__", "numpy", "math", "dataclasses", "typing", "functools", "itertools"}
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for name in _imports(path):
            assert name.split(".")[0] in allowed, (path, name)


def _ignored_top_dirs():
    """Top-level folders .gitignore keeps out of the repository."""
    out = set()
    with open(os.path.join(ROOT, ".gitignore")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#") and line.endswith("/"):
                out.add(line.strip("/").split("/")[0])
    return out


def test_only_tests_smoke_and_bench_run_the_oracle():
    users = set()
    skip = _ignored_top_dirs() | {"oracle"}
    for path in glob.glob(os.path.join(ROOT, "**", "*.py"), recursive=True):
        rel = os.path.relpath(path, ROOT)
        if rel.split(os.sep)[0] in skip:
            continue
        if any(n.split(".")[0] == "oracle" for n in _imports(path)):
            users.add(rel.split(os.sep)[0] if os.sep in rel else rel)
    assert users <= {"tests", "bench.py", "__graft_entry__.py"}, users


def test_no_committed_file_refers_to_the_scratch_folder():
    roots = [PKG, os.path.join(ROOT, "tests"), os.path.join(ROOT, "profiles"),
             os.path.join(ROOT, "include"), os.path.join(ROOT, "oracle")]
    files = [os.path.join(ROOT, f) for f in ("bench.py", "__graft_entry__.py")]
    for r in roots:
        files += [p for p in glob.glob(os.path.join(r, "**", "*"), recursive=True) if os.path.isfile(p)]
    pat = re.compile(r"(^|[^A-Za-z0-9_])_work/")
    for path in files:
        if path.endswith((".so", ".o", ".pyc")) or path == os.path.abspath(__file__):
            continue
        text = open(path, errors="replace").read()
        assert not pat.search(text), path


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """With no compiled library the binding raises; it has nothing to fall
    back on."""
    import pytest
    from paper_2606_00817_gb300 import ddf
    monkeypatch.setattr(ddf, "LIB_PATH", str(tmp_path / "libddf.so"))
    monkeypatch.setattr(ddf, "_LIB", None)
    with pytest.raises(RuntimeError, match="is missing"):
        ddf.lib()
    with pytest.raises(RuntimeError):
        ddf.ddf_param_count(ddf.make_config(6, 128, 4, "bf16"))


def test_every_golden_fixture_states_its_source():
    import json
    files = glob.glob(os.path.join(ROOT, "tests", "golden", "*.json"))
    assert files
    for path in files:
        with open(path) as f:
            src = json.load(f).get("source", "")
        assert isinstance(src, str) and len(src) > 40, path
