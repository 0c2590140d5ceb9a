"""The product path has no CPU fallback: a missing CUDA library raises instead
of computing anything, and nothing in the package imports, links or includes
the oracle."""
import ast
import glob
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2510_01592_gb300")


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2510_01592_gb300 import vm
    missing = os.path.join(ROOT, "no_such_dir", "libvoxmps.so")
    monkeypatch.setattr(vm, "_lib", None)
    monkeypatch.setattr(vm._build, "LIB", missing)
    monkeypatch.setattr(vm._build, "build", lambda *a, **k: missing)  # a build that produced nothing
    with pytest.raises(RuntimeError, match="libvoxmps.so is missing"):
        vm.load(build_if_missing=False)
    with pytest.raises(RuntimeError, match="libvoxmps.so is missing"):
        vm.VoxelMap((8, 8, 8), (0.0, 0.0, 0.0), 0.05)


def test_package_never_reaches_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        tree = ast.parse(open(path).read(), path)
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""] + [a.name for a in node.names]
            else:
                continue
            assert not any("oracle" in n for n in names), (path, names)
        assert "liboracle" not in open(path).read(), path
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        text = open(path).read()
        assert "oracle" not in text.lower(), path
