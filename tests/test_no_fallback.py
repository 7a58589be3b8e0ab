"""The product path has no CPU fallback (CPU checks): a missing library raises, a
machine without a GPU raises instead of computing anything, and no module of the
library package imports the oracle."""
import ast
import os

import pytest

from paper_2604_07980_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2604_07980_gb300")


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(B, "LIB_PATH", os.path.join(PKG, "_build", "no_such_libctm.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(B.CtmError, match="not built"):
        B.lib()


def test_no_gpu_raises_instead_of_computing():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    img = torch.zeros((16, 16), dtype=torch.uint8)
    with pytest.raises((B.CtmError, AssertionError)):
        B.census_build(img, 1, 5, 5, 1)
    with pytest.raises(B.CtmError):
        B._torch()


def test_library_package_never_imports_the_oracle():
    for name in sorted(os.listdir(PKG)):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(PKG, name)).read())
        for node in ast.walk(tree):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            for m in mods:
                assert not m.split(".")[0] == "oracle", f"{name} imports {m}"
    for name in sorted(os.listdir(os.path.join(PKG, "csrc"))):
        src = open(os.path.join(PKG, "csrc", name)).read()
        assert "ctm_oracle" not in src and "orc_" not in src, name
