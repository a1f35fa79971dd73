"""The product path has no CPU fallback (no GPU needed).

Every step of the method runs in the CUDA library libgbs.so.  If that library
is missing, the binding and the solver built on it must refuse to run rather
than compute anything on the host, and no module of the package may reach the
FP64 oracle, which is test infrastructure only.
"""
import ast
import os

import pytest

from paper_1907_11771_gb300 import binding as B
from tests.conftest import ROOT

PKG = os.path.join(ROOT, "paper_1907_11771_gb300")


def test_missing_library_raises_everywhere(monkeypatch, tmp_path):
    from paper_1907_11771_gb300.solver import GBSSolver
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "libgbs.so"))
    with pytest.raises(RuntimeError, match="missing"):
        B.lib()
    pb = B.make_problem(B.GBS_WAVE1D, 1, 4, B.GBS_F64, [(16,)], [(1.0,)])
    for call in (lambda: B.gbs_state_elems(pb), lambda: B.gbs_create(pb),
                 lambda: B.gbs_step_noalloc(pb, None, None, 8, (2, 4, 6, 8), (), (), 1, 1, 0.1, 1),
                 lambda: GBSSolver(B.GBS_WAVE1D, [(16,)], [(1.0,)], precision=B.GBS_F64)):
        with pytest.raises(RuntimeError, match="missing"):
            call()


def test_package_never_imports_the_oracle():
    for name in sorted(os.listdir(PKG)):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(PKG, name)).read(), filename=name)
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            else:
                continue
            for m in mods:
                assert m.split(".")[0] != "oracle", f"{name} imports {m}"
