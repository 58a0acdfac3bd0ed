"""Boundary checks that need no GPU: the library builds, loads and exports
every entry point declared in include/crk.h; the binding fails loudly when the
library is missing; the product package never imports the oracle."""
import ast
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(crk_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libcrk():
    from paper_2202_02840_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("crk_build_cells", "crk_volumes", "crk_corrections", "crk_forces", "crk_step",
                     "crk_compatible", "crk_h_iterate", "crk_create", "crk_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libcrk):
    for name in declared_functions():
        assert hasattr(libcrk, name), name


def test_exports_match_header_exactly(libcrk):
    from paper_2202_02840_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r" T (crk_[a-z_0-9]+)$", out, flags=re.M)))
    assert exported == declared_functions()


def test_variant_count_matches_the_header():
    from paper_2202_02840_gb300 import crk
    txt = open(os.path.join(ROOT, "include", "crk.h")).read()
    assert int(re.search(r"#define CRK_TUNE_NVARIANT (\d+)", txt).group(1)) == crk.CRK_TUNE_NVARIANT


def test_default_params_are_the_papers(libcrk):
    from paper_2202_02840_gb300 import crk
    p = crk.crk_default_params()
    assert abs(p.gamma - 5 / 3) < 1e-15 and p.n_h == 4 and p.N_res == 268
    assert (p.C_l, p.C_q, p.eps) == (2.0, 1.0, 0.1)
    assert abs(p.eta_crit - 0.25) < 1e-15 and abs(p.eta_fold - 0.05) < 1e-15
    assert (p.C_cfl, p.zeta) == (0.25, 4.0)


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_2202_02840_gb300 import build, crk
    monkeypatch.setattr(crk, "_LIB", None)
    monkeypatch.setattr(build, "LIB", os.path.join(ROOT, "does-not-exist", "libcrk.so"))
    with pytest.raises(RuntimeError, match="not built"):
        crk.lib()


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2202_02840_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                tree = ast.parse(open(os.path.join(dirpath, f)).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), f
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", f
            if f.endswith((".cu", ".cuh", ".h")):
                assert "crk_oracle" not in open(os.path.join(dirpath, f)).read(), f
