"""The C-ABI library loads and exports every function include/geoheat.h
declares (no device calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "geoheat.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gh_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1812_06060_gb300 import build
    return build.build()


def test_header_lists_the_binding_exports():
    import paper_1812_06060_gb300 as g
    assert sorted(g.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [name for name in _declared() if not hasattr(lib, name)]
    assert not missing


def test_binding_loads_and_reports_version(libpath):
    import paper_1812_06060_gb300 as g
    g.load_library(libpath)
    assert "sm_103a" in g.gh_version()
    p = g.params()
    assert (p.m, p.gs_sweeps, p.admm_iters, p.mu, p.form) == (1.0, 200, 10, 100.0, g.GH_FORM_EDGE)


def test_missing_library_fails_loudly(tmp_path):
    import paper_1812_06060_gb300 as g
    with pytest.raises(ImportError):
        g._lib, saved = None, g._lib
        try:
            g.load_library(str(tmp_path / "nope.so"))
        finally:
            g._lib = saved


def _header_text():
    return open(os.path.join(ROOT, "include", "geoheat.h")).read()


def test_params_struct_matches_header():
    import paper_1812_06060_gb300 as g
    body = re.search(r"typedef struct \{(.*?)\} gh_params;", _header_text(), re.S).group(1)
    fields = re.findall(r"\b(\w+);", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert [f[0] for f in g.GhParams._fields_] == fields


def test_dump_items_match_header():
    import paper_1812_06060_gb300 as g
    items = re.findall(r"\b(GH_DUMP_\w+) = (\d+)", _header_text())
    assert len(items) >= 25
    for name, val in items:
        assert getattr(g, name) == int(val), name


def test_params_defaults_and_path_constraints_flag(libpath):
    import paper_1812_06060_gb300 as g
    g.load_library(libpath)
    assert g.params().path_constraints == 0
    assert g.params(path_constraints=True).path_constraints == 1
